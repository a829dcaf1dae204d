#!/usr/bin/env python3
"""Throughput of the P3M gravity step on one GB300 (or N independent replicas).

Workload (default): 128^3 particles, 128^3 mesh, box 200 Mpc/h, r_s = 1.25 mesh cells,
cutoff 4.5 r_s, softening 0.02 mean spacings, Einstein-de Sitter, seeded Zel'dovich ICs
(P(k) ~ k^-2 exp(-(k/k_c)^2), k_c = k_Nyq/2, rms displacement 0.2 cells at a = 0.02),
evolved by the GPU path through 64 log-spaced steps a = 0.02 -> 1 to a clustered state
(untimed set-up).  W warm-up and K timed kick-drift-kick steps then continue from a = 1 with
da = 1e-3 a, so that every measured step processes the clustering of the a = 1 snapshot
whatever K is.  One step = one pass of the whole hot path (kick/drift, keys, sort, permute,
CIC deposit, FFT, k-space pass, 3 inverse FFTs, CIC gather, pair sum, kick).

Printed: one JSON line (rank 0).  `value` = particle-updates/s of the whole job with the
state resident in HBM; `e2e` = the same metric through the C ABI with host (pinned) buffers,
host<->device copies of positions, momenta and accelerations inside the timed region.

--impl reference runs the FP64 CPU oracle on the host cores instead (no GPU work): each
step is the oracle's full mesh force at 128^3 plus its pair sum on a sample of particles of
a synthetic clustered 128^3 snapshot, plus the kick/drift of all particles.
"""

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import p3m_synth as S  # noqa: E402

METRIC = "P3M particle-updates/s"
UNIT = "particle-updates/s"
# algorithmic FP32 flops per accepted pair of the short-range sum: the FP32 arithmetic of the
# FP32 kernel's accepted-pair sequence, FMA = 2: d 3 FADD; r^2 3 FFMA; r^2 + eps^2 FADD;
# s^3 = rsqrt * rcp FMUL; r^3 = r^2 sqrt(r^2) FMUL; tau FFMA; the degree-8 Horner chain 8 FFMA;
# g = 1 + r^3 p FFMA; f = g s^3 FMUL; a += f d 3 FFMA  ->  16 FFMA + 7 FADD/FMUL = 39 flops
# (sqrt, rsqrt and rcp run on the MUFU pipe and are not counted)
FLOPS_PER_PAIR = 39
# the same for the FP64 kernel: d 6 DADD (difference plus image); r^2 DMUL + 2 DFMA; r^2 + eps^2
# DADD; r^3 = r^2 (r^2 rsqrt(r^2)) 2 DMUL; tau DFMA; the degree-18 Horner chain 18 DFMA;
# g DFMA; s^3 and g s^3 3 DMUL; a += f d 3 DFMA  ->  25 DFMA + 13 DADD/DMUL = 63 flops
FLOPS_PER_PAIR_FP64 = 63
WORKLOAD = dict(n_p=128, mesh=128, box=200.0, r_s_cells=1.25, cutoff=4.5, softening=0.02,
                a_begin=0.02, a_end=1.0, setup_steps=64, seed=1512)
WORKLOAD_NAME = ("clustered_128: 128^3 particles, 128^3 mesh, box 200 Mpc/h, r_s 1.25 cells, "
                 "cutoff 4.5 r_s, softening 0.02, EdS; seeded Zel'dovich ICs evolved 64 log "
                 "steps a=0.02->1 on the GPU; measured steps from a=1 with da=1e-3 a")
MEASURE_DA = 1e-3  # relative step of the warm-up and measured steps


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- oracle timing (host)


def stratified_targets(x, stride, offset=0):
    """Every stride-th particle along the oracle's cell order (chaining cells, Hilbert order
    inside them): a sample that holds dense and sparse regions in proportion, so that the
    per-target cost of the pair sum, which grows with the local density, averages like the
    whole set's."""
    from oracle import p3m_oracle as O
    w = WORKLOAD
    q = O.Params(w["box"], x.shape[1], w["mesh"], w["r_s_cells"], w["cutoff"], w["softening"],
                 sub_bits=3)
    _, key = O.cell_keys(x, q)
    return np.sort(O.stable_order(key)[offset::stride])


def oracle_step(pos, mom, stride=1, offset=0):
    """One step of the FP64 oracle on this particle set, timed on the host: the full mesh force
    (all particles), the short-range pair sum, and the kick/drift of all particles.  stride = 1:
    the pair sum of every particle.  stride > 1: the pair sum of the stratified sample of every
    stride-th particle, its per-target time scaled by stride (the set-up of cell keys, order and
    ranges of all N particles, timed by a call with one target, is counted once).  Returns a dict
    of seconds per part, the threads the oracle used and accepted pairs per target particle."""
    from oracle import p3m_oracle as O
    w = WORKLOAD
    n = pos.shape[1]
    p = O.Params(w["box"], n, w["mesh"], w["r_s_cells"], w["cutoff"], w["softening"])
    x = O.wrap(pos, w["box"])
    t0 = time.perf_counter()
    lr = O.pm_accel(x, p)
    t1 = time.perf_counter()
    if stride > 1:
        tg = stratified_targets(x, stride, offset)
        t1 = time.perf_counter()
        O.sr_accel(x, p, targets=tg[:1])
        t1b = time.perf_counter()
        _, npairs = O.sr_accel(x, p, targets=tg)
        t2 = time.perf_counter()
        setup = t1b - t1
        pair = setup + max(0.0, (t2 - t1b) - setup) * (n / tg.size)
        nt = tg.size
    else:
        _, npairs = O.sr_accel(x, p)
        t2 = time.perf_counter()
        pair = t2 - t1
        nt = n
    m = mom + lr * O.kick_factor(1.0, 1.02, p)
    x2 = O.wrap(x + m * O.drift_factor(1.0, 1.04, p), w["box"])
    del x2
    t3 = time.perf_counter()
    return {"seconds": (t1 - t0) + pair + (t3 - t2), "mesh_s": t1 - t0, "pair_s": pair,
            "kick_drift_s": t3 - t2, "threads": O.oracle_threads(), "targets": nt,
            "pairs_per_particle": npairs / nt}


def oracle_step_one_core(pos, mom, stride):
    """oracle_step on one host core (a child process with OMP_NUM_THREADS=1; numpy's FFT and
    array arithmetic are single-threaded): the dict of oracle_step, or None if the child failed."""
    import subprocess
    import tempfile
    with tempfile.TemporaryDirectory() as tmp:
        px, pm = os.path.join(tmp, "x.npy"), os.path.join(tmp, "m.npy")
        np.save(px, pos)
        np.save(pm, mom)
        code = (
            "import sys, json, numpy as np\n"
            f"sys.path.insert(0, {ROOT!r})\n"
            "import bench\n"
            f"print(json.dumps(bench.oracle_step(np.load({px!r}), np.load({pm!r}), {stride})))\n")
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=900)
        if r.returncode != 0:
            return None
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return d if d["threads"] == 1 else None


# ---------------------------------------------------------------- replicas across ranks


def aggregate_ranks(dist, ms_local: float, units_per_rank: int, steps: int, device=None):
    """Whole-job rate of independent replicas (weak scaling, no data-path collective): the
    slowest rank's time over all ranks' units.  Returns (value per second, max ms)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    world = 1
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    ms_max = float(t.item())
    return units_per_rank * world * steps / (ms_max / 1e3), ms_max


# ---------------------------------------------------------------- our arm


def run_ours(args, rank, world, local_rank, dist):
    import torch
    from paper_1510_07621_gb300 import P3M, build

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    w = WORKLOAD
    n = w["n_p"] ** 3
    seed = w["seed"] + rank
    pos0, mom0 = S.zeldovich(w["n_p"], w["box"], w["a_begin"], seed)
    extra = {} if args.sub_bits is None else {"sub_bits": args.sub_bits}
    sim = P3M(w["box"], n, w["mesh"], w["r_s_cells"], w["cutoff"], softening=w["softening"],
              precision=args.precision, stream=stream, **extra)
    sim.set_particles(pos0, mom0, a=w["a_begin"])
    a_s = S.log_spaced_steps(w["a_begin"], w["a_end"], w["setup_steps"])
    t_setup = time.perf_counter()
    for i in range(w["setup_steps"]):
        sim.step(a_s[i], a_s[i + 1] - a_s[i])
    torch.cuda.synchronize(dev)
    t_setup = time.perf_counter() - t_setup
    tuned = None
    if args.autotune:  # the library's autotuner on the a = 1 state, before the warm-up
        tuned_b, tuned_ms = sim.autotune()
        tuned = dict(sim.tuning(), ms_per_sub_bits=[None if not np.isfinite(v) else v
                                                     for v in tuned_ms])
    ratio = 1.0 + MEASURE_DA
    a = a_s[-1]
    for _ in range(args.warmup):
        sim.step(a, a * (ratio - 1.0))
        a *= ratio
    torch.cuda.synchronize(dev)

    if args.save_snapshot and rank == 0:
        snap = np.empty((3, n))
        sim.get_particles(snap, np.empty((3, n)))
        np.save(args.save_snapshot, snap.astype(np.float32))
    d0 = sim.diagnostics()
    sim.set_timing(True)
    sim.timings(reset=True)
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    gpu_index = phys[local_rank] if len(phys) > local_rank and phys[local_rank] else local_rank
    clocks = ClockSampler(gpu_index) if rank == 0 else None
    if clocks:
        clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev0, ev1 = evs[0], evs[-1]
    ev0.record(stream)
    for k in range(args.steps):
        sim.step(a, a * (ratio - 1.0))
        a *= ratio
        evs[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    step_ms = sorted(evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps))
    if dist is not None:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    ms_total = ev0.elapsed_time(ev1)
    phases = sim.timings(reset=True)
    sim.set_timing(False)
    d1 = sim.diagnostics()

    value, ms_max = aggregate_ranks(dist, ms_total, n, args.steps, device=dev)

    # ---- kernels and roofline (per launch = per step)
    K = args.steps
    peaks, peak_kind = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    alu_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # FP32 TFLOP/s
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    pairs_per_step = (d1["pairs_total"] - d0["pairs_total"]) / K
    M = w["mesh"]
    nk = M * M * (M // 2 + 1)
    passes = math.ceil(_key_bits(sim) / 8)
    algo_bytes = {  # algorithmic bytes per launch of each HBM-bound phase
        "kick_drift": 124 * n,
        "sort": 16 * passes * n,  # key histogram read (4 B), then per pass key + slot in and out
        "permute": 128 * n,
        # relative coordinates and key (20 B per particle); per node: the accumulator cleared,
        # accumulated once, read by the conversion (8 B each) and the FP32 mesh written (4 B)
        "deposit": 20 * n + 28 * M ** 3,
        "kspace": 32 * nk,
        "gather": 60 * n,
    }
    kernels = {}
    for name, ms in phases.items():
        if ms <= 0:
            continue
        per = ms / K
        entry = {"ms_per_launch": per, "share": ms / sum(phases.values())}
        if name == "pairs":
            wj = [(b - a) / K for a, b in zip(d0["pair_warp_j"], d1["pair_warp_j"])]
            slots = 32.0 * (wj[0] + wj[2])
            entry.update(bound="alu", achieved=pairs_per_step * FLOPS_PER_PAIR / (per / 1e3) / 1e12,
                         peak=alu_peak, unit="TFLOP/s", pairs_per_launch=pairs_per_step,
                         flops_per_pair=FLOPS_PER_PAIR,
                         warp_j_per_launch={"inside_chunks": wj[0], "tested": wj[1],
                                            "tested_accepted": wj[2]},
                         blocks_culled_per_launch=(d1["pair_blocks_culled"] - d0["pair_blocks_culled"]) / K,
                         tiles_per_launch=[(b - a) / K for a, b in zip(d0["pair_tiles"], d1["pair_tiles"])],
                         accepted_per_evaluated_slot=pairs_per_step / slots if slots else None)
        elif name in algo_bytes:
            entry.update(bound="hbm", achieved=algo_bytes[name] / (per / 1e3) / 1e9,
                         peak=hbm_peak, unit="GB/s")
        if "achieved" in entry:
            entry["frac"] = entry["achieved"] / entry["peak"]
        kernels[name] = entry
    top = max(kernels, key=lambda k: kernels[k]["ms_per_launch"])
    tk = kernels[top]
    roofline = None
    if "achieved" in tk:
        roofline = {"kernel": top, "bound": tk["bound"], "achieved": tk["achieved"],
                    "peak": tk["peak"], "unit": tk["unit"], "frac": tk["frac"],
                    "peak_source": f"{peak_kind}: " + ("SMs x 128 FP32 lanes x 2 x max SM clock"
                                                        if tk["bound"] == "alu" else "hbm_gbs"),
                    "traffic": _traffic(top)}

    # measured FMA throughput of this GPU (library probe): cross-check of the derived ALU peak
    from paper_1510_07621_gb300 import measure_fma_peak
    fma32, fma64 = measure_fma_peak(False), measure_fma_peak(True)
    if roofline is not None and roofline["bound"] == "alu":
        roofline["measured_fma_peak"] = fma32
        roofline["frac_of_measured_fma_peak"] = roofline["achieved"] / fma32

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": ms_max / K,
           "ms_per_step_median": step_ms[len(step_ms) // 2], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 forces, f64 positions/momenta" if args.precision == "mixed" else "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME, "particles": n, "mesh": M,
                      "precision": args.precision, "sub_bits": sim.geometry()["sub_bits"], "parallelism": "replicas" if world > 1 else "single",
                      "l2": "per-step working set (~0.5 GB) larger than L2; no flush",
                      "setup_s": t_setup, "tuning": tuned if tuned else sim.tuning()},
           "roofline": roofline, "kernels": kernels,
           "gpu_launches": int(d1["launches"] - d0["launches"]),
           "pairs_per_step": pairs_per_step, "max_cell_count": d1["max_cell_count"],
           "fma_probe_tflops": {"fp32": fma32, "fp64": fma64},
           "clocks": clk}

    # ---- e2e through the C ABI with pinned host buffers: every rank runs its replica, the
    # slowest rank's time over all ranks' particle-updates (as for value)
    if args.e2e_steps > 0:
        hp = torch.empty((3, n), dtype=torch.float64, pin_memory=True)
        hm = torch.empty((3, n), dtype=torch.float64, pin_memory=True)
        ha = torch.empty((3, n), dtype=torch.float64, pin_memory=True)
        sim.get_particles(hp, hm, ha)
        a_e = a
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sim.set_particles(hp, hm, acc=ha, a=a_e)
            sim.step(a_e, a_e * (ratio - 1.0))
            a_e *= ratio
            sim.get_particles(hp, hm, ha)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        e2e_value, _ = aggregate_ranks(dist, 1e3 * dt, n, args.e2e_steps, device=dev)
        out["e2e"] = {"value": e2e_value, "unit": UNIT, "steps": args.e2e_steps,
                      "h2d_bytes_per_step": 72 * n, "d2h_bytes_per_step": 72 * n,
                      "api": "p3m_set_particles(host pos, mom, acc) + p3m_step + "
                             "p3m_get_particles(host pos, mom, acc)"}

    # ---- all-FP64 GPU mode on the same snapshot, and the force difference between the modes
    if rank == 0 and args.fp64_steps > 0 and args.precision == "mixed":
        hp = torch.empty((3, n), dtype=torch.float64, pin_memory=True)
        hm = torch.empty((3, n), dtype=torch.float64, pin_memory=True)
        sim.get_particles(hp, hm)
        f32 = sim.forces(a)
        with P3M(w["box"], n, w["mesh"], w["r_s_cells"], w["cutoff"], softening=w["softening"],
                 precision="fp64", stream=stream) as s64:
            s64.set_particles(hp, hm, a=a)
            f64 = s64.forces(a)
            s64.step(a, a * (ratio - 1.0))
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0 = s64.diagnostics()["pairs_total"]
            e0.record(stream)
            a64 = a * ratio
            for _ in range(args.fp64_steps):
                s64.step(a64, a64 * (ratio - 1.0))
                a64 *= ratio
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms64 = e0.elapsed_time(e1) / args.fp64_steps
            pairs64 = (s64.diagnostics()["pairs_total"] - p0) / args.fp64_steps
        rms = math.sqrt(float(np.sum((f32 - f64) ** 2) / np.sum(f64 ** 2)))
        out["fp64_gpu"] = {"value": n / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                           "steps": args.fp64_steps,
                           "mixed_vs_fp64_force_rel_rms": rms,
                           "pair_tflops": pairs64 * FLOPS_PER_PAIR_FP64 / (ms64 / 1e3) / 1e12,
                           "flops_per_pair": FLOPS_PER_PAIR_FP64,
                           "fp64_fma_peak_measured": fma64,
                           "pair_frac_of_fp64_peak": pairs64 * FLOPS_PER_PAIR_FP64 / (ms64 / 1e3) / 1e12 / fma64,
                           "speedup_mixed_over_fp64": value / world / (n / (ms64 / 1e3))}

    # ---- CPU baseline: the oracle on this machine's host cores (rank 0, N = 1 only), on the
    # synthetic clustered a = 1 stand-in snapshot: no oracle input comes from the GPU path.  The
    # GPU path is timed on the same snapshot too, so that the two rates compare like work.
    if rank == 0 and world == 1 and args.cpu_stride > 0:
        snap_pos, snap_mom = S.clustered(w["n_p"], w["box"], w["seed"])
        sim.set_particles(snap_pos, snap_mom, a=1.0)
        sim.forces(1.0)
        torch.cuda.synchronize(dev)
        d0 = sim.diagnostics()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        a_s = 1.0
        for _ in range(5):
            sim.step(a_s, MEASURE_DA * a_s)
            a_s *= 1.0 + MEASURE_DA
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_si = e0.elapsed_time(e1) / 5
        d1 = sim.diagnostics()
        gpu_stand_in = {"value": n / (ms_si / 1e3), "unit": UNIT, "ms_per_step": ms_si, "steps": 5,
                        "pairs_per_particle": (d1["pairs_total"] - d0["pairs_total"]) / 5 / n}
        full = oracle_step(snap_pos, snap_mom, args.cpu_stride)
        est = oracle_step(snap_pos, snap_mom, 64) if args.cpu_stride == 1 else None
        one = oracle_step_one_core(snap_pos, snap_mom, 64)
        what = ("all particles" if args.cpu_stride == 1 else
                f"the stratified sample of every {args.cpu_stride}th particle in cell order, its "
                "per-target time scaled")
        out["cpu_baseline"] = {
            "value": n / full["seconds"], "unit": UNIT, "cores": full["threads"], "kind": "oracle",
            "sample": (f"one full oracle step of the synthetic clustered a=1 stand-in snapshot "
                       f"({n} particles): mesh force and kick/drift of all particles, short-range "
                       f"pair sum of {what}"),
            "seconds_per_step": full["seconds"],
            "parts_s": {k: full[k] for k in ("mesh_s", "pair_s", "kick_drift_s")},
            "pairs_per_particle": {"stand_in": full["pairs_per_particle"],
                                   "gpu_timed_state": pairs_per_step / n},
            "gpu_on_stand_in": gpu_stand_in,
            "stratified_estimate_64": None if est is None else {
                "value": n / est["seconds"], "targets": est["targets"],
                "pair_s": est["pair_s"]},
            "one_core": None if one is None else {
                "value": n / one["seconds"], "unit": UNIT, "cores": 1,
                "seconds_per_step": one["seconds"],
                "sample": "one oracle step in a one-thread child process: mesh force and "
                          "kick/drift of all particles, pair sum of the stratified sample of "
                          f"every 64th particle ({one['targets']} targets), its per-target time "
                          "scaled by 64"}}
    sim.close()
    return out


def _key_bits(sim):
    g = sim.geometry()
    cells = g["n_c"] ** 3 << (3 * g["sub_bits"])
    return max(1, int(cells - 1).bit_length())


def _traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    source of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = {"pairs": "pair.cu", "deposit": "mesh.cu", "gather": "mesh.cu", "kspace": "mesh.cu",
           "sort": "sort.cu", "permute": "sort.cu", "kick_drift": "sort.cu"}.get(kernel)
    if not src or not os.path.exists(path):
        return None
    with open(os.path.join(ROOT, "paper_1510_07621_gb300", "csrc", src), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    with open(path) as f:
        for line in f:
            kv = dict(x.split("=", 1) for x in line.split() if "=" in x)
            if kv.get("phase") == kernel and kv.get("source_sha") == sha:
                return int(kv["bytes_per_launch"])
    return None


# ---------------------------------------------------------------- batched ensemble


ENSEMBLE_NAME = ("ensemble48: 48 independent EdS simulations, 16 each of 48^3, 64^3 and 96^3 "
                 "particles, mesh = particle grid, box 100 Mpc/h, r_s 1.25 cells, cutoff 4.5 r_s, "
                 "seeded Zel'dovich ICs (seed 4000+k), 20 log-spaced steps a=0.05->1")


def run_ensemble(args):
    """The 48-simulation ensemble advanced a = 0.05 -> 1 in 20 steps: host-issued steps one
    simulation after another; host-issued steps on one stream per simulation; graph replay
    (8-step graphs for the whole ensemble); each ensemble mode with FFTs batched per mesh size
    (one R2C and one C2R per size group and step) or per simulation, and with per-simulation
    pair launches or one batched pair launch per step.  The value is the library's default:
    graph replay with size-grouped FFTs and per-simulation pair launches.  Every mode starts
    from the ICs with their forces known, so no timed region contains a force evaluation of
    the ICs."""
    import torch
    from paper_1510_07621_gb300 import P3M, Ensemble, build

    build.build()
    torch.cuda.set_device(0)
    sizes = [48] * 16 + [64] * 16 + [96] * 16
    box = 100.0
    a = S.log_spaced_steps(0.05, 1.0, 20)
    ics = [S.zeldovich(n_p, box, a[0], 4000 + k) for k, n_p in enumerate(sizes)]
    total = sum(n_p ** 3 for n_p in sizes)

    def fresh():
        sims = [P3M(box, n_p ** 3, n_p, softening=0.02, stream=0) for n_p in sizes]
        for s_, (p, m) in zip(sims, ics):
            s_.set_particles(p, m, a=a[0])
            s_.forces(a[0])
        torch.cuda.synchronize()
        return sims

    out = {}
    # 1. serial host launches, one simulation after another
    sims = fresh()
    t0 = time.perf_counter()
    for k in range(20):
        for s_ in sims:
            s_.step(a[k], a[k + 1] - a[k])
    torch.cuda.synchronize()
    out["serial_host_launches"] = total * 20 / (time.perf_counter() - t0)
    ref = sims[5].get_particles()[0]
    for s_ in sims:
        s_.close()
    # 2.-5. the ensemble: host launches on per-simulation streams or graph replay, each with
    # per-simulation pair launches or one batched pair launch per step
    for mode, use_graph, batched, groups in (
            ("stream_host_launches", False, False, False),
            ("stream_host_launches_fft_groups", False, False, True),
            ("stream_host_launches_batched_pairs", False, True, False),
            ("graph_ensemble", True, False, True),
            ("graph_ensemble_per_context_fft", True, False, False),
            ("graph_ensemble_batched_pairs", True, True, False)):
        sims = fresh()
        with Ensemble(sims, batched=batched, fft_groups=groups) as ens:
            if use_graph:  # capture outside the timed region, then restore the ICs and their
                # forces by the same evaluation as fresh(), so that the particles start from the
                # same slot order (equal sort keys keep it) as in the serial mode
                ens.run(a[:3], use_graph=True)
                torch.cuda.synchronize()
                for s_, (p, m) in zip(sims, ics):
                    s_.set_particles(p, m, a=a[0])
                    s_.forces(a[0])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ens.run(a, use_graph=use_graph)
            torch.cuda.synchronize()
            out[mode] = total * 20 / (time.perf_counter() - t0)
        pos5 = sims[5].get_particles()[0]
        d = pos5 - ref
        d -= box * np.round(d / box)
        out[mode + "_max_dx_vs_serial"] = float(np.max(np.abs(d)))
        for s_ in sims:
            s_.close()
    value = out["graph_ensemble"]
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": 20,
            "warmup": 3, "ms_per_step": 1e3 * total / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 forces, f64 positions/momenta",
            "data": "synthetic",
            "config": {"workload": ENSEMBLE_NAME, "particles": total, "simulations": 48},
            "modes": out,
            "speedup_graph_over_serial": value / out["serial_host_launches"]}


# ---------------------------------------------------------------- differentiable run


ADJOINT_NAME = ("adjoint128: 128^3 particles, 128^3 mesh, box 200 Mpc/h, 20 log steps a=0.05->1, "
                "L2 loss of the final CIC density contrast against a seeded target, gradient with "
                "respect to the 128^3 initial displacement field, checkpoints every 5 steps")


def run_adjoint(args):
    """Forward run + loss, then the reverse sweep (checkpoints every sqrt(20) ~ 5 steps):
    cost of the gradient per step relative to a forward step."""
    import torch
    from paper_1510_07621_gb300 import P3M, build
    from paper_1510_07621_gb300.adjoint import DensityLossRun

    build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n_p, box, mesh = 128, 200.0, 128
    q = torch.from_numpy(S.lattice(n_p, box)).to(dev)
    _, mom = S.zeldovich(n_p, box, 0.05, 1515)
    psi = torch.from_numpy(mom / np.sqrt(0.05)).to(dev)
    a = S.log_spaced_steps(0.05, 1.0, 20)
    target = torch.from_numpy(0.5 * S.gaussian(1516, mesh ** 3)).to(dev)
    sim = P3M(box, n_p ** 3, mesh, softening=0.02)
    # warm-up (plans, first-touch)
    x = psi.clone().requires_grad_(True)
    DensityLossRun.apply(x, sim, q, a[:3], target, 2).backward()
    torch.cuda.synchronize()
    x = psi.clone().requires_grad_(True)
    t0 = time.perf_counter()
    loss = DensityLossRun.apply(x, sim, q, a, target, 5)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = x.grad
    fwd, bwd = (t1 - t0) / 20, (t2 - t1) / 20
    sim.close()
    return {"metric": METRIC, "value": n_p ** 3 / bwd, "unit": UNIT + " (reverse sweep)",
            "n_gpus": 1, "steps": 20, "warmup": 1, "ms_per_step": 1e3 * bwd,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 forces, f64 positions/momenta", "data": "synthetic",
            "config": {"workload": ADJOINT_NAME, "particles": n_p ** 3},
            "forward_ms_per_step": 1e3 * fwd, "adjoint_ms_per_step": 1e3 * bwd,
            "adjoint_over_forward": bwd / fwd, "loss": float(loss.detach()),
            "grad_rms": float(g.pow(2).mean().sqrt())}


# ---------------------------------------------------------------- reference arm (oracle)


def run_reference(args):
    """The oracle as the reference arm: K timed steps (after W untimed ones) on the synthetic
    clustered a=1 stand-in snapshot, each one full oracle step except that the pair sum runs on
    a stratified sample (every stride-th particle in cell order, stride = max(16, 4 K), its
    per-target time scaled; a different offset each step), so that K + W steps end within a few
    minutes.  The same estimator as the cpu_baseline of our arm."""
    w = WORKLOAD
    n = w["n_p"] ** 3
    pos, mom = S.clustered(w["n_p"], w["box"], w["seed"])
    stride = args.ref_stride or max(16, 4 * args.steps)
    for k in range(args.warmup):
        oracle_step(pos, mom, stride, offset=(k + 1) % stride)
    total, executed, threads, ppp = 0.0, 0, 1, 0.0
    for k in range(args.steps):
        d = oracle_step(pos, mom, stride, offset=(k + args.warmup + 1) % stride)
        total += d["seconds"]
        threads = d["threads"]
        ppp = d["pairs_per_particle"]
        executed += 1
    value = n * executed / total
    desc = (f"{executed} oracle steps, each: mesh force and kick/drift of all {n} particles, "
            f"pair sum of the stratified sample of every {stride}th particle in cell order, its "
            "per-target time scaled")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "steps_executed": executed, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / executed,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME.split(";")[0] +
                       "; synthetic clustered a=1 stand-in snapshot (no GPU evolution)",
                       "particles": n, "mesh": w["mesh"], "pair_sample_stride": stride,
                       "pairs_per_particle": ppp},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- 512^3 Zel'dovich


Z512_NAME = ("zeldovich512: 512^3 particles, 512^3 mesh, box 1000 Mpc/h, r_s 1.25 cells, cutoff "
             "4.5 r_s, softening 0.02, EdS; seeded Zel'dovich ICs at a=0.5 (seed 1513), one force "
             "evaluation, then 10 log-spaced steps a=0.5->1")


def run_zeldovich512(args):
    """The largest configuration: 134 M particles, one force evaluation and 10 steps timed
    with CUDA events on the library's stream."""
    import torch
    from paper_1510_07621_gb300 import P3M, build

    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    n_p, box = 512, 1000.0
    n = n_p ** 3
    pos, mom = S.zeldovich(n_p, box, 0.5, 1513)
    a = S.log_spaced_steps(0.5, 1.0, 10)
    out = {}
    extra = {} if args.sub_bits is None else {"sub_bits": args.sub_bits}
    with P3M(box, n, n_p, softening=0.02, stream=stream, **extra) as sim:
        dpos = torch.from_numpy(pos).cuda()
        dmom = torch.from_numpy(mom).cuda()
        del pos, mom
        sim.set_particles(dpos, dmom, a=a[0])
        tuned = None
        if args.autotune:  # the library's autotuner on the ICs, outside the timed region
            tuned_b, tuned_ms = sim.autotune()
            tuned = dict(sim.tuning(), ms_per_sub_bits=[None if not np.isfinite(v) else v
                                                         for v in tuned_ms])
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        sim.set_timing(True)
        sim.timings(reset=True)
        d0 = sim.diagnostics()
        e0.record(stream)
        sim.forces(a[0])
        e1.record(stream)
        for k in range(10):
            sim.step(a[k], a[k + 1] - a[k])
        e2.record(stream)
        torch.cuda.synchronize()
        phases = sim.timings(reset=True)
        d1 = sim.diagnostics()
    ms_force = e0.elapsed_time(e1)
    ms_steps = e1.elapsed_time(e2)
    pairs = d1["pairs_total"] - d0["pairs_total"]
    alu_peak = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 * \
        _peaks()[0].get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    achieved = pairs * FLOPS_PER_PAIR / (phases["pairs"] / 1e3) / 1e12
    value = n * 10 / (ms_steps / 1e3)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": 10,
            "warmup": 0, "ms_per_step": ms_steps / 10, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 forces, f64 positions/momenta",
            "data": "synthetic", "config": {"workload": Z512_NAME, "particles": n, "mesh": n_p,
                                             "tuning": tuned},
            "force_evaluation_ms": ms_force, "phase_ms_total": phases,
            "roofline": {"kernel": "pairs", "bound": "alu", "achieved": achieved,
                         "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                         "traffic": None},
            "pairs_per_step": pairs / 11, "max_cell_count": d1["max_cell_count"],
            "gpu_launches": int(d1["launches"] - d0["launches"])}


# ---------------------------------------------------------------- the other configurations


def other_configs(args):
    """The 512^3 run, the 48-simulation ensemble and the differentiable run, each measured in
    this process after the main workload (N = 1, rank 0): their key figures for the default
    benchmark line."""
    import torch

    def z512():
        z = run_zeldovich512(args)
        r = {k: z[k] for k in ("value", "unit", "ms_per_step", "force_evaluation_ms", "roofline",
                               "pairs_per_step", "gpu_launches")}
        r["workload"] = z["config"]["workload"]
        r["phase_ms_per_evaluation"] = {k: v / 11 for k, v in z["phase_ms_total"].items()}
        return r

    def ens48():
        e = run_ensemble(args)
        return {"value": e["value"], "unit": e["unit"], "workload": e["config"]["workload"],
                "modes": e["modes"], "speedup_graph_over_serial": e["speedup_graph_over_serial"]}

    def adj128():
        d = run_adjoint(args)
        r = {k: d[k] for k in ("value", "unit", "forward_ms_per_step", "adjoint_ms_per_step",
                               "adjoint_over_forward", "loss")}
        r["workload"] = d["config"]["workload"]
        return r

    out = {}
    for name, fn in (("zeldovich512", z512), ("ensemble48", ens48), ("adjoint128", adj128)):
        try:  # one configuration failing (e.g. memory taken by another process) keeps the line
            out[name] = fn()
        except Exception as exc:  # noqa: BLE001 - reported in the line instead
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- profiling cases


PROFILE_CASES = ("evolved_128", "clustered_128", "uniform_128", "eds_32", "zeldovich_256",
                 "zeldovich_512")


def run_profile_case(args):
    """One workload for a profiler (ncu): set-up, then ``--evals`` force evaluations (or steps
    with ``--profile-steps``); prints the per-phase CUDA-event times of those evaluations.

    evolved_128    128^3 Zel'dovich ICs (box 200, mesh 128) evolved 64 log steps a=0.02->1
    clustered_128  the synthetic clustered 128^3 stand-in snapshot (no evolution)
    uniform_128    128^3 Zel'dovich ICs at a = 0.02 (box 200, mesh 128): near-uniform cells
    eds_32         32^3 Zel'dovich ICs at a = 0.02 (box 64, mesh 32)
    zeldovich_256  256^3 Zel'dovich ICs at a = 0.5 (box 500, mesh 256): the 512^3 run's density
    zeldovich_512  512^3 Zel'dovich ICs at a = 0.5 (box 1000, mesh 512)
    """
    import torch

    import p3m_synth as S
    from paper_1510_07621_gb300 import P3M, build

    build.build()
    w = args.profile_case
    if w in ("evolved_128", "clustered_128", "uniform_128"):
        box, n_p, mesh, a = 200.0, 128, 128, 1.0
        if w == "evolved_128":
            pos, mom = S.zeldovich(n_p, box, 0.02, 1512)
        elif w == "uniform_128":
            a = 0.02
            pos, mom = S.zeldovich(n_p, box, a, 1512)
        else:
            pos, mom = S.clustered(n_p, box, 1512)
    elif w == "eds_32":
        box, n_p, mesh, a = 64.0, 32, 32, 0.02
        pos, mom = S.zeldovich(n_p, box, a, 1511)
    elif w == "zeldovich_256":
        box, n_p, mesh, a = 500.0, 256, 256, 0.5
        pos, mom = S.zeldovich(n_p, box, a, 1514)
    else:
        box, n_p, mesh, a = 1000.0, 512, 512, 0.5
        pos, mom = S.zeldovich(n_p, box, a, 1513)
    sim = P3M(box, n_p ** 3, mesh, precision=args.precision)
    if w == "evolved_128":
        sim.set_particles(pos, mom, a=0.02)
        a_s = S.log_spaced_steps(0.02, 1.0, 64)
        for k in range(64):
            sim.step(a_s[k], a_s[k + 1] - a_s[k])
    else:
        sim.set_particles(pos, mom, a=a)
    torch.cuda.synchronize()
    sim.set_timing(True)
    sim.timings(reset=True)
    for _ in range(args.evals):
        if args.profile_steps:
            sim.step(a, 0.01 * a)
            a *= 1.01
        else:
            sim.forces(a)
    t = sim.timings(reset=True)
    d = sim.diagnostics()
    sim.close()
    return {"profile_case": w, "evals": args.evals, "phase_ms": t, "pairs": d["pairs"],
            "max_cell_count": d["max_cell_count"], "pair_warp_j_total": d["pair_warp_j"],
            "pair_blocks_culled_total": d["pair_blocks_culled"], "pair_tiles_total": d["pair_tiles"]}


# ---------------------------------------------------------------- main


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--workload", choices=["clustered_128", "ensemble48", "adjoint128",
                                           "zeldovich512"],
                    default="clustered_128")
    ap.add_argument("--sub-bits", type=int, default=None,
                    help="Hilbert-curve bits per axis inside a chaining cell (library default if unset)")
    ap.add_argument("--autotune", action="store_true",
                    help="run the library's autotuner (sort-key depth, pair tile length) first")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--save-snapshot", default=None,
                    help="write the a=1 positions (float32 .npy) to this path, for offline analysis")
    ap.add_argument("--cpu-stride", type=int, default=1,
                    help="cpu_baseline: the oracle's pair sum runs on every stride-th particle "
                         "in cell order (1: all particles; 0: skip the CPU baseline)")
    ap.add_argument("--ref-stride", type=int, default=0,
                    help="reference arm: pair-sum sample stride (0: max(16, 4 x steps))")
    ap.add_argument("--no-configs", action="store_true",
                    help="leave out the other configurations (512^3 run, 48-simulation ensemble, "
                         "differentiable run) that the default N=1 line carries under 'configs'")
    ap.add_argument("--profile-case", choices=PROFILE_CASES, default=None,
                    help="run one workload for a profiler and print its phase times (no benchmark line)")
    ap.add_argument("--evals", type=int, default=2, help="--profile-case: force evaluations (or steps)")
    ap.add_argument("--profile-steps", action="store_true",
                    help="--profile-case: time kick-drift-kick steps instead of force evaluations")
    args = ap.parse_args()
    if args.profile_case:
        print(json.dumps(run_profile_case(args)), flush=True)
        return
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.workload in ("ensemble48", "adjoint128", "zeldovich512"):
        if rank == 0:
            fn = {"ensemble48": run_ensemble, "adjoint128": run_adjoint,
                  "zeldovich512": run_zeldovich512}[args.workload]
            print(json.dumps(fn(args)), flush=True)
        return

    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        dist = tdist
    out = run_ours(args, rank, world, local_rank, dist)
    if rank == 0 and world == 1 and not args.no_configs:
        out["configs"] = other_configs(args)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
