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
# accepted-pair instruction sequence, FMA = 2: d 3 FADD; r^2 FMUL + 2 FFMA; r = r^2 rsqrt(r^2)
# FMUL; r^3 FMUL; tau FFMA; Q(tau) 10 FFMA; g = 1 + r^3 Q FFMA; r^2 + eps^2 FADD;
# g (r^2+eps^2)^-3/2 3 FMUL; a += f d 3 FFMA  ->  17 FFMA + 10 FADD/FMUL = 44 flops
# (the two rsqrt run on the MUFU pipe and are not counted)
FLOPS_PER_PAIR = 44
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


def oracle_step_time(pos, mom, n_sample, seed, with_pair=False):
    """Seconds the FP64 oracle needs for one step of this particle set: the full mesh force
    (all particles), the pair sum of all particles estimated from n_sample of them, and the
    kick/drift of all particles.  The pair sum's set-up (cell keys, order and ranges of all N
    particles, timed by a call with one target) is counted once; only the per-target part is
    scaled by N / n_sample.  Returns (seconds, threads, description[, pair-sum seconds])."""
    from oracle import p3m_oracle as O
    w = WORKLOAD
    n = pos.shape[1]
    p = O.Params(w["box"], n, w["mesh"], w["r_s_cells"], w["cutoff"], w["softening"])
    x = O.wrap(pos, w["box"])
    t0 = time.perf_counter()
    lr = O.pm_accel(x, p)
    t1 = time.perf_counter()
    tg = np.unique((S.uniform01(seed, n_sample) * n).astype(np.int64) % n)
    O.sr_accel(x, p, targets=tg[:1])
    t1b = time.perf_counter()
    O.sr_accel(x, p, targets=tg)
    t2 = time.perf_counter()
    m = mom + lr * O.kick_factor(1.0, 1.02, p)
    x2 = O.wrap(x + m * O.drift_factor(1.0, 1.04, p), w["box"])
    del x2
    t3 = time.perf_counter()
    setup = t1b - t1
    pair = setup + max(0.0, (t2 - t1b) - setup) * n / tg.size
    total = (t1 - t0) + pair + (t3 - t2)
    desc = (f"full mesh force and kick/drift for all {n} particles; short-range pair sum for "
            f"{tg.size} sampled particles, its per-target time scaled by {n / tg.size:.1f} "
            "(set-up counted once)")
    if with_pair:
        return total, O.oracle_threads(), desc, pair
    return total, O.oracle_threads(), desc


def oracle_pair_time_one_core(x, n_sample, seed):
    """The oracle's pair sum of n_sample sampled particles of the wrapped positions x on one
    host core (a child process with OMP_NUM_THREADS=1): returns (set-up seconds, seconds of the
    per-target work, particles sampled), or (None, None, 0) if the child failed."""
    import subprocess
    import tempfile
    w = WORKLOAD
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "x.npy")
        np.save(path, x)
        code = (
            "import sys, time, numpy as np\n"
            f"sys.path.insert(0, {ROOT!r})\n"
            "import p3m_synth as S\n"
            "from oracle import p3m_oracle as O\n"
            f"x = np.load({path!r}); n = x.shape[1]\n"
            f"p = O.Params({w['box']!r}, n, {w['mesh']!r}, {w['r_s_cells']!r}, {w['cutoff']!r}, "
            f"{w['softening']!r})\n"
            f"tg = np.unique((S.uniform01({seed}, {n_sample}) * n).astype(np.int64) % n)\n"
            "t0 = time.perf_counter(); O.sr_accel(x, p, targets=tg[:1])\n"
            "t1 = time.perf_counter(); O.sr_accel(x, p, targets=tg)\n"
            "t2 = time.perf_counter(); su = t1 - t0\n"
            "print(su, max(0.0, (t2 - t1) - su), tg.size, O.oracle_threads())\n")
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=600)
        if r.returncode != 0:
            return None, None, 0
        setup, work, size, threads = r.stdout.split()[-4:]
        return (float(setup), float(work), int(size)) if int(threads) == 1 else (None, None, 0)


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
        "deposit": 32 * n,
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

    # ---- e2e through the C ABI with pinned host buffers (rank 0 measures, others idle)
    if rank == 0 and args.e2e_steps > 0:
        hp = torch.empty((3, n), dtype=torch.float64, pin_memory=True)
        hm = torch.empty((3, n), dtype=torch.float64, pin_memory=True)
        ha = torch.empty((3, n), dtype=torch.float64, pin_memory=True)
        sim.get_particles(hp, hm, ha)
        a_e = a
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sim.set_particles(hp, hm, acc=ha, a=a_e)
            sim.step(a_e, a_e * (ratio - 1.0))
            a_e *= ratio
            sim.get_particles(hp, hm, ha)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        out["e2e"] = {"value": n * args.e2e_steps / dt, "unit": UNIT, "steps": args.e2e_steps,
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
                           "pair_tflops": pairs64 * FLOPS_PER_PAIR / (ms64 / 1e3) / 1e12,
                           "fp64_fma_peak_measured": fma64,
                           "pair_frac_of_fp64_peak": pairs64 * FLOPS_PER_PAIR / (ms64 / 1e3) / 1e12 / fma64,
                           "speedup_mixed_over_fp64": value / world / (n / (ms64 / 1e3))}

    # ---- CPU baseline: the oracle on this machine's host cores (rank 0, N = 1 only), on the
    # synthetic clustered a = 1 stand-in snapshot: no oracle input comes from the GPU path
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        snap_pos, snap_mom = S.clustered(w["n_p"], w["box"], w["seed"])
        sec, threads, desc, pair_many = oracle_step_time(snap_pos, snap_mom, args.cpu_sample, 99,
                                                         with_pair=True)
        # the same step with the pair sum on one core (mesh part and kick/drift as measured)
        from oracle import p3m_oracle as O
        xw = O.wrap(snap_pos, w["box"])
        n1 = max(2000, args.cpu_sample // 4)
        setup1, work1, size1 = oracle_pair_time_one_core(xw, n1, 98)
        one_core = None
        if work1:
            # the same targets on all cores: the one-core factor of the per-target work
            pp = O.Params(w["box"], n, w["mesh"], w["r_s_cells"], w["cutoff"], w["softening"])
            tg1 = np.unique((S.uniform01(98, n1) * n).astype(np.int64) % n)
            t0 = time.perf_counter()
            O.sr_accel(xw, pp, targets=tg1[:1])
            t1 = time.perf_counter()
            O.sr_accel(xw, pp, targets=tg1)
            t2 = time.perf_counter()
            setup_m, work_m = t1 - t0, max(1e-9, (t2 - t1) - (t1 - t0))
            pair_one = setup1 + (pair_many - setup_m) * work1 / work_m
            sec_one = sec - pair_many + pair_one
            one_core = {"value": n / sec_one, "unit": UNIT, "cores": 1,
                        "sample": f"the multi-core pair-sum estimate times the one-core factor "
                                  f"{work1 / work_m:.1f} of the per-target work, measured on "
                                  f"{size1} sampled particles; mesh force and kick/drift as in "
                                  "the multi-core figure"}
        out["cpu_baseline"] = {"value": n / sec, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "one_core": one_core,
                               "sample": desc + "; on the synthetic clustered a=1 stand-in "
                                                "snapshot of the same size",
                               "seconds_per_step_estimate": sec}
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
    (8-step graphs for the whole ensemble) -- the last two each with per-simulation pair
    launches and with one batched pair launch per step over all simulations.  The value is
    the graph replay with per-simulation launches (the library's default; the batched launch
    is within 1 % of it here).  Every mode starts from the ICs with their forces known, so no
    timed region contains a force evaluation of the ICs."""
    import torch
    from paper_1510_07621_gb300 import P3M, Ensemble, build

    build.build()
    torch.cuda.set_device(0)
    sizes = [48] * 16 + [64] * 16 + [96] * 16
    box = 100.0
    a = S.log_spaced_steps(0.05, 1.0, 20)
    ics = [S.zeldovich(n_p, box, a[0], 4000 + k) for k, n_p in enumerate(sizes)]
    total = sum(n_p ** 3 for n_p in sizes)

    acc0 = [None] * len(sizes)  # the ICs' accelerations, so that a restore needs no evaluation

    def fresh():
        sims = [P3M(box, n_p ** 3, n_p, softening=0.02, stream=0) for n_p in sizes]
        for k, (s_, (p, m)) in enumerate(zip(sims, ics)):
            s_.set_particles(p, m, a=a[0])
            acc0[k] = s_.forces(a[0])
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
    for mode, use_graph, batched in (("stream_host_launches", False, False),
                                     ("stream_host_launches_batched_pairs", False, True),
                                     ("graph_ensemble", True, False),
                                     ("graph_ensemble_batched_pairs", True, True)):
        sims = fresh()
        with Ensemble(sims, batched=batched) as ens:
            if use_graph:  # capture outside the timed region, then restore the ICs and forces
                ens.run(a[:3], use_graph=True)
                torch.cuda.synchronize()
                for s_, (p, m), g in zip(sims, ics, acc0):
                    s_.set_particles(p, m, acc=g, a=a[0])
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
    from oracle import p3m_oracle as O
    w = WORKLOAD
    n = w["n_p"] ** 3
    pos, mom = S.clustered(w["n_p"], w["box"], w["seed"])
    # the pair-sum sample of one step shrinks with the number of steps, so that the whole run
    # (each step also computes the full mesh force, several seconds) ends within minutes
    per_step = max(500, args.cpu_sample // max(1, args.steps))
    for _ in range(args.warmup):
        oracle_step_time(pos, mom, 500, 5)
    total = 0.0
    threads, desc = 1, ""
    for k in range(args.steps):
        sec, threads, desc = oracle_step_time(pos, mom, per_step, 100 + k)
        total += sec
    value = n * args.steps / total
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME.split(";")[0] +
                       "; synthetic clustered a=1 stand-in snapshot (no GPU evolution)",
                       "particles": n, "mesh": w["mesh"]},
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
    with P3M(box, n, n_p, softening=0.02, stream=stream) as sim:
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
    ap.add_argument("--cpu-sample", type=int, default=8000,
                    help="particles whose pair sum the oracle times (0: skip the CPU baseline)")
    args = ap.parse_args()
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
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
