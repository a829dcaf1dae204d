"""Runs one P3M workload for a profiler: set-up, then a few force evaluations or steps.

    python -m paper_1510_07621_gb300.profile_case --workload evolved_128 --evals 2

Workloads (seeded, synthetic):
  evolved_128    128^3 Zel'dovich ICs (box 200, mesh 128) evolved 64 log steps a=0.02->1
  clustered_128  the synthetic clustered 128^3 stand-in snapshot (no evolution)
  uniform_128    128^3 Zel'dovich ICs at a = 0.02 (box 200, mesh 128): near-uniform cells
  eds_32         32^3 Zel'dovich ICs at a = 0.02 (box 64, mesh 32)
  zeldovich_256  256^3 Zel'dovich ICs at a = 0.5 (box 500, mesh 256): the 512^3 run's density
  zeldovich_512  512^3 Zel'dovich ICs at a = 0.5 (box 1000, mesh 512)
Prints the per-phase times (CUDA events) of the evaluations.
"""

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import p3m_synth as S
    from paper_1510_07621_gb300 import P3M, build

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="evolved_128",
                    choices=["evolved_128", "clustered_128", "uniform_128", "eds_32",
                             "zeldovich_256", "zeldovich_512"])
    ap.add_argument("--evals", type=int, default=2)
    ap.add_argument("--steps", action="store_true", help="time steps instead of force evaluations")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args()
    build.build()
    if args.workload in ("evolved_128", "clustered_128", "uniform_128"):
        box, n_p, mesh, a = 200.0, 128, 128, 1.0
        if args.workload == "evolved_128":
            pos, mom = S.zeldovich(n_p, box, 0.02, 1512)
        elif args.workload == "uniform_128":
            a = 0.02
            pos, mom = S.zeldovich(n_p, box, a, 1512)
        else:
            pos, mom = S.clustered(n_p, box, 1512)
    elif args.workload == "eds_32":
        box, n_p, mesh, a = 64.0, 32, 32, 0.02
        pos, mom = S.zeldovich(n_p, box, a, 1511)
    elif args.workload == "zeldovich_256":
        box, n_p, mesh, a = 500.0, 256, 256, 0.5
        pos, mom = S.zeldovich(n_p, box, a, 1514)
    else:
        box, n_p, mesh, a = 1000.0, 512, 512, 0.5
        pos, mom = S.zeldovich(n_p, box, a, 1513)
    sim = P3M(box, n_p ** 3, mesh, precision=args.precision)
    if args.workload == "evolved_128":
        sim.set_particles(pos, mom, a=0.02)
        a_s = S.log_spaced_steps(0.02, 1.0, 64)
        for i in range(64):
            sim.step(a_s[i], a_s[i + 1] - a_s[i])
    else:
        sim.set_particles(pos, mom, a=a)
    torch.cuda.synchronize()
    sim.set_timing(True)
    sim.timings(reset=True)
    for _ in range(args.evals):
        if args.steps:
            sim.step(a, 0.01 * a)
            a *= 1.01
        else:
            sim.forces(a)
    t = sim.timings(reset=True)
    d = sim.diagnostics()
    print(json.dumps({"workload": args.workload, "evals": args.evals, "phase_ms": t,
                      "pairs": d["pairs"], "max_cell_count": d["max_cell_count"],
                      "pair_warp_j_total": d["pair_warp_j"],
                      "pair_blocks_culled_total": d["pair_blocks_culled"],
                      "pair_tiles_total": d["pair_tiles"]}))
    sim.close()


if __name__ == "__main__":
    main()
