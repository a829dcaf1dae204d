"""Compiles the oracle's plain C pair sums (``sr_pairs.c``) into ``libp3m_oracle.so``.

Test infrastructure only: the library is used by tests/, __graft_entry__ and bench.py's
cpu_baseline leg.  Plain ``gcc -O2`` (no fast-math, no -march), OpenMP over particles.
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sr_pairs.c")
LIB = os.path.join(HERE, "libp3m_oracle.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
