"""The deposit's tile flush and the staged gather map a tile index t to its row and column by
FP32 reciprocals instead of integer divisions: row = (int)((t + 1/2) * fl(1/b)) in FP32.  The
rounded quotient is off by at most (t/b + 1) 2^-23, far less than its distance 1/(2b) to an
integer, so the split is exact for every t, b < 2^12 (the largest tile is 4096 nodes).  Checked
here exhaustively with IEEE FP32 arithmetic (numpy float32: correctly rounded division,
multiplication and conversion, as the kernels use them without fast-math)."""

import numpy as np


def test_reciprocal_split_is_exact_below_4096():
    t = np.arange(4096, dtype=np.float32)
    ti = np.arange(4096, dtype=np.int64)
    half = np.float32(0.5)
    for b in range(1, 4097):
        inv = np.float32(1.0) / np.float32(b)
        q = ((t + half) * inv).astype(np.float32).astype(np.int64)
        assert np.array_equal(q, ti // b), b
