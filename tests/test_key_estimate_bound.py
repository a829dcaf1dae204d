"""The chaining-cell key kernel takes the fine index floor(x n_f / L) from an FP32 estimate
(x truncated to its leading 24 significant bits, times n_f / L rounded to FP32) whenever the
estimate lies more than 2^-21 n_f from every integer, and from the correctly rounded FP64
product otherwise.  This checks the error bound that makes the shortcut exact, by emulating
the estimate bit for bit in numpy over random coordinates and every cell face (CPU only)."""

import numpy as np
import pytest


def _estimate(x, inv, nf):
    xb = x.view(np.int64)
    e = ((xb >> 52) & 0x7FF).astype(np.int64) - 1023 + 127
    bits = ((e << 23) | ((xb >> 29) & 0x7FFFFF)).astype(np.int32)
    xf = np.where(e >= 1, bits.view(np.float32), np.float32(0.0))
    p = (xf * np.float32(inv)).astype(np.float32)
    k = np.trunc(p)
    tol = np.float32(nf * 2.0 ** -21)
    ok = (p - k > tol) & (p - k < 1 - tol)
    return np.minimum(k.astype(np.int64), nf - 1), ok


@pytest.mark.parametrize("box,nf", [(200.0, 22 * 8), (1000.0, 90 * 8), (64.0, 1024 * 8),
                                    (37.3, 1000), (500.0, 45 * 32)])
def test_fp32_estimate_is_exact_away_from_faces(box, nf):
    rng = np.random.default_rng(nf)
    inv = nf / box
    faces = np.arange(nf + 1) / inv
    x = np.concatenate([rng.uniform(0.0, box, 400_000), faces,
                        np.nextafter(faces, 0.0), np.nextafter(faces, box), [0.0]])
    x = x[(x >= 0.0) & (x < box)]
    est, ok = _estimate(x, inv, nf)
    exact = np.minimum(np.trunc(x * inv).astype(np.int64), nf - 1)
    assert np.array_equal(est[ok], exact[ok])
    # the shortcut covers almost every random coordinate
    assert ok[:400_000].mean() > 0.99
