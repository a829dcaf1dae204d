"""GPU power spectrum and top-hat sigma (p3m_power_spectrum) against the FP64 oracle, and the
linear growth P(k, a) ~ a^2 of the GPU-evolved Einstein-de Sitter run."""

import numpy as np
import pytest

import p3m_synth as S
from oracle import p3m_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P3M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_07621_gb300 import build
    build.build()
    from paper_1510_07621_gb300 import P3M as cls
    return cls


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-11)])
@pytest.mark.parametrize("case", ["eds32", "clustered48"])
@pytest.mark.parametrize("deconvolve", [True, False])
def test_power_spectrum_matches_oracle(P3M, case, precision, tol, deconvolve):
    if case == "eds32":
        pos, mom = S.zeldovich(32, 64.0, 0.02, 1511)
        box, mesh = 64.0, 32
    else:
        pos, mom = S.clustered(48, 100.0, 4001)
        box, mesh = 100.0, 48
    n = pos.shape[1]
    R = 8.0
    with P3M(box, n, mesh, precision=precision) as sim:
        sim.set_particles(pos, mom, a=1.0)
        k, P, cnt, sig = sim.power_spectrum(deconvolve=deconvolve, tophat_radius=R)
    p = O.Params(box, n, mesh, short_range=False)
    kr, Pr, cr, sr = O.power_spectrum(pos, p, deconvolve=deconvolve, radius=R)
    assert np.array_equal(cnt, cr)
    assert np.max(np.abs(k - kr) / kr) < 1e-13
    assert np.max(np.abs(P - Pr) / Pr) < tol
    assert abs(sig - sr) < tol * sr


def test_linear_growth_of_the_gpu_run(P3M):
    """32^3 EdS run, 10 steps a = 0.02 -> 0.1: the two largest-scale shells grow as D(a)^2 = 25
    (smaller scales are already nonlinear at a = 0.1, where the rms displacement is one cell)."""
    pos, mom = S.zeldovich(32, 64.0, 0.02, 1511)
    a_s = S.log_spaced_steps(0.02, 0.1, 10)
    with P3M(64.0, pos.shape[1], 32) as sim:
        sim.set_particles(pos, mom, a=a_s[0])
        _, P0, _, _ = sim.power_spectrum()
        for i in range(10):
            sim.step(a_s[i], a_s[i + 1] - a_s[i])
        _, P1, _, _ = sim.power_spectrum()
    growth = P1[:2] / P0[:2]
    assert np.all(np.abs(growth / 25.0 - 1.0) < 0.05), growth
