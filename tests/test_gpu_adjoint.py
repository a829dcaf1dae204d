"""GPU reverse-mode derivatives against the FP64 oracle and central finite differences:
the transposed force Jacobian, the density loss and its gradient, and the gradient of a whole
run with respect to the initial displacement field (sqrt(n) checkpointing)."""

import math

import numpy as np
import pytest

import p3m_synth as S
from oracle import p3m_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_07621_gb300 import build
    build.build()
    import paper_1510_07621_gb300 as m
    from paper_1510_07621_gb300.adjoint import DensityLossRun
    return torch, m, DensityLossRun


def rel_rms(a, ref):
    return math.sqrt(float(np.sum((a - ref) ** 2)) / float(np.sum(ref ** 2)))


CASE = dict(n_p=16, box=32.0, mesh=32, soft=0.05)


def _ics(seed=3, a0=0.05, rms=0.3):
    pos, mom = S.zeldovich(CASE["n_p"], CASE["box"], a0, seed, rms_cells=rms)
    return pos, mom


@pytest.mark.parametrize("precision,tol", [("mixed", 2e-5), ("fp64", 1e-10)])
@pytest.mark.parametrize("short_range", [True, False])
def test_force_vjp_matches_oracle(mod, precision, tol, short_range):
    torch, m, _ = mod
    pos, _ = _ics()
    n = pos.shape[1]
    v = S.gaussian(17, 3 * n).reshape(3, n)
    with m.P3M(CASE["box"], n, CASE["mesh"], precision=precision, softening=CASE["soft"],
               short_range=short_range) as sim:
        sim.set_particles(pos, np.zeros_like(pos), a=0.05)
        out = sim.force_vjp(v)
    p = O.Params(CASE["box"], n, CASE["mesh"], softening=CASE["soft"], short_range=short_range)
    ref = O.accel_vjp(pos, v, p)
    assert rel_rms(out, ref) < tol


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-11)])
def test_density_loss_and_gradient(mod, precision, tol):
    torch, m, _ = mod
    pos, _ = _ics()
    n = pos.shape[1]
    target = 0.4 * S.gaussian(5, CASE["mesh"] ** 3)
    with m.P3M(CASE["box"], n, CASE["mesh"], precision=precision) as sim:
        sim.set_particles(pos, np.zeros_like(pos), a=0.05)
        loss, grad = sim.density_loss(target, np.empty((3, n)))
    p = O.Params(CASE["box"], n, CASE["mesh"], short_range=False)
    rl, rg = O.density_loss(pos, target, p)
    assert abs(loss - rl) < tol * rl
    assert rel_rms(grad, rg) < tol


def _run_setup(torch, m, precision):
    n_p, box, mesh = CASE["n_p"], CASE["box"], CASE["mesh"]
    q = S.lattice(n_p, box)
    _, mom = _ics()
    psi = mom / math.sqrt(0.05)
    a = S.log_spaced_steps(0.05, 0.2, 4)
    target = 0.5 * S.gaussian(11, mesh ** 3)
    dev = torch.device("cuda", 0)
    sim = m.P3M(box, n_p ** 3, mesh, precision=precision, softening=CASE["soft"])
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    return sim, q, psi, a, target, t


def test_run_gradient_matches_oracle_and_finite_differences(mod):
    """FP64 mode: the checkpointed reverse sweep equals the oracle's full-storage adjoint, and
    central finite differences of the GPU forward along 8 random directions agree to 1e-4."""
    torch, m, DensityLossRun = mod
    sim, q, psi, a, target, t = _run_setup(torch, m, "fp64")
    psi_t = t(psi).requires_grad_(True)
    loss = DensityLossRun.apply(psi_t, sim, t(q), a, t(target), 2)
    loss.backward()
    g = psi_t.grad.cpu().numpy()
    p = O.Params(CASE["box"], q.shape[1], CASE["mesh"], softening=CASE["soft"])
    rl, rg = O.run_gradient(psi, q, a, target, p)
    assert abs(float(loss.detach()) - rl) < 1e-10 * rl
    assert rel_rms(g, rg) < 1e-8
    eps = 1e-7 * CASE["box"] / CASE["n_p"]
    with torch.no_grad():
        for d in range(8):
            u = S.gaussian(300 + d, psi.size).reshape(psi.shape)
            lp = float(DensityLossRun.apply(t(psi + eps * u), sim, t(q), a, t(target), 2))
            lm = float(DensityLossRun.apply(t(psi - eps * u), sim, t(q), a, t(target), 2))
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - np.sum(g * u)) < 1e-4 * abs(fd), (d, fd, np.sum(g * u))
    sim.close()


def test_mixed_gradient_close_to_fp64(mod):
    torch, m, DensityLossRun = mod
    grads = {}
    for precision in ("fp64", "mixed"):
        sim, q, psi, a, target, t = _run_setup(torch, m, precision)
        psi_t = t(psi).requires_grad_(True)
        DensityLossRun.apply(psi_t, sim, t(q), a, t(target), 2).backward()
        grads[precision] = psi_t.grad.cpu().numpy()
        sim.close()
    assert rel_rms(grads["mixed"], grads["fp64"]) < 1e-3
