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


def test_mixed_gradient_matches_finite_differences(mod):
    """Mixed mode (FP32 forces, FP64 positions), sqrt(n) checkpoints: the gradient's derivative
    along 8 random directions matches central finite differences of the loss within 1e-4.  The
    differences are taken of the FP64 run (the same loss without FP32 rounding, itself pinned to
    the oracle above): the FP32 forces are piecewise constant on the scale of their coordinate
    rounding, so differences of the mixed loss itself do not resolve a derivative."""
    torch, m, DensityLossRun = mod
    grads = {}
    sims = {}
    for precision in ("fp64", "mixed"):
        sim, q, psi, a, target, t = _run_setup(torch, m, precision)
        psi_t = t(psi).requires_grad_(True)
        DensityLossRun.apply(psi_t, sim, t(q), a, t(target), 2).backward()
        grads[precision] = psi_t.grad.cpu().numpy()
        sims[precision] = sim
    eps = 1e-7 * CASE["box"] / CASE["n_p"]
    with torch.no_grad():
        for d in range(8):
            u = S.gaussian(300 + d, psi.size).reshape(psi.shape)
            lp = float(DensityLossRun.apply(t(psi + eps * u), sims["fp64"], t(q), a, t(target), 2))
            lm = float(DensityLossRun.apply(t(psi - eps * u), sims["fp64"], t(q), a, t(target), 2))
            fd = (lp - lm) / (2 * eps)
            gu = float(np.sum(grads["mixed"] * u))
            assert abs(fd - gu) < 1e-4 * abs(fd), (d, fd, gu)
    for s_ in sims.values():
        s_.close()


def test_mixed_gradient_matches_fp64_gradient_48(mod):
    """48^3 particles, box 100 Mpc/h, mesh 48 (216 particles per chaining cell: several pair work
    items per cell and several j tiles per neighbour cell), 4 steps a = 0.05 -> 0.12 with
    checkpoints every 2 steps: the mixed gradient's derivatives along 8 random directions match
    the FP64 gradient's within 1e-4.  Finite differences are no reference at this size: with
    ~4e7 pairs, some pair distance crosses r_c within any step that resolves the derivative, and
    the kick of the discrete step jumps there (reading 13)."""
    torch, m, DensityLossRun = mod
    n_p, box, mesh = 48, 100.0, 48
    q = S.lattice(n_p, box)
    _, mom = S.zeldovich(n_p, box, 0.05, 3, rms_cells=0.3)
    psi = mom / math.sqrt(0.05)
    a = S.log_spaced_steps(0.05, 0.12, 4)
    target = 0.5 * S.gaussian(11, mesh ** 3)
    dev = torch.device("cuda", 0)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    grads = {}
    for precision in ("fp64", "mixed"):
        with m.P3M(box, n_p ** 3, mesh, precision=precision, softening=CASE["soft"]) as sim:
            psi_t = t(psi).requires_grad_(True)
            DensityLossRun.apply(psi_t, sim, t(q), a, t(target), 2).backward()
            grads[precision] = psi_t.grad.cpu().numpy()
            if precision == "mixed":
                assert sim.diagnostics()["max_cell_count"] > 160
    for d in range(8):
        u = S.gaussian(300 + d, psi.size).reshape(psi.shape)
        g64, g32 = float(np.sum(grads["fp64"] * u)), float(np.sum(grads["mixed"] * u))
        assert abs(g32 - g64) < 1e-4 * abs(g64), (d, g32, g64)
