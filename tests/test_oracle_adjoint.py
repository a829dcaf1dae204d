"""Pins of the oracle's reverse-mode derivatives against central finite differences of its own
forward pass (FP64): the transposed force Jacobian through the dot-product identity
w . (A(x + e u) - A(x - e u)) / 2e = (J^T w) . u, the density-loss gradient, and the gradient
of a whole run with respect to the initial displacement field."""

import numpy as np
import pytest

import p3m_synth as S
from oracle import p3m_oracle as O


def _setup(n_p=12, box=30.0, mesh=24, seed=3):
    q = S.lattice(n_p, box)
    pos, mom = S.zeldovich(n_p, box, 0.05, seed, rms_cells=0.3)
    p = O.Params(box, n_p ** 3, mesh, softening=0.05)
    return q, pos, mom, p


@pytest.mark.parametrize("part", ["pm", "sr", "total"])
def test_force_vjp_dot_product_identity(part):
    q, pos, mom, p = _setup()
    n = pos.shape[1]
    u = S.gaussian(71, 3 * n).reshape(3, n)
    w = S.gaussian(72, 3 * n).reshape(3, n)
    f = {"pm": lambda x: O.pm_accel(O.wrap(x, p.box), p),
         "sr": lambda x: O.sr_accel(O.wrap(x, p.box), p)[0],
         "total": lambda x: O.accel(x, p)}[part]
    vjp = {"pm": lambda x, v: O.pm_vjp(O.wrap(x, p.box), v, p),
           "sr": lambda x, v: O.sr_vjp(O.wrap(x, p.box), v, p),
           "total": lambda x, v: O.accel_vjp(x, v, p)}[part]
    eps = 1e-6 * p.box / 12
    fd = np.sum(w * (f(pos + eps * u) - f(pos - eps * u))) / (2 * eps)
    an = np.sum(vjp(pos, w) * u)
    assert abs(fd - an) < 2e-6 * abs(an), (fd, an)


def test_density_loss_gradient():
    q, pos, mom, p = _setup()
    n = pos.shape[1]
    target = 0.3 * S.gaussian(5, p.mesh ** 3)
    loss, grad = O.density_loss(pos, target, p)
    u = S.gaussian(9, 3 * n).reshape(3, n)
    eps = 1e-6 * p.box / 12
    fd = (O.density_loss(pos + eps * u, target, p)[0] - O.density_loss(pos - eps * u, target, p)[0]) / (2 * eps)
    assert abs(fd - np.sum(grad * u)) < 1e-6 * abs(fd)


def test_run_gradient_matches_finite_differences():
    """3 KDK steps a = 0.05 -> 0.2; the loss gradient along 4 random directions of the initial
    displacement field.  The step is 1e-7 of a lattice spacing: the CIC weights are piecewise
    linear and the short-range force jumps at r_c, so larger steps that carry a particle across
    a mesh plane or a pair across the cutoff measure a chord, not the derivative."""
    n_p, box, mesh = 12, 30.0, 24
    q = S.lattice(n_p, box)
    _, mom = S.zeldovich(n_p, box, 0.05, 3, rms_cells=0.3)
    psi = mom / np.sqrt(0.05)  # displacement at a = 0.05
    p = O.Params(box, n_p ** 3, mesh, softening=0.05)
    a = S.log_spaced_steps(0.05, 0.2, 3)
    target = 0.5 * S.gaussian(11, mesh ** 3)
    loss, grad = O.run_gradient(psi, q, a, target, p)
    eps = 1e-7 * box / n_p
    for d in range(4):
        u = S.gaussian(200 + d, 3 * n_p ** 3).reshape(3, -1)
        fd = (O.run_and_loss(psi + eps * u, q, a, target, p)
              - O.run_and_loss(psi - eps * u, q, a, target, p)) / (2 * eps)
        assert abs(fd - np.sum(grad * u)) < 1e-5 * abs(fd), (d, fd, np.sum(grad * u))
