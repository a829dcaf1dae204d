"""Pins of the oracle's potential energy: the Ewald energy's independence of alpha, a
simple-cubic lattice's energy (Madelung constant of the sc lattice with background), and the
P3M potential energy against the Ewald energy of the same periodic particle set."""

import math

import numpy as np

import p3m_synth as S
from oracle import p3m_oracle as O


def test_ewald_energy_alpha_independent():
    pos = S.uniform_random(60, 1.0, 4)
    e1 = O.ewald_potential_energy(pos, 1.0, 1.0, alpha=2.2)
    e2 = O.ewald_potential_energy(pos, 1.0, 1.0, alpha=3.0, nreal=3, kmax=8)
    assert abs(e1 - e2) < 1e-11 * abs(e1)


def test_ewald_energy_of_one_particle_is_the_sc_madelung_energy():
    """One particle per periodic cell of side L with a neutralising background: the Coulomb
    energy of this simple-cubic lattice is (q^2/2) xi / L, xi = -2.837297479 (the Madelung
    constant of the sc Wigner lattice); gravity flips the sign: E = -(Gm/2) xi / L."""
    L = 3.0
    e = O.ewald_potential_energy(np.array([[0.4], [1.1], [2.9]]), L, 1.0)
    assert abs(e - (-0.5) * (-2.837297479480620 / L)) < 1e-10


def test_p3m_energy_of_one_particle_is_exactly_ewald():
    """One particle: the mesh share is replaced by its exact periodic value and the r = 0
    self term removed, so the P3M energy is the Ewald (Madelung) energy to round-off."""
    L = 64.0
    one = np.array([[10.3], [20.7], [33.1]])
    p = O.Params(L, 1, 32, softening=0.0)
    assert abs(O.potential_energy(one, p, 1.0) - O.ewald_potential_energy(one, L, p.gm)) < 1e-12 * 700


def test_p3m_potential_energy_matches_ewald():
    """512 random particles: P3M energy vs Ewald, converging with the cutoff and the mesh."""
    L, n = 64.0, 512
    pos = S.uniform_random(n, L, 21)
    ref = O.ewald_potential_energy(pos, L, O.Params(L, n, 32).gm)
    for cutoff, mesh, tol in ((4.5, 32, 1e-2), (6.0, 64, 1e-3)):
        p = O.Params(L, n, mesh, cutoff=cutoff, softening=0.0)
        w = O.potential_energy(pos, p, a=1.0)
        assert abs(w - ref) < tol * abs(ref), (cutoff, mesh, w, ref)


def test_layzer_irvine_holds_for_the_oracle_dynamics():
    """d[a(K + W)]/da = -K along the oracle's own KDK trajectory of a quasi-linear Zel'dovich
    start: the residual a(K+W) + int K da - a0(K0+W0) stays below 1% of a K (the mesh force
    is not the exact gradient of the interpolated potential, so it does not vanish), while a
    wrong sign or a missing position-dependent term of W would leave O(1) residuals."""
    box, n_p, mesh = 24.0, 12, 24
    pos, mom = S.zeldovich(n_p, box, 0.02, 1512)
    n = pos.shape[1]
    p = O.Params(box, n, mesh, softening=0.02)
    a_s = S.log_spaced_steps(0.02, 0.06, 16)
    x, m = O.wrap(pos, box), mom.copy()
    acc = O.accel(x, p)
    ks = [O.kinetic_energy(m, a_s[0])]
    ws = [O.potential_energy(x, p, a_s[0])]
    for i in range(16):
        x, m, acc = O.step(x, m, acc, a_s[i], a_s[i + 1] - a_s[i], p)
        ks.append(O.kinetic_energy(m, a_s[i + 1]))
        ws.append(O.potential_energy(x, p, a_s[i + 1]))
    ks, ws = np.array(ks), np.array(ws)
    integral = float(np.sum(0.5 * (ks[1:] + ks[:-1]) * np.diff(a_s)))
    res = a_s[-1] * (ks[-1] + ws[-1]) + integral - a_s[0] * (ks[0] + ws[0])
    assert abs(res) < 1e-2 * a_s[-1] * ks[-1], (res, a_s[-1] * ks[-1])
    # the same bookkeeping with W's sign flipped fails by far
    bad = a_s[-1] * (ks[-1] - ws[-1]) + integral - a_s[0] * (ks[0] - ws[0])
    assert abs(bad) > 0.3 * a_s[-1] * ks[-1]
