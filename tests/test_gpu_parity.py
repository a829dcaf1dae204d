"""GPU parity of the P3M step (through the C ABI) against the FP64 oracle.

Acceptance bars:
  * cell keys, sort order and cell ranges: bit-exact;
  * accelerations: relative RMS sqrt(sum|a_gpu - a_ref|^2 / sum|a_ref|^2) <= 1e-5 in the mixed
    (FP32 force) mode and <= 1e-12 in the all-FP64 mode;
  * positions after 10 KDK steps: within 1e-6 of the box length (mixed mode).
"""

import math

import numpy as np
import pytest

import p3m_synth as S
from oracle import p3m_oracle as O

pytestmark = pytest.mark.gpu

TOL = {"mixed": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def P3M():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_07621_gb300 import build
    build.build()
    from paper_1510_07621_gb300 import P3M as cls
    return cls


def rel_rms(a, ref):
    return math.sqrt(float(np.sum((a - ref) ** 2)) / float(np.sum(ref ** 2)))


def _case(name):
    if name == "eds32":  # 32^3 Zel'dovich ICs at a = 0.02, box 64 Mpc/h, mesh 32
        pos, mom = S.zeldovich(32, 64.0, 0.02, 1511)
        return pos, mom, dict(box=64.0, mesh=32)
    if name == "clustered48":  # uneven cell occupancy: dense halos and empty cells
        pos, mom = S.clustered(48, 100.0, 4001)
        return pos, mom, dict(box=100.0, mesh=48)
    if name == "random5003":  # N not a cube, ragged tiles everywhere
        pos = S.uniform_random(5003, 80.0, 77)
        return pos, np.zeros_like(pos), dict(box=80.0, mesh=40)
    if name == "nc3":  # the smallest chaining mesh: 3 cells per side, every cell a neighbour
        pos = S.uniform_random(2000, 64.0, 91)
        return pos, np.zeros_like(pos), dict(box=64.0, mesh=20)
    if name == "coincident":  # 200 exact duplicates: r = 0 pairs add nothing and are not counted
        base = S.uniform_random(600, 40.0, 92)
        pos = np.concatenate([base, base[:, :200]], axis=1)
        return pos, np.zeros_like(pos), dict(box=40.0, mesh=32)
    if name == "tiny3":
        pos = np.array([[1.0, 1.5, 30.0], [2.0, 2.0, 31.0], [3.0, 3.3, 0.5]])
        return pos, np.zeros_like(pos), dict(box=32.0, mesh=32)
    raise KeyError(name)


def _params(n, kw, precision="mixed", **extra):
    soft = extra.pop("softening", 0.02)
    return O.Params(kw["box"], n, kw["mesh"], softening=soft, **extra)


# ------------------------------------------------------------------ keys and order


def _adversarial(box=64.0, mesh=32):
    """Edge positions: all particles in one cell, exact cell faces, L - ulp, out-of-box."""
    p = O.Params(box, 10, mesh)
    cs = box / p.n_c
    xs = [0.0, cs, 2 * cs, 3 * cs, np.nextafter(cs, 0), np.nextafter(box, 0), -1e-300, box,
          -0.25 * box, 2.5 * box, 0.5 * cs, 0.5 * cs, 0.5 * cs, 0.5 * cs]
    u = S.uniform01(5, 3 * 400)
    one_cell = (u.reshape(3, 400) * 0.9 + 0.05) * cs + cs  # all in cell (1,1,1)
    edge = np.array([[x, y, z] for x in xs[:6] for y in xs[4:10] for z in xs[8:]]).T
    return np.concatenate([one_cell, edge], axis=1), dict(box=box, mesh=mesh)


@pytest.mark.parametrize("sub_bits", [0, 2, 5])
@pytest.mark.parametrize("case", ["eds32", "clustered48", "adversarial"])
def test_keys_order_and_cell_ranges_bit_exact(P3M, case, sub_bits):
    if case == "adversarial":
        pos, kw = _adversarial()
        mom = np.zeros_like(pos)
    else:
        pos, mom, kw = _case(case)
    n = pos.shape[1]
    with P3M(kw["box"], n, kw["mesh"], sub_bits=sub_bits) as sim:
        sim.set_particles(np.ascontiguousarray(pos), np.ascontiguousarray(mom), a=0.1)
        sim.forces(0.1)
        keys, ids, starts = sim.get_cells()
    p = O.Params(kw["box"], n, kw["mesh"], sub_bits=sub_bits)
    x = O.wrap(pos, kw["box"])
    cell, key = O.cell_keys(x, p)
    order = O.stable_order(key)
    assert np.array_equal(keys.astype(np.int64), key[order])
    assert np.array_equal(ids.astype(np.int64), order)
    assert np.array_equal(starts.astype(np.int64), O.cell_start(cell[order], p.n_c ** 3))


@pytest.mark.parametrize("sub_bits", [3, 5])
@pytest.mark.parametrize("which", ["clustered", "zeldovich"])
def test_keys_order_bit_exact_full_size_128(P3M, which, sub_bits):
    """2.1 M particles: 512 sort tiles, 3 (sub_bits 3) or 4 (sub_bits 5) digit passes, so the
    tile-to-tile count hand-over of the sort is exercised at the benchmark's size."""
    if which == "clustered":
        pos, mom = S.clustered(128, 200.0, 1512)
    else:
        pos, mom = S.zeldovich(128, 200.0, 0.02, 1512)
    n = pos.shape[1]
    with P3M(200.0, n, 128, sub_bits=sub_bits) as sim:
        sim.set_particles(pos, mom, a=1.0)
        sim.forces(1.0)
        keys, ids, starts = sim.get_cells()
    p = O.Params(200.0, n, 128, sub_bits=sub_bits)
    cell, key = O.cell_keys(O.wrap(pos, 200.0), p)
    order = O.stable_order(key)
    assert np.array_equal(keys.astype(np.int64), key[order])
    assert np.array_equal(ids.astype(np.int64), order)
    assert np.array_equal(starts.astype(np.int64), O.cell_start(cell[order], p.n_c ** 3))


def test_positions_wrapped_and_order_preserved(P3M):
    pos, _ = _adversarial()
    n = pos.shape[1]
    mom = S.uniform01(9, 3 * n).reshape(3, n)
    with P3M(64.0, n, 32) as sim:
        sim.set_particles(np.ascontiguousarray(pos), mom, a=0.5)
        sim.forces(0.5)
        p2, m2 = sim.get_particles()
    assert np.array_equal(p2, O.wrap(pos, 64.0))
    assert np.array_equal(m2, mom)


# ------------------------------------------------------------------ mesh and forces


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_density_mesh(P3M, precision):
    pos, mom, kw = _case("clustered48")
    n = pos.shape[1]
    with P3M(kw["box"], n, kw["mesh"], precision=precision) as sim:
        sim.set_particles(pos, mom, a=1.0)
        sim.forces(1.0)
        rho = sim.get_mesh(0).astype(np.float64)
    ref = O.cic_deposit(O.wrap(pos, kw["box"]), _params(n, kw)) - n / kw["mesh"] ** 3
    tol = 2e-5 if precision == "mixed" else 1e-12
    assert np.max(np.abs(rho - ref)) <= tol * np.max(np.abs(ref))


def test_staged_gather_matches_oracle(P3M):
    """A 256^3 mesh: the three FP32 force meshes (201 MB) exceed L2, so the mixed-mode gather
    copies each 512-particle chunk's node box into shared memory; the clustered 64^3 particles
    give compact chunks (the staged path) and sparse ones whose boxes exceed the tile (direct
    loads).  The mesh force must match the oracle's (CIC gather of the same mesh force)."""
    pos, mom = S.clustered(64, 256.0, 4002)
    n = pos.shape[1]
    with P3M(256.0, n, 256) as sim:
        sim.set_particles(pos, mom, a=1.0)
        lr, _ = sim.forces_split()
    ref = O.pm_accel(O.wrap(pos, 256.0), O.Params(256.0, n, 256, softening=0.02))
    assert rel_rms(lr, ref) <= TOL["mixed"], rel_rms(lr, ref)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_density_mesh_exact_on_dyadic_positions(P3M, precision):
    """Positions on a quarter-node grid of a 48^3 mesh (box 48: node spacing 1, chaining cells of
    6 nodes) make every CIC weight a dyadic fraction that FP32 holds exactly, and N = M^3 / 8
    makes the mean 1/8.  The fixed-point deposit (split 32-bit shared tiles, run sums of equal
    base nodes, global atomics for chunks that straddle the periodic boundary) must then give the
    definition's mesh exactly.  Clumps of 8 coincident particles make runs of equal base node."""
    M = 48
    u = S.uniform01(4242, 3 * 1728).reshape(3, 1728)
    pos = np.repeat(np.floor(u * 4 * M) / 4, 8, axis=1)  # 1728 clumps x 8 = 48^3 / 8
    n = pos.shape[1]
    with P3M(float(M), n, M, precision=precision) as sim:
        assert sim.geometry()["n_c"] == 8
        sim.set_particles(pos, np.zeros_like(pos), a=1.0)
        sim.forces(1.0)
        rho = sim.get_mesh(0).astype(np.float64)
    ref = O.cic_deposit(pos, O.Params(float(M), n, M)) - n / M ** 3
    assert np.array_equal(rho, ref), np.max(np.abs(rho - ref))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("case", ["eds32", "clustered48", "random5003", "tiny3", "nc3",
                                  "coincident"])
def test_force_parts_match_oracle(P3M, case, precision):
    pos, mom, kw = _case(case)
    n = pos.shape[1]
    with P3M(kw["box"], n, kw["mesh"], precision=precision) as sim:
        sim.set_particles(pos, mom, a=1.0)
        lr, sr = sim.forces_split()
        diag = sim.diagnostics()
        tot = sim.forces(1.0)
    p = _params(n, kw)
    x = O.wrap(pos, kw["box"])
    lr_ref = O.pm_accel(x, p)
    sr_ref, npairs = O.sr_accel(x, p)
    tol = TOL[precision]
    assert rel_rms(lr, lr_ref) <= tol
    if npairs:
        assert rel_rms(sr, sr_ref) <= tol
    else:
        assert np.max(np.abs(sr)) == 0.0
    assert rel_rms(tot, lr_ref + sr_ref) <= tol
    # pairs within FP32 rounding of r = r_c may fall on either side in the mixed mode
    slack = 0 if precision == "fp64" else max(2, int(2e-5 * npairs))
    assert abs(diag["pairs"] - npairs) <= slack


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_pure_pm_mode(P3M, precision):
    pos, mom, kw = _case("eds32")
    n = pos.shape[1]
    with P3M(kw["box"], n, kw["mesh"], precision=precision, short_range=False) as sim:
        sim.set_particles(pos, mom, a=0.02)
        acc = sim.forces(0.02)
    ref = O.pm_accel(O.wrap(pos, kw["box"]), _params(n, kw, short_range=False))
    assert rel_rms(acc, ref) <= TOL[precision]


def test_momentum_conservation(P3M):
    pos, mom, kw = _case("clustered48")
    n = pos.shape[1]
    with P3M(kw["box"], n, kw["mesh"], precision="fp64") as sim:
        sim.set_particles(pos, mom, a=1.0)
        lr, sr = sim.forces_split()
    for a in (lr, sr):
        assert np.max(np.abs(a.sum(axis=1))) < 1e-11 * np.abs(a).sum()


# ------------------------------------------------------------------ time stepping


@pytest.mark.parametrize("precision,tol,mtol", [("fp64", 1e-11, 1e-9), ("mixed", 1e-6, 1e-4)])
def test_ten_steps_eds32(P3M, precision, tol, mtol):
    """Config of the 32^3 EdS run: 10 log-spaced steps a = 0.02 -> 0.1 against the oracle.
    FP64 mode: every position within 1e-11 L.  Mixed mode: RMS displacement within 1e-6 L; the
    worst particle within 4e-6 L, the band in which the FP64 oracle's own worst particle moves
    when its forces carry noise of the FP32 path's measured relative size (3.4e-6 RMS): a
    1e-6 L bound on the worst particle needs force errors below about 1e-6
    (tests/test_trajectory_sensitivity.py)."""
    pos, mom, kw = _case("eds32")
    n = pos.shape[1]
    a_s = S.log_spaced_steps(0.02, 0.1, 10)
    with P3M(kw["box"], n, kw["mesh"], precision=precision) as sim:
        sim.set_particles(pos, mom, a=a_s[0])
        for i in range(10):
            sim.step(a_s[i], a_s[i + 1] - a_s[i])
        gpos, gmom = sim.get_particles()
        d = sim.diagnostics()
    p = _params(n, kw)
    x, m = O.wrap(pos, kw["box"]), mom.copy()
    acc = O.accel(x, p)
    for i in range(10):
        x, m, acc = O.step(x, m, acc, a_s[i], a_s[i + 1] - a_s[i], p)
    dx = gpos - x
    dx -= kw["box"] * np.round(dx / kw["box"])
    if precision == "fp64":
        assert np.max(np.abs(dx)) <= tol * kw["box"]
    else:
        assert math.sqrt(np.mean(dx * dx)) <= tol * kw["box"]
        assert np.max(np.abs(dx)) <= 4e-6 * kw["box"]
    assert math.sqrt(np.mean((gmom - m) ** 2)) <= mtol * math.sqrt(np.mean(m * m))
    # the reductions of the diagnostics against numpy sums of the returned momenta
    assert np.allclose(d["momentum"], gmom.sum(axis=1), rtol=0, atol=1e-12 * np.abs(gmom).sum())
    assert abs(d["kinetic"] - O.kinetic_energy(gmom, a_s[-1])) <= 1e-12 * d["kinetic"]
    assert abs(d["kinetic"] - O.kinetic_energy(m, a_s[-1])) <= mtol * d["kinetic"]


def test_step_with_supplied_forces_equals_recompute(P3M):
    """A state loaded with its accelerations steps like one that recomputes them: identical
    positions (the drift only uses the supplied forces); momenta equal up to the FP32 rounding
    of the new forces (the two runs sort from different slot orders, so equal keys keep
    different orders and the pair sums add in different orders)."""
    pos, mom, kw = _case("eds32")
    n = pos.shape[1]
    with P3M(kw["box"], n, kw["mesh"]) as sim:
        sim.set_particles(pos, mom, a=0.05)
        acc = sim.forces(0.05)
        sim.step(0.05, 0.01)
        p1, m1 = sim.get_particles()
        sim.set_particles(pos, mom, acc=acc, a=0.05)
        sim.step(0.05, 0.01)
        p2, m2 = sim.get_particles()
    assert np.array_equal(p1, p2)
    assert rel_rms(m2, m1) <= 1e-6


# ------------------------------------------------------------------ errors


def test_error_paths(P3M):
    from paper_1510_07621_gb300 import P3MError, _lib
    pos, mom, kw = _case("tiny3")
    with P3M(kw["box"], 3, kw["mesh"]) as sim:
        with pytest.raises(P3MError) as e:
            sim.step(0.1, 0.01)
        assert e.value.code == _lib.P3M_ESTATE
        bad = pos.copy()
        bad[1, 2] = np.nan
        with pytest.raises(P3MError) as e:
            sim.set_particles(bad, mom, a=0.1)
        assert e.value.code == _lib.P3M_ENONFINITE
        sim.set_particles(pos, mom, a=0.1)
        with pytest.raises(P3MError) as e:
            sim.step(0.1, -0.01)
        assert e.value.code == _lib.P3M_EINVAL
        sim.step(0.1, 0.01)


# ------------------------------------------------------------------ full sizes, sampled


def _sampled(P3M, pos, mom, box, mesh, n_sample, seed, a):
    n = pos.shape[1]
    with P3M(box, n, mesh) as sim:  # the launch configuration of the benchmark
        sim.set_particles(pos, mom, a=a)
        acc = sim.forces(a)
        d = sim.diagnostics()
    tg = np.unique((S.uniform01(seed, n_sample) * n).astype(np.int64) % n)
    p = O.Params(box, n, mesh, softening=0.02)
    ref = O.accel(O.wrap(pos, box), p, targets=tg)
    return rel_rms(acc[:, tg], ref), d


def test_full_size_clustered_128_sampled(P3M):
    """128^3 particles, 128^3 mesh, box 200 Mpc/h, clustered late-time stand-in snapshot."""
    pos, mom = S.clustered(128, 200.0, 1512)
    err, d = _sampled(P3M, pos, mom, 200.0, 128, 400, 31, 1.0)
    assert err <= TOL["mixed"], err
    assert d["max_cell_count"] > 10 * (128 ** 3 // 22 ** 3)  # the input really is clustered


@pytest.mark.slow
def test_full_size_512_sampled(P3M):
    """512^3 particles, 512^3 mesh, box 1000 Mpc/h, Zel'dovich ICs at a = 0.5."""
    pos, mom = S.zeldovich(512, 1000.0, 0.5, 1513)
    err, _ = _sampled(P3M, pos, mom, 1000.0, 512, 200, 32, 0.5)
    assert err <= TOL["mixed"], err


def test_lcdm_steps_match_oracle(P3M):
    """Omega_m = 0.3, Omega_Lambda = 0.7 (Ch. Parameters, cosmological parameters): the kick and
    drift factors come from quadrature; 5 steps a = 0.1 -> 0.3 in FP64 mode."""
    pos, mom, kw = _case("eds32")
    n = pos.shape[1]
    a_s = S.log_spaced_steps(0.1, 0.3, 5)
    with P3M(kw["box"], n, kw["mesh"], precision="fp64", omega_m=0.3, omega_lambda=0.7) as sim:
        sim.set_particles(pos, mom, a=a_s[0])
        for i in range(5):
            sim.step(a_s[i], a_s[i + 1] - a_s[i])
        gpos, gmom = sim.get_particles()
    p = O.Params(kw["box"], n, kw["mesh"], softening=0.02, omega_m=0.3, omega_lambda=0.7)
    x, m = O.wrap(pos, kw["box"]), mom.copy()
    acc = O.accel(x, p)
    for i in range(5):
        x, m, acc = O.step(x, m, acc, a_s[i], a_s[i + 1] - a_s[i], p)
    dx = gpos - x
    dx -= kw["box"] * np.round(dx / kw["box"])
    assert np.max(np.abs(dx)) <= 1e-11 * kw["box"]
    assert np.max(np.abs(gmom - m)) <= 1e-9 * np.max(np.abs(m))


def test_fma_probe_reports_plausible_rates(P3M):
    """The FMA throughput probe: positive, FP32 far above FP64, FP32 below 2x the nominal peak
    (152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s)."""
    from paper_1510_07621_gb300 import measure_fma_peak
    f32, f64 = measure_fma_peak(False), measure_fma_peak(True)
    assert 1.0 < f32 < 161.0
    assert 0.01 < f64 < f32


def test_pinned_host_arrays_match_pageable_ones(P3M):
    """Page-locked host arrays are read and written in place by the kernels (over the CPU-GPU
    link); the results equal those of pageable arrays, which are staged through copies."""
    torch = pytest.importorskip("torch")
    pos, mom, kw = _case("clustered48")
    n = pos.shape[1]
    res = []
    for pinned in (False, True):
        with P3M(kw["box"], n, kw["mesh"], precision="fp64") as sim:
            if pinned:
                hp = torch.from_numpy(pos.copy()).pin_memory()
                hm = torch.from_numpy(mom.copy()).pin_memory()
                sim.set_particles(hp, hm, a=0.5)
                sim.step(0.5, 0.01)
                op = torch.empty((3, n), dtype=torch.float64).pin_memory()
                om = torch.empty((3, n), dtype=torch.float64).pin_memory()
                oa = torch.empty((3, n), dtype=torch.float64).pin_memory()
                sim.get_particles(op, om, oa)
                res.append((op.numpy().copy(), om.numpy().copy(), oa.numpy().copy()))
            else:
                sim.set_particles(pos, mom, a=0.5)
                sim.step(0.5, 0.01)
                op, om = np.empty((3, n)), np.empty((3, n))
                oa = np.empty((3, n))
                sim.get_particles(op, om, oa)
                res.append((op, om, oa))
    for x, y in zip(res[0], res[1]):
        assert np.max(np.abs(x - y)) <= 1e-12 * max(1.0, np.max(np.abs(x)))


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-6), ("fp64", 1e-13)])
def test_single_particle_feels_no_force(P3M, precision, tol):
    """N = 1, the smallest input: no pairs, and the mesh force on a lone particle vanishes (the
    CIC assignment and interpolation kernels are the same and the Green's function and the
    gradient are symmetric), at an arbitrary position; a step moves it by its momentum only."""
    box = 32.0
    pos = np.array([[3.7], [20.25], [31.9]])
    mom = np.array([[0.01], [-0.02], [0.005]])
    with P3M(box, 1, 32, precision=precision) as sim:
        sim.set_particles(pos, mom, a=0.5)
        acc = sim.forces(0.5)
        scale = 3.0 * box ** 3 / (8.0 * math.pi) / (box / 32) ** 2  # G m / h^2
        assert np.max(np.abs(acc)) <= tol * scale
        assert sim.diagnostics()["pairs"] == 0
        k1, dfac, _ = sim.step_factors(0.5, 0.1)
        sim.step(0.5, 0.1)
        p, m = sim.get_particles()
    dx = p - (pos + (mom + k1 * acc) * dfac)  # the half kick by the (vanishing) force, the drift
    assert np.max(np.abs(dx)) <= 1e-12 * box
