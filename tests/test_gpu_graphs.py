"""Graph-captured steps, ensembles and the autotuner: the same trajectories as steps issued
one kernel at a time.  The mass deposit sums 64-bit fixed-point integers and every other sum
runs in a fixed order, so graph replay, host-issued steps and repeated runs give the same bits."""

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
    return torch, m


def _max_dx(p, q, box):
    d = p - q
    d -= box * np.round(d / box)
    return np.max(np.abs(d))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_steps_follow_host_steps(mod, precision):
    """Graph-replayed steps (device-side step factors, chunked captures, a host step in
    between) and host-issued steps give bit-identical positions and momenta."""
    torch, m = mod
    pos, mom = S.zeldovich(32, 64.0, 0.02, 1511)
    a = S.log_spaced_steps(0.02, 0.1, 14)
    n = pos.shape[1]
    ref = m.P3M(64.0, n, 32, stream=0, precision=precision)
    ref.set_particles(pos, mom, a=a[0])
    for k in range(14):
        ref.step(a[k], a[k + 1] - a[k])
    rp, rm = ref.get_particles()
    s = torch.cuda.Stream()
    with m.P3M(64.0, n, 32, stream=s, precision=precision) as sim:
        sim.set_particles(pos, mom, a=a[0])
        sim.run_steps(a[:4], use_graph=True)     # 3 steps: odd, parity flips
        sim.step(a[3], a[4] - a[3])              # host step in between: graphs recaptured
        sim.run_steps(a[4:], use_graph=True)     # 10 more: an 8-step chunk graph + 2 single
        gp, gm = sim.get_particles()
        d = sim.diagnostics()
    ref.close()
    assert np.array_equal(gp, rp), _max_dx(gp, rp, 64.0)
    assert np.array_equal(gm, rm)
    assert abs(d["a"] - a[-1]) < 1e-15


@pytest.mark.parametrize("fft_groups", [True, False])
def test_ensemble_matches_individual_runs(mod, fft_groups):
    """FP64 ensembles, graph-replayed and host-issued, with the FFTs batched per mesh size (two
    of the three members share mesh 32) or per member: every member's trajectory equals its
    individual run bit for bit, and so do its meshes after the ensemble is freed."""
    torch, m = mod
    specs = [(16, 32.0, 32, 11), (24, 40.0, 24, 12), (32, 64.0, 32, 13)]
    a = S.log_spaced_steps(0.05, 0.2, 12)
    ics = [S.zeldovich(n_p, box, a[0], seed) for n_p, box, mesh, seed in specs]
    refs = []
    for (n_p, box, mesh, seed), (pos, mom) in zip(specs, ics):
        with m.P3M(box, n_p ** 3, mesh, stream=0, precision="fp64") as r:
            r.set_particles(pos, mom, a=a[0])
            for k in range(12):
                r.step(a[k], a[k + 1] - a[k])
            refs.append(r.get_particles())
    for use_graph in (True, False):
        sims = [m.P3M(box, n_p ** 3, mesh, stream=0, precision="fp64")
                for n_p, box, mesh, seed in specs]
        for s_, (pos, mom) in zip(sims, ics):
            s_.set_particles(pos, mom, a=a[0])
        with m.Ensemble(sims, fft_groups=fft_groups) as ens:
            ens.run(a[:3], use_graph=use_graph)   # 2 single-step graphs
            ens.run(a[2:], use_graph=use_graph)   # one 8-step chunk graph, then 2 single steps
            torch.cuda.synchronize()
            dens = [s_.get_mesh(1) for s_ in sims]
        for s_, (n_p, box, mesh, seed), (rp, rm), dm in zip(sims, specs, refs, dens):
            gp, gm = s_.get_particles()
            assert np.array_equal(gp, rp) and np.array_equal(gm, rm), _max_dx(gp, rp, box)
            assert np.array_equal(s_.get_mesh(1), dm)  # the group slices were copied back
            s_.close()


@pytest.mark.parametrize("use_graph,batched", [(True, True), (False, True), (True, False)])
def test_batched_ensemble_matches_individual_runs(mod, use_graph, batched):
    """FP32 ensembles: the batched pair launch (one kernel over all simulations' work items),
    graph replay and per-simulation streams give each simulation its individual trajectory bit
    for bit; afterwards each member's forces match the FP64 oracle's at its positions."""
    torch, m = mod
    specs = [(16, 32.0, 32, 21), (24, 40.0, 24, 22), (32, 64.0, 32, 23), (20, 48.0, 40, 24)]
    a = S.log_spaced_steps(0.05, 0.1, 6)
    ics = [S.zeldovich(n_p, box, a[0], seed) for n_p, box, mesh, seed in specs]
    refs = []
    for (n_p, box, mesh, seed), (pos, mom) in zip(specs, ics):
        with m.P3M(box, n_p ** 3, mesh, stream=0) as r:
            r.set_particles(pos, mom, a=a[0])
            for k in range(6):
                r.step(a[k], a[k + 1] - a[k])
            refs.append(r.get_particles()[0])
    sims = [m.P3M(box, n_p ** 3, mesh, stream=0) for n_p, box, mesh, seed in specs]
    for s_, (pos, mom) in zip(sims, ics):
        s_.set_particles(pos, mom, a=a[0])
    with m.Ensemble(sims, batched=batched) as ens:
        ens.run(a[:2], use_graph=use_graph)
        ens.run(a[1:], use_graph=use_graph)
    for k, (s_, (n_p, box, mesh, seed), rp) in enumerate(zip(sims, specs, refs)):
        gp = s_.get_particles()[0]
        d = s_.diagnostics()
        assert np.array_equal(gp, rp), _max_dx(gp, rp, box)
        assert d["pairs"] > 0
        if k % 2 == 0:  # two members against the oracle at the positions the ensemble reached
            acc = s_.forces(a[-1])
            p = O.Params(box, n_p ** 3, mesh, softening=0.02)
            ref = O.accel(O.wrap(gp, box), p)
            err = math.sqrt(float(np.sum((acc - ref) ** 2) / np.sum(ref ** 2)))
            assert err <= 1e-5, err
        s_.close()


def test_autotune_keeps_forces(mod):
    torch, m = mod
    pos, mom = S.clustered(48, 100.0, 4001)
    n = pos.shape[1]
    with m.P3M(100.0, n, 48) as sim:
        sim.set_particles(pos, mom, a=1.0)
        f0 = sim.forces(1.0)
        b, ms = sim.autotune()
        assert b in (0, 1, 2, 3) and np.isfinite(ms[b]) and ms[b] == np.nanmin(ms)
        t = sim.tuning()
        assert t["sub_bits"] == b and t["tile_blocks"] in (3, 5)
        f1 = sim.forces(1.0)
        keys, ids, starts = sim.get_cells()
    assert math.sqrt(np.sum((f1 - f0) ** 2) / np.sum(f0 ** 2)) < 2e-6
    # after re-sorts with other key depths, equal keys keep their previous relative order:
    # the sorted keys are unique, the ids must be a permutation that carries them
    p = O.Params(100.0, n, 48, sub_bits=b)
    cell, key = O.cell_keys(O.wrap(pos, 100.0), p)
    assert np.array_equal(keys.astype(np.int64), np.sort(key))
    assert np.array_equal(np.sort(ids.astype(np.int64)), np.arange(n))
    assert np.array_equal(key[ids.astype(np.int64)], keys.astype(np.int64))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_repeated_runs_are_bit_identical(mod, precision):
    """Two runs of the same 14-step trajectory on the clustered 48^3 state (dense cells, so the
    deposit's shared-memory tiles and its global atomics both run) give the same bits: forces,
    positions, momenta, the density mesh and the power spectrum."""
    torch, m = mod
    pos, mom = S.clustered(48, 100.0, 4001)
    n = pos.shape[1]
    a = S.log_spaced_steps(0.5, 0.6, 14)
    out = []
    for _ in range(2):
        with m.P3M(100.0, n, 48, precision=precision) as sim:
            sim.set_particles(pos, mom, a=a[0])
            acc = sim.forces(a[0])
            for k in range(14):
                sim.step(a[k], a[k + 1] - a[k])
            p, q = sim.get_particles()
            rho = sim.get_mesh(0)
            ps = sim.power_spectrum(tophat_radius=8.0)
            out.append((acc, p, q, rho, ps[1], ps[3]))
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_fft_groups_toggle_and_energy_tracking(mod):
    """FP32 ensemble of five members (a group of three at mesh 32, a group of two at mesh 24)
    that track the Layzer-Irvine energy: runs with the FFTs batched per group, then per member
    (groups turned off), then grouped again; every member's positions, momenta and energy
    residual equal those of its individual run bit for bit."""
    torch, m = mod
    specs = [(16, 32.0, 32, 41), (16, 32.0, 32, 42), (24, 40.0, 24, 43), (16, 32.0, 32, 44),
             (24, 40.0, 24, 45)]
    a = S.log_spaced_steps(0.05, 0.15, 9)
    ics = [S.zeldovich(n_p, box, a[0], seed) for n_p, box, mesh, seed in specs]
    refs = []
    for (n_p, box, mesh, seed), (pos, mom) in zip(specs, ics):
        with m.P3M(box, n_p ** 3, mesh, stream=0) as r:
            r.set_particles(pos, mom, a=a[0])
            r.track_energy(True)
            for k in range(9):
                r.step(a[k], a[k + 1] - a[k])
            refs.append(r.get_particles() + (r.diagnostics()["layzer_irvine"],))
    sims = [m.P3M(box, n_p ** 3, mesh, stream=0) for n_p, box, mesh, seed in specs]
    for s_, (pos, mom) in zip(sims, ics):
        s_.set_particles(pos, mom, a=a[0])
        s_.track_energy(True)
    with m.Ensemble(sims) as ens:
        ens.run(a[:4], use_graph=True)      # grouped (the default)
        ens._lib.p3m_ensemble_set_fft_groups(ens._e, 0)
        ens.run(a[3:7], use_graph=True)     # per-member FFTs
        ens._lib.p3m_ensemble_set_fft_groups(ens._e, 1)
        ens.run(a[6:], use_graph=False)     # grouped again, host-issued
    for s_, (rp, rm, rli) in zip(sims, refs):
        gp, gm = s_.get_particles()
        assert np.array_equal(gp, rp) and np.array_equal(gm, rm)
        assert s_.diagnostics()["layzer_irvine"] == rli
        s_.close()
