"""The debug build (P3M_DEBUG_CHECKS), which stands in for a memory checker: its kernels test the
indices they compute (mesh nodes of the deposit and gather, source slots of the permute, cell
ranges, the key range, the pair kernels' neighbour ranges) and record a failure instead of
making the access, and every device allocation of p3m_init is followed by guard bytes.  A mixed
and an FP64 run through every phase (forces, steps, power spectrum, force VJP, energies, an
ensemble with graphs) must pass p3m_debug_check and give the release build's results bit for
bit; a guard byte overwritten on purpose (host-side, inside the allocation) must be caught."""

import numpy as np
import pytest

import p3m_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_07621_gb300 import _lib, build
    build.build()
    dbg = _lib.bind(build.build(debug=True))
    return torch, _lib, _lib.load(), dbg


def _run(m, lib, precision):
    pos, mom = S.clustered(32, 64.0, 4005)
    n = pos.shape[1]
    a = S.log_spaced_steps(0.5, 0.6, 3)
    out = []
    with m.P3M(64.0, n, 32, precision=precision, lib=lib) as sim:
        sim.set_particles(pos, mom, a=a[0])
        out.append(sim.forces(a[0]))
        for k in range(3):
            sim.step(a[k], a[k + 1] - a[k])
        out.extend(sim.get_particles())
        out.append(sim.power_spectrum(tophat_radius=8.0)[1])
        out.append(sim.force_vjp(S.gaussian(3, 3 * n).reshape(3, n)))
        out.append(np.array(sim.energy()))
        assert lib.p3m_debug_check(sim._ctx) == 0, lib.p3m_last_error(sim._ctx).decode()
    return out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_debug_build_passes_its_checks_and_matches_release(libs, precision):
    torch, _lib, rel, dbg = libs
    import paper_1510_07621_gb300 as m
    for x, y in zip(_run(m, dbg, precision), _run(m, rel, precision)):
        assert np.array_equal(x, y)


def test_debug_build_staged_gather(libs):
    """A 256^3 mesh, whose three FP32 force meshes exceed L2, takes the staged gather (chunk node
    boxes in shared memory, tile indices from FP32 reciprocals) and the split-tile deposit with
    sparse and dense chunks: every tile index stays in bounds, and the results equal the
    release build's."""
    torch, _lib, rel, dbg = libs
    import paper_1510_07621_gb300 as m
    pos, mom = S.clustered(64, 256.0, 4002)
    out = []
    for lib in (dbg, rel):
        with m.P3M(256.0, pos.shape[1], 256, lib=lib) as sim:
            sim.set_particles(pos, mom, a=1.0)
            out.append(sim.forces_split()[0])
            out.append(sim.get_mesh(0))
            assert lib.p3m_debug_check(sim._ctx) == 0, lib.p3m_last_error(sim._ctx).decode()
    assert np.array_equal(out[0], out[2]) and np.array_equal(out[1], out[3])


def test_debug_build_ensemble_with_graphs(libs):
    torch, _lib, rel, dbg = libs
    import paper_1510_07621_gb300 as m
    specs = [(16, 32.0, 32, 31), (16, 32.0, 32, 32), (24, 40.0, 24, 33)]
    a = S.log_spaced_steps(0.05, 0.1, 10)
    sims = [m.P3M(box, n_p ** 3, mesh, stream=0, lib=dbg) for n_p, box, mesh, seed in specs]
    for s_, (n_p, box, mesh, seed) in zip(sims, specs):
        s_.set_particles(*S.zeldovich(n_p, box, a[0], seed), a=a[0])
    with m.Ensemble(sims) as ens:
        ens.run(a, use_graph=True)
    for s_ in sims:
        assert dbg.p3m_debug_check(s_._ctx) == 0, dbg.p3m_last_error(s_._ctx).decode()
        s_.close()


def test_guard_bytes_catch_an_overwrite(libs):
    torch, _lib, rel, dbg = libs
    import paper_1510_07621_gb300 as m
    with m.P3M(32.0, 16 ** 3, 32, lib=dbg) as sim:
        assert dbg.p3m_debug_check(sim._ctx) == 0
        assert dbg.p3m_debug_poke_canary(sim._ctx, 5) == 0
        assert dbg.p3m_debug_check(sim._ctx) == _lib.P3M_EBOUNDS
        assert "allocation 5" in dbg.p3m_last_error(sim._ctx).decode()
    with m.P3M(32.0, 16 ** 3, 32, lib=rel) as sim:  # the release build has no guard bytes
        assert rel.p3m_debug_poke_canary(sim._ctx, 5) == _lib.P3M_ESTATE
        assert rel.p3m_debug_check(sim._ctx) == 0
