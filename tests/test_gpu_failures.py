"""Failure reporting, tested by injecting the failure on the host (p3m_inject_fault), never by
making the GPU fault: a device allocation or a cuFFT plan of p3m_init that fails, and the
particle sort's bounded look-back wait giving up.  Each failure must come back as its status
code with a message naming the cause, leak nothing, and leave the library (and a context)
usable once the injection is cleared."""

import numpy as np
import pytest

import p3m_synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_07621_gb300 import build
    build.build()
    import paper_1510_07621_gb300 as m
    from paper_1510_07621_gb300 import _lib
    lib = _lib.load()
    yield torch, m, _lib, lib
    lib.p3m_inject_fault(None, _lib.P3M_INJECT_NONE, 0)


@pytest.mark.parametrize("index", [0, 7, 30])
def test_injected_allocation_failure(env, index):
    torch, m, _lib, lib = env
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert lib.p3m_inject_fault(None, _lib.P3M_INJECT_ALLOC, index) == _lib.P3M_OK
    try:
        with pytest.raises(m.P3MError) as e:
            m.P3M(64.0, 16 ** 3, 32)
        assert e.value.code == _lib.P3M_ENOMEM
        msg = lib.p3m_last_error(None).decode()
        assert "cudaMalloc" in msg and "(injected)" in msg
    finally:
        lib.p3m_inject_fault(None, _lib.P3M_INJECT_NONE, 0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (2 << 20)  # what was allocated was freed
    with m.P3M(64.0, 16 ** 3, 32) as sim:  # and the library works again
        pos, mom = S.zeldovich(16, 64.0, 0.1, 5)
        sim.set_particles(pos, mom, a=0.1)
        assert np.all(np.isfinite(sim.forces(0.1)))


def test_injected_fft_plan_failure(env):
    torch, m, _lib, lib = env
    assert lib.p3m_inject_fault(None, _lib.P3M_INJECT_FFT_PLAN, 0) == _lib.P3M_OK
    try:
        with pytest.raises(m.P3MError) as e:
            m.P3M(64.0, 16 ** 3, 32)
        assert e.value.code == _lib.P3M_ECUFFT
        msg = lib.p3m_last_error(None).decode()
        assert "cuFFT" in msg and "(injected)" in msg
    finally:
        lib.p3m_inject_fault(None, _lib.P3M_INJECT_NONE, 0)
    m.P3M(64.0, 16 ** 3, 32).close()


def test_injected_sort_timeout(env):
    """The sort's look-back watches a status word that nothing sets and gives up after 2000
    cycles: the force evaluation returns P3M_ETIMEOUT (it stops right after the sort), the
    positions are unchanged, and after clearing the injection the same context gives the
    forces of a fresh one, bit for bit."""
    torch, m, _lib, lib = env
    pos, mom = S.clustered(32, 64.0, 4004)
    n = pos.shape[1]
    with m.P3M(64.0, n, 32) as ref:
        ref.set_particles(pos, mom, a=1.0)
        f_ref = ref.forces(1.0)
    with m.P3M(64.0, n, 32) as sim:
        sim.set_particles(pos, mom, a=1.0)
        assert lib.p3m_inject_fault(sim._ctx, _lib.P3M_INJECT_SORT_TIMEOUT, 2000) == _lib.P3M_OK
        with pytest.raises(m.P3MError) as e:
            sim.forces(1.0)
        assert e.value.code == _lib.P3M_ETIMEOUT
        assert "wait gave up" in lib.p3m_last_error(sim._ctx).decode()
        p_after, m_after = sim.get_particles()
        assert np.array_equal(p_after, O_wrap(pos, 64.0)) and np.array_equal(m_after, mom)
        assert lib.p3m_inject_fault(sim._ctx, _lib.P3M_INJECT_NONE, 0) == _lib.P3M_OK
        assert np.array_equal(sim.forces(1.0), f_ref)


def O_wrap(pos, box):
    from oracle import p3m_oracle as O
    return O.wrap(pos, box)


def test_inject_fault_rejects_bad_arguments(env):
    torch, m, _lib, lib = env
    assert lib.p3m_inject_fault(None, 99, 0) == _lib.P3M_EINVAL
    assert lib.p3m_inject_fault(None, _lib.P3M_INJECT_ALLOC, -1) == _lib.P3M_EINVAL
    assert lib.p3m_inject_fault(None, _lib.P3M_INJECT_SORT_TIMEOUT, 100) == _lib.P3M_EINVAL
