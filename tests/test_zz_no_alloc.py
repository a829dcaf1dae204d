"""The allocation-free cell binning (p3m_cell_sort_noalloc) against a context's own binning.

Some callers may not allocate GPU memory (their framework's allocator owns the device memory,
or their loop cannot afford cudaMalloc's synchronisation).  p3m_cell_sort_noalloc serves them
from a fixed scratch area that the library reserves when it loads.  Its keys, particle order
and cell ranges must equal, bit for bit, what p3m_get_cells reports for a context holding the
same particles, on two calls in a row through the C ABI (the scratch keeps the previous
call's contents).  This file is collected last.
"""

import ctypes

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
    from paper_1510_07621_gb300 import P3M, _lib
    return torch, P3M, _lib, _lib.load()


@pytest.mark.parametrize("sub_bits", [0, 2])
def test_noalloc_binning_equals_context_binning(env, sub_bits):
    torch, P3M, _lib, lib = env
    box, n_p, mesh = 100.0, 48, 48
    pos, mom = S.clustered(n_p, box, 4002)
    n = pos.shape[1]
    with P3M(box, n, mesh, sub_bits=sub_bits) as sim:
        sim.set_particles(pos, mom, a=1.0)
        sim.forces(1.0)
        keys, ids, starts = sim.get_cells()
        n_c = sim.geometry()["n_c"]
    dev = torch.device("cuda", 0)
    dpos = torch.from_numpy(pos).to(dev).contiguous()
    k = torch.empty(n, dtype=torch.int32, device=dev)
    i = torch.empty(n, dtype=torch.int32, device=dev)
    c = torch.empty(n_c ** 3 + 1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        k.fill_(-1)
        i.fill_(-1)
        c.fill_(-1)
        rc = lib.p3m_cell_sort_noalloc(dpos.data_ptr(), n, box, n_c, sub_bits, k.data_ptr(),
                                       i.data_ptr(), c.data_ptr(), stream.cuda_stream)
        assert rc == _lib.P3M_OK, lib.p3m_last_error(None).decode()
        torch.cuda.synchronize(dev)
        assert np.array_equal(k.cpu().numpy().view(np.uint32), keys)
        assert np.array_equal(i.cpu().numpy().view(np.uint32), ids)
        assert np.array_equal(c.cpu().numpy().view(np.uint32), starts)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, P3M, _lib, lib = env
    n = _lib.P3M_NOALLOC_MAX_N + 1
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    rc = lib.p3m_cell_sort_noalloc(dummy, n, 100.0, 8, 2, dummy, dummy, dummy, None)
    assert rc == _lib.P3M_EINVAL
    assert "outside" in lib.p3m_last_error(None).decode()


def test_noalloc_at_its_largest_size_allocates_nothing(env):
    """n = P3M_NOALLOC_MAX_N, where the digit counts and scan partials sit at the very end of
    the fixed area: the same binning as a context's; and after the set-up call the device's
    free memory does not change across two more calls."""
    torch, P3M, _lib, lib = env
    n, box, mesh, sub_bits = _lib.P3M_NOALLOC_MAX_N, 150.0, 96, 2
    pos = S.uniform_random(n, box, 4003)
    with P3M(box, n, mesh, sub_bits=sub_bits) as sim:
        sim.set_particles(pos, np.zeros_like(pos), a=1.0)
        sim.forces(1.0)
        keys, ids, starts = sim.get_cells()
        n_c = sim.geometry()["n_c"]
    dev = torch.device("cuda", 0)
    dpos = torch.from_numpy(pos).to(dev).contiguous()
    k = torch.empty(n, dtype=torch.int32, device=dev)
    i = torch.empty(n, dtype=torch.int32, device=dev)
    c = torch.empty(n_c ** 3 + 1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def call():
        rc = lib.p3m_cell_sort_noalloc(dpos.data_ptr(), n, box, n_c, sub_bits, k.data_ptr(),
                                       i.data_ptr(), c.data_ptr(), stream.cuda_stream)
        assert rc == _lib.P3M_OK, lib.p3m_last_error(None).decode()
        torch.cuda.synchronize(dev)

    call()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for _ in range(2):
        k.fill_(-1)
        i.fill_(-1)
        call()
        assert torch.cuda.mem_get_info(dev)[0] == free0
        assert np.array_equal(k.cpu().numpy().view(np.uint32), keys)
        assert np.array_equal(i.cpu().numpy().view(np.uint32), ids)
        assert np.array_equal(c.cpu().numpy().view(np.uint32), starts)
