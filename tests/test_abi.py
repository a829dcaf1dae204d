"""The C ABI library builds, loads and exports every entry point include/p3m.h declares.

CPU-only: no call here launches GPU work.  Argument checks that fail before any CUDA call
are exercised through p3m_init.
"""

import ctypes
import os
import re

import pytest

from paper_1510_07621_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "p3m.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(p3m_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = _declared()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} has no Python binding"


def test_default_options_and_phase_names(lib):
    opt = _lib.Options()
    assert lib.p3m_default_options(ctypes.byref(opt)) == 0
    assert opt.precision == _lib.P3M_PREC_MIXED and opt.short_range == 1
    assert abs(opt.softening - 0.02) < 1e-15 and opt.sub_bits == 3
    assert lib.p3m_default_options(None) == _lib.P3M_EINVAL
    names = [lib.p3m_phase_name(i).decode() for i in range(_lib.P3M_NPHASES)]
    assert names[0] == "kick_drift" and names[8] == "pairs"
    assert lib.p3m_phase_name(_lib.P3M_NPHASES) is None


@pytest.mark.parametrize("args,needle", [
    ((64.0, 32768, 32, 1.25, 4.5), None),            # valid -> reaches the device query
    ((64.0, 32768, 31, 1.25, 4.5), "mesh"),          # odd mesh
    ((64.0, 0, 32, 1.25, 4.5), "n must"),            # empty particle set
    ((64.0, 1 << 31, 32, 1.25, 4.5), "n must"),      # too many particles
    ((-1.0, 100, 32, 1.25, 4.5), "box"),
    ((20.0, 100, 16, 1.25, 4.5), "chaining cells"),  # r_c too large: n_c = 2 < 3
    ((64.0, 100, 32, 0.0, 4.5), "r_s"),
    ((64.0, 100, 32, 1.25, float("nan")), "cutoff"),
])
def test_init_argument_checks(lib, args, needle):
    ctx = ctypes.c_void_p()
    rc = lib.p3m_init(ctypes.byref(ctx), *args, None, None)
    msg = lib.p3m_last_error(None).decode()
    if needle is None:
        # no GPU in this container: a valid call stops at the device query
        assert rc in (_lib.P3M_OK, _lib.P3M_ECUDA)
        if rc == _lib.P3M_OK:
            lib.p3m_free(ctx)
    else:
        assert rc == _lib.P3M_EINVAL and needle in msg, msg
        assert not ctx.value


def test_null_context_is_rejected(lib):
    assert lib.p3m_ensemble_set_batched(None, 1) == _lib.P3M_EINVAL
    assert lib.p3m_energy(None, None, None) == _lib.P3M_EINVAL
    assert lib.p3m_track_energy(None, 1) == _lib.P3M_EINVAL
    assert lib.p3m_measure_fma_peak(0, None) == _lib.P3M_EINVAL
    assert lib.p3m_step(None, 0.1, 0.01) == _lib.P3M_EINVAL
    assert lib.p3m_forces(None, 0.1, None, 0) == _lib.P3M_EINVAL
    assert lib.p3m_get_geometry(None, None, None, None, None) == _lib.P3M_EINVAL
    lib.p3m_free(None)
