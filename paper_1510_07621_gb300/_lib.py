"""ctypes binding of ``libp3m.so``: the C ABI of ``include/p3m.h`` under the same names.

Argument marshalling only; every step of the computation runs in the library's CUDA
kernels.  There is no fallback: if the library cannot be loaded, ``load()`` raises.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libp3m.so")

P3M_OK = 0
P3M_EINVAL = -1
P3M_ENOMEM = -2
P3M_ECUDA = -3
P3M_ECUFFT = -4
P3M_ESTATE = -5
P3M_ETIMEOUT = -6
P3M_ENONFINITE = -7
P3M_EBOUNDS = -8
P3M_PREC_MIXED = 0
P3M_PREC_FP64 = 1
P3M_NPHASES = 10
P3M_NOALLOC_MAX_N = 1048576
P3M_INJECT_NONE = 0
P3M_INJECT_ALLOC = 1
P3M_INJECT_FFT_PLAN = 2
P3M_INJECT_SORT_TIMEOUT = 3

# every symbol the header declares, with (restype, argtypes)
_c = ctypes
_vp = _c.c_void_p
_dp = _c.c_void_p  # double*, passed as raw addresses (host or device)


class Cosmology(_c.Structure):
    _fields_ = [("omega_m", _c.c_double), ("omega_lambda", _c.c_double), ("h0", _c.c_double)]


class Options(_c.Structure):
    _fields_ = [("precision", _c.c_int), ("softening", _c.c_double),
                ("deconvolve_cic", _c.c_int), ("short_range", _c.c_int),
                ("sub_bits", _c.c_int), ("stream", _c.c_void_p)]


class Diag(_c.Structure):
    _fields_ = [("momentum", _c.c_double * 3), ("kinetic", _c.c_double),
                ("potential", _c.c_double), ("layzer_irvine", _c.c_double), ("a", _c.c_double),
                ("pairs", _c.c_uint64), ("pairs_total", _c.c_uint64), ("launches", _c.c_uint64),
                ("pair_warp_j", _c.c_uint64 * 3), ("pair_blocks_culled", _c.c_uint64),
                ("pair_tiles", _c.c_uint64 * 2),
                ("n", _c.c_int64), ("n_cells_side", _c.c_int32),
                ("max_cell_count", _c.c_int32)]


SIGNATURES = {
    "p3m_default_options": (_c.c_int, [_c.POINTER(Options)]),
    "p3m_init": (_c.c_int, [_c.POINTER(_vp), _c.c_double, _c.c_int64, _c.c_int, _c.c_double,
                            _c.c_double, _c.POINTER(Cosmology), _c.POINTER(Options)]),
    "p3m_set_particles": (_c.c_int, [_vp, _dp, _dp, _dp, _c.c_double, _c.c_double, _c.c_int]),
    "p3m_forces": (_c.c_int, [_vp, _c.c_double, _dp, _c.c_int]),
    "p3m_forces_split": (_c.c_int, [_vp, _dp, _dp, _c.c_int]),
    "p3m_step": (_c.c_int, [_vp, _c.c_double, _c.c_double]),
    "p3m_power_spectrum": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_double, _vp, _vp, _vp,
                                      _c.POINTER(_c.c_double)]),
    "p3m_get_particles": (_c.c_int, [_vp, _dp, _dp, _dp, _c.c_int]),
    "p3m_diagnostics": (_c.c_int, [_vp, _c.POINTER(Diag)]),
    "p3m_energy": (_c.c_int, [_vp, _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)]),
    "p3m_track_energy": (_c.c_int, [_vp, _c.c_int]),
    "p3m_get_cells": (_c.c_int, [_vp, _vp, _vp, _vp, _c.c_int]),
    "p3m_get_mesh": (_c.c_int, [_vp, _c.c_int, _vp, _c.c_int]),
    "p3m_get_geometry": (_c.c_int, [_vp, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int),
                                    _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "p3m_set_timing": (_c.c_int, [_vp, _c.c_int]),
    "p3m_timings": (_c.c_int, [_vp, _c.POINTER(_c.c_double), _c.c_int, _c.c_int]),
    "p3m_phase_name": (_c.c_char_p, [_c.c_int]),
    "p3m_force_vjp": (_c.c_int, [_vp, _vp, _vp, _c.c_int]),
    "p3m_density_loss": (_c.c_int, [_vp, _vp, _c.POINTER(_c.c_double), _vp, _c.c_int]),
    "p3m_axpy": (_c.c_int, [_vp, _c.c_double, _vp, _vp]),
    "p3m_step_factors": (_c.c_int, [_vp, _c.c_double, _c.c_double, _c.POINTER(_c.c_double),
                                    _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)]),
    "p3m_run_steps": (_c.c_int, [_vp, _vp, _c.c_int, _c.c_int]),
    "p3m_set_stream": (_c.c_int, [_vp, _vp]),
    "p3m_ensemble_create": (_c.c_int, [_c.POINTER(_vp), _vp, _c.c_int, _c.c_int]),
    "p3m_ensemble_run": (_c.c_int, [_vp, _vp, _c.c_int, _c.c_int]),
    "p3m_ensemble_free": (None, [_vp]),
    "p3m_ensemble_set_fft_groups": (_c.c_int, [_vp, _c.c_int]),
    "p3m_ensemble_set_batched": (_c.c_int, [_vp, _c.c_int]),
    "p3m_autotune": (_c.c_int, [_vp, _c.POINTER(_c.c_int), _vp]),
    "p3m_get_tuning": (_c.c_int, [_vp, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "p3m_inject_fault": (_c.c_int, [_vp, _c.c_int, _c.c_int64]),
    "p3m_debug_check": (_c.c_int, [_vp]),
    "p3m_debug_poke_canary": (_c.c_int, [_vp, _c.c_int]),
    "p3m_cell_sort_noalloc": (_c.c_int, [_vp, _c.c_int64, _c.c_double, _c.c_int, _c.c_int,
                                         _vp, _vp, _vp, _vp]),
    "p3m_measure_fma_peak": (_c.c_int, [_c.c_int, _c.POINTER(_c.c_double)]),
    "p3m_last_error": (_c.c_char_p, [_vp]),
    "p3m_free": (None, [_vp]),
}

_lib = None


def bind(path: str):
    """Loads the library at ``path`` with the C ABI's signatures (not cached)."""
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1510_07621_gb300.build.build() "
                           "(the P3M path has no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path: str | None = None):
    """Loads libp3m.so once (building it first is the caller's job: ``build.build()``)."""
    global _lib
    if _lib is None:
        _lib = bind(path or LIB_PATH)
    return _lib


class P3MError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"P3M error {code}: {msg}")
        self.code = code


def check(code: int, ctx=None, lib=None):
    if code != P3M_OK:
        msg = (lib or load()).p3m_last_error(ctx).decode(errors="replace")
        raise P3MError(code, msg)
    return code
