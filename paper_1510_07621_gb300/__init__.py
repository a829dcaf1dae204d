"""GB300 (sm_103a) P3M gravity step of the CONCEPT N-body method, behind a C ABI.

``P3M`` wraps one context of ``libp3m.so`` (``include/p3m.h``).  Particle arrays are
float64 ``(3, N)`` structure-of-arrays, either numpy arrays / CPU torch tensors (host) or
CUDA torch tensors (device).  PyTorch is only used for device memory and the stream; all
arithmetic runs in the library's kernels.  Nothing here falls back to the CPU: without the
compiled library every call raises.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (P3M_PREC_FP64, P3M_PREC_MIXED, Cosmology, Diag, Options, P3MError, check,
                   load)

__all__ = ["P3M", "Ensemble", "P3MError", "load", "P3M_PREC_MIXED", "P3M_PREC_FP64",
           "phase_names"]


def _is_torch(a) -> bool:
    return hasattr(a, "data_ptr") and hasattr(a, "is_cuda")


def _addr(a, shape, dtype_name):
    """(address, on_device) of a C-contiguous array of the given shape and dtype."""
    if a is None:
        return None, None
    if _is_torch(a):
        if str(a.dtype) != f"torch.{dtype_name}" or not a.is_contiguous() or tuple(a.shape) != shape:
            raise ValueError(f"expected a contiguous torch.{dtype_name} tensor of shape {shape}")
        return a.data_ptr(), 1 if a.is_cuda else 0
    if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype_name) or \
            not a.flags["C_CONTIGUOUS"] or a.shape != shape:
        raise ValueError(f"expected a C-contiguous numpy {dtype_name} array of shape {shape}")
    return a.ctypes.data, 0


def _side(*flags):
    f = {x for x in flags if x is not None}
    if len(f) > 1:
        raise ValueError("all arrays of one call must be on the same side (host or device)")
    return f.pop() if f else 0


def phase_names():
    lib = load()
    return [lib.p3m_phase_name(i).decode() for i in range(_lib.P3M_NPHASES)]


def measure_fma_peak(fp64: bool = False) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s (FP32 or FP64)."""
    lib = load()
    t = ctypes.c_double()
    check(lib.p3m_measure_fma_peak(1 if fp64 else 0, ctypes.byref(t)), None)
    return t.value


class P3M:
    """One P3M simulation context (box, N particles, mesh^3 PM grid).

    Parameters follow the guide's (Ch. Parameters): ``box`` (boxsize), ``mesh``
    (PM_gridsize), ``r_s_cells`` (PM_scale, mesh cells), ``cutoff`` (P3M_cutoff, units of the
    scale), ``softening`` (softeningfactors, mean spacings), ``omega_m``/``omega_lambda``.
    """

    def __init__(self, box: float, n: int, mesh: int, r_s_cells: float = 1.25,
                 cutoff: float = 4.5, omega_m: float = 1.0, omega_lambda: float = 0.0,
                 h0: float = 100.0, precision: str = "mixed", softening: float = 0.02,
                 deconvolve: bool = True, short_range: bool = True, sub_bits: int = 3,
                 stream=None, lib=None):
        lib = lib or load()
        self._lib = lib
        self.n = int(n)
        self.box = float(box)
        self.mesh = int(mesh)
        opt = Options()
        lib.p3m_default_options(ctypes.byref(opt))
        opt.precision = {"mixed": P3M_PREC_MIXED, "fp64": P3M_PREC_FP64}[precision]
        opt.softening = float(softening)
        opt.deconvolve_cic = 1 if deconvolve else 0
        opt.short_range = 1 if short_range else 0
        opt.sub_bits = int(sub_bits)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        opt.stream = ctypes.c_void_p(stream or 0)
        self.precision = precision
        cos = Cosmology(float(omega_m), float(omega_lambda), float(h0))
        ctx = ctypes.c_void_p()
        check(lib.p3m_init(ctypes.byref(ctx), self.box, self.n, self.mesh, float(r_s_cells),
                           float(cutoff), ctypes.byref(cos), ctypes.byref(opt)), None, lib)
        self._ctx = ctx

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.p3m_free(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, code):
        return check(code, self._ctx, self._lib)

    # ------------------------------------------------------------------ particles
    def set_particles(self, pos, mom, acc=None, mass: float = 1.0, a: float = 1.0):
        self.mass = float(mass)
        s = (3, self.n)
        p, d1 = _addr(pos, s, "float64")
        m, d2 = _addr(mom, s, "float64")
        q, d3 = _addr(acc, s, "float64")
        self._check(self._lib.p3m_set_particles(self._ctx, p, m, q, float(mass), float(a),
                                                _side(d1, d2, d3)))

    def get_particles(self, pos=None, mom=None, acc=None):
        """Fills the given arrays (caller order); with no arguments returns numpy copies of
        positions and momenta."""
        if pos is None and mom is None and acc is None:
            pos = np.empty((3, self.n))
            mom = np.empty((3, self.n))
            self.get_particles(pos, mom)
            return pos, mom
        s = (3, self.n)
        p, d1 = _addr(pos, s, "float64")
        m, d2 = _addr(mom, s, "float64")
        q, d3 = _addr(acc, s, "float64")
        self._check(self._lib.p3m_get_particles(self._ctx, p, m, q, _side(d1, d2, d3)))
        return pos, mom

    # ------------------------------------------------------------------ forces and steps
    def forces(self, a: float = 1.0, out=None):
        """Evaluates the accelerations; returns them in ``out`` (numpy if not given)."""
        if out is None:
            out = np.empty((3, self.n))
        q, d = _addr(out, (3, self.n), "float64")
        self._check(self._lib.p3m_forces(self._ctx, float(a), q, d or 0))
        return out

    def forces_split(self, lr=None, sr=None):
        if lr is None and sr is None:
            lr, sr = np.empty((3, self.n)), np.empty((3, self.n))
        s = (3, self.n)
        p, d1 = _addr(lr, s, "float64")
        q, d2 = _addr(sr, s, "float64")
        self._check(self._lib.p3m_forces_split(self._ctx, p, q, _side(d1, d2)))
        return lr, sr

    def step(self, a: float, da: float):
        self._check(self._lib.p3m_step(self._ctx, float(a), float(da)))

    def power_spectrum(self, n_bins: int | None = None, deconvolve: bool = True,
                       tophat_radius: float = 0.0):
        """(k_mean, power, n_modes, sigma) of the current positions; see p3m_power_spectrum."""
        nb = self.mesh // 2 if n_bins is None else int(n_bins)
        k = np.empty(nb)
        p = np.empty(nb)
        c = np.empty(nb)
        s = ctypes.c_double(float("nan"))
        self._check(self._lib.p3m_power_spectrum(self._ctx, nb, 1 if deconvolve else 0,
                                                 float(tophat_radius), k.ctypes.data,
                                                 p.ctypes.data, c.ctypes.data, ctypes.byref(s)))
        return k, p, c, (s.value if tophat_radius > 0 else None)

    def force_vjp(self, v, out=None):
        """(dA/dx)^T v at the current positions (v, out: (3, N) float64, host or device)."""
        if out is None:
            out = np.empty((3, self.n)) if not _is_torch(v) else v.new_empty((3, self.n))
        a, d1 = _addr(v, (3, self.n), "float64")
        b, d2 = _addr(out, (3, self.n), "float64")
        self._check(self._lib.p3m_force_vjp(self._ctx, a, b, _side(d1, d2)))
        return out

    def density_loss(self, target, grad=None):
        """(loss, grad): L2 of the CIC density contrast against target (M^3 float64)."""
        t, d1 = _addr(target, (self.mesh ** 3,), "float64")
        g, d2 = _addr(grad, (3, self.n), "float64")
        loss = ctypes.c_double()
        self._check(self._lib.p3m_density_loss(self._ctx, t, ctypes.byref(loss), g, _side(d1, d2)))
        return loss.value, grad

    def axpy(self, alpha: float, x, y):
        """y += alpha x on (3, N) float64 device tensors."""
        a, d1 = _addr(x, (3, self.n), "float64")
        b, d2 = _addr(y, (3, self.n), "float64")
        if not (d1 and d2):
            raise ValueError("axpy works on device tensors")
        self._check(self._lib.p3m_axpy(self._ctx, float(alpha), a, b))

    def step_factors(self, a: float, da: float):
        k1, d, k2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.p3m_step_factors(self._ctx, float(a), float(da), ctypes.byref(k1),
                                               ctypes.byref(d), ctypes.byref(k2)))
        return k1.value, d.value, k2.value

    def run_steps(self, a_list, use_graph: bool = True):
        """Kick-drift-kick steps through the scale factors a_list (len = steps + 1), replayed
        from captured CUDA graphs when use_graph (needs a non-default stream)."""
        a = np.ascontiguousarray(a_list, dtype=np.float64)
        self._check(self._lib.p3m_run_steps(self._ctx, a.ctypes.data, len(a) - 1,
                                            1 if use_graph else 0))

    def set_stream(self, stream):
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
        self._check(self._lib.p3m_set_stream(self._ctx, ctypes.c_void_p(s)))

    def tuning(self) -> dict:
        """Current sort-key Hilbert depth and FP32 pair-kernel tile length (blocks of 32)."""
        b, t = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.p3m_get_tuning(self._ctx, ctypes.byref(b), ctypes.byref(t)))
        return {"sub_bits": b.value, "tile_blocks": t.value}

    def autotune(self):
        """Picks the sort key's Hilbert depth, then the FP32 pair kernel's tile length, by timing
        force evaluations; returns (sub_bits, ms per evaluation for sub_bits 0..3)."""
        b = ctypes.c_int()
        ms = np.full(4, np.nan)
        self._check(self._lib.p3m_autotune(self._ctx, ctypes.byref(b), ms.ctypes.data))
        return b.value, ms

    def energy(self):
        """(K, W): kinetic and peculiar potential energy of the current state."""
        k, w = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.p3m_energy(self._ctx, ctypes.byref(k), ctypes.byref(w)))
        return k.value, w.value

    def track_energy(self, enable: bool = True):
        """Starts (or stops) the Layzer-Irvine bookkeeping: diagnostics() then reports the
        potential energy and the residual a(K + W) + int K da - a0 (K0 + W0)."""
        self._check(self._lib.p3m_track_energy(self._ctx, 1 if enable else 0))

    # ------------------------------------------------------------------ introspection
    def diagnostics(self) -> dict:
        d = Diag()
        self._check(self._lib.p3m_diagnostics(self._ctx, ctypes.byref(d)))
        return {"momentum": np.array(d.momentum[:]), "kinetic": d.kinetic, "a": d.a,
                "potential": d.potential, "layzer_irvine": d.layzer_irvine,
                "pairs": int(d.pairs), "pairs_total": int(d.pairs_total),
                "launches": int(d.launches), "pair_warp_j": [int(v) for v in d.pair_warp_j],
                "pair_blocks_culled": int(d.pair_blocks_culled),
                "pair_tiles": [int(v) for v in d.pair_tiles],
                "n": int(d.n), "n_cells_side": int(d.n_cells_side),
                "max_cell_count": int(d.max_cell_count)}

    def geometry(self) -> dict:
        v = [ctypes.c_int() for _ in range(4)]
        self._check(self._lib.p3m_get_geometry(self._ctx, *[ctypes.byref(x) for x in v]))
        return {"n_c": v[0].value, "mesh": v[1].value, "precision": v[2].value,
                "sub_bits": v[3].value}

    def get_cells(self):
        """(keys, ids, cell_start) of the last sort as numpy uint32 arrays."""
        n_c = self.geometry()["n_c"]
        keys = np.empty(self.n, np.uint32)
        ids = np.empty(self.n, np.uint32)
        cs = np.empty(n_c ** 3 + 1, np.uint32)
        self._check(self._lib.p3m_get_cells(self._ctx, keys.ctypes.data, ids.ctypes.data,
                                            cs.ctypes.data, 0))
        return keys, ids, cs

    def get_mesh(self, which: int) -> np.ndarray:
        dt = np.float32 if self.precision == "mixed" else np.float64
        out = np.empty((self.mesh,) * 3, dt)
        self._check(self._lib.p3m_get_mesh(self._ctx, int(which), out.ctypes.data, 0))
        return out

    def set_timing(self, enable: bool = True):
        self._check(self._lib.p3m_set_timing(self._ctx, 1 if enable else 0))

    def timings(self, reset: bool = True) -> dict:
        ms = (ctypes.c_double * _lib.P3M_NPHASES)()
        self._lib.p3m_timings(self._ctx, ms, _lib.P3M_NPHASES, 1 if reset else 0)
        return dict(zip(phase_names(), list(ms)))


class Ensemble:
    """Independent P3M contexts advanced together through one schedule of scale factors, one
    CUDA graph launch per step for the whole ensemble, FFTs batched per mesh size
    (p3m_ensemble_*)."""

    def __init__(self, sims, own_streams: bool = True, batched: bool | None = None,
                 fft_groups: bool | None = None):
        self._lib = sims[0]._lib if sims else load()
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s._ctx.value for s in self.sims])
        self._arr = arr
        e = ctypes.c_void_p()
        check(self._lib.p3m_ensemble_create(ctypes.byref(e), arr, len(self.sims),
                                            1 if own_streams else 0), None, self._lib)
        self._e = e
        if batched is not None:  # None: the library's default (per-simulation pair launches)
            check(self._lib.p3m_ensemble_set_batched(self._e, 1 if batched else 0), None, self._lib)
        if fft_groups is not None:  # None: the library's default (size-grouped batched FFTs)
            check(self._lib.p3m_ensemble_set_fft_groups(self._e, 1 if fft_groups else 0), None,
                  self._lib)

    def run(self, a_list, use_graph: bool = True):
        a = np.ascontiguousarray(a_list, dtype=np.float64)
        check(self._lib.p3m_ensemble_run(self._e, a.ctypes.data, len(a) - 1,
                                         1 if use_graph else 0), None, self._lib)

    def close(self):
        if getattr(self, "_e", None) is not None and self._e.value:
            self._lib.p3m_ensemble_free(self._e)
            self._e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
