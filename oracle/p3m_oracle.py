"""Plain FP64 CPU oracle of the P3M gravity step -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its cpu_baseline leg and its
``--impl reference`` arm) may import this module.  It shares no code with the CUDA path.

The guide (CONCEPT user's guide, 2015) describes the P3M kick algorithm only through its
parameters (Ch. Parameters: ``boxsize``, ``PM_gridsize``, ``PM_scale``, ``P3M_cutoff``,
``softeningfactors``; cosmological parameters ``H0``, ``Omega_m``, ``Omega_Lambda``;
Ch. Snapshot Formats: comoving positions and momenta).  It prints no equations, so each step
below is the textbook P3M step (Hockney & Eastwood) with the Gaussian/erfc force split,
written in the order the force evaluation runs:

  1. periodic wrap of the positions into [0, L)
  2. chaining-cell keys and the stable order of particles by key
  3. cloud-in-cell (CIC) mass assignment onto the M^3 mesh (nodes at i*h)
  4. forward FFT of the mesh
  5. Green's function -4 pi G / k^2 * exp(-k^2 r_s^2) / W(k)^2 and spectral gradient -i k
  6. three inverse FFTs -> mesh accelerations
  7. CIC interpolation of the mesh accelerations back to the particles
  8. short-range pair sum over the 27 neighbouring chaining cells (plain C, ``sr_pairs.c``)
  9. comoving kick-drift-kick leapfrog

Readings where the guide is silent:
  * split convention g(x) = erfc(x/2) + x/sqrt(pi) exp(-x^2/4), x = r/r_s, with the
    long-range filter exp(-k^2 r_s^2): the only one under which the guide's "cutoff >= 4.8
    leaves < 1 % of the force out" holds (g(4.8) = 0.92 %);
  * mesh nodes at i*h, CIC deconvolution W(k)^-2 with W = prod_d sinc^2(k_d h/2) (option);
  * gradient component k_d set to 0 on the Nyquist plane of axis d;
  * pairs with r = r_c excluded, r = 0 skipped; Plummer softening (r^2 + eps^2)^-3/2 with g
    taken at the unsoftened r;
  * units: H0 = 1 (time unit 1/H0), 4 pi G rho_bar = (3/2) Omega_m H0^2, so the per-particle
    coupling Gm = 3 Omega_m L^3 / (8 pi N);
  * momentum p = m a^2 dx/dt; kick dp = m a_grav * int dt/a, drift dx = p/m * int dt/a^2;
  * inside a chaining cell the particles are ordered by the 3-D Hilbert index of their fine
    sub-cell (Skilling 2004), ties by input order: the guide fixes no order, the GPU path's
    sort reproduces this one bit for bit.

Arrays: positions/momenta/accelerations are float64 SoA of shape (3, N).
"""

from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np
from scipy.special import erfc

from . import build as _build

# --------------------------------------------------------------------------- parameters


@dataclass
class Params:
    """Run parameters, named after the guide's (Ch. Parameters)."""

    box: float                 # boxsize, comoving Mpc/h
    n: int                     # number of particles N
    mesh: int                  # PM_gridsize M
    r_s_cells: float = 1.25    # PM_scale, in PM cells
    cutoff: float = 4.5        # P3M_cutoff, in units of the scale
    softening: float = 0.0     # softeningfactors, units of the mean spacing box/N^(1/3)
    deconvolve: bool = True    # divide the Green's function by W(k)^2
    sub_bits: int = 0          # chaining cells split 2^b per side in the sort key
    short_range: bool = True   # False: pure PM
    omega_m: float = 1.0
    omega_lambda: float = 0.0
    n_c: int = field(init=False)

    def __post_init__(self):
        self.n_c = max(1, int(math.floor(self.box / self.r_c)))

    def check_cells(self):
        if self.n_c < 3:
            raise ValueError("fewer than 3 chaining cells per side: r_c too large for the box")

    @property
    def h(self) -> float:
        return self.box / self.mesh

    @property
    def r_s(self) -> float:
        return self.r_s_cells * (self.box / self.mesh)

    @property
    def r_c(self) -> float:
        return self.cutoff * (self.r_s_cells * (self.box / self.mesh))

    @property
    def eps(self) -> float:
        return self.softening * (self.box / float(np.cbrt(float(self.n))))

    @property
    def gm(self) -> float:
        """G*m from 4 pi G rho_bar = (3/2) Omega_m H0^2, rho_bar = N m / L^3, H0 = 1."""
        return 3.0 * self.omega_m * self.box ** 3 / (8.0 * math.pi * self.n)

    @property
    def n_fine(self) -> int:
        return self.n_c << self.sub_bits

    @property
    def inv_fine(self) -> float:
        return float(self.n_fine) / self.box


# --------------------------------------------------------------------------- 1. wrap


def wrap(pos: np.ndarray, box: float) -> np.ndarray:
    """Periodic wrap into [0, box): fmod (exact in IEEE arithmetic), then one correction each
    way, the second catching -tiny + box rounding up to box."""
    x = np.fmod(pos, box)
    x = np.where(x < 0.0, x + box, x)
    x = np.where(x >= box, x - box, x)
    return x


# --------------------------------------------------------------------------- 2. keys, order


def fine_index(pos: np.ndarray, p: Params) -> np.ndarray:
    """Per-axis fine cell index f_d = min(trunc(x_d * (n_c 2^b / L)), n_c 2^b - 1) of wrapped
    positions: one correctly rounded FP64 multiply, truncation, clamp.  int64 (3, N)."""
    f = np.trunc(pos * p.inv_fine).astype(np.int64)
    return np.minimum(f, p.n_fine - 1)


def hilbert3(sx, sy, sz, bits: int):
    """Index of the point (sx, sy, sz), each in [0, 2^bits), along the 3-D Hilbert curve of that
    order, after Skilling, "Programming the Hilbert curve" (AIP Conf. Proc. 707, 2004): the
    coordinates are turned into the curve's "transposed" index (undo the excess rotations and
    reflections level by level, then Gray-encode), whose bits, read level by level with x as
    the most significant of each triple, form the index.  0 <= index < 8^bits; consecutive
    indices are face-neighbour points."""
    x = [np.asarray(sx, dtype=np.int64).copy(), np.asarray(sy, dtype=np.int64).copy(),
         np.asarray(sz, dtype=np.int64).copy()]
    if bits == 0:
        return np.zeros_like(x[0])
    top = 1 << (bits - 1)
    q = top
    while q > 1:  # undo the excess work, level q
        lowmask = q - 1
        for i in range(3):
            hit = (x[i] & q) != 0
            flipped = x[0] ^ lowmask                    # invert the low bits of x0
            swap = (x[0] ^ x[i]) & lowmask              # or exchange them with x_i
            new0 = np.where(hit, flipped, x[0] ^ swap)
            newi = np.where(hit, x[i], x[i] ^ swap)
            x[0] = new0
            if i:
                x[i] = newi
        q >>= 1
    x[1] ^= x[0]  # Gray encode
    x[2] ^= x[1]
    t = np.zeros_like(x[0])
    q = top
    while q > 1:
        t = np.where((x[2] & q) != 0, t ^ (q - 1), t)
        q >>= 1
    for i in range(3):
        x[i] ^= t
    h = np.zeros_like(x[0])
    for level in range(bits - 1, -1, -1):
        for i in range(3):
            h = (h << 1) | ((x[i] >> level) & 1)
    return h


def cell_keys(pos: np.ndarray, p: Params):
    """Chaining-cell id c = (c_z n_c + c_y) n_c + c_x with c_d = f_d >> b, and the sort key
    (c << 3b) | hilbert(f_x & (2^b-1), f_y & .., f_z & ..).  Returns (cell, key) as int64."""
    p.check_cells()
    f = fine_index(pos, p)
    b = p.sub_bits
    c = f >> b
    cell = (c[2] * p.n_c + c[1]) * p.n_c + c[0]
    mask = (1 << b) - 1
    key = (cell << (3 * b)) | hilbert3(f[0] & mask, f[1] & mask, f[2] & mask, b)
    return cell, key


def stable_order(keys: np.ndarray) -> np.ndarray:
    """Indices that sort the keys ascending, ties kept in index order (stable)."""
    return np.argsort(keys, kind="stable")


def cell_start(sorted_cells: np.ndarray, n_cells: int) -> np.ndarray:
    """cell_start[c] = first sorted position of cell c; cell_start[n_cells] = N."""
    return np.searchsorted(sorted_cells, np.arange(n_cells + 1), side="left").astype(np.int64)


# --------------------------------------------------------------------------- 3. CIC assign


def cic_weights(pos: np.ndarray, p: Params):
    """CIC stencil of each particle: base node i0_d = floor(x_d M/L) and fraction f_d, so that
    the particle gives weight (1-f_d) to node i0_d and f_d to node i0_d + 1 (periodic)."""
    u = pos * (p.mesh / p.box)
    i0 = np.floor(u)
    f = u - i0
    return i0.astype(np.int64) % p.mesh, f


def cic_deposit(pos: np.ndarray, p: Params) -> np.ndarray:
    """Mesh of particle counts n(node) = sum_i prod_d w_d (CIC), shape (M, M, M), z fastest."""
    M = p.mesh
    i0, f = cic_weights(pos, p)
    rho = np.zeros(M ** 3)
    for cx in (0, 1):
        wx = f[0] if cx else 1.0 - f[0]
        ix = (i0[0] + cx) % M
        for cy in (0, 1):
            wy = f[1] if cy else 1.0 - f[1]
            iy = (i0[1] + cy) % M
            for cz in (0, 1):
                wz = f[2] if cz else 1.0 - f[2]
                iz = (i0[2] + cz) % M
                rho += np.bincount((ix * M + iy) * M + iz, weights=wx * wy * wz, minlength=M ** 3)
    return rho.reshape(M, M, M)


def cic_gather(mesh: np.ndarray, pos: np.ndarray, p: Params) -> np.ndarray:
    """Interpolates a (M, M, M) mesh field to the particles with the CIC weights."""
    M = p.mesh
    i0, f = cic_weights(pos, p)
    flat = mesh.ravel()
    out = np.zeros(pos.shape[1])
    for cx in (0, 1):
        wx = f[0] if cx else 1.0 - f[0]
        ix = (i0[0] + cx) % M
        for cy in (0, 1):
            wy = f[1] if cy else 1.0 - f[1]
            iy = (i0[1] + cy) % M
            for cz in (0, 1):
                wz = f[2] if cz else 1.0 - f[2]
                iz = (i0[2] + cz) % M
                out += wx * wy * wz * flat[(ix * M + iy) * M + iz]
    return out


# --------------------------------------------------------------------------- 4-6. k space


def wavenumbers(p: Params):
    """k of the rfft grid along x, y (full) and z (half), Nyquist entries at -pi/h / +pi/h."""
    M = p.mesh
    k1 = 2.0 * np.pi * np.fft.fftfreq(M, d=p.h)
    kz = 2.0 * np.pi * np.fft.rfftfreq(M, d=p.h)
    return k1, k1, kz


def green(p: Params) -> np.ndarray:
    """Long-range Green's function on the rfft grid, acting on the count mesh:
    G(k) = -4 pi (Gm / h^3) exp(-k^2 r_s^2) / k^2 [/ W(k)^2],  G(0) = 0,
    W(k) = prod_d sinc^2(k_d h / 2) (CIC assignment window, sinc(0) = 1).
    Pure PM (no short-range part, the guide's 'PM' kick algorithm) has no Gaussian filter."""
    kx, ky, kz = wavenumbers(p)
    KX, KY, KZ = np.meshgrid(kx, ky, kz, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    rs2 = p.r_s ** 2 if p.short_range else 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(k2 > 0, -4.0 * np.pi * (p.gm / p.h ** 3) * np.exp(-k2 * rs2)
                     / np.where(k2 > 0, k2, 1.0), 0.0)
    if p.deconvolve:
        def sinc(k):
            x = 0.5 * k * p.h
            return np.where(x == 0.0, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))
        w = (sinc(KX) * sinc(KY) * sinc(KZ)) ** 2
        g = g / (w * w)
    return g


def gradient_wavenumbers(p: Params):
    """Spectral-gradient wavenumbers: k_d with the Nyquist entry of each axis set to 0."""
    M = p.mesh
    kx, ky, kz = (k.copy() for k in wavenumbers(p))
    if M % 2 == 0:
        kx[M // 2] = 0.0
        ky[M // 2] = 0.0
        kz[M // 2] = 0.0
    return kx, ky, kz


def pm_force_meshes(pos: np.ndarray, p: Params):
    """Steps 3-6: CIC counts -> rfftn -> G(k) -> -i k_d -> irfftn: the three mesh
    accelerations a_d(node) (numpy's irfftn carries the 1/M^3)."""
    M = p.mesh
    rho = cic_deposit(pos, p)
    rk = np.fft.rfftn(rho)
    phik = green(p) * rk
    gx, gy, gz = gradient_wavenumbers(p)
    GX, GY, GZ = np.meshgrid(gx, gy, gz, indexing="ij")
    return [np.fft.irfftn(-1j * K * phik, s=(M, M, M), axes=(0, 1, 2)) for K in (GX, GY, GZ)], rho


def pm_accel(pos: np.ndarray, p: Params, targets=None) -> np.ndarray:
    """Long-range (PM) accelerations (3, N) at wrapped positions; steps 3-7."""
    meshes, _ = pm_force_meshes(pos, p)
    tp = pos if targets is None else pos[:, targets]
    return np.stack([cic_gather(m, tp, p) for m in meshes])


# --------------------------------------------------------------------------- 8. short range

_lib = None


def _clib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.sr_accel_cells.argtypes = [ctypes.c_int64, dp, ctypes.c_double, ctypes.c_int64,
                                        i64p, i64p, i64p, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, i64p, ctypes.c_int64,
                                        dp, i64p]
        _lib.sr_accel_brute.argtypes = [ctypes.c_int64, dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        i64p, ctypes.c_int64, dp, i64p]
        _lib.oracle_threads.restype = ctypes.c_int
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def oracle_threads() -> int:
    return int(_clib().oracle_threads())


def sr_accel(pos: np.ndarray, p: Params, targets=None, brute: bool = False):
    """Short-range accelerations (3, N or len(targets)) and the number of (target, j) pairs
    inside the cutoff.  Chaining cells from steps 1-2 (sub_bits ignored: cells only), or all
    pairs when ``brute``."""
    lib = _clib()
    x = np.ascontiguousarray(pos, dtype=np.float64)
    n = x.shape[1]
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.size
    acc = np.zeros((3, nt))
    npairs = ctypes.c_int64(0)
    tptr = None if tg is None else _p(tg, ctypes.c_int64)
    if brute:
        if p.r_c >= 0.5 * p.box:
            raise ValueError("minimum-image pair sum needs r_c < box/2")
        lib.sr_accel_brute(n, _p(x, ctypes.c_double), p.box, p.r_s, p.r_c, p.eps, p.gm,
                           tptr, nt, _p(acc, ctypes.c_double), ctypes.byref(npairs))
    else:
        q = Params(p.box, p.n, p.mesh, p.r_s_cells, p.cutoff, p.softening, p.deconvolve, 0,
                   True, p.omega_m, p.omega_lambda)
        cell, _ = cell_keys(x, q)
        order = stable_order(cell).astype(np.int64)
        starts = cell_start(cell[order], q.n_c ** 3)
        cell = np.ascontiguousarray(cell, dtype=np.int64)
        lib.sr_accel_cells(n, _p(x, ctypes.c_double), p.box, q.n_c, _p(cell, ctypes.c_int64),
                           _p(order, ctypes.c_int64), _p(starts, ctypes.c_int64), p.r_s, p.r_c,
                           p.eps, p.gm, tptr, nt, _p(acc, ctypes.c_double), ctypes.byref(npairs))
    return acc, int(npairs.value)


def accel(pos: np.ndarray, p: Params, targets=None) -> np.ndarray:
    """Total P3M acceleration (PM + short range, or PM alone), at wrapped positions."""
    x = wrap(pos, p.box)
    a = pm_accel(x, p, targets)
    if p.short_range:
        a = a + sr_accel(x, p, targets)[0]
    return a


# --------------------------------------------------------------------------- 9. integration


def hubble(a, p: Params):
    """H(a)/H0 for matter, curvature 1 - Omega_m - Omega_Lambda and a cosmological constant."""
    ok = 1.0 - p.omega_m - p.omega_lambda
    return np.sqrt(p.omega_m / a ** 3 + ok / a ** 2 + p.omega_lambda)


def _is_eds(p: Params) -> bool:
    return p.omega_m == 1.0 and p.omega_lambda == 0.0


def kick_factor(a1: float, a2: float, p: Params) -> float:
    """int_{t1}^{t2} dt/a = int_{a1}^{a2} da / (a^2 H(a)); EdS closed form 2(sqrt a2 - sqrt a1)."""
    if _is_eds(p):
        return 2.0 * (math.sqrt(a2) - math.sqrt(a1))
    xg, wg = np.polynomial.legendre.leggauss(48)
    a = 0.5 * (a2 - a1) * xg + 0.5 * (a2 + a1)
    return float(0.5 * (a2 - a1) * np.sum(wg / (a * a * hubble(a, p))))


def drift_factor(a1: float, a2: float, p: Params) -> float:
    """int_{t1}^{t2} dt/a^2 = int da / (a^3 H(a)); EdS closed form 2(a1^-1/2 - a2^-1/2)."""
    if _is_eds(p):
        return 2.0 * (1.0 / math.sqrt(a1) - 1.0 / math.sqrt(a2))
    xg, wg = np.polynomial.legendre.leggauss(48)
    a = 0.5 * (a2 - a1) * xg + 0.5 * (a2 + a1)
    return float(0.5 * (a2 - a1) * np.sum(wg / (a ** 3 * hubble(a, p))))


def step(pos, mom, acc, a: float, da: float, p: Params, mass: float = 1.0):
    """One kick-drift-kick step a -> a + da.  ``acc`` is the acceleration at ``pos`` (from
    the previous step or from ``accel``).  Returns (pos, mom, acc) at a + da."""
    am = a + 0.5 * da
    mom = mom + mass * acc * kick_factor(a, am, p)
    pos = wrap(pos + (mom / mass) * drift_factor(a, a + da, p), p.box)
    acc = accel(pos, p)
    mom = mom + mass * acc * kick_factor(am, a + da, p)
    return pos, mom, acc


# --------------------------------------------------------------------------- checks


def g_split(x):
    """Short-range force factor g(x) = erfc(x/2) + x/sqrt(pi) exp(-x^2/4), x = r/r_s:
    the fraction of the Newtonian pair force the short-range part carries."""
    x = np.asarray(x, dtype=np.float64)
    return erfc(0.5 * x) + x / math.sqrt(math.pi) * np.exp(-0.25 * x * x)


def lr_accel_exact(pos: np.ndarray, p: Params, kmax: int = 12, targets=None) -> np.ndarray:
    """Long-range accelerations without a mesh: the periodic sum over wave vectors
    k = 2 pi n / L, 0 < |n_d| <= kmax, of the Gaussian-filtered Newtonian kernel,
    a_i = -(4 pi Gm / L^3) sum_k k exp(-k^2 r_s^2)/k^2 sum_j sin(k . (x_i - x_j))."""
    L = p.box
    n = np.arange(-kmax, kmax + 1)
    NX, NY, NZ = np.meshgrid(n, n, n, indexing="ij")
    kv = (2.0 * np.pi / L) * np.stack([NX.ravel(), NY.ravel(), NZ.ravel()]).astype(np.float64)
    k2 = np.sum(kv * kv, axis=0)
    keep = k2 > 0
    kv, k2 = kv[:, keep], k2[keep]
    filt = np.exp(-k2 * p.r_s ** 2) / k2
    keep = filt > 1e-30 * filt.max()
    kv, filt = kv[:, keep], filt[keep]
    tp = pos if targets is None else pos[:, targets]
    # S(k) = sum_j exp(-i k.x_j);  sum_j sin(k.(x_i - x_j)) = Im(exp(i k.x_i) S(k))
    s = np.exp(-1j * (kv.T @ pos)).sum(axis=1)
    ph = np.exp(1j * (tp.T @ kv))
    im = (ph * s[None, :]).imag
    return -(4.0 * np.pi * p.gm / L ** 3) * (kv @ (filt[:, None] * im.T))


def ewald_accel(pos: np.ndarray, box: float, gm: float, alpha: float | None = None,
                nreal: int = 2, kmax: int = 6, targets=None) -> np.ndarray:
    """Brute-force periodic Ewald accelerations (infinite periodic lattice of images with a
    uniform neutralising background), for N <= 512:
      real part   Gm sum_j sum_n (d + nL) [erfc(alpha s) + 2 alpha s/sqrt(pi) e^{-alpha^2 s^2}] / s^3,
                  s = |d + nL|, d = minimum image of x_j - x_i, |n_d| <= nreal (the n = 0,
                  j = i term omitted)
      k part      -(4 pi Gm / L^3) sum_{k != 0} k e^{-k^2/(4 alpha^2)}/k^2 sum_j sin(k.(x_i - x_j)).
    The default alpha = 2.6/L with nreal = 2 and kmax = 6 leaves out real-space images at
    s >= 2.5 L (erfc(6.5) ~ 4e-20) and wave vectors with k^2/(4 alpha^2) >= 52 (e^-52 ~ 3e-23)."""
    L = box
    if alpha is None:
        alpha = 2.6 / L
    tp = pos if targets is None else pos[:, targets]
    ti = np.arange(pos.shape[1]) if targets is None else np.asarray(targets)
    acc = np.zeros(tp.shape)
    d0 = pos[:, None, :] - tp[:, :, None]          # (3, nt, N)  x_j - x_i
    d0 = d0 - L * np.round(d0 / L)
    self_mask = ti[:, None] == np.arange(pos.shape[1])[None, :]
    rng = range(-nreal, nreal + 1)
    for nx in rng:
        for ny in rng:
            for nz in rng:
                sh = np.array([nx, ny, nz], dtype=np.float64)[:, None, None] * L
                d = d0 + sh
                s2 = np.sum(d * d, axis=0)
                if nx == 0 and ny == 0 and nz == 0:
                    s2 = np.where(self_mask, 1.0, s2)
                s = np.sqrt(s2)
                f = (erfc(alpha * s) + 2.0 * alpha * s / math.sqrt(math.pi)
                     * np.exp(-alpha * alpha * s2)) / (s2 * s)
                if nx == 0 and ny == 0 and nz == 0:
                    f = np.where(self_mask, 0.0, f)
                acc += gm * np.sum(d * f[None], axis=2)
    n = np.arange(-kmax, kmax + 1)
    NX, NY, NZ = np.meshgrid(n, n, n, indexing="ij")
    kv = (2.0 * np.pi / L) * np.stack([NX.ravel(), NY.ravel(), NZ.ravel()]).astype(np.float64)
    k2 = np.sum(kv * kv, axis=0)
    keep = k2 > 0
    kv, k2 = kv[:, keep], k2[keep]
    filt = np.exp(-k2 / (4.0 * alpha * alpha)) / k2
    s = np.exp(-1j * (kv.T @ pos)).sum(axis=1)
    im = (np.exp(1j * (tp.T @ kv)) * s[None, :]).imag
    acc += -(4.0 * np.pi * gm / L ** 3) * (kv @ (filt[:, None] * im.T))
    return acc


def momentum(mom: np.ndarray) -> np.ndarray:
    """Total momentum sum_i p_i (3,)."""
    return mom.sum(axis=1)


def kinetic_energy(mom: np.ndarray, a: float, mass: float = 1.0) -> float:
    """Peculiar kinetic energy sum_i |p_i|^2 / (2 m a^2)."""
    return float(np.sum(mom * mom) / (2.0 * mass * a * a))


# --------------------------------------------------------------------------- power spectrum
# Ch. Parameters: PM_gridsize is also the grid of the power spectrum, and R_tophat the radius
# of the top-hat sphere for sigma (the rms density variation) computed from the power spectrum.
# Readings: delta = n/n_bar - 1 on the CIC count mesh; delta_k = DFT(delta)/M^3;
# P(k) = L^3 <|delta_k|^2 / W(k)^2> over a shell (the deconvolution optional, no shot-noise
# subtraction); shell b holds the modes with round(|k|/k_f) = b + 1, k_f = 2 pi / L, up to
# b + 1 = M/2; sigma_R^2 = sum over all k != 0 of |delta_k|^2 / W(k)^2 * W_TH(k R)^2 with
# W_TH(x) = 3 (sin x - x cos x) / x^3.


def tophat_window(x):
    """Fourier transform of the unit top-hat sphere, 3 (sin x - x cos x) / x^3, W(0) = 1."""
    x = np.asarray(x, dtype=np.float64)
    small = np.abs(x) < 1e-3
    xs = np.where(small, 1.0, x)
    w = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    return np.where(small, 1.0 - x * x / 10.0, w)


def power_from_mesh(delta: np.ndarray, box: float, deconvolve: bool = True, radius: float = 0.0):
    """Binned power spectrum of a density-contrast mesh (M, M, M): returns (k_mean, P, n_modes,
    sigma_R) with the full complex transform (every mode counted once)."""
    M = delta.shape[0]
    dk = np.fft.fftn(delta) / M ** 3
    k1 = 2.0 * np.pi * np.fft.fftfreq(M, d=box / M)
    KX, KY, KZ = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(KX * KX + KY * KY + KZ * KZ)
    p2 = np.abs(dk) ** 2
    if deconvolve:
        h = box / M

        def sinc(k):
            x = 0.5 * k * h
            return np.where(x == 0.0, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))
        p2 = p2 / (sinc(KX) * sinc(KY) * sinc(KZ)) ** 4
    kf = 2.0 * np.pi / box
    shell = np.floor(kk / kf + 0.5).astype(np.int64) - 1
    nb = M // 2
    sel = (shell >= 0) & (shell < nb)
    cnt = np.bincount(shell[sel], minlength=nb).astype(np.float64)
    psum = np.bincount(shell[sel], weights=p2[sel], minlength=nb)
    ksum = np.bincount(shell[sel], weights=kk[sel], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        kmean = ksum / cnt
        power = box ** 3 * psum / cnt
    sigma = None
    if radius > 0.0:
        nz = kk > 0
        sigma = float(np.sqrt(np.sum(p2[nz] * tophat_window(kk[nz] * radius) ** 2)))
    return kmean, power, cnt, sigma


def power_spectrum(pos: np.ndarray, p: Params, deconvolve: bool = True, radius: float = 0.0):
    """Power spectrum of a particle set: CIC counts -> delta = n / n_bar - 1 -> power_from_mesh."""
    n = cic_deposit(wrap(pos, p.box), p)
    nbar = pos.shape[1] / p.mesh ** 3
    return power_from_mesh(n / nbar - 1.0, p.box, deconvolve, radius)


def cic_shot_noise(k_vec_index, p: Params, n_particles: int, deconvolve: bool = True):
    """Expected power of a Poisson particle set after CIC assignment (Jing 2005, ApJ 620, 559):
    P_shot(k) = (L^3/N) prod_d [1 - (2/3) sin^2(k_d h / 2)], divided by W(k)^2 when
    deconvolved.  k_vec_index: integer mode vectors (3, m)."""
    h = p.h
    k = (2.0 * np.pi / p.box) * np.asarray(k_vec_index, dtype=np.float64)
    s2 = np.sin(0.5 * k * h) ** 2
    ps = (p.box ** 3 / n_particles) * np.prod(1.0 - (2.0 / 3.0) * s2, axis=0)
    if deconvolve:
        x = 0.5 * k * h
        sinc = np.where(x == 0.0, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))
        ps = ps / np.prod(sinc, axis=0) ** 4
    return ps


# --------------------------------------------------------------------------- adjoint
# Reverse-mode derivatives of the step, for gradients of a final-density loss with respect
# to the initial displacement field.  The derivative of a force evaluation is needed as its
# transpose applied to a vector field v ("VJP"): out = (dA/dx)^T v, A the accelerations.


def cic_grad_weights(pos: np.ndarray, p: Params):
    """CIC stencil with the weights and their position derivatives: for each of the 8 corners
    (cx, cy, cz) the node index (N,), weight (N,) and d weight / d x (3, N)."""
    M = p.mesh
    i0, f = cic_weights(pos, p)
    inv_h = p.mesh / p.box
    out = []
    for cx in (0, 1):
        for cy in (0, 1):
            for cz in (0, 1):
                w1 = [f[0] if cx else 1.0 - f[0], f[1] if cy else 1.0 - f[1],
                      f[2] if cz else 1.0 - f[2]]
                dw1 = [(inv_h if c else -inv_h) * np.ones_like(f[0]) for c in (cx, cy, cz)]
                node = (((i0[0] + cx) % M) * M + (i0[1] + cy) % M) * M + (i0[2] + cz) % M
                w = w1[0] * w1[1] * w1[2]
                dw = np.stack([dw1[0] * w1[1] * w1[2], w1[0] * dw1[1] * w1[2],
                               w1[0] * w1[1] * dw1[2]])
                out.append((node, w, dw))
    return out


def pm_vjp(pos: np.ndarray, v: np.ndarray, p: Params) -> np.ndarray:
    """(d a_LR / d x)^T v.  a_LR,i = sum_n W(x_i - n) E(n), E_b = D_b rho, rho(n) = sum_j W(x_j - n)
    with D_b = IFFT(-i k_b G(k) FFT(.)) (real, and D_b^T = -D_b):
      out_k = sum_b v_k,b sum_n grad W(x_k - n) E_b(n)          (interpolation weights)
            + sum_n grad W(x_k - n) psi(n),  psi = -sum_b D_b u_b,  u_b(n) = sum_i W(x_i - n) v_i,b
    (the second term through the deposit)."""
    M = p.mesh
    meshes, _ = pm_force_meshes(pos, p)
    stencil = cic_grad_weights(pos, p)
    u = []
    for b in range(3):
        ub = np.zeros(M ** 3)
        for node, w, dw in stencil:
            ub += np.bincount(node, weights=w * v[b], minlength=M ** 3)
        u.append(ub.reshape(M, M, M))
    gk = green(p)
    gx, gy, gz = gradient_wavenumbers(p)
    GX, GY, GZ = np.meshgrid(gx, gy, gz, indexing="ij")
    psik = sum(1j * K * gk * np.fft.rfftn(ub) for K, ub in zip((GX, GY, GZ), u))
    psi = np.fft.irfftn(psik, s=(M, M, M), axes=(0, 1, 2)).ravel()
    out = np.zeros_like(pos)
    flat = [m.ravel() for m in meshes]
    for node, w, dw in stencil:
        ev = sum(v[b] * flat[b][node] for b in range(3))
        out += dw * (ev + psi[node])[None, :]
    return out


def sr_vjp(pos: np.ndarray, v: np.ndarray, p: Params) -> np.ndarray:
    """(d a_SR / d x)^T v by the plain C pair loop over chaining cells (sr_pairs.c)."""
    lib = _clib()
    if not hasattr(lib, "_vjp_set"):
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.sr_vjp_cells.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_int64,
                                     i64p, i64p, i64p, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, dp]
        lib._vjp_set = True
    x = np.ascontiguousarray(pos, dtype=np.float64)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    n = x.shape[1]
    q = Params(p.box, p.n, p.mesh, p.r_s_cells, p.cutoff, p.softening, p.deconvolve, 0, True,
               p.omega_m, p.omega_lambda)
    cell, _ = cell_keys(x, q)
    order = stable_order(cell).astype(np.int64)
    starts = cell_start(cell[order], q.n_c ** 3)
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    out = np.zeros((3, n))
    lib.sr_vjp_cells(n, _p(x, ctypes.c_double), _p(vv, ctypes.c_double), p.box, q.n_c,
                     _p(cell, ctypes.c_int64), _p(order, ctypes.c_int64),
                     _p(starts, ctypes.c_int64), p.r_s, p.r_c, p.eps, p.gm,
                     _p(out, ctypes.c_double))
    return out


def accel_vjp(pos: np.ndarray, v: np.ndarray, p: Params) -> np.ndarray:
    """(d a / d x)^T v of the total acceleration at wrapped positions."""
    x = wrap(pos, p.box)
    out = pm_vjp(x, v, p)
    if p.short_range:
        out = out + sr_vjp(x, v, p)
    return out


def density_loss(pos: np.ndarray, target: np.ndarray, p: Params):
    """L = sum_n (delta(n) - target(n))^2, delta = n(n)/n_bar - 1 on the CIC mesh, and dL/dx."""
    x = wrap(pos, p.box)
    nbar = pos.shape[1] / p.mesh ** 3
    delta = (cic_deposit(x, p) / nbar - 1.0).ravel()
    r = delta - target.ravel()
    grad = np.zeros_like(x)
    for node, w, dw in cic_grad_weights(x, p):
        grad += dw * (2.0 * r[node] / nbar)[None, :]
    return float(np.sum(r * r)), grad


def zeldovich_state(psi: np.ndarray, q: np.ndarray, a: float, p: Params, mass: float = 1.0):
    """Initial state of a displacement field psi (3, N) on the lattice q: x = q + psi,
    p = m a^(1/2) psi (Einstein-de Sitter linear growth, H0 = 1)."""
    return wrap(q + psi, p.box), mass * math.sqrt(a) * psi


def run_and_loss(psi, q, a_list, target, p: Params, mass: float = 1.0):
    """Forward: Zel'dovich state at a_list[0], KDK steps through a_list, density loss."""
    x, m = zeldovich_state(psi, q, a_list[0], p, mass)
    acc = accel(x, p)
    for k in range(len(a_list) - 1):
        x, m, acc = step(x, m, acc, a_list[k], a_list[k + 1] - a_list[k], p, mass)
    return density_loss(x, target, p)[0]


def run_gradient(psi, q, a_list, target, p: Params, mass: float = 1.0):
    """dL/dpsi by the reverse sweep over stored states (no checkpointing: the oracle keeps all
    states).  Step k maps (x_k, p_k) -> (x_{k+1}, p_{k+1}) with kick factors m K1_k, m K2_k and
    drift factor D_k / m; reverse, with K1_n = 0:
        lam_x += m (K2_k + K1_{k+1}) VJP(x_{k+1}, lam_p);  lam_p += (D_k / m) lam_x
    then lam_x += m K1_0 VJP(x_0, lam_p); dL/dpsi = lam_x + m a_0^(1/2) lam_p."""
    n = len(a_list) - 1
    x, m = zeldovich_state(psi, q, a_list[0], p, mass)
    xs = [x]
    acc = accel(x, p)
    for k in range(n):
        x, m, acc = step(x, m, acc, a_list[k], a_list[k + 1] - a_list[k], p, mass)
        xs.append(x)
    loss, lam_x = density_loss(xs[-1], target, p)
    lam_p = np.zeros_like(lam_x)
    K1 = [kick_factor(a_list[k], a_list[k] + 0.5 * (a_list[k + 1] - a_list[k]), p) for k in range(n)]
    K2 = [kick_factor(a_list[k] + 0.5 * (a_list[k + 1] - a_list[k]), a_list[k + 1], p) for k in range(n)]
    D = [drift_factor(a_list[k], a_list[k + 1], p) for k in range(n)]
    for k in range(n - 1, -1, -1):
        kf = mass * (K2[k] + (K1[k + 1] if k + 1 < n else 0.0))
        lam_x = lam_x + kf * accel_vjp(xs[k + 1], lam_p, p)
        lam_p = lam_p + (D[k] / mass) * lam_x
    lam_x = lam_x + mass * K1[0] * accel_vjp(xs[0], lam_p, p)
    return loss, lam_x + mass * math.sqrt(a_list[0]) * lam_p


# --------------------------------------------------------------------------- energies
# Readings (the guide defines no energy diagnostic; this is the standard cosmic-energy check):
#   comoving potential Phi with nabla^2 Phi = 4 pi G (rho - rho_bar), acceleration -grad Phi;
#   peculiar potential energy W = (1/(2a)) sum_i m Phi(x_i) (self-interaction at r = 0
#   excluded), kinetic energy K = sum_i |p_i|^2 / (2 m a^2);
#   Layzer-Irvine (cosmic energy) equation d[a (K + W)]/da = -K.
# P3M potential of particle i:
#   Phi_i = Phi_LR(x_i) - S_i + (phi_per - phi_iso) + phi_SR,i + 4 pi Gm (N/L^3) r_s^2
#   Phi_LR   the mesh potential IFFT(G(k) FFT(rho)) interpolated by CIC;
#   S_i      the particle's own share of it, sum_{c,c'} w_c w_c' K(n_c - n_c'), K = IFFT(G)
#            (its CIC weights deposited, solved and interpolated back);
#   phi_per  what that share is without a mesh: the periodic long-range potential of a unit
#            particle at its own position, -(4 pi Gm/L^3) sum_{k != 0} exp(-k^2 r_s^2)/k^2;
#   phi_iso  the r = 0 limit of the isolated long-range kernel -Gm erf(r/(2 r_s))/r,
#            -Gm/(sqrt(pi) r_s): the self-interaction, excluded (the interaction with the
#            particle's own periodic images, phi_per - phi_iso, is kept);
#   phi_SR   the pair sum of -Gm erfc(r/(2 r_s)) / sqrt(r^2 + eps^2);
#   the last term: the short-range potential of the neutralising background (density
#            -N m/L^3, and erfc(r/(2 r_s))/r integrates to 4 pi r_s^2 over space).
# With the split at alpha = 1/(2 r_s) this is the Ewald energy term by term for one particle.


def mesh_self_potential(pos: np.ndarray, p: Params) -> np.ndarray:
    """S_i = sum over the 8 x 8 corner pairs of the particle's CIC stencil of
    w_c w_c' K(n_c - n_c'), K = IFFT(G): the particle's own contribution to the mesh potential
    at its position."""
    M = p.mesh
    K = np.fft.irfftn(green(p), s=(M, M, M), axes=(0, 1, 2))
    i0, f = cic_weights(pos, p)
    corners = [(cx, cy, cz) for cx in (0, 1) for cy in (0, 1) for cz in (0, 1)]
    w = {}
    for c in corners:
        w[c] = ((f[0] if c[0] else 1 - f[0]) * (f[1] if c[1] else 1 - f[1])
                * (f[2] if c[2] else 1 - f[2]))
    s = np.zeros(pos.shape[1])
    for c in corners:
        for d in corners:
            s += w[c] * w[d] * K[(c[0] - d[0]) % M, (c[1] - d[1]) % M, (c[2] - d[2]) % M]
    return s


def potential(pos: np.ndarray, p: Params) -> np.ndarray:
    """Comoving potential Phi at each particle (its own contribution removed)."""
    M = p.mesh
    x = wrap(pos, p.box)
    rho = cic_deposit(x, p)
    phi_mesh = np.fft.irfftn(green(p) * np.fft.rfftn(rho), s=(M, M, M), axes=(0, 1, 2))
    phi = cic_gather(phi_mesh, x, p) - mesh_self_potential(x, p)
    if not p.short_range:
        return phi
    kf = 2.0 * math.pi / p.box
    nmax = int(math.ceil(6.5 / (p.r_s * kf)))
    nn = np.arange(-nmax, nmax + 1)
    NX, NY, NZ = np.meshgrid(nn, nn, nn, indexing="ij")
    k2 = kf * kf * (NX * NX + NY * NY + NZ * NZ).astype(np.float64).ravel()
    k2 = k2[k2 > 0]
    phi_per = -(4.0 * math.pi * p.gm / p.box ** 3) * float(np.sum(np.exp(-k2 * p.r_s ** 2) / k2))
    phi_iso = -p.gm / (math.sqrt(math.pi) * p.r_s)
    phi = phi + (phi_per - phi_iso)
    lib = _clib()
    if not hasattr(lib, "_pot_set"):
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.sr_potential_cells.argtypes = [ctypes.c_int64, dp, ctypes.c_double, ctypes.c_int64,
                                           i64p, i64p, i64p, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, dp]
        lib._pot_set = True
    xx = np.ascontiguousarray(x)
    q = Params(p.box, p.n, p.mesh, p.r_s_cells, p.cutoff, p.softening, p.deconvolve, 0, True,
               p.omega_m, p.omega_lambda)
    cell, _ = cell_keys(xx, q)
    order = stable_order(cell).astype(np.int64)
    starts = cell_start(cell[order], q.n_c ** 3)
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    sr = np.zeros(x.shape[1])
    lib.sr_potential_cells(x.shape[1], _p(xx, ctypes.c_double), p.box, q.n_c,
                           _p(cell, ctypes.c_int64), _p(order, ctypes.c_int64),
                           _p(starts, ctypes.c_int64), p.r_s, p.r_c, p.eps, p.gm,
                           _p(sr, ctypes.c_double))
    background = 4.0 * math.pi * p.gm * (x.shape[1] / p.box ** 3) * p.r_s ** 2
    return phi + sr + background


def potential_energy(pos: np.ndarray, p: Params, a: float, mass: float = 1.0) -> float:
    """W = (1/(2a)) sum_i m Phi(x_i)."""
    return float(0.5 * mass * np.sum(potential(pos, p)) / a)


def ewald_potential_energy(pos: np.ndarray, box: float, gm: float, alpha: float | None = None,
                           nreal: int = 2, kmax: int = 6) -> float:
    """Comoving Ewald energy (1/2) m sum_i [sum_{j != i} phi_E(x_i - x_j) + phi_self] of a
    periodic set with a neutralising background, phi_E = -Gm [sum_n erfc(alpha s)/s
    + (4 pi/L^3) sum_{k != 0} e^{-k^2/(4 alpha^2)} cos(k.r)/k^2 - pi/(alpha^2 L^3)], the self
    term taking the images n != 0 and subtracting the r -> 0 limit 2 alpha / sqrt(pi)
    (returned for m = 1 in units where Gm carries the mass)."""
    L = box
    if alpha is None:
        alpha = 2.6 / L
    n_ = pos.shape[1]
    d0 = pos[:, None, :] - pos[:, :, None]
    d0 = d0 - L * np.round(d0 / L)
    offd = ~np.eye(n_, dtype=bool)
    real = 0.0
    rng = range(-nreal, nreal + 1)
    for nx in rng:
        for ny in rng:
            for nz in rng:
                sh = np.array([nx, ny, nz], dtype=np.float64)[:, None, None] * L
                s = np.sqrt(np.sum((d0 + sh) ** 2, axis=0))
                if nx == 0 and ny == 0 and nz == 0:
                    real += np.sum(erfc(alpha * s[offd]) / s[offd])
                else:
                    real += np.sum(erfc(alpha * s) / s)  # includes i = j images
    nn = np.arange(-kmax, kmax + 1)
    NX, NY, NZ = np.meshgrid(nn, nn, nn, indexing="ij")
    kv = (2.0 * np.pi / L) * np.stack([NX.ravel(), NY.ravel(), NZ.ravel()]).astype(np.float64)
    k2 = np.sum(kv * kv, axis=0)
    keep = k2 > 0
    kv, k2 = kv[:, keep], k2[keep]
    sk = np.exp(1j * (kv.T @ pos)).sum(axis=1)
    recip = (4.0 * np.pi / L ** 3) * np.sum(np.exp(-k2 / (4 * alpha ** 2)) / k2 * np.abs(sk) ** 2)
    background = -np.pi / (alpha ** 2 * L ** 3) * n_ * n_
    self_term = -2.0 * alpha / math.sqrt(math.pi) * n_
    return float(-0.5 * gm * (real + recip + background + self_term))
