"""Seeded synthetic particle sets shared by the oracle tests, the GPU tests and the benchmark.

This module only draws random numbers and lays out particle sets.  It holds none of the
P3M arithmetic: no mass assignment, no Green's function, no force and no time integration.
Both the FP64 oracle (``oracle/``) and the CUDA path consume its arrays as plain inputs.

Conventions
-----------
* Positions and momenta are float64 arrays of shape ``(3, N)`` (structure of arrays), in
  comoving length units (Mpc/h) and comoving momenta ``m a^2 dx/dt`` with time in units of
  ``1/H0`` (Ch. Snapshot Formats, the standard snapshot layout: posx..posz, momx..momz).
* Lattice particle ``k = (ix*n + iy)*n + iz`` sits at ``q = (ix, iy, iz) * box/n``.
* Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014) used as a counter-based generator, output ``k`` being the
  finaliser applied to ``seed + (k+1)*0x9E3779B97F4A7C15``; Gaussians by Box-Muller.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64",
    "uniform01",
    "gaussian",
    "lattice",
    "uniform_random",
    "zeldovich",
    "clustered",
    "plane_wave",
    "log_spaced_steps",
    "CONFIGS",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the SplitMix64 stream started at ``seed``."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in (0, 1]: the top 53 bits of each SplitMix64 output, plus one ulp."""
    top = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64)
    return (top + 1.0) * (2.0 ** -53)


def gaussian(seed: int, n: int) -> np.ndarray:
    """Standard normal deviates by the Box-Muller transform of two uniform streams."""
    u1 = uniform01(seed, n, 0)
    u2 = uniform01(seed, n, n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def lattice(n: int, box: float) -> np.ndarray:
    """Simple-cubic lattice of n^3 points at integer multiples of box/n, shape (3, n^3)."""
    i = np.arange(n, dtype=np.float64) * (box / n)
    qx, qy, qz = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([qx.ravel(), qy.ravel(), qz.ravel()])


def uniform_random(n: int, box: float, seed: int) -> np.ndarray:
    """n points uniformly distributed in [0, box)^3, shape (3, n)."""
    u = uniform01(seed, 3 * n) - 2.0 ** -53  # [0, 1)
    return (u * box).reshape(3, n)


def _wavenumbers(n: int, box: float):
    k1 = 2.0 * np.pi * np.fft.fftfreq(n, d=box / n)
    kz = 2.0 * np.pi * np.fft.rfftfreq(n, d=box / n)
    kx, ky, kzz = np.meshgrid(k1, k1, kz, indexing="ij")
    return kx, ky, kzz


def zeldovich(n_p: int, box: float, a_begin: float, seed: int, rms_cells: float = 0.2,
              kc_frac: float = 0.5, mass: float = 1.0, growth: float = 1.0):
    """Zel'dovich initial conditions on an n_p^3 lattice in an Einstein-de Sitter background.

    Recipe: white noise on the lattice -> Fourier space -> multiply by sqrt(P(k)) with
    P(k) = k^-2 exp(-(k/k_c)^2), k_c = kc_frac * k_Nyquist, k = 0 removed -> displacement
    psi_k = i k delta_k / k^2 with each component zeroed on its own Nyquist plane -> real
    space -> scaled so that the rms of |psi| is ``rms_cells`` lattice spacings at ``a_begin``.
    Positions x = q + growth*psi, momenta p = m a^(1/2) psi (linear growth D = a, H0 = 1,
    p = m a^2 dx/dt).  ``growth`` > 1 extrapolates the displacement beyond the linear
    regime (used for clustered test snapshots); momenta are left at the linear value.
    Returns (pos, mom) as float64 arrays of shape (3, N), positions wrapped into [0, box).
    """
    n = n_p
    white = gaussian(seed, n ** 3).reshape(n, n, n)
    dk = np.fft.rfftn(white)
    kx, ky, kz = _wavenumbers(n, box)
    k2 = kx * kx + ky * ky + kz * kz
    kc = kc_frac * np.pi * n / box
    with np.errstate(divide="ignore", invalid="ignore"):
        pk = np.where(k2 > 0, np.exp(-k2 / (kc * kc)) / np.sqrt(np.where(k2 > 0, k2, 1.0)), 0.0)
        dk = dk * np.sqrt(pk)
        inv_k2 = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    nyq = np.pi * n / box
    psi = []
    for kd in (kx, ky, kz):
        kd_g = np.where(np.isclose(np.abs(kd), nyq), 0.0, kd)
        psi.append(np.fft.irfftn(1j * kd_g * dk * inv_k2, s=(n, n, n), axes=(0, 1, 2)).ravel())
    psi = np.stack(psi)
    rms = np.sqrt(np.mean(np.sum(psi * psi, axis=0)))
    psi *= rms_cells * (box / n) / rms
    pos = lattice(n, box) + growth * psi
    pos = np.mod(pos, box)
    pos[pos >= box] -= box
    mom = mass * np.sqrt(a_begin) * psi
    return pos, mom


def clustered(n_p: int, box: float, seed: int, rms_cells: float = 2.0, halo_frac: float = 0.35,
              n_halos: int | None = None, mass: float = 1.0):
    """A strongly clustered particle set standing in for an evolved a = 1 snapshot.

    Zel'dovich displacement of ``rms_cells`` lattice spacings (past shell crossing), after
    which a fraction ``halo_frac`` of the particles is moved into Plummer spheres centred on
    randomly chosen particles.  Halo occupancies follow a power law (dN/dn ~ n^-2 between
    n_min and n_max) and the Plummer scale radius grows as occupancy^(1/3).  Gives the dense
    cells, empty cells and uneven cell occupancies of a late-time snapshot.
    """
    n = n_p ** 3
    pos, mom = zeldovich(n_p, box, 1.0, seed, rms_cells=rms_cells, mass=mass)
    spacing = box / n_p
    n_move = int(halo_frac * n)
    if n_halos is None:
        n_halos = max(1, n_move // 400)
    u = uniform01(seed + 101, 8 * n + 4 * n_halos)
    # occupancy weights ~ power law, normalised to n_move particles in total
    w = 1.0 / np.maximum(u[:n_halos], 1e-3)
    occ = np.floor(w / w.sum() * n_move).astype(np.int64)
    occ[0] += n_move - occ.sum()
    centres = pos[:, (u[n_halos:2 * n_halos] * n).astype(np.int64) % n]
    perm = np.argsort(u[2 * n_halos:2 * n_halos + n], kind="stable")[:n_move]
    owner = np.repeat(np.arange(n_halos), occ)
    r_scale = 0.15 * spacing * np.cbrt(np.maximum(occ, 1) / 100.0)
    v = uniform01(seed + 202, 3 * n_move).reshape(3, n_move)
    xi = np.minimum(v[0], 0.999)
    r = r_scale[owner] / np.sqrt(xi ** (-2.0 / 3.0) - 1.0)
    r = np.minimum(r, 10.0 * r_scale[owner])
    cos_t = 2.0 * v[1] - 1.0
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = 2.0 * np.pi * v[2]
    off = np.stack([r * sin_t * np.cos(phi), r * sin_t * np.sin(phi), r * cos_t])
    pos[:, perm] = centres[:, owner] + off
    pos = np.mod(pos, box)
    pos[pos >= box] -= box
    return pos, mom


def plane_wave(n_p: int, box: float, a_begin: float, amplitude: float, mass: float = 1.0,
               offset_cells: float = 0.0):
    """Single-mode Zel'dovich plane wave along x on an n_p^3 lattice (Einstein-de Sitter).

    The lattice is shifted by ``offset_cells`` lattice spacings along every axis;
    psi(q) = amplitude * sin(2 pi (q_x - shift) / box) x_hat is the displacement at a = 1;
    at a_begin x = q + a_begin psi and p = m a_begin^(3/2) psi.  Returns (q, pos, mom).
    """
    shift = offset_cells * box / n_p
    q = lattice(n_p, box) + shift
    psi = np.zeros_like(q)
    psi[0] = amplitude * np.sin(2.0 * np.pi * (q[0] - shift) / box)
    pos = np.mod(q + a_begin * psi, box)
    mom = mass * a_begin ** 1.5 * psi
    return q, pos, mom


def log_spaced_steps(a_begin: float, a_end: float, n_steps: int) -> np.ndarray:
    """Scale factors of n_steps logarithmically spaced steps from a_begin to a_end (n_steps+1 values)."""
    return np.exp(np.linspace(np.log(a_begin), np.log(a_end), n_steps + 1))


# The five workloads the framework is measured on: particle lattice n_p^3, mesh M^3, box in
# Mpc/h, split scale r_s in mesh cells, cutoff in units of r_s, Einstein-de Sitter background.
CONFIGS = {
    "edS_32": dict(n_p=32, mesh=32, box=64.0, r_s_cells=1.25, cutoff=4.5, a_begin=0.02,
                   a_end=0.1, steps=10, seed=1511),
    "clustered_128": dict(n_p=128, mesh=128, box=200.0, r_s_cells=1.25, cutoff=4.5,
                          a_begin=0.02, a_end=1.0, steps=64, seed=1512),
    "large_512": dict(n_p=512, mesh=512, box=1000.0, r_s_cells=1.25, cutoff=4.5,
                      a_begin=0.5, a_end=1.0, steps=10, seed=1513),
}
