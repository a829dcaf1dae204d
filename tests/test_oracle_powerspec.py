"""Pins of the oracle's power spectrum and top-hat sigma (Ch. Parameters: PM_gridsize,
R_tophat; Ch. Tests: powerspec) against closed forms and a published shot-noise formula."""

import math

import numpy as np

import p3m_synth as S
from oracle import p3m_oracle as O


def test_tophat_window_closed_form():
    assert abs(float(O.tophat_window(0.0)) - 1.0) < 1e-15
    # first zero of tan x = x
    assert abs(float(O.tophat_window(4.493409457909064))) < 1e-13
    x = 0.7
    ref = 3.0 * (math.sin(x) - x * math.cos(x)) / x ** 3
    assert abs(float(O.tophat_window(x)) - ref) < 1e-15


def test_plane_wave_power_and_sigma():
    M, L, m, A = 16, 50.0, 3, 0.3
    x = np.arange(M) * (L / M)
    delta = A * np.cos(2 * np.pi * m * x / L)[:, None, None] * np.ones((1, M, M))
    R = 7.0
    k, P, cnt, sigma = O.power_from_mesh(delta, L, deconvolve=False, radius=R)
    # all the variance A^2/2 sits in the two modes +-m along x, in shell m
    assert abs(P[m - 1] - L ** 3 * (A * A / 2.0) / cnt[m - 1]) < 1e-12 * P[m - 1]
    others = np.delete(P, m - 1)
    assert np.nanmax(np.abs(others)) < 1e-25
    kk = 2 * np.pi * m / L
    assert abs(sigma - A / math.sqrt(2.0) * abs(float(O.tophat_window(kk * R)))) < 1e-13


def test_sigma_small_radius_is_rms_of_the_mesh():
    """R -> 0: W_TH -> 1, so sigma^2 is the variance of the mesh (Parseval)."""
    p = O.Params(40.0, 3000, 20, short_range=False)
    pos = S.uniform_random(3000, 40.0, 3)
    n = O.cic_deposit(pos, p)
    delta = n / (3000 / 20 ** 3) - 1.0
    _, _, _, sig = O.power_from_mesh(delta, 40.0, deconvolve=False, radius=1e-6)
    assert abs(sig ** 2 - np.mean(delta ** 2)) < 1e-10 * np.mean(delta ** 2)


def test_poisson_shot_noise_matches_cic_formula():
    """Poisson particles: the binned power equals the CIC shot-noise spectrum of Jing (2005)
    averaged over each shell, within the shell's sampling error."""
    L, M, N = 100.0, 32, 40000
    p = O.Params(L, N, M, short_range=False)
    for deconvolve in (False, True):
        acc = np.zeros(M // 2)
        reps = 4
        for s in range(reps):
            pos = S.uniform_random(N, L, 100 + s)
            _, P, cnt, _ = O.power_spectrum(pos, p, deconvolve=deconvolve)
            acc += P
        P = acc / reps
        # expected shell averages
        n1 = np.fft.fftfreq(M, d=1.0 / M)
        NX, NY, NZ = np.meshgrid(n1, n1, n1, indexing="ij")
        shell = np.floor(np.sqrt(NX ** 2 + NY ** 2 + NZ ** 2) + 0.5).astype(int) - 1
        ps = O.cic_shot_noise(np.stack([NX.ravel(), NY.ravel(), NZ.ravel()]), p, N, deconvolve)
        for b in range(2, M // 2 - 1):
            sel = shell.ravel() == b
            expect = ps[sel].mean()
            err = 1.0 / math.sqrt(sel.sum() * reps / 2.0)  # exponential |delta_k|^2, paired modes
            assert abs(P[b] / expect - 1.0) < 5 * err + 1e-3, (deconvolve, b, P[b] / expect)


def test_zeldovich_ics_grow_as_a_squared():
    """Zel'dovich displacements scale with D = a, so large-scale power scales with a^2."""
    L, n = 64.0, 32
    p = O.Params(L, n ** 3, n, short_range=False)
    pa, _ = S.zeldovich(n, L, 0.02, 9, rms_cells=0.05)
    pb, _ = S.zeldovich(n, L, 0.02, 9, rms_cells=0.10)
    _, Pa, _, _ = O.power_spectrum(pa, p)
    _, Pb, _, _ = O.power_spectrum(pb, p)
    r = Pb[:4] / Pa[:4]
    assert np.all(np.abs(r / 4.0 - 1.0) < 0.02), r
