"""Pins of the oracle's FFT and Kaiser-Squires inversion (Sec. 4.5).

The FFT is checked against a brute-force DFT and numpy.fft; the KS pair
against the closed-form shear of a plane wave (from the lensing potential:
kappa = lap(psi)/2, gamma1 = (psi_11 - psi_22)/2, gamma2 = psi_12), the
tangential sign of a point mass, forward-then-inverse recovery and the E/B
exchange under gamma -> i gamma.
"""
import numpy as np
import pytest

import oracle
from paper_1204_4293_gb300 import synth


def _naive_dft2(a, inverse=False):
    n = a.shape[0]
    sgn = 1.0 if inverse else -1.0
    idx = np.arange(n)
    out = np.zeros((n, n), dtype=complex)
    for ky in range(n):
        for kx in range(n):
            ph = np.exp(sgn * 2j * np.pi * (np.outer(idx, np.ones(n)) * ky + np.outer(np.ones(n), idx) * kx) / n)
            out[ky, kx] = (a * ph).sum()
    return out / (n * n) if inverse else out


@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_fft2_matches_brute_force_dft(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    assert np.abs(oracle.fft2(a) - _naive_dft2(a)).max() < 1e-12 * n * n
    assert np.abs(oracle.fft2(a, inverse=True) - _naive_dft2(a, inverse=True)).max() < 1e-13 * n


def test_fft2_matches_numpy_at_256():
    rng = np.random.default_rng(7)
    a = rng.standard_normal((256, 256)) + 1j * rng.standard_normal((256, 256))
    ref = np.fft.fft2(a)
    assert np.abs(oracle.fft2(a) - ref).max() / np.abs(ref).max() < 1e-14
    assert np.abs(oracle.fft2(oracle.fft2(a), inverse=True) - a).max() < 1e-13


@pytest.mark.parametrize("k1,k2", [(1, 0), (0, 1), (1, 1), (3, -2), (-5, 7), (8, 8)])
def test_plane_wave_shear_closed_form(k1, k2):
    # psi = cos(k.x): kappa = -|k|^2 psi / 2, gamma1 = -(k1^2 - k2^2) psi / 2,
    # gamma2 = -k1 k2 psi, so gamma = (cos 2 phi_k, sin 2 phi_k) kappa.
    n = 32
    y, x = np.mgrid[0:n, 0:n]
    kappa = np.cos(2 * np.pi * (k1 * x + k2 * y) / n)
    g1, g2 = oracle.ks_forward(kappa)
    phik = np.arctan2(k2, k1)
    assert np.abs(g1 - np.cos(2 * phik) * kappa).max() < 1e-12
    assert np.abs(g2 - np.sin(2 * phik) * kappa).max() < 1e-12
    kE, kB = oracle.ks_invert(g1, g2)
    assert np.abs(kE - kappa).max() < 1e-12
    assert np.abs(kB).max() < 1e-12


def test_point_mass_is_tangential():
    # A positive mass gives tangential shear: gamma_t = -Re(gamma e^{-2i phi}) > 0,
    # so gamma1 < 0 on the +x axis (standard weak-lensing sign).
    n = 64
    kappa = synth.delta_kappa(n)
    g1, g2 = oracle.ks_forward(kappa)
    c = n // 2
    for r in (2, 3, 5, 8):
        assert g1[c, c + r] < 0 and g1[c, c - r] < 0
        assert g1[c + r, c] > 0  # on the y axis the tangential direction flips gamma1
        for ang in np.linspace(0, 2 * np.pi, 16, endpoint=False):
            yy = c + int(round(r * np.sin(ang)))
            xx = c + int(round(r * np.cos(ang)))
            phi = np.arctan2(yy - c, xx - c)
            gt = -(g1[yy, xx] * np.cos(2 * phi) + g2[yy, xx] * np.sin(2 * phi))
            assert gt > 0


def test_forward_then_inverse_recovers_zero_mean_kappa():
    kappa = synth.grf_kappa(128, seed=3)
    kappa = kappa + 0.5  # a mean the inversion cannot see (mass-sheet)
    g1, g2 = oracle.ks_forward(kappa)
    kE, kB = oracle.ks_invert(g1, g2)
    assert np.abs(kE - (kappa - kappa.mean())).max() < 1e-13
    assert np.abs(kB).max() < 1e-13


def test_rotating_shear_by_45_degrees_swaps_E_and_B():
    rng = np.random.default_rng(11)
    g1, g2 = rng.standard_normal((2, 32, 32))
    kE, kB = oracle.ks_invert(g1, g2)
    # gamma -> i gamma: (g1, g2) -> (-g2, g1); then kappa_E' = -kappa_B, kappa_B' = kappa_E
    kE2, kB2 = oracle.ks_invert(-g2, g1)
    assert np.abs(kE2 + kB).max() < 1e-13
    assert np.abs(kB2 - kE).max() < 1e-13


def test_inversion_is_linear_and_unitary_on_nonzero_modes():
    rng = np.random.default_rng(5)
    g1, g2 = rng.standard_normal((2, 64, 64))
    kE, kB = oracle.ks_invert(g1, g2)
    m1, m2 = g1.mean(), g2.mean()
    # |conj(D)| = 1 away from k = 0: power is kept except the mean.
    p_in = ((g1 - m1) ** 2 + (g2 - m2) ** 2).sum()
    p_out = (kE ** 2 + kB ** 2).sum()
    assert p_out == pytest.approx(p_in, rel=1e-12)
