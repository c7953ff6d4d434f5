"""Pins of the oracle's starlet transform (Sec. 3, Sec. 4.2, Fig. 3).

Checked against: exact reconstruction kappa = c_J + sum_j w_j; constant maps;
linearity and (periodic) translation equivariance; an explicit matrix form of
the 1-D filters with holes (mirror and periodic); and the closed-form Fourier
response of the B3 filter bank, whose band responses add up to one (Fig. 3).
"""
import numpy as np
import pytest

import oracle
from paper_1204_4293_gb300 import synth

H = np.array([1, 4, 6, 4, 1]) / 16.0


def _fold(i, n, boundary):
    if boundary == oracle.PERIODIC:
        return i % n
    period = 2 * (n - 1)
    i = i % period
    return period - i if i >= n else i


def _filter_matrix(n, s, boundary):
    """1-D filter h with holes at spacing s as an explicit n x n matrix."""
    m = np.zeros((n, n))
    for i in range(n):
        for k in range(5):
            m[i, _fold(i + (k - 2) * s, n, boundary)] += H[k]
    return m


@pytest.mark.parametrize("boundary", [oracle.MIRROR, oracle.PERIODIC])
@pytest.mark.parametrize("n,J", [(16, 4), (20, 3), (37, 5), (64, 6), (32, 2)])
def test_exact_reconstruction(n, J, boundary):
    kappa = synth.white((n, n), seed=n + J)
    pyr = oracle.starlet(kappa, J, boundary)
    assert pyr.shape == (J, n, n)
    assert np.abs(pyr.sum(axis=0) - kappa).max() <= 1e-12 * np.abs(kappa).max()


@pytest.mark.parametrize("boundary", [oracle.MIRROR, oracle.PERIODIC])
def test_constant_map_has_zero_bands(boundary):
    pyr = oracle.starlet(np.full((24, 24), 3.25), 4, boundary)
    assert np.abs(pyr[:-1]).max() < 1e-14
    assert np.abs(pyr[-1] - 3.25).max() < 1e-14


@pytest.mark.parametrize("boundary", [oracle.MIRROR, oracle.PERIODIC])
@pytest.mark.parametrize("n,J", [(16, 4), (24, 3), (33, 5)])
def test_matches_explicit_matrix_form(n, J, boundary):
    # c_j = A_j c_{j-1} A_j^T with A_j the 1-D filter with holes 2^(j-1).
    kappa = synth.white((n, n), seed=3 * n + J)
    pyr = oracle.starlet(kappa, J, boundary)
    c = kappa.copy()
    for j in range(1, J):
        a = _filter_matrix(n, 2 ** (j - 1), boundary)
        cn = a @ c @ a.T
        assert np.abs(pyr[j - 1] - (c - cn)).max() < 1e-13
        c = cn
    assert np.abs(pyr[J - 1] - c).max() < 1e-13


def test_linearity_and_periodic_shift():
    n, J = 32, 5
    a = synth.white((n, n), seed=1)
    b = synth.white((n, n), seed=2)
    pa = oracle.starlet(a, J, oracle.MIRROR)
    pb = oracle.starlet(b, J, oracle.MIRROR)
    pab = oracle.starlet(2.0 * a - 0.5 * b, J, oracle.MIRROR)
    assert np.abs(pab - (2.0 * pa - 0.5 * pb)).max() < 1e-13
    sh = np.roll(a, (5, -7), axis=(0, 1))
    p1 = oracle.starlet(a, J, oracle.PERIODIC)
    p2 = oracle.starlet(sh, J, oracle.PERIODIC)
    assert np.abs(np.roll(p1, (5, -7), axis=(1, 2)) - p2).max() < 1e-13


def test_fourier_response_closed_form_and_partition_of_unity():
    # Periodic starlet = Fourier multipliers: c_j has response
    # prod_{i<=j} hhat(2^(i-1) w1) hhat(2^(i-1) w2), hhat(w) = (6 + 8 cos w + 2 cos 2w)/16.
    n, J = 32, 5
    delta = np.zeros((n, n))
    delta[0, 0] = 1.0
    pyr = oracle.starlet(delta, J, oracle.PERIODIC)
    w = 2 * np.pi * np.fft.fftfreq(n)

    def hhat(t):
        return (6 + 8 * np.cos(t) + 2 * np.cos(2 * t)) / 16.0

    phi_prev = np.ones((n, n))
    total = np.zeros((n, n), dtype=complex)
    for j in range(1, J):
        s = 2 ** (j - 1)
        phi = phi_prev * np.outer(hhat(s * w), hhat(s * w))
        resp = np.fft.fft2(pyr[j - 1])
        assert np.abs(resp - (phi_prev - phi)).max() < 1e-13
        total += resp
        phi_prev = phi
    resp_c = np.fft.fft2(pyr[J - 1])
    assert np.abs(resp_c - phi_prev).max() < 1e-13
    total += resp_c
    # Fig. 3: w_1 high-pass, w_j band-pass, c_J low-pass; together they pass everything.
    assert np.abs(total - 1.0).max() < 1e-13
    assert abs(resp_c[0, 0] - 1.0) < 1e-14  # low-pass keeps the mean
    assert np.abs(np.fft.fft2(pyr[0])[0, 0]) < 1e-14  # bands are compensated


def test_mean_preserved_by_smooth_array_periodic():
    kappa = synth.grf_kappa(64, seed=9) + 0.3
    pyr = oracle.starlet(kappa, 6, oracle.PERIODIC)
    assert pyr[-1].mean() == pytest.approx(kappa.mean(), abs=1e-14)
    for j in range(5):
        assert abs(pyr[j].mean()) < 1e-15
