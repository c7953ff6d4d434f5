"""Pin of the oracle's shear -> kappa -> starlet composition by the exact,
discrete form of the paper's identity between the aperture mass and the
starlet bands (Sec. 3: M_ap with the starlet-shaped filter is the band at
theta = 2^j).

On a periodic grid every step is a circular convolution, so the band w_j of
the shear field gamma = gamma1 + i gamma2 is a direct sum over the shear
itself: w_j(x) = Re sum_y K_j(x - y) gamma(y), with the complex shear-space
filter K_j whose spectrum is u_j_hat(k) conj(D(k)), u_j the band's impulse
response and D(k) = (k1 + i k2)^2 / |k|^2 (D(0) = 0) the Kaiser-Squires
multiplier (Sec. 4.5).  The sum below runs over shifted copies of the field
(no FFT of the shear), so a wrong sign, conjugate or axis in the oracle's KS,
or a wrong band index or boundary in its starlet, breaks the equality that
otherwise holds to rounding.  The tangential part of K_j is the discrete
counterpart of the paper's starlet Q filter (eq. QU); the continuum Q itself
only converges to the bands (test_oracle_map.py).
"""
import numpy as np
import pytest

import oracle

N, J = 64, 5


def _freqs(n):
    f = np.arange(n)
    return np.where(f < n // 2, f, f - n)


def _conj_ks_multiplier(n):
    k2, k1 = np.meshgrid(_freqs(n), _freqs(n), indexing="ij")  # k1 along x (columns), k2 along y (rows)
    kk = (k1 * k1 + k2 * k2).astype(np.float64)
    d = np.zeros((n, n), dtype=np.complex128)
    nz = kk > 0
    d[nz] = ((k1 - 1j * k2)[nz] ** 2) / kk[nz]
    return d


def _band_impulse_responses(n, J):
    """u_j: the oracle's periodic starlet bands of a unit impulse at pixel 0."""
    delta = np.zeros((n, n))
    delta[0, 0] = 1.0
    return oracle.starlet(delta, J, oracle.PERIODIC)


def _shear_space_sum(K, gamma):
    """Re sum_d K(d) gamma(x - d) over every offset d of the periodic grid."""
    n = gamma.shape[0]
    acc = np.zeros((n, n), dtype=np.complex128)
    for dy in range(n):
        for dx in range(n):
            acc += K[dy, dx] * np.roll(gamma, (dy, dx), axis=(0, 1))
    return acc.real


@pytest.fixture(scope="module")
def field():
    rng = np.random.default_rng(31)
    g1, g2 = rng.standard_normal((2, N, N))
    return g1, g2


@pytest.mark.parametrize("j", [1, 2, 3, 4])
def test_band_equals_direct_sum_with_discrete_shear_filter(field, j):
    g1, g2 = field
    u = _band_impulse_responses(N, J)[j - 1]
    K = np.fft.ifft2(np.fft.fft2(u) * _conj_ks_multiplier(N))
    direct = _shear_space_sum(K, g1 + 1j * g2)
    w = oracle.map_starlet(g1, g2, J, oracle.PERIODIC)[j - 1]
    rms = np.sqrt(np.mean(w ** 2))
    assert np.abs(direct - w).max() / rms <= 1e-12


def test_discrete_shear_filter_is_spin_two_and_compensated():
    # K_j transforms like a spin-2 filter under a 90-degree rotation of the
    # grid (K(R d) = -K(d)) and has no response to a uniform shear (D(0) = 0):
    # the two properties the paper's tangential-shear form relies on
    u = _band_impulse_responses(N, J)[2]
    K = np.fft.ifft2(np.fft.fft2(u) * _conj_ks_multiplier(N))
    assert abs(K.sum()) < 1e-12
    # (y, x) -> (x, -y) on the periodic grid
    idx = np.arange(N)
    rot = K[np.ix_(idx, (-idx) % N)].T
    assert np.abs(rot + K).max() < 1e-12 * np.abs(K).max()
