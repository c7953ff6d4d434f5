"""Pins of the oracle's randomised-shear noise maps (Sec. 1, Sec. 5.1).

* the rotation angle is uniform on [0, pi) (chi-square) and the generator is
  a counter-based SplitMix64 (distinct counters, reproducible);
* rotation keeps |gamma| per pixel;
* the Monte-Carlo variance matches the exact expectation for a uniform phase,
  Var[w_j(x)] = 1/2 sum_y |K_j(x - y)|^2 |gamma(y)|^2, within the chi-square
  spread of a sample variance (periodic boundary, where KS + starlet is a
  convolution with the complex kernel K_j);
* S/N = w_j(data) / sigma_j.
"""
import numpy as np
import pytest

import oracle
from paper_1204_4293_gb300 import synth


def test_splitmix64_counter_properties():
    vals = [oracle.splitmix64(42, i) for i in range(2000)]
    assert len(set(vals)) == len(vals)
    assert vals[:3] == [oracle.splitmix64(42, i) for i in range(3)]
    assert oracle.splitmix64(43, 0) != vals[0]
    # outputs use all 64 bits
    bits = np.array([[(v >> b) & 1 for b in range(64)] for v in vals])
    assert np.all(np.abs(bits.mean(axis=0) - 0.5) < 0.06)


def test_rotation_angle_uniform():
    n = 64
    u = np.array([[oracle.noise_u(7, 3, y, x, n) for x in range(n)] for y in range(n)]).ravel()
    assert u.min() >= 0.0 and u.max() < 1.0
    counts, _ = np.histogram(u, bins=32, range=(0, 1))
    expect = u.size / 32
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 70  # 31 dof; p ~ 1e-4
    # 24-bit grid
    assert np.allclose(u * 2 ** 24, np.round(u * 2 ** 24), atol=0)


def test_rotation_keeps_modulus_and_depends_on_realisation():
    n = 16
    rng = np.random.default_rng(3)
    g1, g2 = rng.standard_normal((2, n, n))
    r1a, r2a = oracle.rotate_shear(g1, g2, 0, 99)
    r1b, r2b = oracle.rotate_shear(g1, g2, 1, 99)
    assert np.allclose(r1a ** 2 + r2a ** 2, g1 ** 2 + g2 ** 2, rtol=1e-14)
    assert np.abs(r1a - r1b).max() > 0.1


def _kernel_modulus2(n, J):
    """|K_j|^2 of the periodic KS + starlet map, from its two impulse responses."""
    z = np.zeros((n, n))
    d = z.copy()
    d[0, 0] = 1.0
    p1 = oracle.map_starlet(d, z, J, oracle.PERIODIC)  # Re K
    p2 = oracle.map_starlet(z, d, J, oracle.PERIODIC)  # Re(i K) = -Im K
    return p1[:-1] ** 2 + p2[:-1] ** 2


def test_monte_carlo_variance_matches_exact_expectation():
    n, J, R = 32, 4, 200
    rng = np.random.default_rng(8)
    g1, g2 = 0.1 * rng.standard_normal((2, n, n))
    var, snr = oracle.map_noise(g1, g2, J, R, seed=5, boundary=oracle.PERIODIC)
    k2 = _kernel_modulus2(n, J)
    mod2 = g1 ** 2 + g2 ** 2
    for j in range(J - 1):
        # periodic convolution of |K_j|^2 with |gamma|^2, halved
        exact = 0.5 * np.real(np.fft.ifft2(np.fft.fft2(k2[j]) * np.fft.fft2(mod2)))
        ratio = var[j] / exact
        # sample variance: relative s.d. sqrt(2 / (R - 1)) = 0.1 per pixel
        assert abs(ratio.mean() - 1.0) < 0.03, (j, ratio.mean())
        assert 0.06 < ratio.std() < 0.14, (j, ratio.std())
    pyr = oracle.map_starlet(g1, g2, J, oracle.PERIODIC)
    assert np.allclose(snr, pyr[:-1] / np.sqrt(var), rtol=1e-14)


def test_noise_is_reproducible_and_seed_dependent():
    n, J, R = 16, 3, 6
    g1, g2 = synth.shape_noise(n, seed=1)
    v1, _ = oracle.map_noise(g1, g2, J, R, seed=11)
    v2, _ = oracle.map_noise(g1, g2, J, R, seed=11)
    v3, _ = oracle.map_noise(g1, g2, J, R, seed=12)
    assert np.array_equal(v1, v2)
    assert np.abs(v1 - v3).max() > 0
