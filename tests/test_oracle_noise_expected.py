"""Pins of the oracle's exact expected noise variance (Sec. 1):
Var[w_j(x)] = 1/2 sum_y |K_j(x - y)|^2 |gamma(y)|^2, periodic boundary.

* Uniform |gamma|^2 = c: Var_j = (c / 2) sum_x |K_j(x)|^2, which by Parseval is
  (c / 2n^2) sum_{k != 0} |H_j(k)|^2 with the band's closed-form response
  H_j = Phi_{j-1} - Phi_j, Phi_j(k) = prod_{i<=j} h_i(k1) h_i(k2),
  h_i(k) = (6 + 8 cos(2 pi k 2^{i-1} / n) + 2 cos(2 pi k 2^i / n)) / 16, and
  |D(k)| = 1 for k != 0, D(0) = 0 (KS, Sec. 4.5);
* the oracle's Monte-Carlo noise maps scatter around it with the chi-square
  spread of a sample variance;
* it scales as |gamma|^2 and is invariant under a rotation of every pixel's
  shear (it sees |gamma| only).
"""
import numpy as np

import oracle


def _band_energy(n, J):
    k = np.arange(n)
    out = []
    phi_prev = np.ones((n, n))
    for j in range(1, J):
        s = 2 ** (j - 1)
        h = (6 + 8 * np.cos(2 * np.pi * k * s / n) + 2 * np.cos(2 * np.pi * k * 2 * s / n)) / 16
        phi = phi_prev * np.outer(h, h)
        H = phi_prev - phi
        H[0, 0] = 0.0  # D(0) = 0
        out.append((H ** 2).sum() / n ** 2)
        phi_prev = phi
    return np.array(out)


def test_uniform_modulus_parseval_closed_form():
    n, J = 32, 5
    rng = np.random.default_rng(2)
    ang = rng.uniform(0, 2 * np.pi, (n, n))
    g1, g2 = 0.3 * np.cos(ang), 0.3 * np.sin(ang)  # |gamma|^2 = 0.09 everywhere
    v = oracle.map_noise_expected(g1, g2, J)
    want = 0.5 * 0.09 * _band_energy(n, J)
    for j in range(J - 1):
        assert np.abs(v[j] - want[j]).max() <= 1e-12 * want[j], (j, v[j].mean(), want[j])


def test_monte_carlo_scatters_around_the_expectation():
    n, J, R = 32, 4, 300
    rng = np.random.default_rng(9)
    g1, g2 = 0.1 * rng.standard_normal((2, n, n))
    g1[:8] *= 3.0  # a non-uniform |gamma| so that position matters
    exact = oracle.map_noise_expected(g1, g2, J)
    var, _ = oracle.map_noise(g1, g2, J, R, seed=11, boundary=oracle.PERIODIC, with_snr=False)
    for j in range(J - 1):
        ratio = var[j] / exact[j]
        sd = np.sqrt(2.0 / (R - 1))  # relative s.d. of a sample variance
        assert abs(ratio.mean() - 1.0) < 3 * sd / 4, (j, ratio.mean())
        assert 0.6 * sd < ratio.std() < 1.4 * sd, (j, ratio.std())


def test_scaling_and_rotation_invariance():
    n, J = 16, 4
    rng = np.random.default_rng(4)
    g1, g2 = rng.standard_normal((2, n, n))
    v = oracle.map_noise_expected(g1, g2, J)
    assert np.allclose(oracle.map_noise_expected(2 * g1, 2 * g2, J), 4 * v, rtol=1e-13, atol=0)
    a = rng.uniform(0, np.pi, (n, n))
    r1 = g1 * np.cos(2 * a) - g2 * np.sin(2 * a)
    r2 = g1 * np.sin(2 * a) + g2 * np.cos(2 * a)
    assert np.allclose(oracle.map_noise_expected(r1, r2, J), v, rtol=1e-12, atol=0)
    # the listed-pixel form equals the full map
    ys, xs = np.array([0, 5, 15]), np.array([3, 0, 15])
    assert np.array_equal(oracle.map_noise_expected_at(g1, g2, J, ys, xs), v[:, ys, xs])
