"""Pins of the oracle's weighted (missing-data) direct M_ap (eq. shearmap with
pixel weights; Sec. 4.3 and Sec. 4.5 on edges, masks and missing data).

M(x) = N_R sum w Q gamma_t / sum w over the in-field offsets 0 < |d| <= R and
coverage = sum w / N_R.  Checked against: a field with one valid pixel (closed
form at offsets where gamma_t reduces to +-gamma1 or -gamma2), the plain
direct map (pinned in test_oracle_map.py) wherever the aperture is unmasked
and inside the field, the aperture pixel count N_R and corner coverage by
lattice counting, the 90-degree symmetry that cancels a uniform shear, and
invariance to the shear under masked pixels and to the weights' scale.
"""
import numpy as np
import pytest

import oracle
from paper_1204_4293_gb300 import synth


def _lattice_count(R, cond=lambda dx, dy: True):
    ri = int(np.floor(R))
    return sum(1 for dy in range(-ri, ri + 1) for dx in range(-ri, ri + 1)
               if 0 < dx * dx + dy * dy <= R * R and cond(dx, dy))


@pytest.mark.parametrize("filt,theta", [(oracle.S98, 5.0), (oracle.STARLET_Q, 3.0), (oracle.JBJ04, 1.5)])
def test_single_valid_pixel_closed_form(filt, theta):
    n = 33
    c = n // 2
    rng = np.random.default_rng(4)
    g1, g2 = rng.standard_normal((2, n, n))
    w = np.zeros((n, n))
    w[c, c] = 1.0
    R = oracle.default_cut(filt) * theta
    n_r = _lattice_count(R)
    m, cov = oracle.map_direct_masked(g1, g2, w, filt, theta)
    # output pixel x sees the valid pixel at offset d = (c - y, c - x)
    for (dy, dx, gt) in [(0, 3, -g1[c, c]), (0, -2, -g1[c, c]), (3, 0, g1[c, c]), (-1, 0, g1[c, c]),
                         (2, 2, -g2[c, c]), (-3, -3, -g2[c, c]), (2, -2, g2[c, c])]:
        y, x = c - dy, c - dx
        r = np.hypot(dx, dy)
        if r > R:
            continue
        q = oracle.q_filter(filt, r, theta)
        assert m[y, x] == pytest.approx(n_r * q * gt, rel=1e-12, abs=1e-300)
        assert cov[y, x] == pytest.approx(1.0 / n_r, rel=1e-14)
    # the valid pixel itself (d = 0 is not in the aperture) and pixels farther than R
    assert m[c, c] == 0.0 and cov[c, c] == 0.0
    ys, xs = np.mgrid[0:n, 0:n]
    far = (ys - c) ** 2 + (xs - c) ** 2 > R * R
    assert np.all(m[far] == 0.0) and np.all(cov[far] == 0.0)


@pytest.mark.parametrize("filt,theta", [(oracle.S98, 4.0), (oracle.STARLET_Q, 2.5)])
def test_unmasked_interior_equals_plain_direct_map(filt, theta):
    n = 40
    g1, g2 = synth.white((2, n, n), seed=8)
    m, cov = oracle.map_direct_masked(g1, g2, np.ones((n, n)), filt, theta)
    plain = oracle.map_direct(g1, g2, filt, theta)
    ri = int(np.floor(oracle.default_cut(filt) * theta))
    inner = (slice(ri, n - ri), slice(ri, n - ri))
    assert np.abs(m[inner] - plain[inner]).max() <= 1e-13 * np.abs(plain[inner]).max()
    assert np.all(cov[inner] == 1.0)
    # at the edges the plain map drops missing pixels, the weighted one rescales them
    assert np.all(cov[0, 0] < 1.0)


def test_corner_and_edge_coverage_by_lattice_count():
    n, theta = 24, 6.0
    R = theta  # S98 cut
    n_r = _lattice_count(R)
    assert n_r == 112  # integer points with 0 < x^2 + y^2 <= 36
    g1, g2 = synth.white((2, n, n), seed=2)
    _, cov = oracle.map_direct_masked(g1, g2, np.ones((n, n)), oracle.S98, theta)
    corner = _lattice_count(R, lambda dx, dy: dx >= 0 and dy >= 0)
    edge = _lattice_count(R, lambda dx, dy: dy >= 0)
    assert cov[0, 0] == pytest.approx(corner / n_r, rel=1e-15)
    assert cov[0, n // 2] == pytest.approx(edge / n_r, rel=1e-15)


def test_uniform_shear_cancels_under_a_fourfold_symmetric_mask():
    # gamma_t of a uniform shear changes sign under a 90-degree rotation of d
    # (cos 2 phi and sin 2 phi do), so a mask invariant under that rotation
    # about x cancels it: M(x) = 0.
    n = 31
    c = n // 2
    rng = np.random.default_rng(6)
    w = (rng.random((n, n)) < 0.6).astype(float)
    w = np.maximum.reduce([w, np.rot90(w, 1), np.rot90(w, 2), np.rot90(w, 3)])
    w[c - 2:c + 3, c + 1] = 0.0
    w = np.minimum.reduce([w, np.rot90(w, 1), np.rot90(w, 2), np.rot90(w, 3)])
    assert np.array_equal(w, np.rot90(w))
    for filt, theta in [(oracle.S98, 7.0), (oracle.STARLET_Q, 3.0)]:
        g1 = np.full((n, n), 0.3)
        g2 = np.full((n, n), -0.2)
        m, cov = oracle.map_direct_masked_at(g1, g2, w, [c], [c], filt, theta)
        assert abs(m[0]) < 1e-14
        assert cov[0] < 1.0


def test_masked_shear_is_ignored_and_weight_scale_cancels():
    n = 28
    g1, g2 = synth.white((2, n, n), seed=12)
    rng = np.random.default_rng(3)
    w = rng.random((n, n)) * (rng.random((n, n)) > 0.3)
    m, cov = oracle.map_direct_masked(g1, g2, w, oracle.S98, 5.0)
    h1, h2 = g1.copy(), g2.copy()
    h1[w == 0] = 1e6
    h2[w == 0] = -3e5
    m2, cov2 = oracle.map_direct_masked(h1, h2, w, oracle.S98, 5.0)
    assert np.abs(m2 - m).max() <= 1e-12 * np.abs(m).max()
    m3, cov3 = oracle.map_direct_masked(g1, g2, 7.5 * w, oracle.S98, 5.0)
    assert np.abs(m3 - m).max() <= 1e-12 * np.abs(m).max()
    assert np.abs(cov3 - 7.5 * cov).max() <= 1e-12


def test_fully_masked_field_gives_zero():
    n = 16
    g1, g2 = synth.white((2, n, n), seed=1)
    m, cov = oracle.map_direct_masked(g1, g2, np.zeros((n, n)), oracle.STARLET_Q, 2.0)
    assert np.all(m == 0.0) and np.all(cov == 0.0)
