"""Pins of the oracle's direct aperture mass (eq. mapdef, eq. shearmap) and of
the paper's identity between M_ap and the starlet bands (Sec. 3).

* eq. shearmap (the oracle, from shear) against eq. mapdef (a brute-force
  convolution of kappa with U, written here) on a smooth periodic field;
* spin-2 consistency: rotating the field by 90 degrees negates the shear and
  rotates the M_ap map;
* support: nothing beyond the cut radius, nothing from outside the field;
* the identity M_ap(starlet Q) ~ w_j (Sec. 3): exact in the continuum only,
  so checked as convergence with theta.
"""
import numpy as np
import pytest

import oracle
from paper_1204_4293_gb300 import synth


def _smooth_kappa(n, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:n, 0:n]
    k = np.zeros((n, n))
    for _ in range(6):
        cy, cx = rng.uniform(0, n, 2)
        amp = rng.normal()
        dy = (y - cy + n / 2) % n - n / 2
        dx = (x - cx + n / 2) % n - n / 2
        k += amp * np.exp(-(dx ** 2 + dy ** 2) / (2 * 7.0 ** 2))
    return k - k.mean()


def _map_from_kappa(kappa, u, R, pts):
    """eq. mapdef by brute force: sum_d U(|d|) kappa(x + d), periodic field."""
    n = kappa.shape[0]
    out = []
    ri = int(np.floor(R))
    d = np.arange(-ri, ri + 1)
    dy, dx = np.meshgrid(d, d, indexing="ij")
    r = np.hypot(dx, dy)
    w = np.where(r <= R, np.vectorize(u)(r), 0.0)
    for (py, px) in pts:
        patch = kappa[np.ix_((py + d) % n, (px + d) % n)]
        out.append((w * patch).sum())
    return np.array(out)


@pytest.mark.parametrize("filt,theta", [(oracle.S98, 12.0), (oracle.STARLET_Q, 6.0)])
def test_shear_form_equals_kappa_form_on_smooth_field(filt, theta):
    n = 128
    kappa = _smooth_kappa(n, seed=4)
    g1, g2 = oracle.ks_forward(kappa)
    if filt == oracle.S98:
        u = lambda v: oracle.u_s98(v, theta, 3)
        R = theta
    else:
        u = lambda v: oracle.u_starlet(v / theta) / theta ** 2
        R = 2 * theta
    rng = np.random.default_rng(1)
    pts = [(int(a), int(b)) for a, b in rng.integers(int(R) + 1, n - int(R) - 1, size=(12, 2))]
    ys, xs = zip(*pts)
    m_shear = oracle.map_direct_at(g1, g2, ys, xs, filt, theta)
    m_kappa = _map_from_kappa(kappa, u, R, pts)
    scale = np.abs(m_kappa).max()
    assert np.abs(m_shear - m_kappa).max() < 0.03 * scale
    assert np.corrcoef(m_shear, m_kappa)[0, 1] > 0.999


@pytest.mark.parametrize("filt", [oracle.STARLET_Q, oracle.S98, oracle.JBJ04])
def test_spin2_rotation(filt):
    n = 24
    rng = np.random.default_rng(2)
    g1, g2 = rng.standard_normal((2, n, n))
    m = oracle.map_direct(g1, g2, filt, 2.0)
    # rotate coordinates by 90 degrees: a spin-2 field changes sign
    m_rot = oracle.map_direct(-np.rot90(g1), -np.rot90(g2), filt, 2.0)
    assert np.abs(m_rot - np.rot90(m)).max() < 1e-13
    # mirror x -> -x: gamma2 changes sign, M_ap is a scalar
    m_flip = oracle.map_direct(g1[:, ::-1], -g2[:, ::-1], filt, 2.0)
    assert np.abs(m_flip - m[:, ::-1]).max() < 1e-13


def test_single_pixel_support_and_field_edge():
    n, theta = 40, 4.0
    g1 = np.zeros((n, n))
    g2 = np.zeros((n, n))
    g1[20, 20] = 1.0
    m = oracle.map_direct(g1, g2, oracle.STARLET_Q, theta)
    y, x = np.mgrid[0:n, 0:n]
    r = np.hypot(x - 20, y - 20)
    assert np.all(m[r > 2 * theta] == 0.0)
    assert m[20, 20] == 0.0  # the d = 0 term is dropped
    assert np.count_nonzero(m) > 0
    # a pixel next to the field edge only sums in-field data: padding the field
    # with zeros does not change it
    g1p = np.pad(g1, 10)
    g2p = np.pad(g2, 10)
    mp = oracle.map_direct(g1p, g2p, oracle.STARLET_Q, theta)
    assert np.abs(mp[10:-10, 10:-10] - m).max() < 1e-15


def test_identity_with_starlet_bands_converges_with_theta():
    # Sec. 3: M_ap with the starlet-shaped Q equals the band w_j at theta = 2^j in
    # the continuum.  On the lattice the mismatch falls with theta.
    n, J = 128, 5
    kappa = synth.grf_kappa(n, seed=2)
    g1, g2 = oracle.ks_forward(kappa)
    pyr = oracle.starlet(oracle.ks_invert(g1, g2)[0], J, oracle.PERIODIC)
    bounds = {1: 0.65, 2: 0.2, 3: 0.06}
    errs = {}
    for j, bound in bounds.items():
        theta = 2.0 ** j
        m = oracle.map_direct(g1, g2, oracle.STARLET_Q, theta)
        cut = int(2 * theta) + 1
        inner = (slice(cut, n - cut), slice(cut, n - cut))
        w = pyr[j - 1][inner]
        rel = np.sqrt(np.mean((m[inner] - w) ** 2)) / np.sqrt(np.mean(w ** 2))
        errs[j] = rel
        assert rel < bound, (j, rel)
        if j >= 2:
            assert np.corrcoef(m[inner].ravel(), w.ravel())[0, 1] > 0.99
    assert errs[3] < errs[2] < errs[1]
