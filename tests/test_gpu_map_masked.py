"""GPU weighted direct M_ap (missing data, Sec. 4.3 and Sec. 4.5) against the
FP64 oracle: masked fields of several tiles with ragged tails, every filter,
shared and per-map weights, the degenerate fields (all masked, smaller than
the aperture) and sampled pixels of a 1024^2 star-masked field.

Error metric.  M = N_R S / D divides by the local weight D, so where few
pixels of the aperture carry data an fp32 rounding of S is amplified by
1/coverage.  The tests therefore bound (a) the coverage, absolutely, (b)
coverage * M = S / 1 (the weighted sum, no division) against its RMS and
(c) M itself against its RMS where coverage >= 0.2.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import rel_err
from paper_1204_4293_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {np.float32: 1e-5, np.float64: 1e-12}


def _fm():
    from paper_1204_4293_gb300 import fastmap
    return fastmap


def _check(m, cov, m_ref, cov_ref, dtype):
    m = np.asarray(m, dtype=np.float64)
    cov = np.asarray(cov, dtype=np.float64)
    tol = TOL[dtype]
    assert np.abs(cov - cov_ref).max() <= (1e-6 if dtype == np.float32 else 1e-14)
    s_ref = m_ref * cov_ref
    if np.abs(s_ref).max() > 0:
        assert rel_err(m * cov, s_ref) <= tol
    good = cov_ref >= 0.2
    if good.any() and np.abs(m_ref[good]).max() > 0:
        assert rel_err(m[good], m_ref[good]) <= tol
    assert np.all(m[cov_ref == 0] == 0)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("filt,theta", [(1, 6.0), (0, 3.0), (2, 2.0), (3, 5.0)])
def test_masked_matches_oracle(filt, theta, dtype):
    fm = _fm()
    n = 96  # 16-row tiles, one partial 256-column tile
    g1, g2 = synth.white((2, n, n), seed=int(theta * 10) + filt, scale=0.1)
    w = synth.star_mask(n, frac=0.2, seed=filt)
    m_ref, cov_ref = oracle.map_direct_masked(g1, g2, w, filt, theta)
    t = lambda a: torch.from_numpy(a.astype(dtype)).cuda()
    m, cov = fm.fm_map_direct_masked(t(g1), t(g2), t(w), filt, theta, coverage=True)
    _check(m.cpu().numpy(), cov.cpu().numpy(), m_ref, cov_ref, dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_masked_batch_shared_and_per_map_weights(dtype):
    fm = _fm()
    n, batch, theta = 70, 3, 4.0
    g = [synth.white((2, n, n), seed=40 + b, scale=0.1) for b in range(batch)]
    ws = [synth.star_mask(n, frac=0.1 + 0.1 * b, seed=b) for b in range(batch)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()
    g1 = t(np.stack([x[0] for x in g]))
    g2 = t(np.stack([x[1] for x in g]))
    # one weight map for the batch
    m, cov = fm.fm_map_direct_masked(g1, g2, t(ws[0]), 1, theta, coverage=True)
    for b in range(batch):
        m_ref, cov_ref = oracle.map_direct_masked(g[b][0], g[b][1], ws[0], 1, theta)
        _check(m[b].cpu().numpy(), cov[b].cpu().numpy(), m_ref, cov_ref, dtype)
    # one weight map per map, fractional weights
    wf = np.stack(ws) * (0.5 + synth.white((batch, n, n), seed=9) ** 2)
    m, cov = fm.fm_map_direct_masked(g1, g2, t(wf), 0, theta / 2, coverage=True)
    for b in range(batch):
        m_ref, cov_ref = oracle.map_direct_masked(g[b][0], g[b][1], wf[b], 0, theta / 2)
        _check(m[b].cpu().numpy(), cov[b].cpu().numpy(), m_ref, cov_ref, dtype)


def test_unit_weights_equal_plain_direct_map_inside():
    fm = _fm()
    n, theta = 128, 8.0
    g1, g2 = (torch.from_numpy(a.astype(np.float32)).cuda() for a in synth.white((2, n, n), seed=5, scale=0.1))
    ones = torch.ones_like(g1)
    m, cov = fm.fm_map_direct_masked(g1, g2, ones, 1, theta, coverage=True)
    plain = fm.fm_map_direct(g1, g2, 1, theta)
    r = int(theta)
    inner = (slice(r, n - r), slice(r, n - r))
    assert torch.all(cov[inner] == 1.0)
    assert rel_err(m[inner].cpu().numpy(), plain[inner].cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("n", [1, 5, 17])
def test_degenerate_fields(n):
    fm = _fm()
    g1, g2 = (torch.from_numpy(a.astype(np.float32)).cuda() for a in synth.white((2, n, n), seed=n, scale=0.1))
    # all masked: zero map, zero coverage
    m, cov = fm.fm_map_direct_masked(g1, g2, torch.zeros_like(g1), 0, 4.0, coverage=True)
    assert torch.all(m == 0) and torch.all(cov == 0)
    # field smaller than the aperture
    w = synth.star_mask(n, frac=0.3, seed=2)
    m, cov = fm.fm_map_direct_masked(g1, g2, torch.from_numpy(w.astype(np.float32)).cuda(), 1, 9.0, coverage=True)
    m_ref, cov_ref = oracle.map_direct_masked(g1.cpu().numpy(), g2.cpu().numpy(), w, 1, 9.0)
    _check(m.cpu().numpy(), cov.cpu().numpy(), m_ref, cov_ref, np.float32)


def test_masked_1024_sampled_pixels():
    # the paper's 1024^2 field with 15 % masked, S98 theta = 16; 3000 sampled
    # pixels (edges, corners and random interior points) against the oracle
    fm = _fm()
    n, theta = 1024, 16.0
    rng = np.random.default_rng(1)
    g1, g2 = (synth.white((n, n), seed=s, scale=0.1) for s in (71, 72))
    w = synth.star_mask(n, frac=0.15, seed=7)
    t = lambda a: torch.from_numpy(a.astype(np.float32)).cuda()
    m, cov = fm.fm_map_direct_masked(t(g1), t(g2), t(w), 1, theta, coverage=True)
    m, cov = m.cpu().numpy(), cov.cpu().numpy()
    ys = np.concatenate([rng.integers(0, n, 2800), [0, 0, n - 1, n - 1], np.full(98, 3)])
    xs = np.concatenate([rng.integers(0, n, 2800), [0, n - 1, 0, n - 1], np.arange(98) * 10])
    m_ref, cov_ref = oracle.map_direct_masked_at(g1, g2, w, ys, xs, 1, theta)
    _check(m[ys, xs], cov[ys, xs], m_ref, cov_ref, np.float32)
