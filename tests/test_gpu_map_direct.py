"""GPU direct M_ap (eq. shearmap, brute force as in Sec. 5.1) against the oracle:
every filter, radii across the paper's range, ragged field sizes, and the
1024^2 theta = 64 case on sampled pixels."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, rel_err, shear

pytestmark = pytest.mark.gpu


def _fm():
    from paper_1204_4293_gb300 import fastmap
    return fastmap


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("filt,theta,n", [(0, 2.0, 64), (0, 4.0, 100), (0, 8.0, 77), (1, 2.0, 64), (1, 8.0, 130),
                                          (1, 16.0, 96), (2, 2.0, 50), (3, 3.0, 33), (0, 1.0, 5)])
def test_map_direct_matches_oracle(filt, theta, n, dtype):
    fm = _fm()
    side = 1 << max(3, (n - 1).bit_length())  # shear is made on a power-of-two grid, then cropped
    g1, g2 = shear(side, seed=int(theta) + n, dtype=dtype)
    g1, g2 = np.ascontiguousarray(g1[:n, :n]), np.ascontiguousarray(g2[:n, :n])
    m = fm.fm_map_direct(torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda(), filt, theta).cpu().numpy()
    ref = oracle.map_direct(g1.astype(np.float64), g2.astype(np.float64), filt, theta)
    assert rel_err(m, ref) <= TOL[dtype]


def test_map_direct_cut_override_and_ell():
    fm = _fm()
    g1, g2 = shear(64, seed=3, dtype=np.float32)
    g1, g2 = np.ascontiguousarray(g1[:48, :48]), np.ascontiguousarray(g2[:48, :48])
    m = fm.fm_map_direct(torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda(), 1, 6.0, ell=1,
                         cut_over_theta=0.5).cpu().numpy()
    ref = oracle.map_direct(g1.astype(np.float64), g2.astype(np.float64), 1, 6.0, ell=1, cut_over_theta=0.5)
    assert rel_err(m, ref) <= 1e-5


@pytest.mark.parametrize("filt,theta,n", [(0, 64.0, 1024), (1, 64.0, 1024), (0, 2.0, 1024), (1, 8.0, 2048),
                                          (2, 8.0, 1024)])
def test_map_direct_paper_size_sampled(filt, theta, n):
    # 2000 random pixels (their oracle RMS stands for the map's RMS) plus the
    # corners and the edges of the 256-column, 16-row tiles
    fm = _fm()
    g1, g2 = shear(n, seed=2, dtype=np.float32)
    m = fm.fm_map_direct(torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda(), filt, theta).cpu().numpy()
    rng = np.random.default_rng(0)
    ys = np.concatenate([rng.integers(0, n, 2000), [0, 0, n - 1, n - 1, 5, n // 2, 15, 16, 3, 4]])
    xs = np.concatenate([rng.integers(0, n, 2000), [0, n - 1, 0, n - 1, n // 2, 3, 255, 256, 511, 512]])
    ref = oracle.map_direct_at(g1.astype(np.float64), g2.astype(np.float64), ys, xs, filt, theta)
    rms = np.sqrt(np.mean(ref[:2000] ** 2))
    assert np.abs(m[ys, xs] - ref).max() / rms <= 1e-5


@pytest.mark.parametrize("filt,theta,n,batch", [(1, 4.0, 300, 3), (0, 8.0, 129, 2), (2, 2.0, 64, 5)])
def test_map_direct_batch_matches_oracle_and_single_calls(filt, theta, n, batch):
    # one launch over a batch of maps (ragged n: partial tiles on both axes)
    # against the oracle map by map, and against single-map calls
    fm = _fm()
    side = 1 << max(3, (n - 1).bit_length())
    maps = []
    for b in range(batch):
        g1, g2 = shear(side, seed=50 + b, dtype=np.float32)
        maps.append((np.ascontiguousarray(g1[:n, :n]), np.ascontiguousarray(g2[:n, :n])))
    t1 = torch.from_numpy(np.stack([m[0] for m in maps])).cuda()
    t2 = torch.from_numpy(np.stack([m[1] for m in maps])).cuda()
    out = fm.fm_map_direct(t1, t2, filt, theta).cpu().numpy()
    for b in range(batch):
        ref = oracle.map_direct(maps[b][0].astype(np.float64), maps[b][1].astype(np.float64), filt, theta)
        assert rel_err(out[b], ref) <= 1e-5
        one = fm.fm_map_direct(t1[b].contiguous(), t2[b].contiguous(), filt, theta).cpu().numpy()
        assert np.array_equal(one, out[b])


@pytest.mark.parametrize("form", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("theta", [6.0, 40.0])
def test_map_direct_kernel_forms_match_oracle(form, theta):
    # every kernel form of the unmasked fp32 sum (scalar FMAs, packed
    # two-lane FMAs in four tile shapes) on a ragged field; theta = 40 splits
    # each tile's input rows into parts summed by a second kernel, written
    # here into an output that is only 4-byte aligned
    fm = _fm()
    n = 160
    g1, g2 = shear(256, seed=61, dtype=np.float32)
    g1, g2 = np.ascontiguousarray(g1[:n, :n]), np.ascontiguousarray(g2[:n, :n])
    ref = oracle.map_direct(g1.astype(np.float64), g2.astype(np.float64), 1, theta)
    t1, t2 = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()
    base = torch.full((n * n + 1,), float("nan"), device="cuda")
    out = base[1:].view(n, n)
    fm.fm_tune(fm.FM_TUNE_DIRECT, form)
    try:
        m = fm.fm_map_direct(t1, t2, 1, theta).cpu().numpy()
        fm.fm_map_direct(t1, t2, 1, theta, out=out)
    finally:
        fm.fm_tune(fm.FM_TUNE_DIRECT, -1)
    assert rel_err(m, ref) <= 1e-5
    assert np.array_equal(out.cpu().numpy(), m)
