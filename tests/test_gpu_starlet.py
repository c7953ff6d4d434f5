"""GPU starlet transform (Sec. 3, Sec. 4.2) against the FP64 oracle.

Sizes span several 64-pixel tiles with ragged tails (n not a multiple of the
tile, n not a power of two), the smallest legal maps (n = 2^J), both
boundaries, every fusion depth, batches, and the degenerate constant map.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, band_errs
from paper_1204_4293_gb300 import synth

pytestmark = pytest.mark.gpu


def _fm():
    from paper_1204_4293_gb300 import fastmap
    return fastmap


CASES = [(4, 2), (8, 3), (16, 4), (37, 5), (64, 6), (100, 6), (200, 7), (256, 5), (130, 7), (128, 7), (512, 8)]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("n,J", CASES)
def test_starlet_matches_oracle(n, J, boundary, dtype):
    fm = _fm()
    kappa = synth.grf_kappa(n, seed=n + J) + synth.white((n, n), seed=J, scale=0.05)
    kappa = kappa.astype(dtype)
    ref = oracle.starlet(kappa.astype(np.float64), J, boundary)
    for fuse in sorted({-1, 1, 2, 3, J - 1}):
        if fuse > J - 1:
            continue
        for large_path in ((0, 1, 2, 3) if 0 < fuse < J - 1 else (0, 3)):
            pyr = fm.fm_starlet_forward(torch.from_numpy(kappa).cuda(), J, boundary=boundary, fuse_depth=fuse,
                                        large_path=large_path)
            errs = band_errs(pyr.cpu().numpy(), ref)
            assert max(errs) <= TOL[dtype], (fuse, large_path, errs)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_starlet_batch_and_reconstruction(dtype):
    fm = _fm()
    n, J, batch = 96, 6, 3
    maps = np.stack([synth.grf_kappa(n, seed=s) for s in range(batch)]).astype(dtype)
    pyr = fm.fm_starlet_forward(torch.from_numpy(maps).cuda(), J).cpu().numpy()
    assert pyr.shape == (batch, J, n, n)
    for b in range(batch):
        ref = oracle.starlet(maps[b].astype(np.float64), J)
        assert max(band_errs(pyr[b], ref)) <= TOL[dtype]
        # kappa = c_J + sum_j w_j (Sec. 3)
        rec = pyr[b].astype(np.float64).sum(axis=0)
        assert np.abs(rec - maps[b]).max() <= 1e-5 * np.abs(maps[b]).max()


def test_constant_map_gives_zero_bands():
    fm = _fm()
    kappa = torch.full((64, 64), 0.75, dtype=torch.float32, device="cuda")
    pyr = fm.fm_starlet_forward(kappa, 5).cpu().numpy()
    assert np.abs(pyr[:-1]).max() < 1e-6
    assert np.abs(pyr[-1] - 0.75).max() < 1e-6


def test_starlet_full_size_paper_config():
    # 1024 x 1024, J = 7 (theta = 2..64 px), a batch of maps as the benchmark runs it
    fm = _fm()
    n, J, batch = 1024, 7, 4
    maps = np.stack([synth.grf_kappa(n, seed=100 + b) for b in range(batch)]).astype(np.float32)
    pyr = fm.fm_starlet_forward(torch.from_numpy(maps).cuda(), J).cpu().numpy()
    for b in (0, batch - 1):
        ref = oracle.starlet(maps[b].astype(np.float64), J)
        errs = band_errs(pyr[b], ref)
        assert max(errs) <= 1e-5, errs


@pytest.mark.parametrize("n,J,dtype", [(2048, 8, np.float32), (4096, 6, np.float64)])
@pytest.mark.parametrize("boundary", [0, 1])
def test_starlet_wide_rows(n, J, dtype, boundary):
    # long rows at large scales (2048 fp32 and 4096 fp64 pixels per row)
    fm = _fm()
    kappa = (synth.grf_kappa(n, seed=n + 1) + synth.white((n, n), seed=3, scale=0.05)).astype(dtype)
    ref = oracle.starlet(kappa.astype(np.float64), J, boundary)
    pyr = fm.fm_starlet_forward(torch.from_numpy(kappa).cuda(), J, boundary=boundary).cpu().numpy()
    assert max(band_errs(pyr, ref)) <= TOL[dtype]


def test_starlet_8192_windows_match_oracle():
    # 8192^2, J = 9: c_8 sees at most 2 (2^8 - 1) = 510 pixels away, so on a
    # 2048^2 crop every pixel >= 510 from a cut edge (a map edge is no cut
    # edge: the crop keeps it and its mirror) equals the full map's value.
    fm = _fm()
    n, J, w, h = 8192, 9, 2048, 510
    kappa = synth.grf_kappa(n, alpha=2.5, seed=57).astype(np.float32)
    pyr = fm.fm_starlet_forward(torch.from_numpy(kappa).cuda(), J)
    for y0, x0 in [(0, 0), (3000, 5000), (n - w, n - w), (0, 4000)]:
        ref = oracle.starlet(kappa[y0:y0 + w, x0:x0 + w].astype(np.float64), J)
        ya = 0 if y0 == 0 else h
        yb = w if y0 + w == n else w - h
        xa = 0 if x0 == 0 else h
        xb = w if x0 + w == n else w - h
        got = pyr[:, y0 + ya:y0 + yb, x0 + xa:x0 + xb].cpu().numpy()
        errs = band_errs(got, ref[:, ya:yb, xa:xb])
        assert max(errs) <= 1e-5, ((y0, x0), errs)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("n,J", [(64, 5), (100, 6), (130, 7), (256, 6)])
def test_tile_kernel_variants(variant, n, J):
    # every fp32 form of the fused small-scale kernel, every fusion depth
    fm = _fm()
    kappa = (synth.grf_kappa(n, seed=n + 3 * J) + synth.white((n, n), seed=J, scale=0.05)).astype(np.float32)
    fm.fm_tune(fm.FM_TUNE_TILE, variant)
    try:
        for boundary in (0, 1):
            ref = oracle.starlet(kappa.astype(np.float64), J, boundary)
            for fuse in range(1, min(4, J - 1) + 1):
                pyr = fm.fm_starlet_forward(torch.from_numpy(kappa).cuda(), J, boundary=boundary, fuse_depth=fuse)
                assert max(band_errs(pyr.cpu().numpy(), ref)) <= TOL[np.float32], (boundary, fuse)
    finally:
        fm.fm_tune(fm.FM_TUNE_TILE, -1)


@pytest.mark.parametrize("n,J,batch,boundary", [(256, 5, 3, 0), (1024, 7, 2, 0), (1024, 7, 2, 1), (200, 4, 1, 0),
                                                 (968, 6, 2, 0), (968, 6, 2, 1), (1000, 7, 1, 1), (4096, 9, 1, 0)])
def test_bulk_copy_halo_equals_thread_loads(n, J, batch, boundary):
    # tiles take their halo box (edge tiles: then folded in shared memory),
    # and interior column-pass row groups their window and c_{j-1} rows, by
    # bulk tensor copies (default) or by per-thread loads: identical
    # pyramids for every fused depth, both boundaries and ragged maps (968:
    # the last tile's far halo folds outside its box), no wait ran out
    fm = _fm()
    maps = np.stack([synth.grf_kappa(n, seed=7 + b) for b in range(batch)]).astype(np.float32)
    kap = torch.from_numpy(maps).cuda()
    for fuse in range(1, min(3, J - 1) + 1):
        fm.fm_tune(fm.FM_TUNE_TMA, 63)
        with_tma = fm.fm_starlet_forward(kap, J, boundary=boundary, fuse_depth=fuse)
        fm.fm_tune(fm.FM_TUNE_TMA, 0)
        try:
            without = fm.fm_starlet_forward(kap, J, boundary=boundary, fuse_depth=fuse)
        finally:
            fm.fm_tune(fm.FM_TUNE_TMA, -1)
        torch.cuda.synchronize()
        assert fm.fm_device_error() == 0
        assert torch.equal(with_tma, without), fuse
    ref = oracle.starlet(maps[batch - 1].astype(np.float64), J, boundary)
    assert max(band_errs(with_tma[batch - 1].cpu().numpy(), ref)) <= 1e-5


@pytest.mark.parametrize("n,J,batch,boundary,dtype", [(1024, 7, 4, 0, np.float32), (2048, 8, 1, 0, np.float32),
                                                      (4096, 9, 1, 0, np.float32), (512, 6, 3, 1, np.float32),
                                                      (1000, 7, 2, 0, np.float32), (512, 7, 2, 0, np.float64),
                                                      (8192, 7, 1, 1, np.float32)])
def test_fused_column_row_pass_is_bit_exact(n, J, batch, boundary, dtype):
    """The column pass of each large scale fused with the next scale's row
    pass (large_path 3; automatic on maps up to 256^2) computes the same sums in the same order as the separate row and column
    kernels (large_path 1): bit-identical pyramids, with the pyramid's
    smooth-array slot used as scratch and then overwritten."""
    fm = _fm()
    kappa = torch.from_numpy(np.stack([synth.grf_kappa(n, seed=7 + b) for b in range(batch)]).astype(dtype)).cuda()
    ref = fm.fm_starlet_forward(kappa, J, boundary=boundary, large_path=1)
    for lp in (0, 3):
        got = fm.fm_starlet_forward(kappa, J, boundary=boundary, large_path=lp)
        assert torch.equal(got, ref), (lp, (got - ref).abs().max().item())
    plain = fm.fm_starlet_forward(kappa, J, boundary=boundary, fuse_depth=-1, large_path=3)
    assert torch.equal(plain, fm.fm_starlet_forward(kappa, J, boundary=boundary, fuse_depth=-1, large_path=1))
    # the oracle on one sampled map
    r = oracle.starlet(kappa[-1].double().cpu().numpy(), J, boundary) if n <= 1024 else None
    if r is not None:
        assert max(band_errs(ref[-1].cpu().numpy(), r)) <= TOL[dtype]


@pytest.mark.parametrize("n,J,batch,boundary", [(4096, 9, 1, 0), (2048, 8, 2, 1), (512, 7, 3, 0), (1024, 7, 2, 1),
                                                (8192, 9, 1, 0)])
def test_one_pass_large_scales_match_two_pass(n, J, batch, boundary):
    # large_path 4 (each large scale in one pass, the row filter from shared
    # memory, bulk tensor copies of the window rows, mirrored or wrapped halo
    # columns at the strip edges) against the row + column passes, and the
    # oracle on the first map where it finishes quickly
    from paper_1204_4293_gb300 import fastmap as fm
    g = torch.Generator(device="cuda").manual_seed(n + J)
    kap = torch.empty((batch, n, n), device="cuda").normal_(0, 0.02, generator=g)
    a = fm.fm_starlet_forward(kap, J, boundary=boundary, large_path=4)
    b = fm.fm_starlet_forward(kap, J, boundary=boundary, large_path=1)
    torch.cuda.synchronize()
    assert fm.fm_device_error() == 0
    for m in range(batch):
        errs = band_errs(a[m].double().cpu().numpy(), b[m].double().cpu().numpy())
        assert max(errs) <= 1e-6, errs
    if n <= 1024:
        ref = oracle.starlet(kap[0].double().cpu().numpy(), J, boundary)
        assert max(band_errs(a[0].cpu().numpy(), ref)) <= 1e-5
