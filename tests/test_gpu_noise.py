"""GPU noise maps by randomised shear (Sec. 1) against the oracle: the same
counter-based generator on both sides makes the realisations identical up to
rounding, so variances agree to the stated 1e-4 (relative to the band's mean
variance) and S/N maps to the fp32 band tolerance."""
import numpy as np
import pytest
import torch

import oracle
from helpers import shear

pytestmark = pytest.mark.gpu


def _fm():
    from paper_1204_4293_gb300 import fastmap
    return fastmap


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,J,R,boundary", [(16, 3, 5, 0), (32, 4, 23, 1), (64, 5, 40, 0)])
def test_noise_matches_oracle(n, J, R, boundary, dtype):
    fm = _fm()
    g1, g2 = shear(n, seed=7, dtype=dtype)
    var, snr = fm.fm_map_noise(torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda(), J, R, seed=1234,
                               boundary=boundary)
    rv, rs = oracle.map_noise(g1.astype(np.float64), g2.astype(np.float64), J, R, 1234, boundary)
    var, snr = var.cpu().numpy(), snr.cpu().numpy()
    tol = 1e-4 if dtype == np.float32 else 1e-10
    for j in range(J - 1):
        assert np.abs(var[j] - rv[j]).max() / rv[j].mean() <= tol
        assert np.abs(snr[j] - rs[j]).max() / np.sqrt(np.mean(rs[j] ** 2)) <= 10 * tol


def test_noise_paper_size_few_realisations():
    # 1024^2 J = 7 in the launch configuration of the noise benchmark, with R = 3
    # so the oracle finishes; the realisation loop is the same at R = 1000.
    fm = _fm()
    n, J, R = 1024, 7, 3
    g1, g2 = shear(n, seed=3, dtype=np.float32)
    var, _ = fm.fm_map_noise(torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda(), J, R, seed=99,
                             with_snr=False)
    rv, _ = oracle.map_noise(g1.astype(np.float64), g2.astype(np.float64), J, R, 99, with_snr=False)
    var = var.cpu().numpy()
    for j in range(J - 1):
        assert np.abs(var[j] - rv[j]).max() / rv[j].mean() <= 1e-4


def test_noise_bench_config_mirror_two_batches():
    # the noise benchmark's configuration (1024^2, J = 7, mirror boundary,
    # one graph-replayed fm_map_noise call) at R = 40: a full batch of 32
    # realisations and a ragged one of 8 in the two alternating pyramid
    # buffers, as in the R = 1000 run, against the oracle
    fm = _fm()
    n, J, R = 1024, 7, 40
    g1, g2 = shear(n, seed=3, dtype=np.float32)
    t1, t2 = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()
    fm.fm_map_noise(t1, t2, J, R, seed=3)  # records the graph
    var, snr = fm.fm_map_noise(t1, t2, J, R, seed=3)  # replays it
    rv, rs = oracle.map_noise(g1.astype(np.float64), g2.astype(np.float64), J, R, 3, oracle.MIRROR)
    var, snr = var.cpu().numpy(), snr.cpu().numpy()
    for j in range(J - 1):
        assert np.abs(var[j] - rv[j]).max() / rv[j].mean() <= 1e-4, j
        assert np.abs(snr[j] - rs[j]).max() / np.sqrt(np.mean(rs[j] ** 2)) <= 1e-3, j
    fm.fm_trim()


def test_noise_graph_replay_matches_eager_launches():
    # fm_map_noise records the whole call into a CUDA graph and replays it;
    # the replay, a second replay and eager launches must agree (the
    # accumulation order is fixed, so in practice bit for bit)
    fm = _fm()
    n, J, R = 128, 5, 40
    g1, g2 = shear(n, seed=9, dtype=np.float32)
    t1, t2 = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()
    var = torch.empty(J - 1, n, n, dtype=torch.float64, device="cuda")
    snr = torch.empty(J - 1, n, n, dtype=torch.float32, device="cuda")
    c = fm._cfg(fm.FM_F32)
    import ctypes
    args = (ctypes.c_void_p(t1.data_ptr()), ctypes.c_void_p(t2.data_ptr()), ctypes.c_void_p(var.data_ptr()),
            ctypes.c_void_p(snr.data_ptr()), n, J, R, ctypes.c_uint64(5), ctypes.byref(c),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert fm.lib.fm_map_noise(*args) == 0
    first = var.clone()
    assert fm.lib.fm_map_noise(*args) == 0  # replay
    second = var.clone()
    fm.fm_tune(fm.FM_TUNE_GRAPHS, 0)
    try:
        assert fm.lib.fm_map_noise(*args) == 0  # eager
    finally:
        fm.fm_tune(fm.FM_TUNE_GRAPHS, -1)
    torch.cuda.synchronize()
    for other in (second, var):
        assert torch.allclose(first, other, rtol=1e-12, atol=0)
    fm.fm_trim()


@pytest.mark.parametrize("n,J,R,boundary", [(32, 4, 23, 1), (64, 5, 40, 0), (1024, 7, 3, 0)])
def test_noise_kahan_fp32_sums_match_oracle(n, J, R, boundary):
    """accum = 1: fp32 running sums with Kahan compensation instead of FP64;
    the variance stays within the same 1e-4 of the FP64 oracle."""
    fm = _fm()
    g1, g2 = shear(n, seed=11, dtype=np.float32)
    var, snr = fm.fm_map_noise(torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda(), J, R, seed=77,
                               boundary=boundary, accum=1)
    rv, rs = oracle.map_noise(g1.astype(np.float64), g2.astype(np.float64), J, R, 77, boundary)
    var, snr = var.cpu().numpy(), snr.cpu().numpy()
    for j in range(J - 1):
        assert np.abs(var[j] - rv[j]).max() / rv[j].mean() <= 1e-4
        if R >= 20:  # with 3 realisations some pixels' sigma is near 0 and S/N is ill-conditioned
            assert np.abs(snr[j] - rs[j]).max() / np.sqrt(np.mean(rs[j] ** 2)) <= 1e-3


def test_noise_kahan_and_fp64_sums_agree_over_many_batches():
    """R = 300 realisations (ten accumulation batches of at most 32): the
    compensated fp32 sums give the FP64 sums' variance to ~1e-6."""
    fm = _fm()
    n, J, R = 256, 5, 300
    g1, g2 = shear(n, seed=12, dtype=np.float32)
    t1, t2 = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()
    v64, _ = fm.fm_map_noise(t1, t2, J, R, seed=5, with_snr=False)
    vk, _ = fm.fm_map_noise(t1, t2, J, R, seed=5, with_snr=False, accum=1)
    for j in range(J - 1):
        rel = ((vk[j] - v64[j]).abs().max() / v64[j].mean()).item()
        assert rel <= 1e-5, (j, rel)
    fm.fm_trim()


def test_noise_in_parts_equals_one_call():
    """Realisations accumulated in parts (checkpoint / resume, or ranges
    split over GPUs: the sums of disjoint ranges add) give fm_map_noise's
    variance and S/N up to the grouping of the fp32 partial sums."""
    fm = _fm()
    n, J, R = 128, 5, 40
    g1, g2 = shear(n, seed=13, dtype=np.float32)
    t1, t2 = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()
    var, snr = fm.fm_map_noise(t1, t2, J, R, seed=21)
    sums = fm.fm_map_noise_accumulate(t1, t2, J, 0, 15, seed=21)  # resume after 15 realisations
    sums = fm.fm_map_noise_accumulate(t1, t2, J, 15, R - 15, seed=21, sums=sums)
    pyr = fm.fm_map_starlet(t1, t2, J)
    v2, s2 = fm.fm_noise_finalize(sums, R, pyramid=pyr)
    a = fm.fm_map_noise_accumulate(t1, t2, J, 0, 20, seed=21)  # two "ranks"
    b = fm.fm_map_noise_accumulate(t1, t2, J, 20, 20, seed=21)
    v3, _ = fm.fm_noise_finalize(a + b, R)
    for j in range(J - 1):
        ref = var[j].mean().item()
        assert (v2[j] - var[j]).abs().max().item() / ref <= 1e-5
        assert (v3[j] - var[j]).abs().max().item() / ref <= 1e-5
        assert (s2[j] - snr[j]).abs().max().item() / snr[j].pow(2).mean().sqrt().item() <= 1e-4
    fm.fm_trim()


def test_noise_accumulate_scratch_excludes_the_sums():
    """A partial accumulation adds to the caller's sums, so its scratch is the
    eager fm_map_noise call's minus the FP64 sums (2 (J-1) n^2 doubles)."""
    fm = _fm()
    n, J, R = 256, 6, 4
    g1, g2 = shear(n, seed=14, dtype=np.float32)
    t1, t2 = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()
    fm.fm_tune(fm.FM_TUNE_GRAPHS, 0)  # the eager call takes one stream-ordered scratch block
    try:
        fm.fm_alloc_stats(reset=True)
        fm.fm_map_noise(t1, t2, J, R, seed=1)
        _, whole = fm.fm_alloc_stats(reset=True)
    finally:
        fm.fm_tune(fm.FM_TUNE_GRAPHS, -1)
    sums = torch.zeros(2, J - 1, n, n, dtype=torch.float64, device="cuda")
    fm.fm_alloc_stats(reset=True)
    fm.fm_map_noise_accumulate(t1, t2, J, 0, R, seed=1, sums=sums)
    count, part = fm.fm_alloc_stats()
    torch.cuda.synchronize()
    assert count == 1
    assert whole - part == 2 * (J - 1) * n * n * 8
