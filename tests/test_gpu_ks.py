"""GPU Kaiser-Squires (Sec. 4.5) against the FP64 oracle, element by element."""
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
@pytest.mark.parametrize("n,batch", [(4, 1), (8, 3), (16, 2), (64, 1), (128, 3), (256, 2), (2048, 1)])
def test_ks_invert_matches_oracle(n, batch, dtype):
    fm = _fm()
    maps = [shear(n, seed=10 + b, dtype=dtype) for b in range(batch)]
    g1 = torch.from_numpy(np.stack([m[0] for m in maps])).cuda()
    g2 = torch.from_numpy(np.stack([m[1] for m in maps])).cuda()
    kE, kB = fm.fm_ks_invert(g1, g2, with_b=True)
    kE, kB = kE.cpu().numpy(), kB.cpu().numpy()
    for b in range(batch):
        rE, rB = oracle.ks_invert(maps[b][0].astype(np.float64), maps[b][1].astype(np.float64))
        assert rel_err(kE[b], rE) <= TOL[dtype]
        # B-mode: shape noise only, same scale as E
        assert rel_err(kB[b], rB) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", [8, 64, 512, 2048])
def test_ks_forward_matches_oracle(n, dtype):
    fm = _fm()
    from paper_1204_4293_gb300 import synth
    kappa = synth.grf_kappa(n, seed=n).astype(dtype)
    g1, g2 = fm.fm_ks_forward(torch.from_numpy(kappa).cuda())
    r1, r2 = oracle.ks_forward(kappa.astype(np.float64))
    assert rel_err(g1.cpu().numpy(), r1) <= TOL[dtype]
    assert rel_err(g2.cpu().numpy(), r2) <= TOL[dtype]


def test_ks_8192_round_trip():
    # largest supported size, GPU against itself: forward then inverse gives
    # kappa back and no B-mode (the oracle comparison at this size is in
    # test_gpu_pipeline.py)
    fm = _fm()
    from paper_1204_4293_gb300 import synth
    n = 8192
    kappa = torch.from_numpy(synth.grf_kappa(n, alpha=2.5, seed=56).astype(np.float32)).cuda()
    g1, g2 = fm.fm_ks_forward(kappa)
    kE, kB = fm.fm_ks_invert(g1, g2, with_b=True)
    rms = kappa.double().pow(2).mean().sqrt().item()
    assert (kE - kappa).abs().max().item() / rms < 1e-5
    assert kB.abs().max().item() / rms < 1e-5


@pytest.mark.parametrize("n,batch", [(64, 3), (256, 2), (1024, 2), (2048, 1), (4096, 1), (8192, 1)])
def test_bulk_copy_rows_equal_thread_loads(n, batch):
    # the FFT kernels take their rows (row passes) and column strips (column
    # pass) by bulk tensor copies or by per-thread loads: identical results,
    # also for the rotated noise rows (one broadcast input map), and no wait
    # ran out
    fm = _fm()
    g1 = torch.empty((batch, n, n), device="cuda").normal_(0, 0.1)
    g2 = torch.empty_like(g1).normal_(0, 0.1)
    outs = {}
    for tma in (127, 0):
        fm.fm_tune(fm.FM_TUNE_TMA, tma)
        try:
            kE, kB = fm.fm_ks_invert(g1, g2, with_b=True)
            var, _ = fm.fm_map_noise(g1[0], g2[0], 4, 3, seed=5, with_snr=False)
            outs[tma] = (kE, kB, var)
        finally:
            fm.fm_tune(fm.FM_TUNE_TMA, -1)
    torch.cuda.synchronize()
    assert fm.fm_device_error() == 0
    for a, b in zip(outs[127], outs[0]):
        assert torch.equal(a, b)


@pytest.mark.parametrize("n,batch", [(32, 2), (64, 3), (128, 1), (256, 2), (512, 2), (1024, 2), (2048, 1), (4096, 1),
                                     (8192, 1)])
def test_ks_invert_real_output_matches_oracle(n, batch):
    # kappa_E alone takes the real-output inverse (half spectrum, Nyquist row
    # and column by conj(D) Gamma1, complex-to-real rows): against the FP64
    # oracle, and against the complex inverse's real part (FM_TUNE_KS_REAL 0)
    fm = _fm()
    maps = [shear(n, seed=70 + b, dtype=np.float32) for b in range(batch)]
    g1 = torch.from_numpy(np.stack([m[0] for m in maps])).cuda()
    g2 = torch.from_numpy(np.stack([m[1] for m in maps])).cuda()
    try:
        fm.fm_tune(fm.FM_TUNE_KS_REAL, 1)  # every size that has it (n >= 64)
        kE, kB = fm.fm_ks_invert(g1, g2)
        fm.fm_tune(fm.FM_TUNE_KS_REAL, 0)
        kC, _ = fm.fm_ks_invert(g1, g2)
    finally:
        fm.fm_tune(fm.FM_TUNE_KS_REAL, -1)
    assert kB is None
    torch.cuda.synchronize()
    assert fm.fm_device_error() == 0
    kE, kC = kE.cpu().numpy(), kC.cpu().numpy()
    for b in range(batch):
        rE, _ = oracle.ks_invert(maps[b][0].astype(np.float64), maps[b][1].astype(np.float64))
        assert rel_err(kE[b], rE) <= TOL[np.float32]
        assert rel_err(kE[b], kC[b]) <= 2e-6


def test_ks_real_output_nyquist_and_corner_modes():
    # shear made of single Fourier modes on the Nyquist row and column, at the
    # corners and on the axes (where the Hermitian part of conj(D) gamma_hat
    # departs from Re(D) Gamma1 + Im(D) Gamma2), plus a generic mode
    fm = _fm()
    n = 256
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    maps = []
    for (kx, ky) in ((n // 2, 3), (5, n // 2), (n // 2, n // 2), (n // 2, 0), (0, n // 2), (0, 7), (9, 0), (17, 40)):
        ph = 2 * np.pi * (kx * x + ky * y) / n
        maps.append((np.cos(ph + 0.3), np.sin(2 * ph + 1.1) + 0.5 * np.cos(ph - 0.7)))
    g1 = torch.from_numpy(np.stack([m[0] for m in maps]).astype(np.float32)).cuda()
    g2 = torch.from_numpy(np.stack([m[1] for m in maps]).astype(np.float32)).cuda()
    fm.fm_tune(fm.FM_TUNE_KS_REAL, 1)
    try:
        kE, _ = fm.fm_ks_invert(g1, g2)
    finally:
        fm.fm_tune(fm.FM_TUNE_KS_REAL, -1)
    kE = kE.cpu().numpy()
    for b, m in enumerate(maps):
        rE, _ = oracle.ks_invert(m[0], m[1])
        scale = max(np.sqrt(np.mean(rE ** 2)), 1e-3)
        assert np.abs(kE[b] - rE).max() / scale <= 1e-5, b


@pytest.mark.parametrize("n,batch", [(64, 3), (256, 2), (1024, 2), (4096, 1), (8192, 1)])
def test_real_output_bulk_copies_equal_thread_loads(n, batch):
    fm = _fm()
    g1 = torch.empty((batch, n, n), device="cuda").normal_(0, 0.1)
    g2 = torch.empty_like(g1).normal_(0, 0.1)
    outs = {}
    fm.fm_tune(fm.FM_TUNE_KS_REAL, 1)
    for tma in (127, 0):
        fm.fm_tune(fm.FM_TUNE_TMA, tma)
        try:
            outs[tma] = fm.fm_ks_invert(g1, g2)[0]
        finally:
            fm.fm_tune(fm.FM_TUNE_TMA, -1)
    fm.fm_tune(fm.FM_TUNE_KS_REAL, -1)
    torch.cuda.synchronize()
    assert fm.fm_device_error() == 0
    assert torch.equal(outs[127], outs[0])


@pytest.mark.parametrize("n,J,batch", [(1024, 7, 9), (256, 5, 3)])
def test_pipeline_real_output_inverse_matches_complex(n, J, batch):
    # the batched KS + starlet chunks (graph replay, two streams) and a noise
    # map with the real-output inverse forced on, against the complex inverse
    fm = _fm()
    g1 = torch.empty((batch, n, n), device="cuda").normal_(0, 0.1)
    g2 = torch.empty_like(g1).normal_(0, 0.1)
    out = {}
    for real in (1, 0):
        fm.fm_tune(fm.FM_TUNE_KS_REAL, real)
        try:
            pyr = fm.fm_map_starlet(g1, g2, J)
            var, _ = fm.fm_map_noise(g1[0], g2[0], J, 5, seed=8, with_snr=False)
            out[real] = (pyr.double().cpu().numpy(), var.cpu().numpy())
        finally:
            fm.fm_tune(fm.FM_TUNE_KS_REAL, -1)
    for b in range(batch):
        for j in range(J):
            a, c = out[1][0][b, j], out[0][0][b, j]
            assert np.abs(a - c).max() / np.sqrt(np.mean(c ** 2)) <= 1e-5
    for j in range(J - 1):
        a, c = out[1][1][j], out[0][1][j]
        assert np.abs(a - c).max() / c.mean() <= 1e-5
    fm.fm_trim()
