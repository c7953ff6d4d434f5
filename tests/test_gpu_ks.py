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
