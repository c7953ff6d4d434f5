"""GPU autotuner: fm_autotune times candidate plans of the batched KS +
starlet call and keeps the fastest; the automatic configuration then runs
that plan, and its results match the oracle and the same plan requested
explicitly."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, band_errs, shear

pytestmark = pytest.mark.gpu


@pytest.fixture
def fm():
    from paper_1204_4293_gb300 import fastmap
    fastmap.fm_autotune_clear()
    yield fastmap
    fastmap.fm_autotune_clear()


@pytest.mark.parametrize("n,J,batch,dtype", [(256, 6, 8, np.float32), (128, 5, 3, np.float64),
                                             (1024, 7, 4, np.float32)])
def test_autotuned_plan_is_used_and_matches_oracle(fm, n, J, batch, dtype):
    prec = fm.FM_F32 if dtype == np.float32 else fm.FM_F64
    plan = fm.fm_autotune(n, J, batch, precision=prec)
    fmax = min(4 if dtype == np.float32 else 3, J - 1)
    assert 1 <= plan["fuse_depth"] <= fmax and plan["large_path"] in (1, 3, 4) and plan["tile"] in (0, 1)
    assert plan["chunk_mb"] in (24, 36, 48, 64, 96)
    assert 0 < plan["ms"] <= plan["default_ms"]  # the built-in plan is the first candidate
    assert fm.fm_autotune_get(n, J, prec) == plan
    assert fm.fm_starlet_fuse_depth(n, J, precision=prec) == plan["fuse_depth"]

    g1, g2 = shear(n, seed=21, dtype=np.float64)
    g1b = np.stack([np.roll(g1, 7 * b, axis=0) for b in range(batch)]).astype(dtype)
    g2b = np.stack([np.roll(g2, 7 * b, axis=0) for b in range(batch)]).astype(dtype)
    t1, t2 = torch.from_numpy(g1b).cuda(), torch.from_numpy(g2b).cuda()
    auto = fm.fm_map_starlet(t1, t2, J)
    explicit = fm.fm_map_starlet(t1, t2, J, fuse_depth=plan["fuse_depth"], large_path=plan["large_path"])
    assert torch.equal(auto, explicit)
    kappa = oracle.ks_invert(g1b[-1].astype(np.float64), g2b[-1].astype(np.float64))[0]
    ref = oracle.starlet(kappa, J)
    assert max(band_errs(auto[-1].cpu().numpy(), ref)) <= TOL[dtype]


def test_hand_set_plan_drives_every_automatic_choice(fm):
    """A plan entered by hand (shared-buffer tile form, fused column/row
    path, 40 MiB chunks, one fused scale) is what the automatic
    configuration runs: bit-identical to the same choices made explicitly,
    within tolerance of the oracle, and for the noise maps too."""
    n, J, batch = 512, 6, 6
    g1, g2 = shear(n, seed=5, dtype=np.float32)
    t1 = torch.from_numpy(np.stack([np.roll(g1, 11 * b, axis=1) for b in range(batch)])).cuda()
    t2 = torch.from_numpy(np.stack([np.roll(g2, 11 * b, axis=1) for b in range(batch)])).cuda()
    fm.fm_autotune_set(n, J, fuse_depth=1, large_path=3, tile=0, chunk_mb=40)
    auto = fm.fm_map_starlet(t1, t2, J)
    fm.fm_autotune_clear()
    fm.fm_tune(fm.FM_TUNE_TILE, 0)
    fm.fm_tune(fm.FM_TUNE_CHUNK_BYTES, 40 << 20)
    try:
        explicit = fm.fm_map_starlet(t1, t2, J, fuse_depth=1, large_path=3)
    finally:
        fm.fm_tune(fm.FM_TUNE_TILE, -1)
        fm.fm_tune(fm.FM_TUNE_CHUNK_BYTES, -1)
    assert torch.equal(auto, explicit)
    kappa = oracle.ks_invert(np.roll(g1, 11 * (batch - 1), axis=1).astype(np.float64),
                             np.roll(g2, 11 * (batch - 1), axis=1).astype(np.float64))[0]
    assert max(band_errs(auto[-1].cpu().numpy(), oracle.starlet(kappa, J))) <= TOL[np.float32]
    # noise maps follow the plan as well and stay within the variance bound
    fm.fm_autotune_set(n, J, fuse_depth=1, large_path=3, tile=0, chunk_mb=40)
    var, _ = fm.fm_map_noise(t1[0], t2[0], J, 5, seed=8, with_snr=False)
    rv, _ = oracle.map_noise(g1.astype(np.float64), g2.astype(np.float64), J, 5, 8, with_snr=False)
    var = var.cpu().numpy()
    for j in range(J - 1):
        assert np.abs(var[j] - rv[j]).max() / rv[j].mean() <= 1e-4
