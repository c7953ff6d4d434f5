"""Statistics of the aperture-mass maps on the GPU (Sec. 2.2, Sec. 4.4):
fm_band_moments against numpy, band variances against the discrete eq.
varmap at a larger size than the oracle check, and the Fig. 2 spectral
pattern from the GPU's direct M_ap maps."""
import numpy as np
import pytest
import torch

import oracle
from helpers import rel_err
from paper_1204_4293_gb300 import synth
from test_oracle_fig2_varmap import band_variance_prediction, check_fig2, fig2_maps

pytestmark = pytest.mark.gpu


def _fm():
    from paper_1204_4293_gb300 import fastmap
    return fastmap


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_band_moments_match_numpy(dtype):
    fm = _fm()
    n, J, batch = 200, 5, 3
    kap = torch.from_numpy(np.stack([synth.grf_kappa(n, seed=60 + b) + synth.white((n, n), seed=b, scale=0.01)
                                     for b in range(batch)])).to(dtype).cuda()
    pyr = fm.fm_starlet_forward(kap, J)
    mom = fm.fm_band_moments(pyr).cpu().numpy()
    x = pyr.double().cpu().numpy().reshape(batch, J, -1)
    mean = x.mean(-1)
    d = x - mean[..., None]
    var = (d ** 2).mean(-1)
    skew = (d ** 3).mean(-1) / var ** 1.5
    kurt = (d ** 4).mean(-1) / var ** 2 - 3
    tol = 2e-5 if dtype == torch.float32 else 1e-9
    assert np.allclose(mom[..., 1], var, rtol=tol * 10)
    assert np.allclose(mom[..., 0], mean, atol=tol * np.sqrt(var).max())
    assert np.allclose(mom[..., 2], skew, atol=1e-3)
    assert np.allclose(mom[..., 3], kurt, atol=1e-3)


def test_band_variance_follows_eq_varmap_gpu():
    fm = _fm()
    n, J, alpha, maps = 512, 7, 2.0, 8
    pred = band_variance_prediction(n, J, alpha)
    kap = torch.from_numpy(np.stack([synth.grf_kappa(n, alpha=alpha, rms=None, seed=900 + s)
                                     for s in range(maps)])).float().cuda()
    pyr = fm.fm_starlet_forward(kap, J, boundary=fm.FM_PERIODIC)
    got = fm.fm_band_moments(pyr)[..., 1].mean(0).cpu().numpy()
    rtol = [0.01, 0.02, 0.04, 0.08, 0.15, 0.3, 0.5]
    for j in range(J):
        assert abs(got[j] / pred[j] - 1) < rtol[j], (j, got / pred)


def test_fig2_oscillations_gpu_direct_maps():
    fm = _fm()
    n = 128
    g1, g2 = oracle.ks_forward(synth.delta_kappa(n))
    t1 = torch.from_numpy(g1.astype(np.float32)).cuda()
    t2 = torch.from_numpy(g2.astype(np.float32)).cuda()

    def gpu_map(a, b, f, theta, ell, cut):
        return fm.fm_map_direct(t1, t2, f, theta, ell=ell, cut_over_theta=cut).double().cpu().numpy()

    band2 = fm.fm_map_starlet(t1, t2, 4, boundary=fm.FM_PERIODIC)[1].double().cpu().numpy()
    maps = fig2_maps(g1, g2, gpu_map, band2)
    ref = fig2_maps(g1, g2, lambda a, b, f, t, l, c: oracle.map_direct(a, b, f, t, ell=l, cut_over_theta=c),
                    oracle.map_starlet(g1.astype(np.float32).astype(np.float64),
                                       g2.astype(np.float32).astype(np.float64), 4, oracle.PERIODIC)[1])
    for k in maps:
        if k != "starlet_band":
            assert rel_err(maps[k], ref[k]) <= 1e-4, k  # inputs differ by the fp32 rounding of the shear
    assert rel_err(maps["starlet_band"], ref["starlet_band"]) <= 1e-5
    check_fig2(maps)
