"""GPU exact expected noise variance (Sec. 1; periodic boundary) against the
FP64 oracle: full maps at small sizes (the generic FFT path below n = 32 and
the radix-32 path above), sampled pixels of a 1024^2 map, the Parseval closed
form for a uniform |gamma|, and the GPU's own Monte-Carlo noise maps, which
must scatter around it with the spread of a sample variance.

Error metric: max |var_gpu - var_oracle| / mean(var_oracle) per band, bound
1e-4 in fp32 (the variance bound of the noise maps) and 1e-10 in fp64.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1204_4293_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {np.float32: 1e-4, np.float64: 1e-10}


def _fm():
    from paper_1204_4293_gb300 import fastmap
    return fastmap


def _shear(n, seed, dtype):
    g1, g2 = oracle.ks_forward(synth.grf_kappa(n, seed=seed))
    s1, s2 = synth.shape_noise(n, 0.1, seed=seed)
    g1, g2 = g1 + s1, g2 + s2
    g1[: n // 4] *= 2.0  # position-dependent |gamma|
    return g1.astype(dtype), g2.astype(dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,J", [(16, 3), (64, 5), (128, 6)])
def test_expected_variance_matches_oracle(n, J, dtype):
    fm = _fm()
    g1, g2 = _shear(n, n + J, dtype)
    ref = oracle.map_noise_expected(g1.astype(np.float64), g2.astype(np.float64), J)
    var = fm.fm_map_noise_expected(torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda(), J).cpu().numpy()
    for j in range(J - 1):
        err = np.abs(var[j] - ref[j]).max() / ref[j].mean()
        assert err <= TOL[dtype], (j, err)


def test_expected_variance_1024_sampled():
    fm = _fm()
    n, J = 1024, 7
    g1, g2 = _shear(n, 3, np.float32)
    var = fm.fm_map_noise_expected(torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda(), J).cpu().numpy()
    rng = np.random.default_rng(0)
    ys = np.concatenate([rng.integers(0, n, 60), [0, n - 1, 255, 256]])
    xs = np.concatenate([rng.integers(0, n, 60), [0, n - 1, 7, 1000]])
    ref = oracle.map_noise_expected_at(g1.astype(np.float64), g2.astype(np.float64), J, ys, xs)
    for j in range(J - 1):
        err = np.abs(var[j][ys, xs] - ref[j]).max() / ref[j].mean()
        assert err <= TOL[np.float32], (j, err)


def test_uniform_modulus_closed_form_on_gpu():
    # |gamma|^2 = c everywhere: Var_j = (c / 2n^2) sum_{k != 0} H_j(k)^2 (Parseval)
    fm = _fm()
    n, J = 256, 6
    ang = np.random.default_rng(1).uniform(0, 2 * np.pi, (n, n))
    g1, g2 = (0.2 * np.cos(ang)).astype(np.float32), (0.2 * np.sin(ang)).astype(np.float32)
    var = fm.fm_map_noise_expected(torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda(), J).cpu().numpy()
    k = np.arange(n)
    phi_prev = np.ones((n, n))
    for j in range(1, J):
        s = 2 ** (j - 1)
        h = (6 + 8 * np.cos(2 * np.pi * k * s / n) + 2 * np.cos(2 * np.pi * k * 2 * s / n)) / 16
        phi = phi_prev * np.outer(h, h)
        H = phi_prev - phi
        H[0, 0] = 0.0
        want = 0.5 * 0.04 * (H ** 2).sum() / n ** 2
        assert np.abs(var[j - 1] - want).max() <= 1e-4 * want, j
        phi_prev = phi


def test_gpu_monte_carlo_scatters_around_expectation():
    fm = _fm()
    n, J, R = 256, 5, 400
    g1, g2 = _shear(n, 8, np.float32)
    t1, t2 = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()
    exp = fm.fm_map_noise_expected(t1, t2, J).double().cpu().numpy()
    mc, _ = fm.fm_map_noise(t1, t2, J, R, seed=21, boundary=fm.FM_PERIODIC, with_snr=False)
    mc = mc.cpu().numpy()
    sd = np.sqrt(2.0 / (R - 1))
    for j in range(J - 1):
        ratio = mc[j] / exp[j]
        assert abs(ratio.mean() - 1.0) < 0.5 * sd, (j, ratio.mean())
        assert 0.8 * sd < ratio.std() < 1.2 * sd, (j, ratio.std())


def test_mirror_boundary_is_refused():
    fm = _fm()
    g = torch.zeros((64, 64), device="cuda")
    c = fm._cfg(0, fm.FM_MIRROR)
    var = torch.empty((3, 64, 64), device="cuda")
    st = fm.lib.fm_map_noise_expected(fm._ptr(g), fm._ptr(g), fm._ptr(var), 64, 4, fm.ctypes.byref(c), None)
    assert st == fm.FM_EINVAL


def test_noise_maps_at_the_benchmark_size_match_the_expectation():
    # the noise configuration the benchmark times (1024^2, J = 7, R = 1000, one
    # CUDA-graph launch), periodic boundary: the Monte-Carlo variance scatters
    # around the exact expectation (itself checked against the oracle at
    # sampled 1024^2 pixels above) with the spread of a sample variance
    fm = _fm()
    n, J, R = 1024, 7, 1000
    g1, g2 = _shear(n, 5, np.float32)
    t1, t2 = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()
    exp = fm.fm_map_noise_expected(t1, t2, J).double()
    var, snr = fm.fm_map_noise(t1, t2, J, R, seed=9, boundary=fm.FM_PERIODIC)
    assert fm.fm_device_error() == 0
    sd = np.sqrt(2.0 / (R - 1))
    for j in range(J - 1):
        ratio = (var[j] / exp[j]).cpu().numpy()
        assert abs(ratio.mean() - 1.0) < 0.5 * sd, (j, ratio.mean())
        assert 0.8 * sd < ratio.std() < 1.2 * sd, (j, ratio.std())
    assert torch.isfinite(snr).all()
