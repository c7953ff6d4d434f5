"""C-ABI behaviour on the GPU: errors come back as status codes, launches are
counted, the profiling hook times a selected kernel, and serving gives each
request the same result alone and in a concurrent mix."""
import ctypes

import numpy as np
import pytest
import torch

from helpers import shear

pytestmark = pytest.mark.gpu


def _fm():
    from paper_1204_4293_gb300 import fastmap
    return fastmap


def test_invalid_arguments_return_einval():
    fm = _fm()
    x = torch.zeros(2, 48, 48, device="cuda")
    with pytest.raises(fm.FastmapError) as e:
        fm.fm_ks_invert(x, x)  # 48 is not a power of two
    assert e.value.status == fm.FM_EINVAL
    with pytest.raises(fm.FastmapError):
        fm.fm_starlet_forward(torch.zeros(16, 16, device="cuda"), 5)  # n < 2^J
    c = fm._cfg(0)
    assert fm.lib.fm_map_direct(None, None, None, 16, 9, 2.0, 3, 0.0, ctypes.byref(c), None) == fm.FM_EINVAL
    # the context is still healthy
    y = fm.fm_starlet_forward(torch.ones(32, 32, device="cuda"), 3)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()


def test_launch_count_and_profile_hook():
    fm = _fm()
    g1 = torch.randn(4, 256, 256, device="cuda")
    g2 = torch.randn(4, 256, 256, device="cuda")
    fm.fm_map_starlet(g1, g2, 6)
    c0 = fm.fm_launch_count()
    fm.fm_profile_select("fft_cols_ks")
    for _ in range(3):
        fm.fm_map_starlet(g1, g2, 6)
    ms, cnt = fm.fm_profile_read()
    fm.fm_profile_select(0)
    assert cnt == 3 and ms > 0
    assert fm.fm_launch_count() - c0 >= 3 * 5


def test_serving_mix_equals_alone():
    fm = _fm()
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(10):
        n = int(rng.choice([64, 128, 256]))
        J = int(np.log2(n)) - 2
        R = int(rng.choice([0, 0, 4]))
        g1, g2 = shear(n, seed=30 + i, dtype=np.float32)
        reqs.append((torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda(), J, R))
    alone = []
    for g1, g2, J, R in reqs:
        pyr = fm.fm_map_starlet(g1, g2, J)
        var = fm.fm_map_noise(g1, g2, J, R, seed=77, with_snr=False)[0] if R else None
        alone.append((pyr, var))
    torch.cuda.synchronize()
    with fm.Server(mem_budget_bytes=64 << 20, max_slots=4) as sv:
        outs, tickets = [], []
        for g1, g2, J, R in reqs:
            n = g1.shape[-1]
            pyr = torch.empty(J, n, n, device="cuda")
            var = torch.empty(J - 1, n, n, dtype=torch.float64, device="cuda") if R else None
            tickets.append(sv.submit(g1, g2, J, pyr, R=R, seed=77, out_var=var))
            outs.append((pyr, var))
        res = [sv.wait(t, 60.0) for t in tickets]
    assert all(r.status == fm.FM_OK for r in res)
    assert all(r.t_submit_ns <= r.t_admit_ns <= r.t_done_ns for r in res)
    for (pa, va), (pb, vb) in zip(alone, outs):
        assert torch.equal(pa, pb)
        if va is not None:
            assert torch.allclose(va, vb, rtol=1e-12, atol=0)


def test_serving_rejects_over_budget():
    fm = _fm()
    g1 = torch.zeros(512, 512, device="cuda")
    pyr = torch.empty(7, 512, 512, device="cuda")
    with fm.Server(mem_budget_bytes=1 << 20, max_slots=2) as sv:
        res = sv.wait(sv.submit(g1, g1, 7, pyr), 30.0)
    assert res.status == fm.FM_EBUDGET


def test_graph_cache_eviction_and_trim_keep_results():
    # more batched calls with distinct keys than the cache keeps (LRU
    # eviction), then fm_trim and a replay: every result equals the eager one
    from paper_1204_4293_gb300 import fastmap as fm
    n, J = 256, 5
    per_map = n * n * 4 * 5
    fm.fm_tune(fm.FM_TUNE_CHUNK_BYTES, 2 * per_map)  # chunks of 2 maps: every call below is multi-chunk
    try:
        calls = []
        for batch in (3, 4, 5, 6, 7, 8):
            g1 = torch.empty((batch, n, n), device="cuda").normal_(0, 0.1)
            g2 = torch.empty_like(g1).normal_(0, 0.1)
            calls.append((g1, g2))
        fm.fm_tune(fm.FM_TUNE_GRAPHS, 0)
        eager = [fm.fm_map_starlet(g1, g2, J) for g1, g2 in calls]
        fm.fm_tune(fm.FM_TUNE_GRAPHS, 1)
        for _ in range(2):  # record (evicting), then replay what is left
            for (g1, g2), ref in zip(calls, eager):
                assert torch.equal(fm.fm_map_starlet(g1, g2, J), ref)
        fm.fm_trim()
        g1, g2 = calls[0]
        assert torch.equal(fm.fm_map_starlet(g1, g2, J), eager[0])
    finally:
        for knob in (fm.FM_TUNE_CHUNK_BYTES, fm.FM_TUNE_GRAPHS):
            fm.fm_tune(knob, -1)
        fm.fm_trim()


def test_noise_graph_cache_eviction():
    # three noise calls with distinct keys (the cache keeps two) recorded and
    # replayed; each equals the eager call on the same inputs
    from paper_1204_4293_gb300 import fastmap as fm
    n, J = 128, 4
    g1 = torch.empty((n, n), device="cuda").normal_(0, 0.1)
    g2 = torch.empty_like(g1).normal_(0, 0.1)
    keys = [(10, 1), (12, 2), (10, 3)]
    fm.fm_tune(fm.FM_TUNE_GRAPHS, 0)
    try:
        eager = [fm.fm_map_noise(g1, g2, J, R, seed=s) for R, s in keys]
    finally:
        fm.fm_tune(fm.FM_TUNE_GRAPHS, -1)
    for _ in range(2):
        for (R, s), (v_ref, snr_ref) in zip(keys, eager):
            v, snr = fm.fm_map_noise(g1, g2, J, R, seed=s)
            assert torch.equal(v, v_ref) and torch.equal(snr, snr_ref)
    fm.fm_trim()


def test_bounded_wait_runs_out_and_is_reported():
    """Failure detection without a GPU fault: the FM_TUNE_WAIT_TEST hook makes
    the fused tile kernel's halo copy announce more bytes than it delivers,
    so every interior tile's bounded wait runs out.  The call still returns
    FM_OK, the device stays usable, fm_device_error reports the timeout once,
    and the next call is exact again."""
    import time

    import numpy as np

    from paper_1204_4293_gb300 import synth
    fm = _fm()
    kap = torch.from_numpy(synth.grf_kappa(512, seed=3).astype(np.float32)).cuda()
    ref = fm.fm_starlet_forward(kap, 5)
    torch.cuda.synchronize()
    assert fm.fm_device_error() == 0
    fm.fm_tune(fm.FM_TUNE_WAIT_TEST, 1)
    try:
        t0 = time.time()
        fm.fm_starlet_forward(kap, 5)
        torch.cuda.synchronize()
        dt = time.time() - t0
    finally:
        fm.fm_tune(fm.FM_TUNE_WAIT_TEST, 0)
    assert fm.fm_device_error() == 1
    assert fm.fm_device_error() == 0  # reading cleared it
    assert dt < 30.0
    again = fm.fm_starlet_forward(kap, 5)
    torch.cuda.synchronize()
    assert torch.equal(again, ref) and fm.fm_device_error() == 0


@pytest.mark.parametrize("merge", [16, 1])
def test_serving_merged_runs_equal_alone(merge):
    # 24 pyramid-only requests of three shapes submitted at once (plus two
    # noise requests between them): the server merges queued requests of one
    # shape into batched runs (or, with merging off, runs each alone); every
    # pyramid equals its single fm_map_starlet call bit for bit
    fm = _fm()
    rng = np.random.default_rng(9)
    reqs = []
    for i in range(26):
        n = int(rng.choice([128, 256, 512]))
        J = int(np.log2(n)) - 2
        R = 3 if i in (5, 17) else 0
        g1 = torch.empty(n, n, device="cuda").normal_(0, 0.1)
        g2 = torch.empty_like(g1).normal_(0, 0.1)
        reqs.append((g1, g2, J, R))
    alone = [fm.fm_map_starlet(g1, g2, J) for g1, g2, J, _ in reqs]
    fm.fm_tune(fm.FM_TUNE_SERVE_MERGE, merge)
    try:
        with fm.Server(mem_budget_bytes=2 << 30, max_slots=2) as sv:
            outs, tickets = [], []
            for g1, g2, J, R in reqs:
                n = g1.shape[-1]
                pyr = torch.full((J, n, n), float("nan"), device="cuda")
                var = torch.empty(J - 1, n, n, dtype=torch.float64, device="cuda") if R else None
                tickets.append(sv.submit(g1, g2, J, pyr, R=R, seed=3, out_var=var))
                outs.append(pyr)
            res = [sv.wait(t, 60.0) for t in tickets]
    finally:
        fm.fm_tune(fm.FM_TUNE_SERVE_MERGE, -1)
    assert all(r.status == fm.FM_OK for r in res)
    for a, b in zip(alone, outs):
        assert torch.equal(a, b)
