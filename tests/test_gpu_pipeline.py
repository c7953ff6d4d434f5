"""GPU shear -> KS -> starlet (the fast aperture-mass maps) against the oracle,
at the small configuration (256^2, J = 5), at the paper's 1024^2 J = 7 in the
benchmark's batched launch, and through the host-buffer entry point."""
import numpy as np
import pytest
import torch

import oracle
from helpers import TOL, band_errs, rel_err, shear

pytestmark = pytest.mark.gpu


def _fm():
    from paper_1204_4293_gb300 import fastmap
    return fastmap


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,J,batch", [(16, 3, 2), (64, 5, 1), (256, 5, 2)])
def test_map_starlet_matches_oracle(n, J, batch, dtype):
    fm = _fm()
    maps = [shear(n, seed=20 + b, dtype=dtype) for b in range(batch)]
    g1 = torch.from_numpy(np.stack([m[0] for m in maps])).cuda()
    g2 = torch.from_numpy(np.stack([m[1] for m in maps])).cuda()
    pyr = fm.fm_map_starlet(g1, g2, J).cpu().numpy()
    for b in range(batch):
        ref = oracle.map_starlet(maps[b][0].astype(np.float64), maps[b][1].astype(np.float64), J)
        assert max(band_errs(pyr[b], ref)) <= TOL[dtype]


def test_map_starlet_paper_size_batched():
    # the benchmark's workload and launch configuration: 32 1024^2 fp32 shear
    # maps, J = 7, in L2-sized chunks on two streams, recorded into a CUDA
    # graph and replayed; the oracle checks the first and the last map in full
    fm = _fm()
    n, J, batch = 1024, 7, 32
    maps = [shear(n, seed=2 + b, dtype=np.float32) for b in (0, batch - 1)]
    g1 = torch.empty((batch, n, n), dtype=torch.float32, device="cuda")
    g2 = torch.empty_like(g1)
    g1.normal_(0, 0.1)
    g2.normal_(0, 0.1)
    g1[0], g2[0] = torch.from_numpy(maps[0][0]), torch.from_numpy(maps[0][1])
    g1[-1], g2[-1] = torch.from_numpy(maps[1][0]), torch.from_numpy(maps[1][1])
    pyr = fm.fm_map_starlet(g1, g2, J)  # records the graph
    pyr = fm.fm_map_starlet(g1, g2, J, out=torch.full_like(pyr, float("nan")))  # replays it
    assert fm.fm_device_error() == 0
    for idx, m in ((0, maps[0]), (batch - 1, maps[1])):
        ref = oracle.map_starlet(m[0].astype(np.float64), m[1].astype(np.float64), J)
        errs = band_errs(pyr[idx].cpu().numpy(), ref)
        assert max(errs) <= 1e-5, errs


def test_map_starlet_host_equals_device():
    fm = _fm()
    n, J, batch = 128, 6, 3
    g1 = torch.randn(batch, n, n, dtype=torch.float32).mul_(0.1).pin_memory()
    g2 = torch.randn(batch, n, n, dtype=torch.float32).mul_(0.1).pin_memory()
    out = torch.empty(batch, J, n, n, dtype=torch.float32).pin_memory()
    fm.fm_map_starlet_host(g1, g2, J, out)
    torch.cuda.synchronize()
    dev = fm.fm_map_starlet(g1.cuda(), g2.cuda(), J).cpu()
    assert torch.equal(out, dev)


def test_map_starlet_large_field_4096_j9():
    # the large-field configuration: 4096^2, P(k) ~ k^-2.5, J = 9, a batch of
    # two; the oracle checks the first map in full
    fm = _fm()
    n, J = 4096, 9
    g1, g2 = shear(n, seed=40, alpha=2.5, dtype=np.float32)
    t1 = torch.from_numpy(np.stack([g1, g1[::-1].copy()])).cuda()
    t2 = torch.from_numpy(np.stack([g2, g2[::-1].copy()])).cuda()
    pyr = fm.fm_map_starlet(t1, t2, J)
    ref = oracle.map_starlet(g1.astype(np.float64), g2.astype(np.float64), J)
    errs = band_errs(pyr[0].cpu().numpy(), ref)
    assert max(errs) <= 1e-5, errs


def test_ks_and_starlet_8192_match_oracle():
    # the largest field of the large-field workload (one 8192^2 map, P(k) ~
    # k^-2.5, J = 9) in the launch the benchmark times (fm_map_starlet, batch
    # of one), and the KS inversion alone, against the FP64 oracle in full:
    # the four-step column strips and their bulk tensor stores exist only at
    # this size
    fm = _fm()
    n, J = 8192, 9
    g1, g2 = shear(n, seed=56, alpha=2.5, dtype=np.float32)
    t1, t2 = torch.from_numpy(g1).cuda(), torch.from_numpy(g2).cuda()
    kE, kB = fm.fm_ks_invert(t1.unsqueeze(0), t2.unsqueeze(0), with_b=True)
    pyr = fm.fm_map_starlet(t1.unsqueeze(0), t2.unsqueeze(0), J)
    torch.cuda.synchronize()
    assert fm.fm_device_error() == 0
    d1, d2 = g1.astype(np.float64), g2.astype(np.float64)
    rE, rB = oracle.ks_invert(d1, d2)
    assert rel_err(kE[0].cpu().numpy(), rE) <= 1e-5
    assert rel_err(kB[0].cpu().numpy(), rB) <= 1e-5
    del kE, kB, rB
    ref = oracle.starlet(rE, J)  # the oracle's map_starlet is ks_invert then starlet
    del rE
    errs = [rel_err(pyr[0, j].cpu().numpy(), ref[j]) for j in range(J)]
    assert max(errs) <= 1e-5, errs


def test_map_starlet_8192_reconstruction_and_ks():
    # the largest field: the pyramid sums back to kappa_E (exact reconstruction)
    fm = _fm()
    n, J = 8192, 9
    from paper_1204_4293_gb300 import synth
    kap = torch.from_numpy(synth.grf_kappa(n, alpha=2.5, seed=56).astype(np.float32)).cuda()
    g1, g2 = fm.fm_ks_forward(kap)
    pyr = fm.fm_map_starlet(g1, g2, J)
    kE, _ = fm.fm_ks_invert(g1, g2)
    rms = kap.double().pow(2).mean().sqrt().item()
    assert (pyr.double().sum(0) - kE.double()).abs().max().item() / rms < 1e-5
    assert (kE - kap).abs().max().item() / rms < 1e-5


@pytest.mark.parametrize("streams", [1, 2, 3, 4])
@pytest.mark.parametrize("graphs", [0, 1])
def test_chunk_plans_give_identical_pyramids(streams, graphs):
    # 7 maps in chunks of 2 (a ragged last chunk) on 1..4 streams, replayed
    # from a graph or launched eagerly: bit-identical to one unchunked pass
    fm = _fm()
    n, J, batch = 256, 6, 7
    g1 = torch.empty((batch, n, n), device="cuda").normal_(0, 0.1)
    g2 = torch.empty_like(g1).normal_(0, 0.1)
    fm.fm_tune(fm.FM_TUNE_CHUNK_BYTES, 0)
    try:
        ref = fm.fm_map_starlet(g1, g2, J)
        per_map = n * n * 4 * 5  # complex work buffer, kappa, two starlet scratch arrays
        fm.fm_tune(fm.FM_TUNE_CHUNK_BYTES, 2 * per_map + per_map // 2)  # chunks of 2 maps
        fm.fm_tune(fm.FM_TUNE_CHUNK_STREAMS, streams)
        fm.fm_tune(fm.FM_TUNE_GRAPHS, graphs)
        out = torch.full_like(ref, float("nan"))
        for _ in range(2):  # record, then replay
            fm.fm_map_starlet(g1, g2, J, out=out)
        assert torch.equal(out, ref)
    finally:
        for knob in (fm.FM_TUNE_CHUNK_BYTES, fm.FM_TUNE_CHUNK_STREAMS, fm.FM_TUNE_GRAPHS):
            fm.fm_tune(knob, -1)
        fm.fm_trim()
    o = oracle.map_starlet(g1[batch - 1].double().cpu().numpy(), g2[batch - 1].double().cpu().numpy(), J)
    assert max(band_errs(ref[batch - 1].cpu().numpy(), o)) <= 1e-5


@pytest.mark.parametrize("streams", [1, 2, 4])
@pytest.mark.parametrize("dtype,pinned", [(torch.float32, True), (torch.float64, True), (torch.float32, False)])
def test_host_pipeline_over_chunk_slots(streams, dtype, pinned):
    # 7 maps in chunks of 2 through 1, 2 or 4 slots: copy in, compute and copy
    # out per chunk; equals the device-buffer call
    fm = _fm()
    n, J, batch = 128, 5, 7
    g1 = torch.randn(batch, n, n, dtype=dtype).mul_(0.1)
    g2 = torch.randn(batch, n, n, dtype=dtype).mul_(0.1)
    out = torch.full((batch, J, n, n), float("nan"), dtype=dtype)
    if pinned:
        g1, g2, out = g1.pin_memory(), g2.pin_memory(), out.pin_memory()
    es = 8 if dtype == torch.float64 else 4
    per_map = n * n * es * 5
    fm.fm_tune(fm.FM_TUNE_CHUNK_BYTES, 2 * per_map + per_map // 2)
    fm.fm_tune(fm.FM_TUNE_CHUNK_STREAMS, streams)
    try:
        fm.fm_map_starlet_host(g1, g2, J, out)
        torch.cuda.synchronize()
    finally:
        fm.fm_tune(fm.FM_TUNE_CHUNK_BYTES, -1)
        fm.fm_tune(fm.FM_TUNE_CHUNK_STREAMS, -1)
    dev = fm.fm_map_starlet(g1.cuda(), g2.cuda(), J).cpu()
    assert torch.equal(out, dev)


@pytest.mark.parametrize("n,J,batch", [(256, 5, 3), (1024, 7, 5)])
def test_unaligned_buffers_take_the_scalar_paths(n, J, batch):
    # shear, kappa and pyramid views starting one float into their storage
    # (4-byte aligned only): no 16-byte vector load or bulk tensor copy may
    # touch them; results equal the aligned call's up to rounding order
    fm = _fm()
    def offset_like(shape, fill=None):
        total = int(np.prod(shape))
        base = torch.empty(total + 1, device="cuda")
        view = base[1:].view(*shape)
        if fill is not None:
            view.copy_(fill)
        return view
    g1 = torch.empty((batch, n, n), device="cuda").normal_(0, 0.1)
    g2 = torch.empty_like(g1).normal_(0, 0.1)
    u1, u2 = offset_like(g1.shape, g1), offset_like(g2.shape, g2)
    assert u1.data_ptr() % 16 == 4
    out = offset_like((batch, J, n, n))
    ref = fm.fm_map_starlet(g1, g2, J)
    fm.fm_map_starlet(u1, u2, J, out=out)
    kap, _ = fm.fm_ks_invert(g1, g2)
    uk = offset_like(kap.shape, kap)
    st_ref = fm.fm_starlet_forward(kap, J)
    st_out = offset_like((batch, J, n, n))
    fm.fm_starlet_forward(uk, J, out=st_out)
    torch.cuda.synchronize()
    assert fm.fm_device_error() == 0
    for a, b in ((out, ref), (st_out, st_ref)):
        a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
        for m in range(batch):
            assert max(band_errs(a[m], b[m])) <= 1e-6
