"""CPU-side checks of the C ABI: the library builds and loads, exports every
function include/fastmap.h declares, and rejects invalid arguments before it
touches a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastmap.h")


@pytest.fixture(scope="module")
def fm():
    from paper_1204_4293_gb300 import build
    build.build()
    from paper_1204_4293_gb300 import fastmap
    return fastmap


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(fm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fm_ks_invert", "fm_starlet_forward", "fm_map_direct", "fm_map_noise", "fm_serve_create",
                     "fm_serve_submit", "fm_serve_poll", "fm_serve_destroy", "fm_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(fm):
    lib = ctypes.CDLL(fm.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(fm):
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert fm.lib.fm_status_string(code)
    assert fm.lib.fm_status_string(-99) == b"unknown status"


def test_validation_before_any_device_work(fm):
    c = fm._cfg(0)
    cfg = ctypes.byref(c)
    lib = fm.lib
    assert lib.fm_ks_invert(None, None, None, None, 48, 1, cfg, None) == fm.FM_EINVAL
    assert lib.fm_ks_invert(None, None, None, None, 16384, 1, cfg, None) == fm.FM_EINVAL
    assert lib.fm_ks_forward(None, None, None, 64, 0, cfg, None) == fm.FM_EINVAL
    assert lib.fm_starlet_forward(None, None, 16, 5, 1, cfg, None) == fm.FM_EINVAL
    assert lib.fm_starlet_forward(None, None, 64, 1, 1, cfg, None) == fm.FM_EINVAL
    assert lib.fm_map_starlet(None, None, None, 64, 3, 1, cfg, None) == fm.FM_EINVAL  # null pointers
    assert lib.fm_map_direct(None, None, None, 64, 7, 2.0, 3, 0.0, cfg, None) == fm.FM_EINVAL
    assert lib.fm_map_direct(None, None, None, 64, 0, -1.0, 3, 0.0, cfg, None) == fm.FM_EINVAL
    assert lib.fm_map_noise(None, None, None, None, 64, 4, 1, 0, cfg, None) == fm.FM_EINVAL
    assert lib.fm_map_noise_expected(1, 1, 1, 64, 4, cfg, None) == fm.FM_EINVAL  # mirror boundary
    assert b"PERIODIC" in lib.fm_last_error()
    per = fm._cfg(0, fm.FM_PERIODIC)
    assert lib.fm_map_noise_expected(1, 1, 1, 48, 4, ctypes.byref(per), None) == fm.FM_EINVAL
    assert lib.fm_map_noise_expected(None, 1, 1, 64, 4, ctypes.byref(per), None) == fm.FM_EINVAL
    assert lib.fm_map_direct_masked(None, None, None, 0, None, None, 64, 1, 1, 4.0, 3, 0.0, cfg, None) == fm.FM_EINVAL
    assert lib.fm_map_direct_masked(1, 1, 1, -1, 1, None, 64, 1, 1, 4.0, 3, 0.0, cfg, None) == fm.FM_EINVAL
    assert lib.fm_map_direct_masked(1, 1, 1, 0, 1, None, 64, 0, 1, 4.0, 3, 0.0, cfg, None) == fm.FM_EINVAL
    assert lib.fm_map_direct_masked(1, 1, 1, 0, 1, None, 64, 1, 1, 0.5, 3, 0.0, cfg, None) == fm.FM_EINVAL
    bad = fm._cfg(2)
    assert lib.fm_starlet_forward(None, None, 64, 3, 1, ctypes.byref(bad), None) == fm.FM_EINVAL
    assert b"precision" in lib.fm_last_error()
    for acc, prec in ((2, 0), (1, 1)):  # accum 2 does not exist; Kahan fp32 sums need fp32 maps
        bad = fm._cfg(prec, accum=acc)
        assert lib.fm_map_noise(1, 1, 1, None, 64, 4, 8, 0, ctypes.byref(bad), None) == fm.FM_EINVAL
        assert b"accum" in lib.fm_last_error()
    assert lib.fm_map_noise_accumulate(1, 1, None, 64, 4, 0, 3, 0, cfg, None) == fm.FM_EINVAL  # null sums
    assert lib.fm_map_noise_accumulate(1, 1, 1, 64, 4, -1, 3, 0, cfg, None) == fm.FM_EINVAL  # r0 < 0
    assert lib.fm_map_noise_accumulate(1, 1, 1, 64, 4, 0, 0, 0, cfg, None) == fm.FM_EINVAL  # R < 1
    assert lib.fm_noise_finalize(1, None, 1, 1, 64, 4, 10, cfg, None) == fm.FM_EINVAL  # S/N without pyramid
    assert lib.fm_noise_finalize(1, None, 1, None, 64, 4, 1, cfg, None) == fm.FM_EINVAL  # R_total < 2
    assert lib.fm_noise_finalize(1, None, 1, None, 48, 4, 10, cfg, None) == fm.FM_EINVAL  # no sums exist for n = 48
    kahan = fm._cfg(0, accum=1)
    assert lib.fm_map_noise_accumulate(1, 1, 1, 64, 4, 0, 3, 0, ctypes.byref(kahan), None) == fm.FM_EINVAL
    # the allocation-free KS takes the configs fm_ks_invert takes, and n up to
    # 2048 (a batch of one fills its static buffer)
    for bad in (fm._cfg(0, large_path=5), fm._cfg(0, boundary=5), fm._cfg(1)):
        assert lib.fm_ks_invert_noalloc(1, 1, 1, None, 256, 1, ctypes.byref(bad), None) == fm.FM_EINVAL
    assert lib.fm_ks_invert_noalloc(1, 1, 1, None, 4096, 1, cfg, None) == fm.FM_EINVAL
    assert b"[32, 2048]" in lib.fm_last_error()
    bad = fm._cfg(0, large_path=5)
    assert lib.fm_starlet_forward(1, 1, 64, 3, 1, ctypes.byref(bad), None) == fm.FM_EINVAL
    h = ctypes.c_void_p()
    assert lib.fm_serve_create(0, 2, ctypes.byref(h)) == fm.FM_EINVAL
    assert lib.fm_serve_poll(None, 1, None) == fm.FM_EINVAL


def test_alloc_stats_read_and_reset(fm):
    count, largest = fm.fm_alloc_stats(reset=True)
    assert count >= 0 and largest >= 0
    assert fm.fm_alloc_stats() == (0, 0)


def test_request_scratch_bytes_is_monotone(fm):
    small = fm.Server.scratch_bytes(256, 6)
    big = fm.Server.scratch_bytes(1024, 8)
    noisy = fm.Server.scratch_bytes(1024, 8, R=100, with_var=True)
    assert 0 < small < big <= noisy


def test_request_scratch_bytes_counts_work_buffer_and_kappa(fm):
    # a single map's KS + starlet scratch: the complex FFT work buffer (2 n^2
    # values), which also holds the starlet's two scratch maps, and kappa
    # (n^2), each rounded to 256 bytes
    for n, J, prec, es in ((1024, 7, fm.FM_F32, 4), (512, 6, fm.FM_F64, 8), (4096, 9, fm.FM_F32, 4)):
        got = fm.Server.scratch_bytes(n, J, precision=prec)
        assert 3 * n * n * es <= got <= 3 * n * n * es + 3 * 256, (n, got)


def test_fuse_depth_rule(fm):
    """The automatic fused depth (host only): two scales for fp32 maps of
    512^2 to 2048^2, three otherwise; bounded by J - 1 and the tile's
    shared-memory limit (4 in fp32, 3 in fp64); -1 turns fusion off."""
    d = fm.fm_starlet_fuse_depth
    assert [d(n, 7) for n in (256, 512, 1024, 2048, 4096, 8192)] == [3, 2, 2, 2, 3, 3]
    assert d(1024, 7, precision=fm.FM_F64) == 3
    assert d(1024, 3) == 2 and d(256, 3) == 2 and d(256, 2) == 1
    assert d(1024, 7, fuse_depth=4) == 4 and d(1024, 7, fuse_depth=8) == 4
    assert d(1024, 7, precision=fm.FM_F64, fuse_depth=4) == 3
    assert d(1000, 7) == 2 and d(400, 7) == 3  # non-power-of-two starlet sizes follow the same rule
    assert d(1024, 7, fuse_depth=-1) == 0
    with pytest.raises(fm.FastmapError):
        d(16, 5)  # n < 2^J
    with pytest.raises(fm.FastmapError):
        d(1024, 7, fuse_depth=9)


def test_autotune_table_roundtrip(fm, tmp_path):
    """The autotuner's table (host only): a plan entered for (n, J,
    precision) drives the automatic fused depth; it saves to JSON, loads
    back, rejects malformed files and invalid plans, and clears."""
    import json
    fm.fm_autotune_clear()
    try:
        assert fm.fm_autotune_get(1024, 7) is None
        assert fm.fm_starlet_fuse_depth(1024, 7) == 2  # built-in rule
        fm.fm_autotune_set(1024, 7, fuse_depth=4, large_path=3, tile=0, chunk_mb=60)
        fm.fm_autotune_set(512, 6, precision=fm.FM_F64, fuse_depth=1, large_path=1, tile=1, chunk_mb=0)
        got = fm.fm_autotune_get(1024, 7)
        assert (got["fuse_depth"], got["large_path"], got["tile"], got["chunk_mb"]) == (4, 3, 0, 60)
        assert fm.fm_starlet_fuse_depth(1024, 7) == 4
        assert fm.fm_starlet_fuse_depth(1024, 7, fuse_depth=3) == 3  # an explicit depth wins
        assert fm.fm_starlet_fuse_depth(1024, 7, precision=fm.FM_F64) == 3  # other precision: built-in
        assert fm.fm_starlet_fuse_depth(512, 6, precision=fm.FM_F64) == 1
        path = tmp_path / "plans.json"
        fm.fm_autotune_save(path)
        doc = json.loads(path.read_text())
        assert doc["fastmap_autotune"] == 1 and len(doc["entries"]) == 2
        fm.fm_autotune_clear()
        assert fm.fm_autotune_get(1024, 7) is None and fm.fm_starlet_fuse_depth(1024, 7) == 2
        fm.fm_autotune_load(path)
        assert fm.fm_autotune_get(1024, 7)["chunk_mb"] == 60
        assert fm.fm_autotune_get(512, 6, fm.FM_F64)["fuse_depth"] == 1
        bad = tmp_path / "bad.json"
        bad.write_text('{"fastmap_autotune": 1, "entries": [{"n": 1024, "J": 7, "precision": 0, "fuse_depth": 9, '
                       '"large_path": 1, "tile": 1, "chunk_mb": 80}]}')
        with pytest.raises(fm.FastmapError):
            fm.fm_autotune_load(bad)
        assert fm.fm_autotune_get(1024, 7)["fuse_depth"] == 4  # unchanged
        bad.write_text('{"entries": []}')
        with pytest.raises(fm.FastmapError):
            fm.fm_autotune_load(bad)
        for kw in ({"fuse_depth": 5}, {"large_path": 2}, {"tile": 2}, {"chunk_mb": -1}):
            args = dict(fuse_depth=3, large_path=1, tile=1, chunk_mb=0)
            args.update(kw)
            with pytest.raises(fm.FastmapError):
                fm.fm_autotune_set(256, 5, **args)
        with pytest.raises(fm.FastmapError):
            fm.fm_autotune_set(256, 5, precision=fm.FM_F64, fuse_depth=4)
        with pytest.raises(fm.FastmapError):
            fm.fm_autotune(48, 4, 1)  # not a power of two: refused before any device work
    finally:
        fm.fm_autotune_clear()


def test_autotune_json_is_tolerant_of_layout(fm, tmp_path):
    """The plan table loads JSON written by other tools: any whitespace and key
    order, numbers in exponent form, the timing fields optional."""
    fm.fm_autotune_clear()
    try:
        path = tmp_path / "hand.json"
        path.write_text('{\n "entries": [ { "J" : 6, "n": 512, "precision": 0,\n "chunk_mb": 4e1, "tile": 1,'
                        ' "large_path": 3, "fuse_depth": 2 } ],\n "fastmap_autotune": 1 }\n')
        fm.fm_autotune_load(path)
        got = fm.fm_autotune_get(512, 6)
        assert (got["fuse_depth"], got["large_path"], got["tile"], got["chunk_mb"]) == (2, 3, 1, 40)
        assert got["ms"] == 0.0 and got["default_ms"] == 0.0
        assert fm.fm_starlet_fuse_depth(512, 6) == 2
        path.write_text('{"fastmap_autotune": 1, "entries": []}')
        fm.fm_autotune_load(path)  # an empty table file merges nothing
        assert fm.fm_autotune_get(512, 6)["fuse_depth"] == 2
        missing = tmp_path / "missing.json"
        with pytest.raises(fm.FastmapError):
            fm.fm_autotune_load(missing)
    finally:
        fm.fm_autotune_clear()


def test_ks_real_output_size_rule(fm):
    """Host rule of the inverse KS form (no GPU needed): the real-output
    (half spectrum) inverse from 512^2 up, in fm_ks_invert and in the
    batched pipeline alike, the complex one below; FM_TUNE_KS_REAL forces
    either (the real form exists from 64^2 up)."""
    try:
        for batched in (False, True):
            assert [fm.fm_ks_real_output(n, batched) for n in (64, 128, 256, 512, 1024, 4096, 8192)] == \
                [False, False, False, True, True, True, True]
        fm.fm_tune(fm.FM_TUNE_KS_REAL, 1)
        assert fm.fm_ks_real_output(64) and fm.fm_ks_real_output(256) and not fm.fm_ks_real_output(32)
        fm.fm_tune(fm.FM_TUNE_KS_REAL, 0)
        assert not any(fm.fm_ks_real_output(n) for n in (512, 1024, 8192))
    finally:
        fm.fm_tune(fm.FM_TUNE_KS_REAL, -1)
