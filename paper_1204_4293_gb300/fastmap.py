"""Thin Python binding of libfastmap (include/fastmap.h) over torch tensors.

Argument marshalling only: every function here checks shapes, dtypes and
devices, allocates outputs with torch (device memory is torch's job) and
calls the C entry point of the same name on torch's current CUDA stream.
All compute runs in the library's CUDA kernels; there is no CPU fallback.
Importing this module fails if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfastmap.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1204_4293_gb300.build` "
                      "(or __graft_entry__.build()); there is no fallback implementation")

_lib = ctypes.CDLL(LIB_PATH)

# ---- constants (mirror include/fastmap.h) ------------------------------------
FM_OK, FM_PENDING = 0, 1
FM_EINVAL, FM_ENOMEM, FM_EBUDGET, FM_ETIMEOUT, FM_ECUDA, FM_ENOTFOUND, FM_EBUSY = -1, -2, -3, -4, -5, -6, -7
FM_F32, FM_F64 = 0, 1
FM_MIRROR, FM_PERIODIC = 0, 1
FM_FILTER_STARLET, FM_FILTER_S98, FM_FILTER_JBJ04, FM_FILTER_VW98 = 0, 1, 2, 3
KERNEL_IDS = {"fft_rows_fwd": 1, "fft_cols_ks": 2, "fft_rows_inv": 3, "starlet_tile": 4, "starlet_row": 5,
              "starlet_col": 6, "map_direct": 7, "noise_final": 8, "noise_accum": 9, "starlet_colrow": 10}


class fm_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("boundary", ctypes.c_int), ("accum", ctypes.c_int),
                ("fuse_depth", ctypes.c_int), ("large_path", ctypes.c_int)]


class fm_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("J", ctypes.c_int), ("R", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int), ("g1", ctypes.c_void_p), ("g2", ctypes.c_void_p),
                ("out_pyramid", ctypes.c_void_p), ("out_var", ctypes.c_void_p)]


class fm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64)]


class fm_plan(ctypes.Structure):
    _fields_ = [("fuse_depth", ctypes.c_int), ("large_path", ctypes.c_int), ("tile", ctypes.c_int),
                ("chunk_mb", ctypes.c_int), ("ms", ctypes.c_double), ("default_ms", ctypes.c_double)]


_P, _I, _D, _U64, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_size_t
_CFG = ctypes.POINTER(fm_config)
_SIGS = {
    "fm_ks_invert": (_I, [_P, _P, _P, _P, _I, _I, _CFG, _P]),
    "fm_ks_forward": (_I, [_P, _P, _P, _I, _I, _CFG, _P]),
    "fm_ks_invert_noalloc": (_I, [_P, _P, _P, _P, _I, _I, _CFG, _P]),
    "fm_starlet_forward": (_I, [_P, _P, _I, _I, _I, _CFG, _P]),
    "fm_starlet_fuse_depth": (_I, [_I, _I, _CFG]),
    "fm_map_starlet": (_I, [_P, _P, _P, _I, _I, _I, _CFG, _P]),
    "fm_map_starlet_host": (_I, [_P, _P, _P, _I, _I, _I, _CFG, _P]),
    "fm_map_direct": (_I, [_P, _P, _P, _I, _I, _D, _I, _D, _CFG, _P]),
    "fm_map_direct_batch": (_I, [_P, _P, _P, _I, _I, _I, _D, _I, _D, _CFG, _P]),
    "fm_map_direct_masked": (_I, [_P, _P, _P, ctypes.c_long, _P, _P, _I, _I, _I, _D, _I, _D, _CFG, _P]),
    "fm_map_noise": (_I, [_P, _P, _P, _P, _I, _I, _I, _U64, _CFG, _P]),
    "fm_map_noise_expected": (_I, [_P, _P, _P, _I, _I, _CFG, _P]),
    "fm_map_noise_accumulate": (_I, [_P, _P, _P, _I, _I, _I, _I, _U64, _CFG, _P]),
    "fm_noise_finalize": (_I, [_P, _P, _P, _P, _I, _I, _I, _CFG, _P]),
    "fm_band_moments": (_I, [_P, _P, _I, _I, _I, _CFG, _P]),
    "fm_serve_create": (_I, [_SZ, _I, ctypes.POINTER(ctypes.c_void_p)]),
    "fm_serve_submit": (_I, [_P, ctypes.POINTER(fm_request), ctypes.POINTER(ctypes.c_uint64)]),
    "fm_serve_poll": (_I, [_P, _U64, ctypes.POINTER(fm_result)]),
    "fm_serve_wait": (_I, [_P, _U64, ctypes.POINTER(fm_result), _D]),
    "fm_serve_destroy": (_I, [_P]),
    "fm_request_scratch_bytes": (_SZ, [ctypes.POINTER(fm_request)]),
    "fm_status_string": (ctypes.c_char_p, [_I]),
    "fm_last_error": (ctypes.c_char_p, []),
    "fm_launch_count": (ctypes.c_int64, []),
    "fm_ks_real_output": (_I, [_I, _I]),
    "fm_measure_bandwidth": (_I, [_SZ, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "fm_alloc_stats": (_I, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _I]),
    "fm_device_error": (_I, []),
    "fm_profile_select": (_I, [_I]),
    "fm_tune": (_I, [_I, ctypes.c_int64]),
    "fm_trim": (_I, []),
    "fm_autotune": (_I, [_I, _I, _I, _CFG, ctypes.POINTER(fm_plan)]),
    "fm_autotune_get": (_I, [_I, _I, _I, ctypes.POINTER(fm_plan)]),
    "fm_autotune_set": (_I, [_I, _I, _I, ctypes.POINTER(fm_plan)]),
    "fm_autotune_save": (_I, [ctypes.c_char_p]),
    "fm_autotune_load": (_I, [ctypes.c_char_p]),
    "fm_autotune_clear": (_I, []),
    "fm_profile_read": (_I, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

lib = _lib  # raw ctypes handle (C-ABI calls with plain pointers)


class FastmapError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.fm_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_lib.fm_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def _check(status: int, where: str) -> int:
    if status < 0:
        raise FastmapError(status, where)
    return status


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _prec(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return FM_F32
    if t.dtype == torch.float64:
        return FM_F64
    raise TypeError(f"maps must be float32 or float64, got {t.dtype}")


def _cfg(precision, boundary=FM_MIRROR, fuse_depth=0, large_path=0, accum=0):
    c = fm_config()
    c.precision, c.boundary, c.accum, c.fuse_depth, c.large_path = precision, boundary, accum, fuse_depth, large_path
    return c


def _maps(*ts, device=True):
    """Validate a set of same-shape [batch, n, n] or [n, n] contiguous maps."""
    ref = ts[0]
    for t in ts:
        if t.shape != ref.shape or t.dtype != ref.dtype:
            raise ValueError("maps must share shape and dtype")
        if device and not t.is_cuda:
            raise ValueError("maps must be CUDA tensors")
        if not t.is_contiguous():
            raise ValueError("maps must be contiguous")
    if ref.dim() not in (2, 3) or ref.shape[-1] != ref.shape[-2]:
        raise ValueError("maps are [n, n] or [batch, n, n]")
    n = ref.shape[-1]
    batch = 1 if ref.dim() == 2 else ref.shape[0]
    return n, batch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


# ---- entry points ----------------------------------------------------------------
def fm_ks_invert(g1, g2, with_b=False, stream=None):
    """(kappa_E, kappa_B or None) from shear (Kaiser-Squires, Sec. 4.5)."""
    n, batch = _maps(g1, g2)
    kE = torch.empty_like(g1)
    kB = torch.empty_like(g1) if with_b else None
    c = _cfg(_prec(g1))
    _check(_lib.fm_ks_invert(_ptr(g1), _ptr(g2), _ptr(kE), _ptr(kB), n, batch, ctypes.byref(c), _stream(stream)),
           "fm_ks_invert")
    return kE, kB


def fm_ks_forward(kappa, stream=None):
    """(gamma1, gamma2) of a convergence map (forward Kaiser-Squires)."""
    n, batch = _maps(kappa)
    g1, g2 = torch.empty_like(kappa), torch.empty_like(kappa)
    c = _cfg(_prec(kappa))
    _check(_lib.fm_ks_forward(_ptr(kappa), _ptr(g1), _ptr(g2), n, batch, ctypes.byref(c), _stream(stream)),
           "fm_ks_forward")
    return g1, g2


def _pyr_out(ref, J, out):
    shape = ((J,) if ref.dim() == 2 else (ref.shape[0], J)) + tuple(ref.shape[-2:])
    if out is None:
        return torch.empty(shape, dtype=ref.dtype, device=ref.device)
    if tuple(out.shape) != shape or out.dtype != ref.dtype or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous {ref.dtype} tensor of shape {shape}")
    return out


def fm_starlet_forward(kappa, J, boundary=FM_MIRROR, fuse_depth=0, out=None, stream=None, large_path=0):
    """Starlet pyramid [.., J, n, n]: w_1..w_{J-1}, smooth (Sec. 3)."""
    n, batch = _maps(kappa)
    pyr = _pyr_out(kappa, J, out)
    c = _cfg(_prec(kappa), boundary, fuse_depth, large_path)
    _check(_lib.fm_starlet_forward(_ptr(kappa), _ptr(pyr), n, J, batch, ctypes.byref(c), _stream(stream)),
           "fm_starlet_forward")
    return pyr


def fm_starlet_fuse_depth(n, J, precision=FM_F32, boundary=FM_MIRROR, fuse_depth=0, large_path=0) -> int:
    """Scales the fused tile kernel computes for an n x n map, J scales (host only)."""
    c = _cfg(precision, boundary, fuse_depth, large_path)
    return _check(_lib.fm_starlet_fuse_depth(int(n), int(J), ctypes.byref(c)), "fm_starlet_fuse_depth")


def fm_map_starlet(g1, g2, J, boundary=FM_MIRROR, fuse_depth=0, out=None, stream=None, large_path=0):
    """KS inversion then starlet: all aperture-mass bands from shear."""
    n, batch = _maps(g1, g2)
    pyr = _pyr_out(g1, J, out)
    c = _cfg(_prec(g1), boundary, fuse_depth, large_path)
    _check(_lib.fm_map_starlet(_ptr(g1), _ptr(g2), _ptr(pyr), n, J, batch, ctypes.byref(c), _stream(stream)),
           "fm_map_starlet")
    return pyr


def fm_map_starlet_host(g1, g2, J, out, boundary=FM_MIRROR, fuse_depth=0, stream=None):
    """fm_map_starlet from and to HOST tensors (pinned for speed); asynchronous."""
    n, batch = _maps(g1, g2, device=False)
    if g1.is_cuda or out.is_cuda:
        raise ValueError("fm_map_starlet_host takes host tensors")
    _pyr_out(g1, J, out)
    c = _cfg(_prec(g1), boundary, fuse_depth)
    _check(_lib.fm_map_starlet_host(_ptr(g1), _ptr(g2), _ptr(out), n, J, batch, ctypes.byref(c), _stream(stream)),
           "fm_map_starlet_host")
    return out


def fm_map_direct(g1, g2, filt, theta, ell=3, cut_over_theta=0.0, out=None, stream=None):
    """Brute-force M_ap map from tangential shear (eq. shearmap): one [n, n]
    map (fm_map_direct) or a batch [batch, n, n] in one launch
    (fm_map_direct_batch)."""
    n, batch = _maps(g1, g2)
    m = torch.empty_like(g1) if out is None else out
    if m.shape != g1.shape or m.dtype != g1.dtype or not m.is_contiguous():
        raise ValueError("out must be a contiguous tensor of the maps' shape and dtype")
    c = _cfg(_prec(g1))
    if g1.dim() == 2:
        _check(_lib.fm_map_direct(_ptr(g1), _ptr(g2), _ptr(m), n, int(filt), float(theta), int(ell),
                                  float(cut_over_theta), ctypes.byref(c), _stream(stream)), "fm_map_direct")
    else:
        _check(_lib.fm_map_direct_batch(_ptr(g1), _ptr(g2), _ptr(m), n, batch, int(filt), float(theta), int(ell),
                                        float(cut_over_theta), ctypes.byref(c), _stream(stream)),
               "fm_map_direct_batch")
    return m


def fm_map_direct_masked(g1, g2, weight, filt, theta, ell=3, cut_over_theta=0.0, coverage=False, out=None,
                         stream=None):
    """Weighted direct M_ap for fields with missing data: (map, coverage or
    None).  g1, g2 are [n, n] or [batch, n, n]; weight is [n, n] (one mask
    for the batch) or the maps' shape; weights >= 0, 0 = masked."""
    n, batch = _maps(g1, g2)
    if weight.dtype != g1.dtype or not weight.is_cuda or not weight.is_contiguous():
        raise ValueError("weight must be a contiguous CUDA tensor of the maps' dtype")
    if weight.shape == g1.shape:
        wbs = n * n if g1.dim() == 3 else 0
    elif weight.shape == (n, n):
        wbs = 0
    else:
        raise ValueError("weight is [n, n] or the maps' shape")
    m = torch.empty_like(g1) if out is None else out
    cov = torch.empty_like(g1) if coverage else None
    c = _cfg(_prec(g1))
    _check(_lib.fm_map_direct_masked(_ptr(g1), _ptr(g2), _ptr(weight), wbs, _ptr(m), _ptr(cov), n, batch, int(filt),
                                     float(theta), int(ell), float(cut_over_theta), ctypes.byref(c),
                                     _stream(stream)), "fm_map_direct_masked")
    return m, cov


def fm_map_noise_expected(g1, g2, J, out=None, stream=None):
    """Exact expected noise variance of bands 1..J-1 (periodic boundary):
    [J-1, n, n] in the maps' dtype."""
    n, batch = _maps(g1, g2)
    if batch != 1 or g1.dim() != 2:
        raise ValueError("fm_map_noise_expected takes one [n, n] map")
    var = torch.empty((J - 1, n, n), dtype=g1.dtype, device=g1.device) if out is None else out
    c = _cfg(_prec(g1), FM_PERIODIC)
    _check(_lib.fm_map_noise_expected(_ptr(g1), _ptr(g2), _ptr(var), n, J, ctypes.byref(c), _stream(stream)),
           "fm_map_noise_expected")
    return var


def fm_map_noise(g1, g2, J, R, seed, boundary=FM_MIRROR, with_snr=True, fuse_depth=0, stream=None, accum=0):
    """(variance [J-1, n, n] float64, S/N or None) over R rotated realisations.
    accum: 0 = FP64 running sums, 1 = fp32 running sums with Kahan compensation."""
    n, batch = _maps(g1, g2)
    if batch != 1 or g1.dim() != 2:
        raise ValueError("fm_map_noise takes one [n, n] map")
    var = torch.empty((J - 1, n, n), dtype=torch.float64, device=g1.device)
    snr = torch.empty((J - 1, n, n), dtype=g1.dtype, device=g1.device) if with_snr else None
    c = _cfg(_prec(g1), boundary, fuse_depth, accum=accum)
    _check(_lib.fm_map_noise(_ptr(g1), _ptr(g2), _ptr(var), _ptr(snr), n, J, int(R),
                             ctypes.c_uint64(int(seed) & (2**64 - 1)), ctypes.byref(c), _stream(stream)),
           "fm_map_noise")
    return var, snr


def fm_map_noise_accumulate(g1, g2, J, r0, R, seed, sums=None, boundary=FM_MIRROR, stream=None):
    """Add realisations r0 .. r0 + R - 1 to `sums` ([2, J-1, n, n] float64,
    zeros when None) and return it."""
    n, batch = _maps(g1, g2)
    if batch != 1 or g1.dim() != 2:
        raise ValueError("fm_map_noise_accumulate takes one [n, n] map")
    if sums is None:
        sums = torch.zeros((2, J - 1, n, n), dtype=torch.float64, device=g1.device)
    if sums.shape != (2, J - 1, n, n) or sums.dtype != torch.float64 or not sums.is_contiguous():
        raise ValueError("sums must be a contiguous [2, J-1, n, n] float64 tensor")
    c = _cfg(_prec(g1), boundary)
    _check(_lib.fm_map_noise_accumulate(_ptr(g1), _ptr(g2), _ptr(sums), n, J, int(r0), int(R),
                                        ctypes.c_uint64(int(seed) & (2**64 - 1)), ctypes.byref(c), _stream(stream)),
           "fm_map_noise_accumulate")
    return sums


def fm_noise_finalize(sums, R_total, pyramid=None, dtype=torch.float32, stream=None):
    """(variance [J-1, n, n] float64, S/N or None) from sums of R_total
    realisations; S/N when the data's pyramid [J, n, n] is given."""
    if sums.dim() != 4 or sums.shape[0] != 2 or sums.dtype != torch.float64 or not sums.is_contiguous():
        raise ValueError("sums must be a contiguous [2, J-1, n, n] float64 tensor")
    J, n = sums.shape[1] + 1, sums.shape[2]
    var = torch.empty((J - 1, n, n), dtype=torch.float64, device=sums.device)
    snr = None
    prec = _prec(pyramid) if pyramid is not None else (FM_F64 if dtype == torch.float64 else FM_F32)
    if pyramid is not None:
        if pyramid.shape != (J, n, n) or not pyramid.is_contiguous():
            raise ValueError("pyramid must be a contiguous [J, n, n] tensor")
        snr = torch.empty((J - 1, n, n), dtype=pyramid.dtype, device=sums.device)
    c = _cfg(prec)
    _check(_lib.fm_noise_finalize(_ptr(sums), _ptr(pyramid), _ptr(var), _ptr(snr), n, J, int(R_total),
                                  ctypes.byref(c), _stream(stream)), "fm_noise_finalize")
    return var, snr


FM_TUNE_CHUNK_BYTES, FM_TUNE_GRAPHS, FM_TUNE_CHUNK_STREAMS, FM_TUNE_PDL, FM_TUNE_TILE, FM_TUNE_TMA = 1, 2, 3, 4, 5, 6
FM_TUNE_WAIT_TEST = 7
FM_TUNE_DIRECT = 8
FM_TUNE_KS_REAL = 9
FM_TUNE_SERVE_MERGE = 10
FM_TUNE_SERVE_HEAVY = 11


def fm_tune(knob: int, value: int) -> None:
    """Process-wide tuning knob (FM_TUNE_*); value < 0 restores the default."""
    _check(_lib.fm_tune(int(knob), int(value)), "fm_tune")


def fm_band_moments(pyramid, stream=None):
    """[.., J, 4] float64: mean, variance, skewness, excess kurtosis of each
    pyramid array over its pixels (Sec. 2.2)."""
    if pyramid.dim() not in (3, 4) or not pyramid.is_cuda or not pyramid.is_contiguous():
        raise ValueError("pyramid is a contiguous CUDA tensor [J, n, n] or [batch, J, n, n]")
    batch = 1 if pyramid.dim() == 3 else pyramid.shape[0]
    J, n = pyramid.shape[-3], pyramid.shape[-1]
    out = torch.empty(tuple(pyramid.shape[:-2]) + (4,), dtype=torch.float64, device=pyramid.device)
    c = _cfg(_prec(pyramid))
    _check(_lib.fm_band_moments(_ptr(pyramid), _ptr(out), n, J, batch, ctypes.byref(c), _stream(stream)),
           "fm_band_moments")
    return out


def _plan_dict(p: fm_plan) -> dict:
    return {"fuse_depth": p.fuse_depth, "large_path": p.large_path, "tile": p.tile, "chunk_mb": p.chunk_mb,
            "ms": p.ms, "default_ms": p.default_ms}


def fm_autotune(n, J, batch, precision=FM_F32, boundary=FM_MIRROR) -> dict:
    """Time candidate plans of fm_map_starlet for `batch` n x n maps and keep
    the fastest for (n, J, precision) in the library's table."""
    c = _cfg(precision, boundary)
    p = fm_plan()
    _check(_lib.fm_autotune(int(n), int(J), int(batch), ctypes.byref(c), ctypes.byref(p)), "fm_autotune")
    return _plan_dict(p)


def fm_autotune_get(n, J, precision=FM_F32):
    """The table's plan for (n, J, precision), or None."""
    p = fm_plan()
    st = _lib.fm_autotune_get(int(n), int(J), int(precision), ctypes.byref(p))
    if st == FM_ENOTFOUND:
        return None
    _check(st, "fm_autotune_get")
    return _plan_dict(p)


def fm_autotune_set(n, J, precision=FM_F32, fuse_depth=3, large_path=1, tile=1, chunk_mb=0) -> None:
    p = fm_plan(fuse_depth=fuse_depth, large_path=large_path, tile=tile, chunk_mb=chunk_mb)
    _check(_lib.fm_autotune_set(int(n), int(J), int(precision), ctypes.byref(p)), "fm_autotune_set")


def fm_autotune_save(path) -> None:
    _check(_lib.fm_autotune_save(os.fsencode(path)), "fm_autotune_save")


def fm_autotune_load(path) -> None:
    _check(_lib.fm_autotune_load(os.fsencode(path)), "fm_autotune_load")


def fm_autotune_clear() -> None:
    _check(_lib.fm_autotune_clear(), "fm_autotune_clear")


def fm_trim() -> None:
    """Free the library's cached CUDA graphs and their scratch."""
    _check(_lib.fm_trim(), "fm_trim")


def fm_launch_count() -> int:
    return int(_lib.fm_launch_count())


def fm_ks_real_output(n: int, batched: bool = True) -> bool:
    """Whether the inverse KS of n x n fp32 maps (kappa_E only) takes the
    real-output path: in the batched pipeline's chunks, or in fm_ks_invert."""
    return bool(_lib.fm_ks_real_output(int(n), 1 if batched else 0))


def fm_measure_bandwidth(nbytes: int, reps: int = 20):
    """(read GB/s, copy GB/s) of streaming kernels over a working set of
    nbytes on the current device (32 MiB: L2; GiBs: HBM)."""
    r, c = ctypes.c_double(0), ctypes.c_double(0)
    _check(_lib.fm_measure_bandwidth(int(nbytes), int(reps), ctypes.byref(r), ctypes.byref(c)),
           "fm_measure_bandwidth")
    return r.value, c.value


def fm_alloc_stats(reset: bool = False):
    """(count, largest bytes) of the device allocations the library made
    since the last reset; reset=True zeroes them after reading."""
    c, m = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(_lib.fm_alloc_stats(ctypes.byref(c), ctypes.byref(m), 1 if reset else 0), "fm_alloc_stats")
    return int(c.value), int(m.value)


def fm_device_error() -> int:
    """1 if a kernel gave up waiting for a bulk copy since the last call."""
    v = int(_lib.fm_device_error())
    if v < 0:
        _check(v, "fm_device_error")
    return v


def fm_profile_select(kernel: str | int) -> None:
    kid = KERNEL_IDS[kernel] if isinstance(kernel, str) else int(kernel)
    _check(_lib.fm_profile_select(kid), "fm_profile_select")


def fm_profile_read():
    ms = ctypes.c_double(0)
    cnt = ctypes.c_int64(0)
    _check(_lib.fm_profile_read(ctypes.byref(ms), ctypes.byref(cnt)), "fm_profile_read")
    return ms.value, cnt.value


class Server:
    """Continuous-batching server (fm_serve_*): submit, poll, wait."""

    def __init__(self, mem_budget_bytes: int, max_slots: int = 4):
        h = ctypes.c_void_p()
        _check(_lib.fm_serve_create(int(mem_budget_bytes), int(max_slots), ctypes.byref(h)), "fm_serve_create")
        self._h = h
        self._keep = {}

    def submit(self, g1, g2, J, out_pyramid, R=0, seed=0, out_var=None) -> int:
        n, batch = _maps(g1, g2)
        if batch != 1 or g1.dim() != 2:
            raise ValueError("one [n, n] map per request")
        r = fm_request(n=n, J=J, R=int(R), seed=int(seed) & (2**64 - 1), precision=_prec(g1),
                       g1=g1.data_ptr(), g2=g2.data_ptr(), out_pyramid=out_pyramid.data_ptr(),
                       out_var=out_var.data_ptr() if out_var is not None else None)
        t = ctypes.c_uint64()
        _check(_lib.fm_serve_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "fm_serve_submit")
        self._keep[t.value] = (g1, g2, out_pyramid, out_var)  # keep buffers alive until done
        return t.value

    def poll(self, ticket: int):
        res = fm_result()
        st = _lib.fm_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(res))
        if st == FM_PENDING:
            return None
        _check(st, "fm_serve_poll")
        self._keep.pop(ticket, None)
        return res

    def wait(self, ticket: int, timeout_s: float = 60.0):
        res = fm_result()
        st = _lib.fm_serve_wait(self._h, ctypes.c_uint64(ticket), ctypes.byref(res), float(timeout_s))
        _check(st, "fm_serve_wait")
        self._keep.pop(ticket, None)
        return res

    @staticmethod
    def scratch_bytes(n, J, R=0, precision=FM_F32, with_var=False) -> int:
        r = fm_request(n=n, J=J, R=R, seed=0, precision=precision, g1=None, g2=None, out_pyramid=None,
                       out_var=1 if with_var else None)
        return int(_lib.fm_request_scratch_bytes(ctypes.byref(r)))

    def close(self):
        if self._h:
            _check(_lib.fm_serve_destroy(self._h), "fm_serve_destroy")
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
