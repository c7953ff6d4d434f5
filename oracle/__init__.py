"""FP64 CPU oracle for the fast aperture-mass pipeline (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.  It
wraps ``oracle.c`` (plain C, FP64) through ctypes and shares nothing with the
CUDA path.

Each wrapper names the paper passage its C function follows:
  ks_forward / ks_invert   Sec. 4.5 (Kaiser-Squires in Fourier space)
  starlet                  Sec. 3 and Sec. 4.2 (a trous B3-spline starlet)
  map_direct               eq. shearmap (Sec. 2.1), brute force as in Sec. 5.1
  map_direct_masked        eq. shearmap with pixel weights for missing data
                           (Sec. 4.3, Sec. 4.5)
  map_noise                Sec. 1 and Sec. 5.1 (randomised-data noise maps)
  map_noise_expected       Sec. 1: exact expectation of that variance (periodic)
  u_/q_ filters            eq. sch, eq. mexhat, the starlet U and Q (Sec. 4)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# Flags: no FMA contraction and no fast-math, so x86 and Arm give the same
# FP64 results for the same operation order.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc); return the path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        c_int, c_double, c_u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        sigs = {
            "oracle_phi_b3": (c_double, [c_double]),
            "oracle_starlet_taps": (None, [_D]),
            "oracle_u_starlet": (c_double, [c_double]),
            "oracle_q_starlet": (c_double, [c_double]),
            "oracle_u_s98": (c_double, [c_double, c_double, c_int]),
            "oracle_q_s98": (c_double, [c_double, c_double, c_int]),
            "oracle_u_gauss": (c_double, [c_double, c_double, c_double]),
            "oracle_q_gauss": (c_double, [c_double, c_double, c_double]),
            "oracle_q_filter": (c_double, [c_int, c_double, c_double, c_int]),
            "oracle_default_cut": (c_double, [c_int]),
            "oracle_fft2": (None, [_D, c_int, c_int]),
            "oracle_ks_forward": (None, [_D, _D, _D, c_int]),
            "oracle_ks_invert": (None, [_D, _D, _D, _D, c_int]),
            "oracle_starlet": (None, [_D, _D, c_int, c_int, c_int]),
            "oracle_map_starlet": (None, [_D, _D, _D, c_int, c_int, c_int]),
            "oracle_map_direct": (None, [_D, _D, _D, c_int, c_int, c_double, c_int, c_double]),
            "oracle_map_direct_at": (None, [_D, _D, _I, _I, c_int, _D, c_int, c_int, c_double, c_int, c_double]),
            "oracle_map_direct_masked_at": (None, [_D, _D, _D, _I, _I, c_int, _D, _D, c_int, c_int, c_double, c_int,
                                                    c_double]),
            "oracle_map_noise_expected_at": (None, [_D, _D, _I, _I, c_int, _D, c_int, c_int]),
            "oracle_splitmix64": (c_u64, [c_u64, c_u64]),
            "oracle_noise_u": (c_double, [c_u64, c_int, c_int, c_int, c_int]),
            "oracle_rotate_shear": (None, [_D, _D, _D, _D, c_int, c_int, c_u64]),
            "oracle_map_noise": (None, [_D, _D, _D, _D, c_int, c_int, c_int, c_u64, c_int]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _in(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.shape != (n, n):
        raise ValueError(f"expected shape {(n, n)}, got {a.shape}")
    return a


def _p(a):
    return a.ctypes.data_as(_D)


def _n_of(a):
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("maps are square n x n")
    return a.shape[0]


def _pow2_n(a):
    n = _n_of(a)
    if n < 1 or n & (n - 1):
        raise ValueError("the radix-2 FFT needs n a power of two")
    return n


MIRROR, PERIODIC = 0, 1
STARLET_Q, S98, JBJ04, VW98 = 0, 1, 2, 3


# --- filters (Sec. 4) ------------------------------------------------------
def phi_b3(x):
    return _load().oracle_phi_b3(float(x))


def starlet_taps():
    h = np.zeros(5)
    _load().oracle_starlet_taps(_p(h))
    return h


def u_starlet(eta):
    return _load().oracle_u_starlet(float(eta))


def q_starlet(eta):
    return _load().oracle_q_starlet(float(eta))


def u_s98(v, theta, ell=3):
    return _load().oracle_u_s98(float(v), float(theta), int(ell))


def q_s98(v, theta, ell=3):
    return _load().oracle_q_s98(float(v), float(theta), int(ell))


def u_gauss(v, theta, b):
    return _load().oracle_u_gauss(float(v), float(theta), float(b))


def q_gauss(v, theta, b):
    return _load().oracle_q_gauss(float(v), float(theta), float(b))


def q_filter(filt, v, theta, ell=3):
    return _load().oracle_q_filter(int(filt), float(v), float(theta), int(ell))


def default_cut(filt):
    return _load().oracle_default_cut(int(filt))


# --- transforms --------------------------------------------------------------
def fft2(a, inverse=False):
    """2-D FFT (forward unnormalised, inverse / n^2) of a complex n x n array."""
    a = np.ascontiguousarray(a, dtype=np.complex128).copy()
    n = _pow2_n(a)
    _load().oracle_fft2(a.view(np.float64).ctypes.data_as(_D), n, 1 if inverse else 0)
    return a


def ks_forward(kappa):
    """gamma1, gamma2 = KS forward of kappa (Sec. 4.5)."""
    k = _in(kappa)
    n = _pow2_n(k)
    g1, g2 = np.empty_like(k), np.empty_like(k)
    _load().oracle_ks_forward(_p(k), _p(g1), _p(g2), n)
    return g1, g2


def ks_invert(g1, g2):
    """(kappa_E, kappa_B) = KS inverse of the shear (Sec. 4.5)."""
    a = _in(g1)
    n = _pow2_n(a)
    b = _in(g2, n)
    kE, kB = np.empty_like(a), np.empty_like(a)
    _load().oracle_ks_invert(_p(a), _p(b), _p(kE), _p(kB), n)
    return kE, kB


def starlet(kappa, J, boundary=MIRROR):
    """(J, n, n) pyramid: w_1 .. w_{J-1}, then the smooth array (Sec. 3)."""
    k = _in(kappa)
    n = _n_of(k)
    pyr = np.empty((J, n, n))
    _load().oracle_starlet(_p(k), _p(pyr), n, int(J), int(boundary))
    return pyr


def map_starlet(g1, g2, J, boundary=MIRROR):
    """KS inversion then the starlet of kappa_E."""
    a = _in(g1)
    n = _pow2_n(a)
    b = _in(g2, n)
    pyr = np.empty((J, n, n))
    _load().oracle_map_starlet(_p(a), _p(b), _p(pyr), n, int(J), int(boundary))
    return pyr


def map_direct(g1, g2, filt, theta, ell=3, cut_over_theta=0.0):
    """Brute-force M_ap map from tangential shear (eq. shearmap)."""
    a = _in(g1)
    n = _n_of(a)
    b = _in(g2, n)
    m = np.empty_like(a)
    _load().oracle_map_direct(_p(a), _p(b), _p(m), n, int(filt), float(theta), int(ell), float(cut_over_theta))
    return m


def map_direct_at(g1, g2, ys, xs, filt, theta, ell=3, cut_over_theta=0.0):
    a = _in(g1)
    n = _n_of(a)
    b = _in(g2, n)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.empty(len(ys))
    _load().oracle_map_direct_at(_p(a), _p(b), ys.ctypes.data_as(_I), xs.ctypes.data_as(_I), len(ys), _p(out), n,
                                 int(filt), float(theta), int(ell), float(cut_over_theta))
    return out


def map_direct_masked_at(g1, g2, w, ys, xs, filt, theta, ell=3, cut_over_theta=0.0):
    """Weighted direct M_ap (missing data, Sec. 4.3 and 4.5) at listed pixels:
    returns (M, coverage) with M = N_R sum w Q gamma_t / sum w."""
    a = _in(g1)
    n = _n_of(a)
    b = _in(g2, n)
    c = _in(w, n)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    m = np.empty(len(ys))
    cov = np.empty(len(ys))
    _load().oracle_map_direct_masked_at(_p(a), _p(b), _p(c), ys.ctypes.data_as(_I), xs.ctypes.data_as(_I), len(ys),
                                        _p(m), _p(cov), n, int(filt), float(theta), int(ell), float(cut_over_theta))
    return m, cov


def map_direct_masked(g1, g2, w, filt, theta, ell=3, cut_over_theta=0.0):
    """Weighted direct M_ap over the whole map: (M, coverage), each n x n."""
    n = _n_of(_in(g1))
    ys, xs = np.mgrid[0:n, 0:n]
    m, cov = map_direct_masked_at(g1, g2, w, ys.ravel(), xs.ravel(), filt, theta, ell, cut_over_theta)
    return m.reshape(n, n), cov.reshape(n, n)


def splitmix64(seed, index):
    return int(_load().oracle_splitmix64(int(seed) & (2**64 - 1), int(index) & (2**64 - 1)))


def noise_u(seed, r, y, x, n):
    return _load().oracle_noise_u(int(seed) & (2**64 - 1), int(r), int(y), int(x), int(n))


def rotate_shear(g1, g2, r, seed):
    a = _in(g1)
    n = _pow2_n(a)
    b = _in(g2, n)
    o1, o2 = np.empty_like(a), np.empty_like(a)
    _load().oracle_rotate_shear(_p(a), _p(b), _p(o1), _p(o2), n, int(r), int(seed) & (2**64 - 1))
    return o1, o2


def map_noise(g1, g2, J, R, seed, boundary=MIRROR, with_snr=True):
    """(var, snr): per-band variance over R rotated realisations and S/N."""
    a = _in(g1)
    n = _pow2_n(a)
    b = _in(g2, n)
    var = np.empty((J - 1, n, n))
    snr = np.empty((J - 1, n, n)) if with_snr else None
    _load().oracle_map_noise(_p(a), _p(b), _p(var), _p(snr) if with_snr else None, n, int(J), int(R),
                             int(seed) & (2**64 - 1), int(boundary))
    return var, snr


def map_noise_expected_at(g1, g2, J, ys, xs):
    """Exact expected noise variance of bands 1..J-1 (periodic boundary) at
    listed pixels: [J-1, npts]."""
    a = _in(g1)
    n = _pow2_n(a)
    b = _in(g2, n)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    out = np.empty((J - 1, len(ys)))
    _load().oracle_map_noise_expected_at(_p(a), _p(b), ys.ctypes.data_as(_I), xs.ctypes.data_as(_I), len(ys),
                                         _p(out), n, int(J))
    return out


def map_noise_expected(g1, g2, J):
    """Exact expected noise variance over the whole map: [J-1, n, n]."""
    n = _pow2_n(_in(g1))
    ys, xs = np.mgrid[0:n, 0:n]
    return map_noise_expected_at(g1, g2, J, ys.ravel(), xs.ravel()).reshape(J - 1, n, n)
