"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and shapes them into Gaussian random
fields; it holds none of the pipeline's arithmetic (no shear/convergence
relation, no wavelet filter).  The tests and the benchmark both take their
inputs from here.

Recipe (the paper analyses 1024 x 1024 pixel maps, Sec. 5.1, and gives no
data set; a Gaussian random field stands in for its convergence maps):
  kappa_hat(k) = |k|^(-alpha/2) (a + i b) / sqrt(2), a, b ~ N(0, 1) iid,
  |k| in integer frequency units, kappa_hat(0) = 0;
  kappa = Re IFFT2(kappa_hat), rescaled to the requested RMS (default 0.02);
  shape noise: N(0, sigma^2) per pixel per shear component (default 0.1);
  masks (missing data: bright stars, bad pixels): 0/1 weights with discs of
  log-uniform radius at uniform centres until the masked fraction is reached,
  plus one bad column strip.
The shear of a field is obtained by the caller through a forward
Kaiser-Squires transform (the oracle's in tests, the library's on the GPU).
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def grf_kappa(n: int, alpha: float = 2.0, rms: float | None = 0.02, seed: int = 1) -> np.ndarray:
    """n x n float64 Gaussian random field with P(k) proportional to k^-alpha
    (exactly |kappa_hat(k)|^2 = |k|^-alpha in expectation when rms is None;
    otherwise rescaled to the given sample RMS)."""
    rng = _rng(seed)
    f = np.fft.fftfreq(n) * n
    k = np.sqrt(f[None, :] ** 2 + f[:, None] ** 2)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (-alpha / 2.0)
    a = rng.standard_normal((n, n))
    b = rng.standard_normal((n, n))
    field = np.real(np.fft.ifft2(amp * (a + 1j * b) / np.sqrt(2.0)))
    field -= field.mean()
    if rms is None:
        return field
    std = field.std()
    return field * (rms / std) if std > 0 else field


def shape_noise(n: int, sigma: float = 0.1, seed: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """Two n x n float64 maps of iid N(0, sigma^2) shape noise."""
    rng = _rng(seed + 0x5EED)
    return sigma * rng.standard_normal((n, n)), sigma * rng.standard_normal((n, n))


def delta_kappa(n: int, amplitude: float = 1.0) -> np.ndarray:
    """A null convergence map with one central delta (the Fig. 2 input)."""
    k = np.zeros((n, n))
    k[n // 2, n // 2] = amplitude
    return k


def white(shape, seed: int = 1, scale: float = 1.0) -> np.ndarray:
    """iid N(0, scale^2) values (generic test input)."""
    return scale * _rng(seed).standard_normal(shape)


def star_mask(n: int, frac: float = 0.15, r_min: float = 2.0, r_max: float | None = None, seed: int = 1) -> np.ndarray:
    """n x n float64 weights: 1 for data, 0 inside masked discs (stars) and one
    bad 2-pixel column strip, drawn until about `frac` of the field is masked."""
    rng = _rng(seed + 0xA5C)
    r_max = max(r_min, n / 32.0) if r_max is None else r_max
    w = np.ones((n, n))
    yy, xx = np.mgrid[0:n, 0:n]
    if n >= 8:
        c = int(rng.integers(0, n - 2))
        w[:, c:c + 2] = 0.0
    for _ in range(100000):
        if 1.0 - w.mean() >= frac:
            break
        cy, cx = rng.random(2) * n
        r = float(np.exp(rng.uniform(np.log(r_min), np.log(r_max))))
        w[(yy - cy) ** 2 + (xx - cx) ** 2 <= r * r] = 0.0
    return w
