"""Shared test helpers: seeded shear inputs and the per-band error metric."""
import numpy as np

import oracle
from paper_1204_4293_gb300 import synth

# max |gpu - oracle| / RMS(oracle band): the fp32 bound is the one the
# method's accuracy target states; fp64 is bounded by FP64 rounding of the
# O(log n) FFT depth and the a-trous sums.
TOL = {np.float32: 1e-5, np.float64: 1e-12}


def shear(n, seed=1, alpha=2.0, sigma=0.1, dtype=np.float64):
    """gamma1, gamma2 of a GRF convergence (oracle forward KS) plus shape noise."""
    kappa = synth.grf_kappa(n, alpha=alpha, seed=seed)
    g1, g2 = oracle.ks_forward(kappa)
    n1, n2 = synth.shape_noise(n, sigma=sigma, seed=seed)
    return (g1 + n1).astype(dtype), (g2 + n2).astype(dtype)


def rel_err(got, ref):
    ref = np.asarray(ref, dtype=np.float64)
    rms = np.sqrt(np.mean(ref ** 2))
    return float(np.abs(np.asarray(got, dtype=np.float64) - ref).max() / rms)


def band_errs(got, ref):
    """Per-array max|diff| / RMS(oracle array) over the last two axes."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return [rel_err(got[j], ref[j]) for j in range(ref.shape[0])]
