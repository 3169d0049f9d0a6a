"""Comparison helpers shared by the GPU parity tests."""
import numpy as np


def fwd_err(gpu, orc, amb=None):
    """max |gpu - oracle| beyond the ambiguity allowance, relative to max|oracle|.

    ``amb`` (from the oracle) bounds, per output, what a sample whose TOF
    window decision sits within the FP32/FP64 rounding band can contribute;
    either decision is correct there."""
    gpu = np.asarray(gpu, dtype=np.float64)
    orc = np.asarray(orc, dtype=np.float64)
    scale = max(np.abs(orc).max(), 1e-30)
    d = np.abs(gpu - orc)
    if amb is not None:
        d = np.maximum(d - np.asarray(amb, dtype=np.float64), 0.0)
    return float(d.max() / scale) if d.size else 0.0


def rel_l2(gpu, orc):
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    orc = np.asarray(orc, dtype=np.float64).ravel()
    n = np.linalg.norm(orc)
    return float(np.linalg.norm(gpu - orc) / max(n, 1e-30))


FWD_TOL = 1e-5   # max|err| <= 1e-5 * max|oracle|
BACK_TOL = 1e-4  # relative L2
AMB_EPS = 1e-3   # mm: TOF truncation decisions within this band are ambiguous
