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


def _edge_weight(tof):
    """Largest untruncated TOF bin weight of a sample within AMB_EPS of the
    truncation radius R = n_sigmas sigma + D / 2 (Sec. 2.1, 2.6): the
    weight falls with |dist| there, so its value at R - AMB_EPS."""
    import math
    R = tof.n_sigmas * tof.sigma + 0.5 * tof.bin_width
    k = 1.0 / (math.sqrt(2.0) * tof.sigma)
    d = R - AMB_EPS
    return 0.5 * (math.erf((d + 0.5 * tof.bin_width) * k) - math.erf((d - 0.5 * tof.bin_width) * k))


def amb_check(amb, xs, xe, geom, tof, img_absmax, max_frac=0.01):
    """Bounds what the ambiguity allowance of ``fwd_err`` can absorb.

    Per output at most two samples (one per edge of the TOF window; plane
    samples lie w0 >= v_a apart along the LOR, far more than 2 AMB_EPS) can
    fall in the band, each contributing at most w0 * edge weight * max|f|.
    Also the outputs with a nonzero allowance must be rare (the band is
    2 AMB_EPS wide per edge).  Prints and returns (fraction of outputs with
    amb > 0, max amb / (w0 * max|f|))."""
    xs = np.asarray(xs, np.float64).reshape(-1, 3)
    xe = np.asarray(xe, np.float64).reshape(-1, 3)
    amb = np.asarray(amb, np.float64).reshape(len(xs), -1)
    d = xe - xs
    L = np.linalg.norm(d, axis=1)
    a = np.argmax(np.abs(d), axis=1)
    da = np.abs(d[np.arange(len(d)), a])
    v = np.asarray(geom.voxsize, np.float64)
    w0 = np.where(da > 0, v[a] * L / np.maximum(da, 1e-300), 0.0)
    scale = np.maximum(w0 * float(img_absmax), 1e-300)[:, None]
    ratio = float((amb / scale).max()) if amb.size else 0.0
    frac = float(np.count_nonzero(amb) / max(amb.size, 1))
    print(f"TOF-edge allowance: {frac:.2e} of outputs, max {ratio:.3e} x w0 max|f| "
          f"(bound 2 x {_edge_weight(tof):.3e})")
    assert frac <= max_frac
    assert ratio <= 2.0 * _edge_weight(tof) * (1.0 + 1e-9)
    return frac, ratio
