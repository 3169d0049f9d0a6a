"""FP64 image-based resolution model.  TEST INFRASTRUCTURE ONLY (see the
package docstring).

Paper Sec. 2.6 (listmode OSEM set-up): every listmode OSEM reconstruction
models the scanner resolution with a shift-invariant, isotropic 3D Gaussian
of 4.5 mm FWHM applied in image space; Sec. 4 counts two such convolutions
per subset (one before the forward projection, one after the back
projection).  The paper does not fix the discretisation; this module reads it
as follows (the same reading the CUDA path implements):

  * sigma = FWHM / sqrt(8 ln 2), per axis in mm (an anisotropic FWHM is
    allowed; the paper's case is 4.5 mm on every axis);
  * axis a uses the Gaussian sampled at the voxel-centre offsets t * d_a,
    t = -R_a .. R_a with R_a = ceil(truncate * sigma_a / d_a) (truncate = 4
    by default), normalised so that the R_a taps sum to 1; sigma_a = 0 gives
    the single tap 1 (identity);
  * the 3D kernel is the product of the three axis kernels;
  * the image is zero outside its grid, so the operator H is the plain
    truncated correlation and its adjoint H^T is the correlation with the
    reversed taps (equal to H, as the taps are symmetric).

With the resolution model the listmode OSEM subset update (paper Sec. 2.6
and 3) reads
    x <- x / (s' / n_sub) * H^T A_S^T ( 1 / (A_S H x + b) ),  s' = H^T A^T 1,
and x = 0 where s' = 0.
"""
from __future__ import annotations

import math

import numpy as np


def sigma_from_fwhm(fwhm_mm):
    """Gaussian sigma (mm) of a given FWHM: FWHM = sqrt(8 ln 2) sigma."""
    return float(fwhm_mm) / math.sqrt(8.0 * math.log(2.0))


def gauss_taps(fwhm_mm, voxsize, truncate=4.0, _mutant=0):
    """Per-axis taps [w_0, w_1, w_2] (each of length 2 R_a + 1, FP64).

    ``fwhm_mm`` is a scalar or three per-axis values.  ``_mutant`` plants a
    known mistake (used only by the pin test that checks the pins catch it):
    1 = taps not normalised, 2 = sigma taken as FWHM / 2, 3 = taps offset by
    one sample."""
    f = np.broadcast_to(np.asarray(fwhm_mm, dtype=np.float64), (3,))
    taps = []
    for a in range(3):
        s = sigma_from_fwhm(f[a]) if _mutant != 2 else float(f[a]) / 2.0
        d = float(voxsize[a])
        if s <= 0.0:
            taps.append(np.ones(1))
            continue
        r = int(math.ceil(truncate * s / d))
        t = np.arange(-r, r + 1, dtype=np.float64)
        if _mutant == 3:
            t = t + 1.0
        w = np.exp(-0.5 * (t * d / s) ** 2)
        if _mutant != 1:
            w = w / w.sum()
        taps.append(w)
    return taps


def _shifted(x, sh):
    """y[i] = x[i + sh] along all three axes, zero where i + sh is outside."""
    y = np.zeros_like(x)
    src, dst = [], []
    for n, s in zip(x.shape, sh):
        if abs(s) >= n:
            return y
        src.append(slice(max(0, s), min(n, n + s)))
        dst.append(slice(max(0, -s), min(n, n - s)))
    y[tuple(dst)] = x[tuple(src)]
    return y


def gauss3d(img, geom, fwhm_mm, truncate=4.0, adjoint=False, _mutant=0):
    """(H x)_i = sum_t w_0[t_0] w_1[t_1] w_2[t_2] x_{i + t - R}, x = 0 off the
    grid: the 3D correlation written out over every tap of the product kernel
    (no separable shortcut).  ``adjoint`` applies H^T (the reversed taps).
    ``img`` is one image of ``geom.shape`` or a stack of them."""
    x = np.asarray(img, dtype=np.float64)
    if x.ndim == 4:
        return np.stack([gauss3d(xi, geom, fwhm_mm, truncate, adjoint, _mutant) for xi in x])
    taps = gauss_taps(fwhm_mm, geom.voxsize, truncate, _mutant)
    if _mutant == 4:  # axes 0 and 1 exchanged
        taps = [taps[1], taps[0], taps[2]]
    if adjoint:
        taps = [w[::-1] for w in taps]
    r = [(len(w) - 1) // 2 for w in taps]
    out = np.zeros_like(x)
    for t0, w0 in enumerate(taps[0]):
        for t1, w1 in enumerate(taps[1]):
            for t2, w2 in enumerate(taps[2]):
                out += (w0 * w1 * w2) * _shifted(x, (t0 - r[0], t1 - r[1], t2 - r[2]))
    return out
