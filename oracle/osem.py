"""FP64 listmode OSEM and log-likelihood gradient on top of the oracle
projector.  TEST INFRASTRUCTURE ONLY (see package docstring).

Listmode OSEM (paper Sec. 2.6 and 3, Fig. 6 caption): with sensitivity image
s = A^T 1 over all possible LORs, subset S of n_sub event subsets, additive
background b and unit event values,
    x <- x / (s / n_sub) * A_S^T ( 1 / (A_S x + b) ),   x = 0 where s = 0.
Subset m holds the events e with e mod n_sub == m.

Sinogram OSEM (``sino_osem_subset_update``) uses per-subset sensitivities
s_S = A_S^T 1 and an additive contamination sinogram c:
    x <- x / s_S * A_S^T ( y / (A_S x + c) ).

With the image-based resolution model H (``fwhm_mm`` > 0, see
``resolution.py``) the update is
    x <- x / (s' / n_sub) * H^T A_S^T ( 1 / (A_S H x + b) )
and ``sens`` is the caller's s' = H^T A^T 1.
"""
from __future__ import annotations

import numpy as np

from . import joseph, resolution


def _subset(arrs, m, n_sub, contiguous=False):
    if contiguous:  # planted mistake: a block of events instead of e mod n_sub
        n = len(arrs[0])
        blk = -(-n // n_sub)
        return [None if a is None else np.asarray(a)[m * blk:(m + 1) * blk] for a in arrs]
    return [None if a is None else np.asarray(a)[m::n_sub] for a in arrs]


def lm_osem_subset_update(x, xs, xe, tof_bin, geom, tof, sens, b, m, n_sub, threads=1, fwhm_mm=0.0,
                          truncate=4.0, sigma=None, _mutant=0):
    """One subset update of TOF listmode OSEM (double precision), with the
    resolution model when ``fwhm_mm`` > 0 and per-event TOF sigma when
    ``sigma`` is given.

    ``_mutant`` plants a known mistake (used only by the pin test that checks
    the pins catch it): 1 = sensitivity not divided by n_sub, 2 = background
    dropped from the ratio, 3 = a contiguous block of events as the subset,
    4 = H^T not applied to the back projection."""
    sxs, sxe, stb, ssg = _subset([xs, xe, tof_bin, sigma], m, n_sub, contiguous=(_mutant == 3))
    res = np.any(np.asarray(fwhm_mm, dtype=np.float64) > 0)
    y = resolution.gauss3d(x, geom, fwhm_mm, truncate) if res else x
    p = joseph.fwd(sxs, sxe, y, geom, mode="tof_lm", tof=tof, tof_bin=stb, threads=threads, sigma=ssg)
    q = 1.0 / p if _mutant == 2 else 1.0 / (p + b)
    bp = joseph.back(sxs, sxe, q, geom, mode="tof_lm", tof=tof, tof_bin=stb, threads=threads, sigma=ssg)
    if res and _mutant != 4:
        bp = resolution.gauss3d(bp, geom, fwhm_mm, truncate, adjoint=True)
    s = np.asarray(sens, dtype=np.float64) / (1 if _mutant == 1 else n_sub)
    out = np.zeros_like(np.asarray(x, dtype=np.float64))
    pos = s > 0
    out[pos] = np.asarray(x, dtype=np.float64)[pos] * bp[pos] / s[pos]
    return out


def lm_osem(xs, xe, tof_bin, geom, tof, sens, b, n_iter, n_sub, threads=1, x0=None, fwhm_mm=0.0,
            truncate=4.0, sigma=None):
    """Full TOF listmode OSEM: x0 = 1 on voxels with s > 0 (else 0)."""
    sens = np.asarray(sens, dtype=np.float64)
    x = (sens > 0).astype(np.float64) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    for _ in range(n_iter):
        for m in range(n_sub):
            x = lm_osem_subset_update(x, xs, xe, tof_bin, geom, tof, sens, b, m, n_sub, threads, fwhm_mm,
                                      truncate, sigma)
    return x


def sino_osem_subset_update(x, xs, xe, y, c, sens, geom, mode="nontof", tof=None, threads=1, _mutant=0):
    """One sinogram OSEM subset update (paper Sec. 2.6: an OSEM subset update
    with 34 subsets of equally spaced views; the emission and contamination
    sinograms of Sec. 4).  For the subset's LORs (xs, xe), emission counts y
    and additive contamination c (both [n] non-TOF or [n, n_bins] TOF
    sinogram) and subset sensitivity sens = A_S^T 1:
        x <- x / sens * A_S^T ( y / (A_S x + c) ),   x = 0 where sens = 0,
    reading y / (A_S x + c) as 0 where A_S x + c = 0 (no expected counts).

    ``_mutant`` (pin test only): 5 = contamination dropped from the
    denominator, 6 = the ratio inverted."""
    p = joseph.fwd(xs, xe, x, geom, mode=mode, tof=tof, threads=threads)
    den = p + (0.0 if _mutant == 5 else np.asarray(c, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64)
    q = np.zeros_like(den)
    nz = den > 0
    q[nz] = den[nz] / y[nz] if _mutant == 6 else y[nz] / den[nz]
    bp = joseph.back(xs, xe, q, geom, mode=mode, tof=tof, threads=threads)
    s = np.asarray(sens, dtype=np.float64)
    out = np.zeros_like(np.asarray(x, dtype=np.float64))
    pos = s > 0
    out[pos] = np.asarray(x, dtype=np.float64)[pos] * bp[pos] / s[pos]
    return out


def poisson_loglik_grad(x, xs, xe, tof_bin, geom, tof, w, b, threads=1, _mutant=0):
    """f(x) = sum_e w_e log((A x)_e + b) and its gradient A^T (w / (A x + b)).
    ``_mutant`` (pin test only): 7 = the weights dropped from the gradient."""
    p = joseph.fwd(xs, xe, x, geom, mode="tof_lm", tof=tof, tof_bin=tof_bin, threads=threads)
    w = np.asarray(w, dtype=np.float64)
    val = float(np.sum(w * np.log(p + b)))
    g = joseph.back(xs, xe, (1.0 if _mutant == 7 else w) / (p + b), geom, mode="tof_lm", tof=tof,
                    tof_bin=tof_bin, threads=threads)
    return val, g
