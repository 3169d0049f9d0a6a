"""ctypes wrapper around the FP64 C oracle (``joseph_oracle.c``).

TEST INFRASTRUCTURE ONLY (see package docstring).  Inputs are promoted to
double exactly; outputs are double.  Geometry objects only need ``shape``,
``origin`` and ``voxsize`` attributes; TOF objects ``bin_width``, ``sigma``,
``n_sigmas`` and ``n_bins``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "joseph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
MODES = {"nontof": 0, "tof_sino": 1, "tof_lm": 2}
_libs = {}
_lock = threading.Lock()


def _libpath(mutant: int) -> str:
    return os.path.join(_BUILD, "liboracle.so" if mutant == 0 else f"liboracle_m{mutant}.so")


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _libpath(mutant)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           "-fno-fast-math", f"-DOR_MUTANT={int(mutant)}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(mutant: int = 0):
    with _lock:
        if mutant in _libs:
            return _libs[mutant]
        lib = ctypes.CDLL(build(mutant))
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.or_fwd.argtypes = [P, P, I64, P, P, P, ctypes.c_int, P, I64, P, P, P, P, P, ctypes.c_int]
        lib.or_fwd.restype = ctypes.c_int
        lib.or_back.argtypes = [P, P, I64, P, P, P, ctypes.c_int, P, I64, P, P, P, P, ctypes.c_int]
        lib.or_back.restype = ctypes.c_int
        D = ctypes.c_double
        lib.or_fwd_ex.argtypes = [P, P, I64, P, P, P, ctypes.c_int, P, I64, P, P, P, P, I64, D, P, P, P,
                                  ctypes.c_int]
        lib.or_fwd_ex.restype = ctypes.c_int
        lib.or_back_ex.argtypes = [P, P, I64, P, P, P, ctypes.c_int, P, I64, P, P, P, P, I64, D, P, P,
                                   ctypes.c_int]
        lib.or_back_ex.restype = ctypes.c_int
        lib.or_tof_weight.argtypes = [ctypes.c_double] * 5
        lib.or_tof_weight.restype = ctypes.c_double
        lib.or_principal_axis.argtypes = [P, P]
        lib.or_principal_axis.restype = ctypes.c_int
        _libs[mutant] = lib
        return lib


def _d(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _geom(geom):
    n = np.ascontiguousarray(np.asarray(geom.shape, dtype=np.int64))
    o = _d(geom.origin)
    v = _d(geom.voxsize)
    return n, o, v


def _tof(tof, amb_eps):
    if tof is None:
        return None, 0
    return _d([tof.bin_width, tof.sigma, tof.n_sigmas, amb_eps]), int(tof.n_bins)


def _table(tof):
    """(table, nodes, half width) of a tabulated TOF kernel, or (None, 0, 0)."""
    kernel = getattr(tof, "kernel", None) if tof is not None else None
    if kernel is None:
        return None, 0, 0.0
    t = _d(kernel)
    return t, int(t.size), float(tof.kernel_half_width)


def _common(xs, xe, mode, tof_bin, delta):
    xs = _d(xs).reshape(-1, 3)
    xe = _d(xe).reshape(-1, 3)
    if xs.shape != xe.shape:
        raise ValueError("xs/xe shape mismatch")
    n = xs.shape[0]
    tb = None if tof_bin is None else np.ascontiguousarray(np.asarray(tof_bin, dtype=np.int64).reshape(n))
    de = None if delta is None else _d(delta).reshape(n)
    m = MODES[mode]
    return xs, xe, n, m, tb, de


def fwd(xs, xe, img, geom, mode="nontof", tof=None, tof_bin=None, delta=None,
        threads=1, amb_eps=0.0, return_amb=False, mutant=0, sigma=None):
    """Forward projection (FP64).  Returns [n] or [n, n_bins] (TOF sinogram);
    with ``return_amb`` also the per-output ambiguity magnitude.  ``sigma``:
    optional per-LOR Gaussian sigma; a tabulated kernel comes with ``tof``."""
    lib = load(mutant)
    xs, xe, n, m, tb, de = _common(xs, xe, mode, tof_bin, delta)
    sg = None if sigma is None else _d(sigma).reshape(n)
    tab, tn, thw = _table(tof)
    ng, og, vg = _geom(geom)
    img = _d(img).reshape(-1)
    if img.size != int(np.prod(ng)):
        raise ValueError("image size does not match geometry")
    tp, nb = _tof(tof, amb_eps)
    nout = nb if m == 1 else 1
    out = np.zeros(n * nout, dtype=np.float64)
    amb = np.zeros(n * nout, dtype=np.float64) if return_amb else None
    rc = lib.or_fwd_ex(_ptr(xs), _ptr(xe), n, _ptr(ng), _ptr(og), _ptr(vg), m, _ptr(tp), nb,
                       _ptr(tb), _ptr(de), _ptr(sg), _ptr(tab), tn, thw, _ptr(img), _ptr(out), _ptr(amb),
                       int(threads))
    if rc != 0:
        raise ValueError(f"or_fwd failed ({rc})")
    shape = (n, nout) if m == 1 else (n,)
    if return_amb:
        return out.reshape(shape), amb.reshape(shape)
    return out.reshape(shape)


def back(xs, xe, y, geom, mode="nontof", tof=None, tof_bin=None, delta=None, threads=1,
         mutant=0, sigma=None):
    """Back projection A^T y (FP64), returned as an image of ``geom.shape``."""
    lib = load(mutant)
    xs, xe, n, m, tb, de = _common(xs, xe, mode, tof_bin, delta)
    sg = None if sigma is None else _d(sigma).reshape(n)
    tab, tn, thw = _table(tof)
    ng, og, vg = _geom(geom)
    tp, nb = _tof(tof, 0.0)
    nin = nb if m == 1 else 1
    y = _d(y).reshape(-1)
    if y.size != n * nin:
        raise ValueError("y size mismatch")
    img = np.zeros(int(np.prod(ng)), dtype=np.float64)
    rc = lib.or_back_ex(_ptr(xs), _ptr(xe), n, _ptr(ng), _ptr(og), _ptr(vg), m, _ptr(tp), nb,
                        _ptr(tb), _ptr(de), _ptr(sg), _ptr(tab), tn, thw, _ptr(y), _ptr(img), int(threads))
    if rc != 0:
        raise ValueError(f"or_back failed ({rc})")
    return img.reshape(tuple(int(s) for s in ng))


def tof_weight(tau, centre, bin_width, sigma, n_sigmas, mutant=0):
    """The oracle's TOF bin weight g (Sec. 2.1: Gaussian convolved with a
    bin-wide rect, truncated)."""
    return load(mutant).or_tof_weight(float(tau), float(centre), float(bin_width),
                                      float(sigma), float(n_sigmas))


def principal_axis(xs, xe, mutant=0):
    xs = _d(xs).reshape(3)
    xe = _d(xe).reshape(3)
    return int(load(mutant).or_principal_axis(_ptr(xs), _ptr(xe)))
