"""Thin ctypes binding of libjoseph (declared in include/joseph.h).

Argument marshalling only: every function converts torch CUDA tensors into
device pointers, passes the current CUDA stream and raises ``JosephError``
on a non-zero status.  All compute runs in the library's CUDA kernels; there
is no CPU path.  Function names mirror the C entry points (``jp_fwd`` ...);
short aliases (``fwd`` ...) are provided for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import torch

from . import build as _build

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
F32 = ctypes.c_float

TOF_MODES = {"nontof": 0, "tof_sino": 1, "tof_lm": 2}
JP_PLAN_KEEP_ORDER = 1
JP_PLAN_TOF_EXACT = 2
JP_PLAN_INTERLEAVED = 4
JP_PLAN_TILES = 8
OSEM_PATHS = {"auto": 0, "quads": 1, "direct": 2}
OSEM_DIRECT_VOXELS_PER_EVENT = 24  # JP_OSEM_DIRECT_VOXELS_PER_EVENT


class JosephError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libjoseph error {code}: {msg}")
        self.code = code


class ImageGeomC(ctypes.Structure):
    _fields_ = [("n", I32 * 3), ("origin", F32 * 3), ("voxsize", F32 * 3)]


class TofC(ctypes.Structure):
    _fields_ = [("bin_width", F32), ("sigma", F32), ("n_sigmas", F32), ("n_bins", I32),
                ("kernel", P), ("kernel_nodes", I32), ("kernel_half_width", F32)]


class ResolutionC(ctypes.Structure):
    _fields_ = [("fwhm_mm", F32 * 3), ("truncate", F32)]


class PlanOptsC(ctypes.Structure):
    _fields_ = [("block", I32), ("slope_bins", I32), ("offset_bins", I32), ("window_bins", I32),
                ("tof_bin_width", F32), ("lors_per_warp", I32), ("flags", I32), ("zoff_bins", I32),
                ("max_ctas_per_sm", I32), ("tile_lors", I32)]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "jp_plan_create_batch": [ctypes.POINTER(P), P, P, P, P, P, I32, P, P, P],
    "jp_plan_create": [ctypes.POINTER(P), P, P, P, P, I64, P, P, P],
    "jp_plan_rebind": [P, P, P, P, P, P, I32, P],
    "jp_plan_destroy": [P],
    "jp_plan_set_event_sigma": [P, P, P],
    "jp_plan_create_batch_det": [ctypes.POINTER(P), P, P, P, I32, P, P, P, I32, P, P, P],
    "jp_plan_rebind_det": [P, P, P, P, I32, P, P, P, I32, P],
    "jp_plan_info": [P, P, P, P, P],
    "jp_fwd": [P, P, I64, P, P],
    "jp_back": [P, P, P, I64, P],
    "jp_fwd_tof_sino": [P, P, I64, P, P, P],
    "jp_back_tof_sino": [P, P, P, P, I64, P],
    "jp_fwd_tof_lm": [P, P, I64, P, P, P],
    "jp_back_tof_lm": [P, P, P, P, I64, P],
    "jp_fwd_lors": [P, P, P, P, I64, P, I32, P, P, P, P],
    "jp_back_lors": [P, P, P, P, I64, P, I32, P, P, P, P],
    "jp_osem_ratio": [P, P, P, P, I64, P],
    "jp_osem_update": [P, P, P, F32, I64, I32, I64, I64, P],
    "jp_osem_ratio_sino": [P, P, P, P, I64, P],
    "jp_sum_f64": [P, I64, P, P],
    "jp_count_samples": [P, I32, P, P, P],
    "jp_count_red_requests": [P, I32, P, P, P],
    "jp_bench_tof_bins": [P, I32, I32, P, P, P],
    "jp_osem_subset_tof_lm": [P, I32, I32, P, P, F32, F32, P, P],
    "jp_osem_init": [P, P, I64, P],
    "jp_osem_subset_tof_lm_dev": [P, I32, I32, P, P, F32, P, P, P],
    "jp_osem_subset_tof_lm_ex": [P, I32, I32, P, P, F32, F32, P, P, P, I32, P, P],
    "jp_gauss3d": [P, P, P, I32, P, P, P],
    "jp_poisson_loglik_value": [P, P, P, P, I64, P, P, P],
    "jp_poisson_loglik_grad": [P, P, P, P, P, I64, P, P],
    "jp_back_tof_lm_noalloc": [P, P, P, P, I64, P, P, P, P, P],
    "jp_bench_red": [P, I64, I32, I32, P, P],
    "jp_bench_red_pattern": [P, I64, I32, I32, I32, P, P],
}


def lib_path() -> str:
    return _build.LIB


def load():
    """Loads the in-tree libjoseph.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libjoseph is not built ({path}); run paper_2212_12519_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.jp_launch_count.restype = ctypes.c_uint64
        lib.jp_launch_count.argtypes = []
        lib.jp_last_error.restype = ctypes.c_char_p
        lib.jp_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        raise JosephError(rc, load().jp_last_error().decode())


def _stream(stream=None) -> P:
    s = torch.cuda.current_stream() if stream is None else stream
    return P(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor], dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return P(t.data_ptr())


def image_geom(geom) -> ImageGeomC:
    g = ImageGeomC()
    for i in range(3):
        g.n[i] = int(geom.shape[i])
        g.origin[i] = float(geom.origin[i])
        g.voxsize[i] = float(geom.voxsize[i])
    return g


def resolution(fwhm_mm, truncate: float = 4.0) -> ResolutionC:
    """jp_resolution of a scalar (isotropic) or per-axis FWHM in mm."""
    f = [float(fwhm_mm)] * 3 if isinstance(fwhm_mm, (int, float)) else [float(v) for v in fwhm_mm]
    if len(f) != 3:
        raise ValueError("fwhm_mm must be a scalar or three values")
    r = ResolutionC()
    for i in range(3):
        r.fwhm_mm[i] = f[i]
    r.truncate = float(truncate)
    return r


_kernel_tables: dict = {}


def _kernel_table(values, device) -> torch.Tensor:
    """Device copy of a tabulated TOF kernel, made once per table and device."""
    key = (tuple(values), str(device))
    t = _kernel_tables.get(key)
    if t is None:
        t = torch.tensor(values, dtype=torch.float32, device=device)
        _kernel_tables[key] = t
    return t


def tof_params(tof) -> TofC:
    kernel = getattr(tof, "kernel", None)
    if kernel is None:
        return TofC(float(tof.bin_width), float(tof.sigma), float(tof.n_sigmas), int(tof.n_bins), None, 0, 0.0)
    tab = _kernel_table(kernel, torch.device("cuda", torch.cuda.current_device()))
    return TofC(float(tof.bin_width), float(tof.sigma), float(tof.n_sigmas), int(tof.n_bins),
                P(tab.data_ptr()), int(tab.numel()), float(tof.kernel_half_width))


def _lors(xs, xe):
    if xs.dim() != 2 or xs.shape[1] != 3 or xs.shape != xe.shape:
        raise ValueError("xstart/xend must be [n, 3]")
    return _ptr(xs, torch.float32, "xstart"), _ptr(xe, torch.float32, "xend")


# ---------------------------------------------------------------------------
# plans
# ---------------------------------------------------------------------------
class Plan:
    """Owns a libjoseph plan (sorted, packed LORs of one or more frames)."""

    def __init__(self, handle: int, geom, n: int, n_frames: int, frame_offsets: Sequence[int],
                 has_tof_bin: bool):
        self._h = P(handle)
        self.geom = geom
        self.n = n
        self.n_frames = n_frames
        self.frame_offsets = list(frame_offsets)
        self.has_tof_bin = has_tof_bin

    @property
    def handle(self):
        if self._h is None or not self._h.value:
            raise RuntimeError("plan has been destroyed")
        return self._h

    def perm(self, stream=None) -> torch.Tensor:
        """A copy of the plan's permutation (binned position -> caller index)."""
        out = torch.empty(self.n, dtype=torch.int32, device="cuda")
        _check(load().jp_plan_info(self.handle, None, None, _ptr(out, torch.int32, "perm"), _stream(stream)))
        return out

    def destroy(self):
        if self._h is not None and self._h.value:
            _check(load().jp_plan_destroy(self._h))
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _opts(block=0, slope_bins=0, offset_bins=0, window_bins=0, tof_bin_width=0.0, keep_order=False,
          tof_exact=False, lors_per_warp=0, interleaved=False, zoff_bins=0, max_ctas_per_sm=0, tiles=False,
          tile_lors=0):
    flags = ((JP_PLAN_KEEP_ORDER if keep_order else 0) | (JP_PLAN_TOF_EXACT if tof_exact else 0)
             | (JP_PLAN_INTERLEAVED if interleaved else 0) | (JP_PLAN_TILES if tiles else 0))
    return PlanOptsC(int(block), int(slope_bins), int(offset_bins), int(window_bins),
                     float(tof_bin_width), int(lors_per_warp), flags, int(zoff_bins), int(max_ctas_per_sm),
                     int(tile_lors))


def jp_plan_create_batch(xs, xe, geom, frame_offsets, tof_bin=None, delta=None, stream=None,
                         **opts) -> Plan:
    pxs, pxe = _lors(xs, xe)
    off = (ctypes.c_int64 * len(frame_offsets))(*[int(v) for v in frame_offsets])
    h = P()
    g = image_geom(geom)
    o = _opts(**opts)
    _check(load().jp_plan_create_batch(ctypes.byref(h), pxs, pxe, _ptr(tof_bin, torch.int16, "tof_bin"),
                                       _ptr(delta, torch.float32, "delta"), off, len(frame_offsets) - 1,
                                       ctypes.byref(g), ctypes.byref(o), _stream(stream)))
    return Plan(h.value, geom, int(frame_offsets[-1]), len(frame_offsets) - 1, frame_offsets,
                tof_bin is not None)


def jp_plan_create(xs, xe, geom, tof_bin=None, delta=None, stream=None, **opts) -> Plan:
    return jp_plan_create_batch(xs, xe, geom, [0, int(xs.shape[0])], tof_bin, delta, stream, **opts)


def jp_plan_create_subsets(xs, xe, geom, n_subsets, tof_bin=None, delta=None, stream=None, **opts) -> Plan:
    """Plan whose frames are the listmode OSEM subsets e mod n_subsets
    (JP_PLAN_INTERLEAVED); all subsets share one image."""
    n = int(xs.shape[0])
    off = [0] * n_subsets + [n]
    plan = jp_plan_create_batch(xs, xe, geom, off, tof_bin, delta, stream, interleaved=True, **opts)
    plan.frame_offsets = [sum(n // n_subsets + (1 if f < n % n_subsets else 0) for f in range(m))
                          for m in range(n_subsets + 1)]
    return plan


def _det(det_start, det_end, det_xyz):
    if det_start.dim() != 1 or det_start.shape != det_end.shape:
        raise ValueError("det_start/det_end must be 1-D of equal length")
    if det_xyz.dim() != 2 or det_xyz.shape[1] != 3:
        raise ValueError("det_xyz must be [n_det, 3]")
    return (_ptr(det_start, torch.int32, "det_start"), _ptr(det_end, torch.int32, "det_end"),
            _ptr(det_xyz, torch.float32, "det_xyz"), int(det_xyz.shape[0]))


def jp_plan_create_batch_det(det_start, det_end, det_xyz, geom, frame_offsets, tof_bin=None, delta=None,
                             stream=None, **opts) -> Plan:
    """Plan from detector-index listmode events: LOR j runs from
    det_xyz[det_start[j]] to det_xyz[det_end[j]] (int32 indices, float32
    [n_det, 3] table, all on the device)."""
    pds, pde, pxyz, nd = _det(det_start, det_end, det_xyz)
    off = (ctypes.c_int64 * len(frame_offsets))(*[int(v) for v in frame_offsets])
    h = P()
    g = image_geom(geom)
    o = _opts(**opts)
    _check(load().jp_plan_create_batch_det(ctypes.byref(h), pds, pde, pxyz, nd,
                                           _ptr(tof_bin, torch.int16, "tof_bin"),
                                           _ptr(delta, torch.float32, "delta"), off, len(frame_offsets) - 1,
                                           ctypes.byref(g), ctypes.byref(o), _stream(stream)))
    return Plan(h.value, geom, int(frame_offsets[-1]), len(frame_offsets) - 1, frame_offsets,
                tof_bin is not None)


def jp_plan_rebind_det(plan: Plan, det_start, det_end, det_xyz, frame_offsets=None, tof_bin=None, delta=None,
                       stream=None):
    """Rebinds a plan to detector-index events (no allocation)."""
    pds, pde, pxyz, nd = _det(det_start, det_end, det_xyz)
    if frame_offsets is None:
        frame_offsets = [0, int(det_start.shape[0])]
    off = (ctypes.c_int64 * len(frame_offsets))(*[int(v) for v in frame_offsets])
    _check(load().jp_plan_rebind_det(plan.handle, pds, pde, pxyz, nd, _ptr(tof_bin, torch.int16, "tof_bin"),
                                     _ptr(delta, torch.float32, "delta"), off, len(frame_offsets) - 1,
                                     _stream(stream)))
    plan.n = int(frame_offsets[-1])
    plan.n_frames = len(frame_offsets) - 1
    plan.frame_offsets = list(frame_offsets)
    plan.has_tof_bin = tof_bin is not None
    return plan


def jp_plan_set_event_sigma(plan: Plan, sigma, stream=None):
    """Per-event TOF sigma (mm, float32 [n], caller order) for the plan's
    bound listmode events; None clears it.  Rebinding clears it too."""
    if sigma is not None and sigma.numel() != plan.n:
        raise ValueError("sigma must hold one value per bound event")
    _check(load().jp_plan_set_event_sigma(plan.handle, _ptr(sigma, torch.float32, "sigma"), _stream(stream)))
    return plan


def jp_plan_rebind(plan: Plan, xs, xe, frame_offsets=None, tof_bin=None, delta=None, stream=None):
    pxs, pxe = _lors(xs, xe)
    if frame_offsets is None:
        frame_offsets = [0, int(xs.shape[0])]
    off = (ctypes.c_int64 * len(frame_offsets))(*[int(v) for v in frame_offsets])
    _check(load().jp_plan_rebind(plan.handle, pxs, pxe, _ptr(tof_bin, torch.int16, "tof_bin"),
                                 _ptr(delta, torch.float32, "delta"), off, len(frame_offsets) - 1,
                                 _stream(stream)))
    plan.n = int(frame_offsets[-1])
    plan.n_frames = len(frame_offsets) - 1
    plan.frame_offsets = list(frame_offsets)
    plan.has_tof_bin = tof_bin is not None


def jp_plan_destroy(plan: Plan):
    plan.destroy()


# ---------------------------------------------------------------------------
# projections
# ---------------------------------------------------------------------------
def _img_stride(plan: Plan, img: torch.Tensor, img_stride):
    if img_stride is not None:
        return int(img_stride)
    nvox = int(plan.geom.shape[0] * plan.geom.shape[1] * plan.geom.shape[2])
    if img.numel() == nvox:
        return 0
    if img.numel() == nvox * plan.n_frames:
        return nvox
    raise ValueError("image size matches neither one image nor one per frame")


def _out_size(out, n, what="out"):
    if out.numel() < n:
        raise ValueError(f"{what} holds {out.numel()} elements, the plan needs {n}")


def jp_fwd(plan: Plan, img, out=None, img_stride=None, stream=None):
    out = torch.empty(plan.n, dtype=torch.float32, device=img.device) if out is None else out
    _out_size(out, plan.n)
    _check(load().jp_fwd(plan.handle, _ptr(img, torch.float32, "img"), _img_stride(plan, img, img_stride),
                         _ptr(out, torch.float32, "proj"), _stream(stream)))
    return out


def jp_back(plan: Plan, proj, img_accum, img_stride=None, stream=None):
    _out_size(proj, plan.n, "proj")
    _check(load().jp_back(plan.handle, _ptr(proj, torch.float32, "proj"),
                          _ptr(img_accum, torch.float32, "img_accum"),
                          _img_stride(plan, img_accum, img_stride), _stream(stream)))
    return img_accum


def jp_fwd_tof_sino(plan: Plan, img, tof, out=None, img_stride=None, stream=None):
    if out is None:
        out = torch.empty((plan.n, int(tof.n_bins)), dtype=torch.float32, device=img.device)
    _out_size(out, plan.n * int(tof.n_bins))
    t = tof_params(tof)
    _check(load().jp_fwd_tof_sino(plan.handle, _ptr(img, torch.float32, "img"),
                                  _img_stride(plan, img, img_stride), ctypes.byref(t),
                                  _ptr(out, torch.float32, "proj"), _stream(stream)))
    return out


def jp_back_tof_sino(plan: Plan, proj, tof, img_accum, img_stride=None, stream=None):
    _out_size(proj, plan.n * int(tof.n_bins), "proj")
    t = tof_params(tof)
    _check(load().jp_back_tof_sino(plan.handle, _ptr(proj, torch.float32, "proj"), ctypes.byref(t),
                                   _ptr(img_accum, torch.float32, "img_accum"),
                                   _img_stride(plan, img_accum, img_stride), _stream(stream)))
    return img_accum


def jp_fwd_tof_lm(plan: Plan, img, tof, out=None, img_stride=None, stream=None):
    out = torch.empty(plan.n, dtype=torch.float32, device=img.device) if out is None else out
    _out_size(out, plan.n)
    t = tof_params(tof)
    _check(load().jp_fwd_tof_lm(plan.handle, _ptr(img, torch.float32, "img"),
                                _img_stride(plan, img, img_stride), ctypes.byref(t),
                                _ptr(out, torch.float32, "proj"), _stream(stream)))
    return out


def jp_back_tof_lm(plan: Plan, proj, tof, img_accum, img_stride=None, stream=None):
    _out_size(proj, plan.n, "proj")
    t = tof_params(tof)
    _check(load().jp_back_tof_lm(plan.handle, _ptr(proj, torch.float32, "proj"), ctypes.byref(t),
                                 _ptr(img_accum, torch.float32, "img_accum"),
                                 _img_stride(plan, img_accum, img_stride), _stream(stream)))
    return img_accum


def jp_fwd_lors(xs, xe, img, geom, tof_mode="nontof", tof=None, tof_bin=None, delta=None, out=None,
                stream=None):
    m = TOF_MODES[tof_mode]
    n = int(xs.shape[0])
    if out is None:
        shape = (n, int(tof.n_bins)) if m == 1 else (n,)
        out = torch.empty(shape, dtype=torch.float32, device=img.device)
    pxs, pxe = _lors(xs, xe)
    g = image_geom(geom)
    t = tof_params(tof) if tof is not None else None
    _check(load().jp_fwd_lors(pxs, pxe, _ptr(tof_bin, torch.int16, "tof_bin"), _ptr(delta, torch.float32, "delta"),
                              n, ctypes.byref(g), m, ctypes.byref(t) if t is not None else None,
                              _ptr(img, torch.float32, "img"), _ptr(out, torch.float32, "proj"), _stream(stream)))
    return out


def jp_back_lors(xs, xe, proj, geom, img_accum, tof_mode="nontof", tof=None, tof_bin=None, delta=None,
                 stream=None):
    m = TOF_MODES[tof_mode]
    pxs, pxe = _lors(xs, xe)
    g = image_geom(geom)
    t = tof_params(tof) if tof is not None else None
    _check(load().jp_back_lors(pxs, pxe, _ptr(tof_bin, torch.int16, "tof_bin"), _ptr(delta, torch.float32, "delta"),
                               int(xs.shape[0]), ctypes.byref(g), m, ctypes.byref(t) if t is not None else None,
                               _ptr(proj, torch.float32, "proj"), _ptr(img_accum, torch.float32, "img_accum"),
                               _stream(stream)))
    return img_accum


def jp_back_tof_lm_noalloc(xs, xe, proj, geom, img_accum, tof, tof_bin, delta=None, stream=None):
    """img_accum += A^T proj (TOF listmode) without any device allocation:
    the workspace is fixed inside the library (images up to
    sum_a n_a' (n_b+2)(n_c+2) <= 2^20, n_a' = n_a rounded up to even).
    Overlapping calls race."""
    pxs, pxe = _lors(xs, xe)
    g = image_geom(geom)
    t = tof_params(tof)
    _check(load().jp_back_tof_lm_noalloc(pxs, pxe, _ptr(tof_bin, torch.int16, "tof_bin"),
                                         _ptr(delta, torch.float32, "delta"), int(xs.shape[0]), ctypes.byref(g),
                                         ctypes.byref(t), _ptr(proj, torch.float32, "proj"),
                                         _ptr(img_accum, torch.float32, "img_accum"), _stream(stream)))
    return img_accum


# ---------------------------------------------------------------------------
# OSEM element-wise steps and FP64 check sum
# ---------------------------------------------------------------------------
def jp_osem_ratio(plan: Optional[Plan], proj, b, out=None, stream=None):
    out = proj if out is None else out
    _check(load().jp_osem_ratio(plan.handle if plan is not None else None, _ptr(proj, torch.float32, "proj"),
                                _ptr(b, torch.float32, "b"), _ptr(out, torch.float32, "q"), int(proj.numel()),
                                _stream(stream)))
    return out


def jp_osem_update(x, bp, sens, scale, nvox, n_frames=1, img_stride=None, s_stride=0, stream=None):
    img_stride = nvox if img_stride is None else img_stride
    _check(load().jp_osem_update(_ptr(x, torch.float32, "x"), _ptr(bp, torch.float32, "bp"),
                                 _ptr(sens, torch.float32, "sens"), float(scale), int(nvox), int(n_frames),
                                 int(img_stride), int(s_stride), _stream(stream)))
    return x


def jp_osem_ratio_sino(proj, y, c=None, out=None, stream=None):
    """q = y / (proj + c) (0 where proj + c <= 0); ``out`` may be ``proj``."""
    out = torch.empty_like(proj) if out is None else out
    if y.numel() != proj.numel() or out.numel() != proj.numel() or (c is not None and c.numel() != proj.numel()):
        raise ValueError("proj, y, c and out must have the same number of elements")
    _check(load().jp_osem_ratio_sino(_ptr(proj, torch.float32, "proj"), _ptr(y, torch.float32, "y"),
                                     _ptr(c, torch.float32, "c"), _ptr(out, torch.float32, "out"),
                                     int(proj.numel()), _stream(stream)))
    return out


def jp_osem_subset_tof_lm(plan: Plan, f0: int, f1: int, x, sens, sens_scale: float, b: float, tof,
                          stream=None):
    """x <- x / (sens*sens_scale) * A_S^T (1/(A_S x + b)) for the events of
    subset frames [f0, f1) of an interleaved plan (one fused pass per event)."""
    t = tof_params(tof)
    _check(load().jp_osem_subset_tof_lm(plan.handle, int(f0), int(f1), _ptr(x, torch.float32, "x"),
                                        _ptr(sens, torch.float32, "sens"), float(sens_scale), float(b),
                                        ctypes.byref(t), _stream(stream)))
    return x


def jp_osem_subset_tof_lm_dev(plan: Plan, f0: int, f1: int, x, sens, sens_scale: float, b_dev, tof,
                              stream=None):
    """As jp_osem_subset_tof_lm with b in device memory and the subset range
    read on the device: a captured graph of these calls stays valid when the
    plan is rebound and b is rewritten."""
    t = tof_params(tof)
    _check(load().jp_osem_subset_tof_lm_dev(plan.handle, int(f0), int(f1), _ptr(x, torch.float32, "x"),
                                            _ptr(sens, torch.float32, "sens"), float(sens_scale),
                                            _ptr(b_dev, torch.float32, "b"), ctypes.byref(t), _stream(stream)))
    return x


def jp_osem_subset_tof_lm_ex(plan: Plan, f0: int, f1: int, x, sens, sens_scale: float, b, tof, fwhm_mm=0.0,
                             work=None, truncate: float = 4.0, path: str = "auto", stream=None):
    """Subset update, general form: with the resolution model H (Gaussian of
    ``fwhm_mm``; 0 = none) x <- x / (sens*sens_scale) * H^T A_S^T
    (1/(A_S H x + b)), sens = H^T A^T 1.  ``b`` is a float, or a device
    float tensor (read when the kernels run, capturable in a CUDA graph);
    ``work`` holds 2 images (needed with the resolution model); ``path`` is
    "auto", "quads" or "direct"."""
    t = tof_params(tof)
    r = None if (isinstance(fwhm_mm, (int, float)) and float(fwhm_mm) == 0.0) else resolution(fwhm_mm, truncate)
    if r is not None and work is None:
        raise ValueError("the resolution model needs a work tensor of 2 images")
    if path not in OSEM_PATHS:
        raise ValueError(f"path must be one of {sorted(OSEM_PATHS)}")
    b_dev = b if isinstance(b, torch.Tensor) else None
    _check(load().jp_osem_subset_tof_lm_ex(plan.handle, int(f0), int(f1), _ptr(x, torch.float32, "x"),
                                           _ptr(sens, torch.float32, "sens"), float(sens_scale),
                                           0.0 if b_dev is not None else float(b),
                                           _ptr(b_dev, torch.float32, "b"), ctypes.byref(t),
                                           None if r is None else ctypes.byref(r), OSEM_PATHS[path],
                                           _ptr(work, torch.float32, "work"), _stream(stream)))
    return x


def jp_osem_subset_tof_lm_res(plan: Plan, f0: int, f1: int, x, sens, sens_scale: float, b, tof, fwhm_mm,
                              work, truncate: float = 4.0, path: str = "auto", stream=None):
    """jp_osem_subset_tof_lm_ex with the resolution model of ``fwhm_mm``."""
    return jp_osem_subset_tof_lm_ex(plan, f0, f1, x, sens, sens_scale, b, tof, fwhm_mm, work, truncate, path,
                                    stream)


def jp_gauss3d(img, geom, fwhm_mm, truncate: float = 4.0, out=None, work=None, stream=None):
    """out = H img: separable Gaussian resolution model of ``fwhm_mm`` (zero
    outside the grid; H^T = H).  ``img`` is one image of ``geom.shape`` or a
    stack [n, *geom.shape]."""
    shape = tuple(int(v) for v in geom.shape)
    if tuple(img.shape[-3:]) != shape or img.dim() not in (3, 4):
        raise ValueError("img must be [*geom.shape] or [n, *geom.shape]")
    n = 1 if img.dim() == 3 else int(img.shape[0])
    out = torch.empty_like(img) if out is None else out
    work = torch.empty_like(img) if work is None else work
    if out.shape != img.shape or work.numel() < img.numel():
        raise ValueError("out must match img and work must hold as many voxels")
    g = image_geom(geom)
    r = resolution(fwhm_mm, truncate)
    _check(load().jp_gauss3d(_ptr(img, torch.float32, "img"), _ptr(out, torch.float32, "out"),
                             _ptr(work, torch.float32, "work"), n, ctypes.byref(g), ctypes.byref(r),
                             _stream(stream)))
    return out


LOGLIK_BLOCKS = 1024  # JP_LOGLIK_BLOCKS


def jp_poisson_loglik_value(plan: Optional[Plan], proj, w, b, out=None, work=None, stream=None):
    """sum_e w_e log(p_e + b_frame(e)) as a device float (0-dim tensor),
    an FP32 compensated sum; ``work`` is scratch of 2 * LOGLIK_BLOCKS floats."""
    out = torch.empty((), dtype=torch.float32, device=proj.device) if out is None else out
    work = torch.empty(2 * LOGLIK_BLOCKS, dtype=torch.float32, device=proj.device) if work is None else work
    if work.numel() < 2 * LOGLIK_BLOCKS:
        raise ValueError("work needs 2 * LOGLIK_BLOCKS floats")
    _check(load().jp_poisson_loglik_value(plan.handle if plan is not None else None, _ptr(proj, torch.float32, "proj"),
                                          _ptr(w, torch.float32, "w"), _ptr(b, torch.float32, "b"), int(proj.numel()),
                                          _ptr(out, torch.float32, "value"), _ptr(work, torch.float32, "work"),
                                          _stream(stream)))
    return out


def jp_poisson_loglik_grad(plan: Optional[Plan], proj, w, b, scale=None, out=None, stream=None):
    """grad_e = scale * w_e / (p_e + b_frame(e)) (scale: device float or None)."""
    out = torch.empty_like(proj) if out is None else out
    _check(load().jp_poisson_loglik_grad(plan.handle if plan is not None else None, _ptr(proj, torch.float32, "proj"),
                                         _ptr(w, torch.float32, "w"), _ptr(b, torch.float32, "b"),
                                         _ptr(scale, torch.float32, "scale"), int(proj.numel()),
                                         _ptr(out, torch.float32, "grad"), _stream(stream)))
    return out


def jp_osem_init(x, sens, stream=None):
    """x = sens > 0 ? 1 : 0 (listmode OSEM start image)."""
    _check(load().jp_osem_init(_ptr(x, torch.float32, "x"), _ptr(sens, torch.float32, "sens"), int(x.numel()),
                               _stream(stream)))
    return x


def jp_sum_f64(x, out=None, stream=None):
    out = torch.empty((), dtype=torch.float64, device=x.device) if out is None else out
    _check(load().jp_sum_f64(_ptr(x, torch.float32, "x"), int(x.numel()), _ptr(out, torch.float64, "out"),
                             _stream(stream)))
    return out


def jp_count_samples(plan: Plan, tof_mode="nontof", tof=None, stream=None) -> int:
    """Plane samples visited by the projector for the plan's LORs (exact);
    tof_mode "tof_sino": the TOF bin evaluations over those samples."""
    out = torch.zeros((), dtype=torch.int64, device="cuda")
    t = tof_params(tof) if tof is not None else None
    _check(load().jp_count_samples(plan.handle, TOF_MODES[tof_mode], ctypes.byref(t) if t is not None else None,
                                   _ptr(out, None, "out"), _stream(stream)))
    return int(out.item())


def jp_count_red_requests(plan: Plan, tof_mode="nontof", tof=None, stream=None) -> int:
    """L2 reduction requests (32-byte sector operations) of the plan's
    quad-image back projection with every LOR live (device-side replay)."""
    out = torch.zeros((), dtype=torch.int64, device="cuda")
    t = tof_params(tof) if tof is not None else None
    _check(load().jp_count_red_requests(plan.handle, TOF_MODES[tof_mode], ctypes.byref(t) if t is not None else None,
                                        _ptr(out, None, "out"), _stream(stream)))
    return int(out.item())


def jp_bench_tof_bins(tof, direction: int = 0, per_thread: int = 256, stream=None) -> dict:
    """Ceiling of the TOF-sinogram per-bin work (measurement helper): bin
    evaluations per second of the forward's (direction 0) or the back
    projection's (direction 1) table-and-accumulate operation."""
    ms = ctypes.c_float()
    out = torch.zeros((), dtype=torch.int64, device="cuda")
    t = tof_params(tof)
    _check(load().jp_bench_tof_bins(ctypes.byref(t), int(direction), int(per_thread), ctypes.byref(ms),
                                    _ptr(out, None, "bins"), _stream(stream)))
    bins = int(out.item())
    return {"bins_per_s": bins / (ms.value / 1e3), "ms": ms.value, "bins": bins, "direction": int(direction)}


def jp_bench_red(n_entries: int = 3_000_000, per_thread: int = 64, iters: int = 5, pattern: int = 0,
                 stream=None) -> dict:
    """Scattered 16-byte reduction ceiling of the device (measurement helper):
    reductions per second over an L2-resident buffer of n_entries float4.
    pattern 0: one random sector per reduction; 1: two reductions per random
    sector; 2: a warp on 512 contiguous bytes; 3 / 4: 4 / 8 lanes on one
    random 128-byte line."""
    buf = torch.zeros((n_entries, 4), dtype=torch.float32, device="cuda")
    ms = ctypes.c_float()
    _check(load().jp_bench_red_pattern(_ptr(buf, torch.float32, "buf"), int(n_entries), int(per_thread),
                                       int(iters), int(pattern), ctypes.byref(ms), _stream(stream)))
    blocks = torch.cuda.get_device_properties(buf.device).multi_processor_count * 32
    ops_ = blocks * 256 * per_thread
    sectors_per_red = {0: 1.0, 1: 0.5, 2: 0.5, 3: 0.5, 4: 0.5}[int(pattern)]
    rate = ops_ / (ms.value / 1e3)
    return {"reductions_per_s": rate, "sectors_per_s": rate * sectors_per_red, "ms": ms.value,
            "buffer_bytes": n_entries * 16, "pattern": int(pattern)}


def jp_launch_count() -> int:
    """Kernels launched by libjoseph so far in this process."""
    return int(load().jp_launch_count())


def jp_version() -> str:
    return load().jp_version().decode()


# short aliases
plan_create = jp_plan_create
plan_create_batch = jp_plan_create_batch
plan_create_subsets = jp_plan_create_subsets
osem_subset_tof_lm = jp_osem_subset_tof_lm
plan_rebind = jp_plan_rebind
fwd = jp_fwd
back = jp_back
fwd_tof_sino = jp_fwd_tof_sino
back_tof_sino = jp_back_tof_sino
fwd_tof_lm = jp_fwd_tof_lm
back_tof_lm = jp_back_tof_lm
fwd_lors = jp_fwd_lors
back_lors = jp_back_lors
osem_ratio = jp_osem_ratio
osem_update = jp_osem_update
sum_f64 = jp_sum_f64
