"""Listmode OSEM on the GPU (paper Sec. 2.6 and 3: TOF listmode OSEM,
x <- x / s_sub * A_S^T (1 / (A_S x + b)), subsets of the event stream).

With the image-based resolution model of Sec. 2.6 (a 3D Gaussian of
``fwhm_mm``, 4.5 mm in the paper) the projector is A H and the update
x <- x / s'_sub * H^T A_S^T (1 / (A_S H x + b)) uses s' = H^T A^T 1
(``resolution_sensitivity``); one call of jp_osem_subset_tof_lm_ex runs both
convolutions, the fused projections and the update.

Each subset update takes one of two paths (``path``): the plan's quad
images (one 16-byte access per sample, an image-sized quad build / clear /
fold per update) or the direct path (image gathers and scalar atomics, no
quad traffic), which is cheaper for small subsets; "auto" picks by the
subset's event count.

The sensitivity image s = A^T 1 is the non-TOF back projection of every LOR
of the scanner's span-1 sinogram; a frame's events are held in one plan
whose frames are the subsets e mod n_sub; one subset update is one call of
jp_osem_subset_tof_lm (forward, ratio, back projection fused per event, then
the multiplicative update).  A full reconstruction (n_iter x n_sub updates)
can be captured once into a CUDA graph and replayed.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Tuple

import torch

from . import ops, synth


def sensitivity(geom: synth.ImageGeom, spec: synth.SinoSpec = synth.SINO_CLINICAL, device="cuda",
                plane_chunk: int = 1296, check: bool = True) -> Tuple[torch.Tensor, Optional[dict]]:
    """s = A^T 1 over every LOR of the sinogram (non-TOF), plus the FP64
    normalisation check sum_j s_j == sum_i (A 1)_i computed on the GPU."""
    s = torch.zeros(geom.shape, dtype=torch.float32, device=device)
    ones_img = torch.ones(geom.shape, dtype=torch.float32, device=device) if check else None
    tot_back = torch.zeros((), dtype=torch.float64, device=device)
    tot_fwd = torch.zeros((), dtype=torch.float64, device=device)
    for p0 in range(0, spec.n_planes, plane_chunk):
        p1 = min(spec.n_planes, p0 + plane_chunk)
        xs, xe = synth.sinogram_lors(spec, device=device, plane_range=(p0, p1))
        plan = ops.jp_plan_create(xs, xe, geom)
        ones = torch.ones(xs.shape[0], dtype=torch.float32, device=device)
        ops.jp_back(plan, ones, s)
        if check:
            p = ops.jp_fwd(plan, ones_img)
            tot_fwd += ops.jp_sum_f64(p)
        plan.destroy()
        del xs, xe, ones
    info = None
    if check:
        tot_back = ops.jp_sum_f64(s)
        a, b = float(tot_back), float(tot_fwd)
        info = {"sum_sens_f64": a, "sum_fwd_ones_f64": b, "rel_gap": abs(a - b) / max(abs(b), 1e-300)}
    return s, info


def resolution_sensitivity(sens: torch.Tensor, geom: synth.ImageGeom, fwhm_mm: float) -> torch.Tensor:
    """s' = H^T s for the resolution model (H^T = H: symmetric taps, zero
    outside the grid)."""
    if fwhm_mm <= 0:
        return sens
    return ops.jp_gauss3d(sens.contiguous(), geom, fwhm_mm)


# Sort granularity of a frame's subset plan: the subsets multiply the key
# space, so coarser bins than a single-frame plan keep the histogram small.
# One event per warp pass (32 lanes over its planes) gives the fused subset
# kernel the most parallelism for small and medium subsets and ties with 8
# lanes per event for subsets of 1-2M events (measured on 200x200x71).
OSEM_PLAN_OPTS = dict(slope_bins=64, offset_bins=128, window_bins=16, zoff_bins=4, lors_per_warp=1)


@dataclass
class FrameSpec:
    """One listmode frame: events on the device plus its reconstruction setup."""
    xs: torch.Tensor
    xe: torch.Tensor
    tof_bin: torch.Tensor
    geom: synth.ImageGeom
    b: float
    n_iter: int = 3
    n_sub: int = 8
    fwhm_mm: float = 0.0    # resolution model (0: none); sens must then be H^T A^T 1
    path: str = "auto"      # subset update path: "auto", "quads" or "direct"
    sigma: Optional[torch.Tensor] = None  # per-event TOF sigma (mm), caller order


class LMOSEMFrame:
    """Device-resident state of one frame's reconstruction."""

    def __init__(self, spec: FrameSpec, sens: torch.Tensor, tof: synth.TofParams,
                 stream: Optional[torch.cuda.Stream] = None, plan: Optional[ops.Plan] = None,
                 **plan_opts):
        """``plan``: an interleaved plan of this grid to rebind (no device
        allocation); otherwise a new plan is created and owned."""
        self.spec, self.sens, self.tof = spec, sens, tof
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.own_plan = plan is None
        n = int(spec.xs.shape[0])
        with torch.cuda.stream(self.stream):
            if plan is None:
                opts = dict(OSEM_PLAN_OPTS)
                opts.update(plan_opts)
                self.plan = ops.jp_plan_create_subsets(spec.xs, spec.xe, spec.geom, spec.n_sub,
                                                       tof_bin=spec.tof_bin, tof_bin_width=tof.bin_width,
                                                       **opts)
            else:
                if plan.n_frames != spec.n_sub and plan.frame_offsets is None:
                    raise ValueError("plan/subset mismatch")
                ops.jp_plan_rebind(plan, spec.xs, spec.xe, [0] * spec.n_sub + [n], tof_bin=spec.tof_bin)
                plan.frame_offsets = [sum(n // spec.n_sub + (1 if f < n % spec.n_sub else 0) for f in range(m))
                                      for m in range(spec.n_sub + 1)]
                self.plan = plan
            if spec.sigma is not None:
                ops.jp_plan_set_event_sigma(self.plan, spec.sigma)
            self.x = torch.empty(spec.geom.shape, dtype=torch.float32, device=spec.xs.device)
            self.work = (torch.empty((2,) + tuple(spec.geom.shape), dtype=torch.float32, device=spec.xs.device)
                         if spec.fwhm_mm > 0 else None)
            ops.jp_osem_init(self.x, sens)
        self.graph = None

    def _updates(self, n_iter):
        for _ in range(n_iter):
            for m in range(self.spec.n_sub):
                ops.jp_osem_subset_tof_lm_ex(self.plan, m, m + 1, self.x, self.sens, 1.0 / self.spec.n_sub,
                                             self.spec.b, self.tof, self.spec.fwhm_mm, self.work,
                                             path=self.spec.path)

    def run(self):
        """All n_iter x n_sub subset updates, launched on the frame's stream."""
        with torch.cuda.stream(self.stream):
            self._updates(self.spec.n_iter)
        return self.x

    def capture(self):
        """Captures one iteration (n_sub updates) into a CUDA graph (on a
        side stream when the frame runs on the default stream)."""
        self.graph = torch.cuda.CUDAGraph()
        cap = self.stream
        if cap == torch.cuda.default_stream(cap.device):
            cap = torch.cuda.Stream(device=cap.device)
            cap.wait_stream(self.stream)
        with torch.cuda.graph(self.graph, stream=cap):
            self._updates(1)
        if cap is not self.stream:
            self.stream.wait_stream(cap)
        return self.graph

    def run_graph(self):
        """Replays the captured iteration n_iter times (x restarts from x0)."""
        if self.graph is None:
            self.capture()
            with torch.cuda.stream(self.stream):
                ops.jp_osem_init(self.x, self.sens)
        with torch.cuda.stream(self.stream):
            for _ in range(self.spec.n_iter):
                self.graph.replay()
        return self.x

    def nbytes(self) -> int:
        return estimate_bytes(self.spec.xs.shape[0], self.spec.geom, self.spec.n_sub)

    def release(self):
        if self.own_plan:
            self.plan.destroy()
        self.graph = None


def estimate_bytes(n_events: int, geom: synth.ImageGeom, n_sub: int = 8,
                   slope_bins=64, offset_bins=128, window_bins=16, zoff_bins=4) -> int:
    """Device bytes a frame holds while it is being reconstructed: its
    events, its plan (packed events, permutation, keys, histogram) and the
    image workspace (with the resolution model's two scratch images)."""
    n0, n1, n2 = geom.shape
    quad = 16 * (n0 * (n1 + 2) * (n2 + 2) + n1 * (n0 + 2) * (n2 + 2) + n2 * (n0 + 2) * (n1 + 2))
    hist = 4 * n_sub * 3 * slope_bins * offset_bins * window_bins * zoff_bins
    return int(n_events * (26 + 36 + 4) + 2 * quad + hist + 16 * n0 * n1 * n2)


def reconstruct_plain(spec: FrameSpec, sens: torch.Tensor, tof: synth.TofParams) -> torch.Tensor:
    """Sequential plain per-frame OSEM: the planless one-thread-per-event
    kernels (the paper's own parallelisation), subset by subset, with the
    element-wise ratio and update kernels (and, with a resolution model, a
    separate convolution before the forward and after the back projection)."""
    xs_s = [spec.xs[m::spec.n_sub].contiguous() for m in range(spec.n_sub)]
    xe_s = [spec.xe[m::spec.n_sub].contiguous() for m in range(spec.n_sub)]
    tb_s = [spec.tof_bin[m::spec.n_sub].contiguous() for m in range(spec.n_sub)]
    x = torch.empty(spec.geom.shape, dtype=torch.float32, device=spec.xs.device)
    ops.jp_osem_init(x, sens)
    bp = torch.empty_like(x)
    bvec = torch.full((1,), spec.b, dtype=torch.float32, device=x.device)
    nvox = x.numel()
    res = spec.fwhm_mm > 0
    y = torch.empty_like(x) if res else x
    work = torch.empty_like(x) if res else None
    for _ in range(spec.n_iter):
        for m in range(spec.n_sub):
            if res:
                ops.jp_gauss3d(x, spec.geom, spec.fwhm_mm, out=y, work=work)
            p = ops.jp_fwd_lors(xs_s[m], xe_s[m], y, spec.geom, "tof_lm", tof, tof_bin=tb_s[m])
            ops.jp_osem_ratio(None, p, bvec)
            bp.zero_()
            ops.jp_back_lors(xs_s[m], xe_s[m], p, spec.geom, bp, "tof_lm", tof, tof_bin=tb_s[m])
            if res:
                ops.jp_gauss3d(bp, spec.geom, spec.fwhm_mm, out=y, work=work)
                ops.jp_osem_update(x, y, sens, 1.0 / spec.n_sub, nvox)
            else:
                ops.jp_osem_update(x, bp, sens, 1.0 / spec.n_sub, nvox)
    return x
