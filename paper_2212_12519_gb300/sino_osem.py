"""Sinogram OSEM on the GPU (paper Sec. 2.6: OSEM subset updates with 34
subsets of equally spaced views of a span-1 sinogram; Sec. 4: the emission
sinogram, its forward projection and the additive contamination sinogram are
held in device memory).

Subset m holds the views m, m + n_sub, ... .  Each subset has its own plan
(binned LORs), its own sensitivity s_m = A_m^T 1 (TOF: summed over the TOF
bins), and device-resident emission counts y_m and contamination c_m.  One
subset update is

    x <- x / s_m * A_m^T ( y_m / (A_m x + c_m) ),   x = 0 where s_m = 0,

four library calls: forward projection (jp_fwd or jp_fwd_tof_sino), the
ratio (jp_osem_ratio_sino, in place), back projection and the multiplicative
update (jp_osem_update).  With the image-based resolution model (``fwhm_mm``
> 0) the projector is A H: x is convolved before the forward projection, the
back projection before the update, and s_m = H^T A_m^T 1.
"""
from __future__ import annotations

from typing import List, Optional

import torch

from . import ops, synth


class SinoOSEM:
    def __init__(self, spec: synth.SinoSpec, geom: synth.ImageGeom, n_sub: int = 34,
                 tof: Optional[synth.TofParams] = None, fwhm_mm: float = 0.0, order: str = "PVR",
                 device="cuda", **plan_opts):
        self.spec, self.geom, self.n_sub, self.tof, self.fwhm = spec, geom, n_sub, tof, fwhm_mm
        self.device = torch.device(device)
        self.nb = tof.n_bins if tof is not None else 1
        self.plans: List[ops.Plan] = []
        self.sens: List[torch.Tensor] = []
        self.n: List[int] = []
        for m in range(n_sub):
            xs, xe = synth.sinogram_lors(spec.subset(m, n_sub), device=self.device, order=order)
            plan = ops.jp_plan_create(xs, xe, geom, **plan_opts)
            del xs, xe
            self.plans.append(plan)
            self.n.append(plan.n)
        nmax = max(self.n)
        self.p = torch.empty(nmax * self.nb, dtype=torch.float32, device=self.device)
        self.bp = torch.empty(geom.shape, dtype=torch.float32, device=self.device)
        self.hx = torch.empty_like(self.bp) if fwhm_mm > 0 else None
        self.work = torch.empty_like(self.bp) if fwhm_mm > 0 else None
        ones = torch.ones(nmax * self.nb, dtype=torch.float32, device=self.device)
        for m, plan in enumerate(self.plans):
            s = torch.zeros(geom.shape, dtype=torch.float32, device=self.device)
            self._back(m, ones[: self.n[m] * self.nb], s)
            if fwhm_mm > 0:
                s = ops.jp_gauss3d(s, geom, fwhm_mm)
            self.sens.append(s)
        del ones
        self.y: List[Optional[torch.Tensor]] = [None] * n_sub
        self.c: List[Optional[torch.Tensor]] = [None] * n_sub

    # -- projections of subset m -------------------------------------------
    def _shape(self, m):
        return (self.n[m], self.nb) if self.tof is not None else (self.n[m],)

    def fwd(self, m: int, x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """A_m x (sinogram of subset m in its LOR order; TOF: [n_m, n_bins])."""
        if self.tof is not None:
            return ops.jp_fwd_tof_sino(self.plans[m], x, self.tof, out=out)
        return ops.jp_fwd(self.plans[m], x, out=out)

    def _back(self, m: int, q: torch.Tensor, img: torch.Tensor):
        if self.tof is not None:
            ops.jp_back_tof_sino(self.plans[m], q.view(self.n[m], self.nb), self.tof, img)
        else:
            ops.jp_back(self.plans[m], q.view(self.n[m]), img)

    # -- data ----------------------------------------------------------------
    def set_data(self, y: List[torch.Tensor], c: List[Optional[torch.Tensor]]):
        """Per-subset emission counts and contamination (float32, subset
        shape); c[m] may be None (no contamination)."""
        for m in range(self.n_sub):
            if tuple(y[m].shape) != self._shape(m) or (c[m] is not None and tuple(c[m].shape) != self._shape(m)):
                raise ValueError(f"subset {m}: data must have shape {self._shape(m)}")
        self.y, self.c = list(y), list(c)

    def simulate(self, x_true: torch.Tensor, contamination: float = 0.2, seed: int = 0, noise: bool = True):
        """Synthetic data: c_m = contamination * mean(A x_true) (uniform, as
        randoms are uniform over LORs and TOF bins), y_m ~ Poisson(A_m x_true
        + c_m) (or its mean when ``noise`` is False)."""
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        projs = [self.fwd(m, H(x_true, self.geom, self.fwhm)).clone() for m in range(self.n_sub)]
        mean = float(sum(float(p.double().sum()) for p in projs) / sum(p.numel() for p in projs))
        ys, cs = [], []
        for p in projs:
            c = torch.full_like(p, contamination * mean)
            lam = p + c
            ys.append(torch.poisson(lam, generator=gen) if noise else lam)
            cs.append(c)
        self.set_data(ys, cs)

    # -- OSEM ----------------------------------------------------------------
    def subset_update(self, x: torch.Tensor, m: int) -> torch.Tensor:
        if self.y[m] is None:
            raise RuntimeError("no data: call set_data or simulate first")
        n = self.n[m] * self.nb
        xin = x
        if self.fwhm > 0:
            xin = ops.jp_gauss3d(x, self.geom, self.fwhm, out=self.hx, work=self.work)
        p = self.p[:n].view(self._shape(m))
        self.fwd(m, xin, out=p)
        ops.jp_osem_ratio_sino(p, self.y[m], self.c[m], out=p)
        self.bp.zero_()
        self._back(m, p, self.bp)
        bp = self.bp
        if self.fwhm > 0:
            bp = ops.jp_gauss3d(self.bp, self.geom, self.fwhm, out=self.hx, work=self.work)
        ops.jp_osem_update(x, bp, self.sens[m], 1.0, x.numel())
        return x

    def run(self, n_iter: int, x0: Optional[torch.Tensor] = None) -> torch.Tensor:
        """n_iter iterations of all subsets from x0 (default: 1 where the
        total sensitivity is > 0)."""
        if x0 is None:
            x = torch.empty(self.geom.shape, dtype=torch.float32, device=self.device)
            ops.jp_osem_init(x, sum(self.sens))
        else:
            x = x0.clone()
        for _ in range(n_iter):
            for m in range(self.n_sub):
                self.subset_update(x, m)
        return x

    def close(self):
        for p in self.plans:
            p.destroy()
        self.plans.clear()


def H(x: torch.Tensor, geom: synth.ImageGeom, fwhm_mm: float) -> torch.Tensor:
    return ops.jp_gauss3d(x.contiguous(), geom, fwhm_mm) if fwhm_mm > 0 else x
