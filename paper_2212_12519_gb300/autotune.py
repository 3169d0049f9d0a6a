"""Autotuner for the projection launch parameters.

Tunes, per device and workload shape, the plan options that the paper's
design leaves to the implementation: threads per CTA, LORs per warp (one LOR
per thread, or 8/16/32 lanes stepping through one LOR's planes) and the sort
granularity of the LOR binning (slope / offset / TOF-window bins).  Each
candidate builds a plan on a sample of the LORs and is timed over forward +
back projection with CUDA events; the fastest is cached as JSON (path from
$JP_AUTOTUNE_CACHE, default ~/.cache/paper_2212_12519_gb300/autotune.json).
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Callable, Dict, List, Optional

import torch

# block 0: the library's per-kernel defaults (256 threads per CTA for the back
# projections, 128 for the non-TOF and TOF-listmode forwards, 512 for the
# TOF-sinogram forward).  512 threads for every kernel is left out: on the
# 10M-event sample it can time as fast, but on the 8 x 40M batch its
# forward takes 45.3 ms against 41.6 ms.
CANDIDATES: List[dict] = [
    dict(block=b, lors_per_warp=l, slope_bins=s, offset_bins=o, window_bins=w, zoff_bins=z)
    for b in (0, 256)
    for l in (0, 4, 32)
    for (s, o, w, z) in ((128, 256, 16, 8), (128, 256, 64, 1), (128, 256, 32, 4), (64, 64, 16, 1))
]

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("JP_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2212_12519_gb300", "autotune.json")


def _load() -> Dict[str, dict]:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d: Dict[str, dict]):
    path = cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def key(device: str, mode: str, n: int, shape, n_frames: int = 1) -> str:
    bucket = 0 if n <= 0 else int(math.log2(n))
    return f"{device}|{mode}|n2^{bucket}|{'x'.join(str(int(s)) for s in shape)}|f{n_frames}"


def tune(xs: torch.Tensor, xe: torch.Tensor, geom, mode: str = "tof_lm", tof=None,
         tof_bin: Optional[torch.Tensor] = None, sample: int = 10_000_000,
         candidates: Optional[List[dict]] = None, reps: int = 2, use_cache: bool = True,
         timer: Optional[Callable[[dict], float]] = None) -> dict:
    """Best plan options for this device/workload (cached).  ``timer``
    replaces the GPU measurement (it maps options to milliseconds)."""
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    k = key(dev, mode, int(xs.shape[0]), geom.shape)
    if use_cache:
        with _lock:
            hit = _load().get(k)
        if hit is not None:
            return dict(hit["opts"])
    cands = candidates if candidates is not None else CANDIDATES
    if timer is None:
        timer = _gpu_timer(xs, xe, geom, mode, tof, tof_bin, sample, reps)
    results = [(timer(dict(c)), c) for c in cands]
    ms, best = min(results, key=lambda r: r[0])
    if use_cache:
        with _lock:
            d = _load()
            d[k] = {"opts": best, "ms": ms, "tried": len(results)}
            _save(d)
    return dict(best)


def _gpu_timer(xs, xe, geom, mode, tof, tof_bin, sample, reps):
    from . import ops
    m = min(int(xs.shape[0]), sample)
    sx, se = xs[:m], xe[:m]
    stb = tof_bin[:m] if tof_bin is not None else None
    img = torch.rand(geom.shape, device=xs.device)
    nb = tof.n_bins if (mode == "tof_sino") else 1
    y = torch.rand((m, nb) if nb > 1 else (m,), device=xs.device)
    out = torch.zeros(geom.shape, device=xs.device)

    def run(plan):
        if mode == "tof_lm":
            ops.jp_fwd_tof_lm(plan, img, tof)
            ops.jp_back_tof_lm(plan, y, tof, out)
        elif mode == "tof_sino":
            ops.jp_fwd_tof_sino(plan, img, tof)
            ops.jp_back_tof_sino(plan, y, tof, out)
        else:
            ops.jp_fwd(plan, img)
            ops.jp_back(plan, y, out)

    def timer(opts):
        extra = dict(tof_bin=stb, tof_bin_width=tof.bin_width) if mode == "tof_lm" else {}
        plan = ops.jp_plan_create(sx, se, geom, **extra, **opts)
        run(plan)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            run(plan)
        b.record()
        torch.cuda.synchronize()
        plan.destroy()
        return a.elapsed_time(b) / reps

    return timer
