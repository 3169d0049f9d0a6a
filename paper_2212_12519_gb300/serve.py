"""Served listmode OSEM: a request loop with continuous batching.

Each request is one frame (TOF listmode events, an image grid, a background
b) to reconstruct with n_iter x n_sub subset updates (paper Sec. 2.6 and 3,
listmode OSEM; Sec. 4 on reconstructions within seconds and short frames).
Requests arrive over time; the server keeps up to ``max_slots`` frames in
flight, each on its own CUDA stream, so work of frames that arrived while
others were running overlaps on the device.  A frame is admitted when a
slot is free and the device-memory budget holds its events, plan and
workspace; it leaves as soon as its image is ready.

Two execution modes are compared on the same arrival process:
  * ``batched``:   binned plan per frame, fused per-event OSEM subset kernel,
                   one iteration captured in a CUDA graph and replayed,
                   several frames concurrently;
  * ``sequential``: one frame at a time with the planless one-thread-per-
                   event kernels and separate ratio/update kernels.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np
import torch

from . import ops, osem, synth


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    spec: osem.FrameSpec
    start: Optional[float] = None
    finish: Optional[float] = None
    x: Optional[torch.Tensor] = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


class OSEMServer:
    def __init__(self, sens: Dict[tuple, torch.Tensor], tof: synth.TofParams, mode: str = "batched",
                 max_slots: int = 8, hbm_budget: Optional[int] = None, use_graphs: bool = True,
                 poll_s: float = 20e-6, plan_opts: Optional[dict] = None):
        if mode not in ("batched", "sequential"):
            raise ValueError(mode)
        self.sens = sens
        self.tof = tof
        self.mode = mode
        self.max_slots = 1 if mode == "sequential" else max_slots
        self.budget = hbm_budget
        self.use_graphs = use_graphs
        self.poll_s = poll_s
        self.plan_opts = plan_opts or {}
        self.streams = [torch.cuda.Stream() for _ in range(self.max_slots)]
        self.admission_waits = 0
        self.peak_bytes = 0
        self.plans: Dict[tuple, ops.Plan] = {}
        self.slot_graphs: Dict[tuple, "SlotGraph"] = {}

    def reserve(self, max_events: int, geoms: List[synth.ImageGeom], n_sub: int = 8, fwhm_mm: float = 0.0):
        """Pre-creates one interleaved plan per (slot, image grid) with room
        for ``max_events`` events, so admitting a frame only rebinds it (no
        device allocation, no device-wide synchronisation)."""
        if self.mode != "batched":
            return
        for slot in range(self.max_slots):
            for g in geoms:
                if (slot, g.shape) in self.plans:
                    continue
                xs = torch.zeros((max_events, 3), dtype=torch.float32, device="cuda")
                xs[:, 0] = 1.0
                tb = torch.zeros(max_events, dtype=torch.int16, device="cuda")
                opts = dict(osem.OSEM_PLAN_OPTS)
                opts.update(self.plan_opts)
                with torch.cuda.stream(self.streams[slot]):
                    self.plans[(slot, g.shape)] = ops.jp_plan_create_subsets(
                        xs, torch.zeros_like(xs), g, n_sub, tof_bin=tb, tof_bin_width=self.tof.bin_width,
                        **opts)
                torch.cuda.synchronize()
                del xs, tb
                if self.use_graphs:
                    self.slot_graphs[(slot, g.shape)] = SlotGraph(
                        self.plans[(slot, g.shape)], self.sens[g.shape], self.tof, g, n_sub, self.streams[slot],
                        fwhm_mm)

    def close(self):
        self.slot_graphs.clear()
        for p in self.plans.values():
            p.destroy()
        self.plans.clear()

    def _start(self, req: Request, slot: int):
        st = self.streams[slot]
        sens = self.sens[req.spec.geom.shape]
        if self.mode == "batched":
            sg = self.slot_graphs.get((slot, req.spec.geom.shape))
            if sg is not None:
                fr = None
                x = sg.run(req.spec)
            else:
                plan = self.plans.get((slot, req.spec.geom.shape))
                fr = osem.LMOSEMFrame(req.spec, sens, self.tof, stream=st, plan=plan, **self.plan_opts)
                fr.run()
                x = fr.x
        else:
            fr = None
            with torch.cuda.stream(st):
                x = osem.reconstruct_plain(req.spec, sens, self.tof)
        ev = torch.cuda.Event()
        ev.record(st)
        return fr, x, ev

    def run(self, requests: List[Request]) -> dict:
        reqs = sorted(requests, key=lambda r: r.arrival)
        n = len(reqs)
        pending: deque = deque()
        active: Dict[int, tuple] = {}
        free = list(range(self.max_slots))[::-1]
        used = 0
        done = 0
        nxt = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while done < n:
            now = time.perf_counter() - t0
            progressed = False
            while nxt < n and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
                progressed = True
            for slot in list(active.keys()):
                req, fr, x, ev, nbytes = active[slot]
                if ev.query():
                    req.finish = time.perf_counter() - t0
                    req.x = x
                    if fr is not None:
                        fr.release()
                    used -= nbytes
                    free.append(slot)
                    del active[slot]
                    done += 1
                    progressed = True
            while pending and free:
                req = pending[0]
                nbytes = osem.estimate_bytes(req.spec.xs.shape[0], req.spec.geom, req.spec.n_sub)
                if self.budget is not None and active and used + nbytes > self.budget:
                    self.admission_waits += 1
                    break
                pending.popleft()
                slot = free.pop()
                req.start = time.perf_counter() - t0
                fr, x, ev = self._start(req, slot)
                used += nbytes
                self.peak_bytes = max(self.peak_bytes, used)
                active[slot] = (req, fr, x, ev, nbytes)
                progressed = True
            if not progressed:
                if not active and nxt < n:
                    wait = reqs[nxt].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                else:
                    time.sleep(self.poll_s)
        makespan = max(r.finish for r in reqs) - min(r.arrival for r in reqs)
        lat = np.array([r.latency for r in reqs])
        ev_total = sum(int(r.spec.xs.shape[0]) for r in reqs)
        iters = sum(r.spec.n_iter for r in reqs)
        return {"mode": self.mode, "requests": n, "frames_per_s": n / makespan,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "makespan_s": makespan,
                "events_per_s": ev_total * (iters / n) / makespan,
                "admission_waits": self.admission_waits, "peak_bytes": self.peak_bytes}


class SlotGraph:
    """One OSEM iteration (n_sub subset updates) captured once per slot and
    image grid, replayed for every frame the slot serves.  The captured
    kernels read the subset ranges and b from device memory, so rebinding
    the slot's plan to a new frame keeps the graph valid.  Two graphs are
    captured, one per subset-update path (quad images / direct); a frame
    replays the direct one when its subsets are small."""

    def __init__(self, plan: ops.Plan, sens: torch.Tensor, tof: synth.TofParams, geom: synth.ImageGeom,
                 n_sub: int, stream: torch.cuda.Stream, fwhm_mm: float = 0.0):
        self.plan, self.sens, self.tof, self.n_sub, self.stream = plan, sens, tof, n_sub, stream
        self.fwhm_mm = fwhm_mm
        self.x = torch.zeros(geom.shape, dtype=torch.float32, device="cuda")
        self.b = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.work = (torch.empty((2,) + tuple(geom.shape), dtype=torch.float32, device="cuda")
                     if fwhm_mm > 0 else None)
        self.graphs = {}
        torch.cuda.synchronize()
        for path in ("quads", "direct"):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for m in range(n_sub):
                    ops.jp_osem_subset_tof_lm_ex(plan, m, m + 1, self.x, sens, 1.0 / n_sub, self.b, tof, fwhm_mm,
                                                 self.work, path=path)
            self.graphs[path] = g
        torch.cuda.synchronize()

    def run(self, spec: osem.FrameSpec) -> torch.Tensor:
        n = int(spec.xs.shape[0])
        if spec.n_sub != self.n_sub:
            raise ValueError("subset count differs from the captured graph")
        if spec.fwhm_mm != self.fwhm_mm:
            raise ValueError("resolution model differs from the captured graph")
        path = spec.path
        if path == "auto":
            nvox = int(np.prod(spec.geom.shape))
            path = "direct" if n < (nvox // ops.OSEM_DIRECT_VOXELS_PER_EVENT) * spec.n_sub else "quads"
        graph = self.graphs[path]
        with torch.cuda.stream(self.stream):
            ops.jp_plan_rebind(self.plan, spec.xs, spec.xe, [0] * spec.n_sub + [n], tof_bin=spec.tof_bin)
            self.b.fill_(float(spec.b))
            ops.jp_osem_init(self.x, self.sens)
            for _ in range(spec.n_iter):
                graph.replay()
            return self.x.clone()


# ---------------------------------------------------------------------------
# synthetic frame stream
# ---------------------------------------------------------------------------
def make_event_pools(tof: synth.TofParams, pool_events: int = 20_000_000, device="cuda", seed: int = 5000):
    """One pool of TOF listmode events per image size (the listmode batch recipe):
    frames take seeded random windows of their pool."""
    pools = {}
    for k, (geom, ph_spec) in enumerate([(synth.GEOM_OSEM_SMALL, synth.PHANTOM_OSEM_SMALL),
                                          (synth.GEOM_CLINICAL, synth.PHANTOM_CLINICAL)]):
        ph = synth.ellipsoid_phantom(geom, ph_spec, seed + 10 * k, device=device)
        xs, xe, tb = synth.lm_events(ph, geom, synth.SCANNER_CLINICAL, tof, pool_events,
                                     seed=seed + 10 * k + 1, device=device)
        pools[geom.shape] = dict(geom=geom, phantom=ph, xs=xs, xe=xe, tb=tb,
                                 b=synth.background_level(ph, tof))
    return pools


def make_requests(pools: dict, n_requests: int, rate: float, seed: int = 5001,
                  ev_min: float = 1e5, ev_max: float = 2e7, n_iter: int = 3, n_sub: int = 8,
                  fwhm_mm: float = 0.0) -> List[Request]:
    """Poisson arrivals at ``rate`` frames/s; events log-uniform in
    [ev_min, ev_max]; image 128x128x71 or 200x200x71 with probability 1/2;
    resolution model of ``fwhm_mm`` (0: none)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    keys = list(pools.keys())
    reqs = []
    for i in range(n_requests):
        pool = pools[keys[int(rng.integers(0, len(keys)))]]
        ne = int(math.exp(rng.uniform(math.log(ev_min), math.log(ev_max))))
        npool = pool["xs"].shape[0]
        ne = min(ne, npool)
        off = int(rng.integers(0, npool - ne + 1))
        spec = osem.FrameSpec(pool["xs"][off:off + ne], pool["xe"][off:off + ne], pool["tb"][off:off + ne],
                              pool["geom"], pool["b"], n_iter=n_iter, n_sub=n_sub, fwhm_mm=fwhm_mm)
        reqs.append(Request(i, float(arrivals[i]), spec))
    return reqs


def reset(requests: List[Request]):
    for r in requests:
        r.start = r.finish = None
        r.x = None
