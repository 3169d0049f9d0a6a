"""Benchmark: TOF listmode Joseph forward + back projection, events/s.

Workload (default): 8 images of 200x200x71 voxels (2 mm), 40M synthetic TOF
listmode events each (320M events), clinical scanner (36 rings x 672
crystals, R = 400 mm), 29 TOF bins of 28 mm, FWHM 57.7 mm, 3 sigma.  One
step = sort/pack all events into the plan (binning) + forward projection of
the batch through the autograd Function + the loss sum(w log(Ax + b)) (fused
value / gradient kernels) + its backward (the adjoint kernel).  events/s = events in the batch / step time.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own batch (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FRAMES = 8
EVENTS_PER_FRAME = 40_000_000
METRIC = "TOF listmode fwd+back events/s"
UNIT = "events/s"

# DRAM traffic of the TOF-listmode back projection per event (ncu
# dram__bytes_read.sum + dram__bytes_write.sum of the quad-image group back
# kernel on one 10M-event frame, 200x200x71), scaled to a launch by its
# events: the traffic grows with the events; the per-frame image terms are
# small.
BACK_DRAM_BYTES_PER_EVENT = (606_467_072 + 77_018_880) / 10_000_000


# ---------------------------------------------------------------------------
# environment helpers
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples nvidia-smi clocks/throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def plan_opts(args) -> dict:
    """Plan options from the command line (0 = the library default)."""
    o = dict(tile_lors=args.tile_lors, block=args.block, max_ctas_per_sm=args.ctas_per_sm,
             lors_per_warp=args.lors_per_warp)
    if args.path == "tiles":
        o["tiles"] = True
    return o


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_tof_lm_batch(rank: int, n_frames: int, events: int, device):
    """8 phantoms x ``events`` TOF listmode events each (seeded per frame and
    rank), as recorded listmode data: two detector indices and a TOF bin per
    event, plus the scanner's detector table (the LOR endpoints are kept
    too, for the oracle sample and the autotuner)."""
    from paper_2212_12519_gb300 import synth
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    imgs, xs_l, xe_l, tb_l, ds_l, de_l, bvals = [], [], [], [], [], [], []
    for f in range(n_frames):
        seed = 4001 + f + 1000 * 100 * rank
        ph = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, seed, device=device)
        xs, xe, tb, ds, de = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, events, seed=seed + 50,
                                             device=device, return_det=True)
        imgs.append(ph)
        xs_l.append(xs)
        xe_l.append(xe)
        tb_l.append(tb)
        ds_l.append(ds)
        de_l.append(de)
        bvals.append(synth.background_level(ph, tof))
    xs = torch.cat(xs_l)
    xe = torch.cat(xe_l)
    tb = torch.cat(tb_l)
    ds = torch.cat(ds_l)
    de = torch.cat(de_l)
    del xs_l, xe_l, tb_l, ds_l, de_l
    w = synth.loss_weights(xs.shape[0], 4999 + rank, device=device)
    offsets = [events * f for f in range(n_frames + 1)]
    bvec = torch.repeat_interleave(torch.tensor(bvals, dtype=torch.float32, device=device),
                                   torch.full((n_frames,), events, device=device))
    x = torch.stack(imgs).contiguous()
    bframe = torch.tensor(bvals, dtype=torch.float32, device=device)
    return dict(geom=g, tof=tof, xs=xs.contiguous(), xe=xe.contiguous(), tb=tb.contiguous(),
                ds=ds.contiguous(), de=de.contiguous(), det=synth.SCANNER_CLINICAL.crystal_table(device),
                w=w, bvec=bvec.contiguous(), bframe=bframe, x=x, offsets=offsets, bvals=bvals)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch.distributed as dist
    from paper_2212_12519_gb300 import ops
    from paper_2212_12519_gb300.autograd import JosephNonTOF, JosephTOFLM, PoissonLogLik
    from paper_2212_12519_gb300 import build as jbuild

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    jbuild.build()
    ops.load()
    n_frames, epf = args.frames, args.events
    nontof = args.workload == "nontof_lm"
    W = make_tof_lm_batch(rank, n_frames, epf, dev)
    g, tof = W["geom"], W["tof"]
    n_total = W["xs"].shape[0]
    if nontof:
        # same events without their TOF bins
        W["tb"] = None
    opts = plan_opts(args)
    if not args.no_autotune:
        from paper_2212_12519_gb300 import autotune
        if args.workload == "nontof_lm":
            opts = autotune.tune(W["xs"][:epf], W["xe"][:epf], g, mode="nontof")
        else:
            opts = autotune.tune(W["xs"][:epf], W["xe"][:epf], g, mode="tof_lm", tof=tof, tof_bin=W["tb"][:epf])
    if args.path == "tiles":
        opts = dict(opts, tiles=True)
    plan = ops.jp_plan_create_batch_det(W["ds"], W["de"], W["det"], g, W["offsets"], tof_bin=W["tb"],
                                        tof_bin_width=0.0 if nontof else tof.bin_width, **opts)
    if nontof:
        # background: 10 % of each frame's mean non-TOF projection
        p0 = ops.jp_fwd(plan, W["x"]).view(n_frames, epf).mean(dim=1)
        W["bvals"] = [float(0.1 * v) for v in p0.cpu()]
        W["bframe"] = torch.tensor(W["bvals"], dtype=torch.float32, device=dev)
        del p0
    x = W["x"].clone().requires_grad_(True)
    stream = torch.cuda.current_stream()
    sigma_e = None
    if args.event_sigma and not nontof:
        # per-event TOF resolution: three timing classes around the scanner's
        gen = torch.Generator(device=dev)
        gen.manual_seed(4998 + rank)
        cls = torch.randint(0, 3, (n_total,), generator=gen, device=dev)
        sigma_e = (tof.sigma * torch.tensor([0.85, 1.0, 1.2], device=dev)[cls]).float().contiguous()

    timers = {"fwd": [], "back": [], "bin": []}

    def timed(name, fn):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        r = fn()
        e.record(stream)
        timers[name].append((s, e))
        return r

    class TimedTOFLM(torch.autograd.Function):
        @staticmethod
        def forward(ctx, xx):
            ctx.shape = xx.shape
            if nontof:
                return timed("fwd", lambda: ops.jp_fwd(plan, xx.contiguous()))
            return timed("fwd", lambda: ops.jp_fwd_tof_lm(plan, xx.contiguous(), tof))

        @staticmethod
        def backward(ctx, gp):
            gx = torch.zeros(ctx.shape, dtype=torch.float32, device=gp.device)
            if nontof:
                timed("back", lambda: ops.jp_back(plan, gp.contiguous(), gx))
            else:
                timed("back", lambda: ops.jp_back_tof_lm(plan, gp.contiguous(), tof, gx))
            return gx

    def step(record=True):
        if record:
            timed("bin", lambda: ops.jp_plan_rebind_det(plan, W["ds"], W["de"], W["det"], W["offsets"],
                                                        tof_bin=W["tb"]))
        else:
            ops.jp_plan_rebind_det(plan, W["ds"], W["de"], W["det"], W["offsets"], tof_bin=W["tb"])
        if sigma_e is not None:
            ops.jp_plan_set_event_sigma(plan, sigma_e)
        x.grad = None
        if record:
            p = TimedTOFLM.apply(x)
        else:
            p = JosephNonTOF.apply(x, plan) if nontof else JosephTOFLM.apply(x, plan, tof)
        loss = PoissonLogLik.apply(p, plan, W["w"], W["bframe"])
        loss.backward()
        return loss

    for _ in range(args.warmup):
        step(record=False)
    torch.cuda.synchronize()
    for k in timers:
        timers[k].clear()
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ops.jp_launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    rng_id = torch.cuda.nvtx.range_start("timed")  # process-wide: covers the autograd thread too
    t0.record(stream)
    for _ in range(args.steps):
        loss = step()
    t1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_end(rng_id)
    launches = ops.jp_launch_count() - launches0
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    if ws > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    kern = {k: statistics.mean(s.elapsed_time(e) for s, e in v) for k, v in timers.items() if v}

    # exact algorithmic work of one launch, counted on the device
    mode = "nontof" if nontof else "tof_lm"
    samples = ops.jp_count_samples(plan, mode, tof)
    requests = ops.jp_count_red_requests(plan, mode, tof)
    value = n_total * ws / (ms / 1e3)

    # ---- e2e through the public API with host buffers --------------------
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, W, plan, g, tof, dev, ws, nontof)
    # L2 reduction ceiling (one 16-byte RED per plane sample bounds the back projection)
    red = {pt: ops.jp_bench_red(pattern=pt) for pt in (0, 1, 2, 3, 4)}
    cpu_sample = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu_sample = _oracle_events(W, min(W["xs"].shape[0], 8_000_000))
    plan.destroy()
    extra_nontof = None
    if not args.no_extra and rank == 0 and ws == 1 and not nontof:
        # the same events without their TOF bins, while they are resident
        extra_nontof = measure_nontof_lm_batch(W, 5, 3)
    del W["xs"], W["xe"], W["ds"], W["de"], W["w"], W["bvec"]
    W["tb"] = None
    torch.cuda.empty_cache()
    workloads = None
    if not args.no_extra and rank == 0 and ws == 1 and not nontof:
        # the other workloads at one GPU: the three sinogram configurations,
        # non-TOF listmode and the paper's 34-subset iteration
        workloads = {name: measure_sino(name, 5, 3) for name in ("sino_small", "sino_clinical", "tof_sino")}
        workloads["nontof_lm"] = extra_nontof
        workloads["lm_osem_iter"] = measure_lm_osem_iter(5, 3, args.fwhm)
    serving = None
    if not args.no_serving and rank == 0 and not nontof:
        rates = [float(r) for r in args.serving_rates.split(",")]
        serving = run_serving(n_requests=args.serving_requests, rates=rates, max_slots=args.serving_slots,
                              fwhm_mm=args.fwhm)

    if rank == 0:
        peaks, peak_kind = measured_peaks()
        nvox = int(np.prod(g.shape))
        # HBM view of the back projection (30 B per event + the images)
        alg_bytes = n_total * (24 + (0 if nontof else 2) + 4) + n_frames * nvox * 4 * 2
        achieved = alg_bytes / (kern["back"] / 1e3) / 1e9
        # binding resource: the back projection's L2 reduction requests (counted
        # on the device for this launch) against the reduction ceiling
        # measured in this run
        sec_rate = requests / (kern["back"] / 1e3)
        sec_peak = max(r["sectors_per_s"] for r in red.values())
        kname = "back_nontof_lm" if nontof else "back_tof_lm"
        line = {
            "metric": METRIC if not nontof else "non-TOF listmode fwd+back events/s",
            "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{'nontof' if nontof else 'tof'}_lm_batch{n_frames}x{epf // 1_000_000}M_200x200x71"
                                   + ("_event_sigma" if sigma_e is not None else ""),
                       "frames_per_gpu": n_frames, "events_per_frame": epf, "image": list(g.shape),
                       "tof_bins": 0 if nontof else tof.n_bins,
                       "input": "listmode as recorded: int32 detector-index pairs"
                                + ("" if nontof else " + int16 TOF bin") + " per event, float32 detector table",
                       "l2": "inputs (>10 GB/step) larger than L2, no flush",
                       "parallelism": f"dp{ws} (independent batches)", "plan_opts": opts},
            "kernel_ms": kern,
            "samples_per_step": samples,
            "events_per_s_excl_binning": n_total * ws / ((ms - kern.get("bin", 0.0)) / 1e3),
            "roofline": {"bound": "l2", "kernel": kname,
                         "resource": "L2 reduction requests (32-byte sector operations of the 16-byte "
                                     "vector reductions, one per plane sample)",
                         "achieved": sec_rate, "peak": sec_peak, "unit": "sectors/s", "frac": sec_rate / sec_peak,
                         "traffic": (BACK_DRAM_BYTES_PER_EVENT * n_total if not nontof else None),
                         "requests_per_launch": requests, "requests_per_sample": requests / max(samples, 1),
                         "peak_patterns": {str(k): v["sectors_per_s"] for k, v in red.items()},
                         "lane_reductions_per_s_patterns": {str(k): v["reductions_per_s"] for k, v in red.items()},
                         "peak_source": "jp_bench_red_pattern (measured in this run), max over patterns"},
            "hbm_roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved,
                             "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                             "peak_source": peak_kind, "alg_bytes_per_launch": alg_bytes},
            "clocks": clk,
            "gpu_launches": int(launches),
            "e2e": e2e,
            "workloads": workloads,
            "serving": serving,
        }
        if cpu_sample is not None:
            line["cpu_baseline"] = cpu_baseline(cpu_sample, W["bvals"][0], g, None if nontof else tof, n_total,
                                                target_s=args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def measure_nontof_lm_batch(W, steps, warmup):
    """Non-TOF listmode on the batch's events (their TOF bins dropped): one
    step is the rebind from detector indices, the forward projection, the
    Poisson loss with a background of 10% of each frame's mean projection
    and its backward (the back projection), as the TOF step."""
    from paper_2212_12519_gb300 import ops
    from paper_2212_12519_gb300.autograd import JosephNonTOF, PoissonLogLik
    g = W["geom"]
    n_frames = len(W["offsets"]) - 1
    epf = W["offsets"][1]
    plan = ops.jp_plan_create_batch_det(W["ds"], W["de"], W["det"], g, W["offsets"])
    p0 = ops.jp_fwd(plan, W["x"]).view(n_frames, epf).mean(dim=1)
    bframe = (0.1 * p0).float().contiguous()
    del p0
    x = W["x"].clone().requires_grad_(True)

    def step():
        ops.jp_plan_rebind_det(plan, W["ds"], W["de"], W["det"], W["offsets"])
        x.grad = None
        p = JosephNonTOF.apply(x, plan)
        loss = PoissonLogLik.apply(p, plan, W["w"], bframe)
        loss.backward()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    samples = ops.jp_count_samples(plan, "nontof")
    n = W["ds"].shape[0]
    plan.destroy()
    del x
    return {"metric": "non-TOF listmode fwd+back events/s", "value": n / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms, "steps": steps, "warmup": warmup, "higher_is_better": True,
            "samples_per_step": samples,
            "config": {"workload": f"nontof_lm_batch{n_frames}x{epf // 1_000_000}M_200x200x71",
                       "input": "the TOF batch's detector-index pairs without their TOF bins",
                       "step": "bin + fwd + loss + back"}}


def run_e2e(args, W, plan, g, tof, dev, ws, nontof=False):
    """Same step through the public API with the inputs copied from pinned
    host memory and the loss and gradient images read back, every step.
    NB device buffer sets (--e2e-buffers): the inputs of step k + NB - 1 are
    copied on a side stream while steps k .. k + NB - 2 compute (and step
    k's results are read back on it), so the copies overlap the compute and
    a copy may take up to NB - 1 steps; the timed region holds all of them."""
    import torch.distributed as dist
    from paper_2212_12519_gb300 import ops
    from paper_2212_12519_gb300.autograd import JosephNonTOF, JosephTOFLM, PoissonLogLik
    keys = ("ds", "de", "det", "w", "bframe", "x") if nontof else ("ds", "de", "det", "tb", "w", "bframe", "x")
    host = {k: W[k].cpu().pin_memory() for k in keys}
    nb = max(2, int(args.e2e_buffers))
    dbuf = [{k: torch.empty_like(W[k]) for k in keys} for _ in range(nb)]
    out_grad = [torch.empty(W["x"].shape, dtype=torch.float32).pin_memory() for _ in range(nb)]
    out_loss = [torch.empty((), dtype=torch.float32).pin_memory() for _ in range(nb)]
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = out_grad[0].numel() * 4 + 4
    comp = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(nb)]
    done = [torch.cuda.Event() for _ in range(nb)]
    results = [None] * nb

    def h2d_into(b):
        with torch.cuda.stream(copy):
            copy.wait_event(done[b])  # buffer set b is free once its last step finished
            for k in keys:
                dbuf[b][k].copy_(host[k], non_blocking=True)
            copied[b].record(copy)

    def compute(b):
        comp.wait_event(copied[b])
        d = dbuf[b]
        ops.jp_plan_rebind_det(plan, d["ds"], d["de"], d["det"], W["offsets"], tof_bin=d.get("tb"))
        x = d["x"].detach().requires_grad_(True)
        p = JosephNonTOF.apply(x, plan) if nontof else JosephTOFLM.apply(x, plan, tof)
        loss = PoissonLogLik.apply(p, plan, d["w"], d["bframe"])
        loss.backward()
        results[b] = (x.grad, loss.detach())
        done[b].record(comp)
        with torch.cuda.stream(copy):
            copy.wait_event(done[b])
            out_grad[b].copy_(results[b][0], non_blocking=True)
            out_loss[b].copy_(results[b][1], non_blocking=True)

    def run(nsteps):
        for k in range(min(nb - 1, nsteps)):
            h2d_into(k)
        for k in range(nsteps):
            if k + nb - 1 < nsteps:
                h2d_into((k + nb - 1) % nb)  # the set step k - 1 used
            compute(k % nb)
        comp.wait_stream(copy)

    for e in done:
        e.record(comp)
    run(max(1, min(args.warmup, 2)))
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    n = max(2, args.steps)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(comp)
    run(n)
    t1.record(comp)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / n
    if ws > 1:
        # the slowest rank sets the whole job's time, as for the device-resident step
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    return {"value": W["xs"].shape[0] * ws / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "steps": n, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "copies": f"pinned host <-> device every step, overlapped with compute ({nb} buffer sets)"}


# ---------------------------------------------------------------------------
# sinogram workloads: small non-TOF, clinical non-TOF, TOF sinogram
# ---------------------------------------------------------------------------
SINO_WORKLOADS = {
    # name: (sino spec, image geom, phantom, seed base, tof?)
    "sino_small": ("SINO_SMALL", "GEOM_SMALL", "PHANTOM_SMALL", 1000, False),
    "sino_clinical": ("SINO_CLINICAL", "GEOM_CLINICAL", "PHANTOM_CLINICAL", 2000, False),
    "tof_sino": ("SINO_TOF", "GEOM_CLINICAL", "PHANTOM_CLINICAL", 3000, True),
}


def measure_sino(workload, steps, warmup, opts=None, cpu_lors=0):
    """One step = forward + back projection of every LOR of the sinogram
    (LOR endpoints and their plan are computed once, outside the timed
    region, as the paper excludes LOR set-up).  Returns the bench line:
    LORs projected forward and back per second, per-kernel CUDA-event times,
    and the binding roofline of each kernel from work counted on the device
    against a ceiling measured in the same run (non-TOF: L2 reduction
    requests of the back projection vs the reduction ceiling; TOF: bin
    evaluations vs the per-bin operation's ceiling)."""
    from paper_2212_12519_gb300 import ops, synth
    dev = torch.device("cuda")
    spec_n, geom_n, ph_n, sb, is_tof = SINO_WORKLOADS[workload]
    spec, g, phs = getattr(synth, spec_n), getattr(synth, geom_n), getattr(synth, ph_n)
    tof = synth.TOF_CLINICAL if is_tof else None
    img = synth.ellipsoid_phantom(g, phs, sb + 1, device=dev)
    xs, xe = synth.sinogram_lors(spec, device=dev)
    n = xs.shape[0]
    gen = torch.Generator(device=dev)
    gen.manual_seed(sb + 2)
    if is_tof:
        y = torch.poisson(torch.full((n, tof.n_bins), 2.0, device=dev), generator=gen)
    else:
        y = torch.rand(n, generator=gen, device=dev)
    plan = ops.jp_plan_create(xs, xe, g, **(opts or {}))
    out = torch.zeros(g.shape, device=dev)
    stream = torch.cuda.current_stream()
    tim = {"fwd": [], "back": []}

    def rec(name, fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        tim[name].append((a, b))

    f = (lambda: ops.jp_fwd_tof_sino(plan, img, tof)) if is_tof else (lambda: ops.jp_fwd(plan, img))
    bk = (lambda: ops.jp_back_tof_sino(plan, y, tof, out)) if is_tof else (lambda: ops.jp_back(plan, y, out))
    for _ in range(warmup):
        f()
        bk()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = ops.jp_launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    rng_id = torch.cuda.nvtx.range_start("timed")
    t0.record(stream)
    for _ in range(steps):
        rec("fwd", f)
        rec("back", bk)
    t1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_end(rng_id)
    launches = ops.jp_launch_count() - launches0
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / steps
    kern = {k: statistics.mean(a.elapsed_time(b) for a, b in v) for k, v in tim.items()}
    samples = ops.jp_count_samples(plan, "nontof")
    peaks, peak_kind = measured_peaks()
    nb = tof.n_bins if is_tof else 1
    dom = "back" if kern["back"] >= kern["fwd"] else "fwd"
    nvox = int(np.prod(g.shape))
    alg = n * (24 + 4 * nb) + nvox * 4 * (2 if dom == "back" else 1)
    hbm = alg / (kern[dom] / 1e3) / 1e9
    hbm_line = {"bound": "hbm", "kernel": f"{dom}_{workload}", "achieved": hbm, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": hbm / peaks["hbm_gbs"], "traffic": None, "peak_source": peak_kind,
                "alg_bytes_per_launch": alg}
    if is_tof:
        bins = ops.jp_count_samples(plan, "tof_sino", tof)
        binding = {}
        for dname, direction in (("fwd", 0), ("back", 1)):
            ceil = ops.jp_bench_tof_bins(tof, direction)["bins_per_s"]
            ach = bins / (kern[dname] / 1e3)
            binding[dname] = {"kernel": f"{dname}_tof_sino", "resource": "TOF bin evaluations (table read, "
                              "interpolation and accumulation per bin)", "bound": "alu", "achieved": ach,
                              "peak": ceil, "unit": "bins/s", "frac": ach / ceil, "bins_per_launch": bins,
                              "bins_per_sample": bins / max(samples, 1),
                              "peak_source": "jp_bench_tof_bins (measured in this run)"}
        roofline = dict(binding["back"])
    else:
        req = ops.jp_count_red_requests(plan, "nontof")
        red = {pt: ops.jp_bench_red(pattern=pt) for pt in (0, 1, 2)}
        peak = max(r["sectors_per_s"] for r in red.values())
        ach = req / (kern["back"] / 1e3)
        roofline = {"bound": "l2", "kernel": f"back_{workload}",
                    "resource": "L2 reduction requests (32-byte sector operations)", "achieved": ach,
                    "peak": peak, "unit": "sectors/s", "frac": ach / peak, "traffic": None,
                    "requests_per_launch": req, "requests_per_sample": req / max(samples, 1),
                    "peak_source": "jp_bench_red_pattern (measured in this run), max over patterns"}
        binding = None
    line = {"metric": "LOR projections (fwd+back)/s", "value": n / (ms / 1e3), "unit": "LOR/s",
            "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload, "lors": n, "image": list(g.shape), "tof_bins": nb,
                       "l2": "LOR arrays larger than L2" if n * 24 > 200e6 else "small case, L2-resident"},
            "kernel_ms": kern, "samples_per_step": samples, "roofline": roofline, "hbm_roofline": hbm_line,
            "clocks": clk, "gpu_launches": int(launches)}
    if binding is not None:
        line["binding_roofline"] = binding
    if cpu_lors:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        m = min(n, cpu_lors)
        sx, se = xs[:m].cpu().numpy(), xe[:m].cpu().numpy()
        yy = y[:m].cpu().numpy()
        im = img.cpu().numpy()
        mode = "tof_sino" if is_tof else "nontof"
        t = time.perf_counter()
        oracle.fwd(sx, se, im, g, mode, tof, threads=threads)
        oracle.back(sx, se, yy, g, mode, tof, threads=threads)
        dt = time.perf_counter() - t
        line["cpu_baseline"] = {"value": m / dt, "unit": "LOR/s", "cores": threads, "kind": "oracle",
                                "sample": f"first {m} of {n} LORs, FP64 fwd+back, {dt:.1f} s"}
    plan.destroy()
    del xs, xe, y, out, img
    torch.cuda.empty_cache()
    return line


def run_sino(args):
    from paper_2212_12519_gb300 import build as jbuild, ops
    torch.cuda.set_device(dist_env()[2])
    jbuild.build()
    ops.load()
    line = measure_sino(args.workload, args.steps, args.warmup, plan_opts(args),
                        0 if args.no_cpu_baseline else args.cpu_lors)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# sinogram OSEM (34 view subsets, emission + contamination sinograms)
# ---------------------------------------------------------------------------
def run_sino_osem(args):
    """One step = one OSEM iteration over all 34 view subsets of the TOF
    sinogram (68.1M LORs x 29 bins, 200x200x71), data y ~ Poisson(A x + c)
    with a uniform contamination c (20 % of the mean projection), all
    device-resident; with --fwhm > 0 the resolution model wraps A."""
    from paper_2212_12519_gb300 import build as jbuild, ops, sino_osem, synth
    jbuild.build()
    ops.load()
    dev = torch.device("cuda")
    g, tof = synth.GEOM_CLINICAL, synth.TOF_CLINICAL
    spec = synth.SINO_TOF
    t0 = time.perf_counter()
    so = sino_osem.SinoOSEM(spec, g, n_sub=34, tof=tof, fwhm_mm=args.fwhm)
    x_true = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, 9001, device=dev)
    so.simulate(x_true, contamination=0.2, seed=9002)
    setup_s = time.perf_counter() - t0
    x = torch.empty(g.shape, dtype=torch.float32, device=dev)
    ops.jp_osem_init(x, sum(so.sens))
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        for m in range(so.n_sub):
            so.subset_update(x, m)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = ops.jp_launch_count()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        for m in range(so.n_sub):
            so.subset_update(x, m)
    b.record(stream)
    torch.cuda.synchronize()
    launches = ops.jp_launch_count() - launches0
    clk = clocks.stop()
    ms = a.elapsed_time(b) / args.steps
    n_lor = sum(so.n)
    data_gb = 2 * n_lor * tof.n_bins * 4 / 1e9
    line = {"metric": "sinogram OSEM iterations/s (34 subsets)", "value": 1e3 / ms, "unit": "iterations/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "sino_osem_tof_68M_x29_200x200x71", "subsets": so.n_sub, "lors": n_lor,
                       "tof_bins": tof.n_bins, "resolution_fwhm_mm": args.fwhm,
                       "device_data_gb": data_gb, "l2": "sinograms (>15 GB) larger than L2"},
            "lor_bins_per_s": n_lor * tof.n_bins / (ms / 1e3), "setup_s": setup_s,
            "clocks": clk, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)
    so.close()


def measure_lm_osem_iter(steps, warmup, fwhm):
    """The paper's LM-OSEM timing (Sec. 3, discussed in Sec. 4): one TOF
    listmode OSEM iteration (34 subset updates, each with the two
    resolution-model convolutions when fwhm > 0) for one frame of 40e6 and
    of 1.25e6 events on the 200x200x71 grid.  The frame's subset plan
    (binning) is built once before its iterations and timed separately; one
    iteration is a replayed CUDA graph."""
    from paper_2212_12519_gb300 import osem, synth
    dev = torch.device("cuda")
    g, tof = synth.GEOM_CLINICAL, synth.TOF_CLINICAL
    s_raw, _ = osem.sensitivity(g, check=False)
    sens = osem.resolution_sensitivity(s_raw, g, fwhm)
    ph = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, 9201, device=dev)
    b = synth.background_level(ph, tof)
    out = []
    for n_ev in (40_000_000, 1_250_000):
        xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, n_ev, seed=9202, device=dev)
        spec = osem.FrameSpec(xs, xe, tb, g, b, n_iter=1, n_sub=34, fwhm_mm=fwhm)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fr = osem.LMOSEMFrame(spec, sens, tof)
        e.record()
        torch.cuda.synchronize()
        bin_ms = a.elapsed_time(e)
        fr.run_graph()  # capture + one iteration
        for _ in range(warmup):
            fr.run_graph()
        torch.cuda.synchronize()
        a.record(fr.stream)
        for _ in range(steps):
            fr.run_graph()
        e.record(fr.stream)
        torch.cuda.synchronize()
        it_ms = a.elapsed_time(e) / steps
        out.append({"events": n_ev, "subsets": 34, "iteration_ms": it_ms, "plan_ms": bin_ms,
                    "convolutions_per_iteration": 68 if fwhm > 0 else 0,
                    "paper_gpu_iteration_ms": 600.0 if n_ev == 40_000_000 else 57.0})
        fr.release()
        del fr, xs, xe, tb, spec
        torch.cuda.empty_cache()
    del sens, s_raw, ph
    torch.cuda.empty_cache()
    return {"metric": "TOF LM-OSEM ms per iteration (34 subsets)",
            "config": {"workload": "lm_osem_iteration_200x200x71", "resolution_fwhm_mm": fwhm,
                       "steps": steps, "warmup": warmup},
            "rows": out}


def run_lm_osem_iter(args):
    from paper_2212_12519_gb300 import build as jbuild, ops
    jbuild.build()
    ops.load()
    print(json.dumps(measure_lm_osem_iter(args.steps, args.warmup, args.fwhm)), flush=True)


def run_layout_study(args):
    """The paper's memory-layout benchmark (Sec. 2.6 and 3): forward + back projection of one
    34-subset sinogram (one view subset of the clinical span-1 sinogram,
    ~4M LORs, paper: 415 x 8 x 1292) for every sinogram order (PVR, VRP,
    RVP) x image symmetry axis (0, 1, 2), non-TOF and TOF, through the
    binned plan and through the one-thread-per-LOR planless kernels in the
    caller's order.  Prints the time of each and the slowest / fastest
    ratio per path (the paper's GPU spread: 7.6 non-TOF, 3.6 TOF)."""
    from paper_2212_12519_gb300 import build as jbuild, ops, synth
    jbuild.build()
    ops.load()
    dev = torch.device("cuda")
    g0, tof = synth.GEOM_CLINICAL, synth.TOF_CLINICAL
    spec = synth.SINO_CLINICAL.subset(0, 34)
    img0 = synth.ellipsoid_phantom(g0, synth.PHANTOM_CLINICAL, 9101, device=dev)
    rows = []

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    for order in synth.SINO_ORDERS:
        xs0, xe0 = synth.sinogram_lors(spec, device=dev, order=order)
        n = xs0.shape[0]
        for axis in (0, 1, 2):
            g, xs, xe = synth.symmetry_axis(g0, xs0, xe0, axis)
            perm = {2: (0, 1, 2), 0: (2, 0, 1), 1: (0, 2, 1)}[axis]
            img = img0.permute(*perm).contiguous()
            out = torch.zeros(g.shape, device=dev)
            plan = ops.jp_plan_create(xs, xe, g)
            for mode in ("nontof", "tof_sino"):
                t = tof if mode == "tof_sino" else None
                y = torch.rand((n, tof.n_bins) if t else (n,), device=dev)
                if t:
                    planned = lambda: (ops.jp_fwd_tof_sino(plan, img, t), ops.jp_back_tof_sino(plan, y, t, out))
                    direct = lambda: (ops.jp_fwd_lors(xs, xe, img, g, "tof_sino", t),
                                      ops.jp_back_lors(xs, xe, y, g, out, "tof_sino", t))
                else:
                    planned = lambda: (ops.jp_fwd(plan, img), ops.jp_back(plan, y, out))
                    direct = lambda: (ops.jp_fwd_lors(xs, xe, img, g), ops.jp_back_lors(xs, xe, y, g, out))
                rows.append({"order": order, "symmetry_axis": axis, "mode": mode, "lors": n,
                             "planned_ms": timed(planned, args.steps), "planless_ms": timed(direct, args.steps)})
                del y
            plan.destroy()
    spread = {}
    for mode in ("nontof", "tof_sino"):
        for path in ("planned_ms", "planless_ms"):
            v = [r[path] for r in rows if r["mode"] == mode]
            spread[f"{mode}_{path[:-3]}"] = {"min_ms": min(v), "max_ms": max(v), "max_over_min": max(v) / min(v)}
    print(json.dumps({"metric": "layout study: fwd+back ms per order x symmetry axis",
                      "config": {"workload": "layout_study_sino_subset", "lors": rows[0]["lors"],
                                 "image": list(g0.shape), "tof_bins": tof.n_bins},
                      "spread": spread, "rows": rows}), flush=True)


# ---------------------------------------------------------------------------
# small cases for ncu captures
# ---------------------------------------------------------------------------
def run_profile_osem(args):
    """One frame (--events events, 200x200x71), one iteration of 34 subsets
    (with the --fwhm resolution model) through direct launches, for the ncu
    launch list."""
    from paper_2212_12519_gb300 import build as jbuild, ops, osem, synth
    jbuild.build()
    ops.load()
    dev = torch.device("cuda")
    g, tof = synth.GEOM_CLINICAL, synth.TOF_CLINICAL
    ph = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, 5010, device=dev)
    xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, args.events, seed=5011, device=dev)
    sens = torch.ones(g.shape, device=dev)
    spec = osem.FrameSpec(xs, xe, tb, g, synth.background_level(ph, tof), n_iter=1, n_sub=34, fwhm_mm=args.fwhm)
    fr = osem.LMOSEMFrame(spec, sens, tof)
    fr.run()
    torch.cuda.synchronize()
    rng = torch.cuda.nvtx.range_start("timed")
    t0 = time.perf_counter()
    fr = osem.LMOSEMFrame(spec, sens, tof, plan=fr.plan)
    fr.run()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_end(rng)
    print(json.dumps({"profile_osem": args.events, "ms": (time.perf_counter() - t0) * 1e3}))


def run_profile_tof_sino(args):
    """One view subset (1 of 34) of the TOF sinogram: 2.0M LORs x 29 bins,
    forward and back twice, for ncu captures of the TOF-sinogram kernels."""
    from paper_2212_12519_gb300 import build as jbuild, ops, synth
    jbuild.build()
    ops.load()
    dev = torch.device("cuda")
    g, tof = synth.GEOM_CLINICAL, synth.TOF_CLINICAL
    img = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, 3001, device=dev)
    xs, xe = synth.sinogram_lors(synth.SINO_TOF.subset(0, 34), device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(3002)
    y = torch.poisson(torch.full((xs.shape[0], tof.n_bins), 2.0, device=dev), generator=gen)
    plan = ops.jp_plan_create(xs, xe, g)
    out = torch.zeros(g.shape, device=dev)
    for _ in range(2):
        ops.jp_fwd_tof_sino(plan, img, tof)
        ops.jp_back_tof_sino(plan, y, tof, out)
    torch.cuda.synchronize()
    print(json.dumps({"profile_tof_sino": int(xs.shape[0]), "tof_bins": tof.n_bins,
                      "samples": ops.jp_count_samples(plan, "nontof")}))
    plan.destroy()


def run_profile_case(args):
    """One frame of --events listmode events (200x200x71, TOF unless
    --lm-mode nontof; from coordinates, or with --det from detector indices):
    the plan (key, scan x3, scatter, flags), then three times forward + back
    projection (each timed with CUDA events), then a rebind."""
    from paper_2212_12519_gb300 import build as jbuild, ops, synth
    jbuild.build()
    ops.load()
    dev = torch.device("cuda")
    g, tof = synth.GEOM_CLINICAL, synth.TOF_CLINICAL
    nontof = args.lm_mode == "nontof"
    ph = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, 4001, device=dev)
    xs, xe, tb, ds, de = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, args.events, seed=4051, device=dev,
                                         return_det=True)
    det = synth.SCANNER_CLINICAL.crystal_table(dev)
    y = torch.rand(args.events, device=dev)
    img = torch.zeros(g.shape, device=dev)
    popts = plan_opts(args)
    tb_arg = None if nontof else tb
    if args.det:
        # listmode as recorded: detector-index pairs and the detector table
        plan = ops.jp_plan_create_batch_det(ds, de, det, g, [0, args.events], tof_bin=tb_arg,
                                            tof_bin_width=0.0 if nontof else tof.bin_width, **popts)
    elif nontof:
        plan = ops.jp_plan_create(xs, xe, g, **popts)
    else:
        plan = ops.jp_plan_create(xs, xe, g, tof_bin=tb, tof_bin_width=tof.bin_width, **popts)
    if nontof:
        fwd, back = (lambda: ops.jp_fwd(plan, ph)), (lambda: ops.jp_back(plan, y, img))
    else:
        fwd, back = (lambda: ops.jp_fwd_tof_lm(plan, ph, tof)), (lambda: ops.jp_back_tof_lm(plan, y, tof, img))
    ms = {"fwd": [], "back": []}
    for _ in range(3):
        for name, fn in (("fwd", fwd), ("back", back)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            ms[name].append((a, b))
    if args.det:
        ops.jp_plan_rebind_det(plan, ds, de, det, [0, args.events], tof_bin=tb_arg)
    else:
        ops.jp_plan_rebind(plan, xs, xe, tof_bin=tb_arg)
    torch.cuda.synchronize()
    mode = "nontof" if nontof else "tof_lm"
    print(json.dumps({"profile_case": mode, "events": args.events, "det": bool(args.det), "path": args.path,
                      "plan_opts": popts,
                      "ms": {k: [a.elapsed_time(b) for a, b in v] for k, v in ms.items()},
                      "samples": ops.jp_count_samples(plan, mode, tof)}))
    plan.destroy()


def run_profile_sino(args):
    """One view subset (1 of 34, 10 views) of the clinical non-TOF sinogram:
    4,056,480 LORs (their endpoints and plan records exceed L2), forward and
    back projection three times, for ncu captures of the non-TOF sinogram
    kernels."""
    from paper_2212_12519_gb300 import build as jbuild, ops, synth
    jbuild.build()
    ops.load()
    dev = torch.device("cuda")
    g = synth.GEOM_CLINICAL
    img = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, 2001, device=dev)
    xs, xe = synth.sinogram_lors(synth.SINO_CLINICAL.subset(0, 34), device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2002)
    y = torch.rand(xs.shape[0], generator=gen, device=dev)
    plan = ops.jp_plan_create(xs, xe, g, **plan_opts(args))
    out = torch.zeros(g.shape, device=dev)
    for _ in range(3):
        ops.jp_fwd(plan, img)
        ops.jp_back(plan, y, out)
    torch.cuda.synchronize()
    print(json.dumps({"profile_sino": int(xs.shape[0]), "samples": ops.jp_count_samples(plan, "nontof"),
                      "red_requests": ops.jp_count_red_requests(plan, "nontof")}))
    plan.destroy()


# ---------------------------------------------------------------------------
# served listmode OSEM (frame stream): batched vs sequential plain
# ---------------------------------------------------------------------------
def time_gauss3d(g, fwhm_mm, reps=200):
    """Device time of one resolution-model convolution H x (three separable
    passes) of one image, and the bytes each pass moves at minimum (read +
    write of the image; the image stays in L2 between passes)."""
    from paper_2212_12519_gb300 import ops
    x = torch.rand(g.shape, device="cuda")
    out, work = torch.empty_like(x), torch.empty_like(x)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            ops.jp_gauss3d(x, g, fwhm_mm, out=out, work=work)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    # captured in a CUDA graph, as the OSEM iterations run, so host launch
    # cost does not enter the device time
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        for _ in range(reps):
            ops.jp_gauss3d(x, g, fwhm_mm, out=out, work=work)
    graph.replay()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    graph.replay()
    b.record()
    torch.cuda.synchronize()
    us = a.elapsed_time(b) * 1e3 / reps
    nbytes = 3 * 2 * 4 * x.numel()
    return {"image": list(g.shape), "us_per_convolution": us, "passes": 3,
            "min_bytes_per_convolution": nbytes, "GBps_effective": nbytes / (us * 1e-6) / 1e9}


def run_serving(n_requests=200, rates=(1.0,), pool_events=20_000_000, max_slots=4, budget_gb=None,
                use_graphs=True, seed=5001, fwhm_mm=4.5, extra_arms=True, control_rates=(1.0, 1.5, 3.0)):
    """Served listmode OSEM (config 5): the batched server (binned plans,
    graph-replayed iterations, continuous batching over max_slots
    concurrent frames) against sequential plain per-frame projection, at
    arrival rates given as multiples of the sequential capacity mu_seq.
    With extra_arms: the batched server with one slot (binned kernels and
    graphs, no overlap of frames), its capacity and at control_rates (the
    last close to the batched capacity, where the sequential server is long
    saturated and is not run), which separates what continuous batching
    buys from what the binned kernels buy; and, when fwhm_mm > 0, the same
    comparison without the resolution model."""
    from paper_2212_12519_gb300 import serve, synth
    tof = synth.TOF_CLINICAL
    t0 = time.perf_counter()
    pools = serve.make_event_pools(tof, pool_events=pool_events)
    geoms = [p["geom"] for p in pools.values()]
    budget = None if budget_gb is None else int(budget_gb * 2 ** 30)

    def arm(fwhm, arm_rates, one_slot_rates):
        from paper_2212_12519_gb300 import osem
        sens, checks = {}, {}
        for shape, pool in pools.items():
            s_, checks[str(shape)] = osem.sensitivity(pool["geom"])
            sens[shape] = osem.resolution_sensitivity(s_, pool["geom"], fwhm)
        res_model = time_gauss3d(synth.GEOM_CLINICAL, fwhm) if fwhm > 0 else None
        # mu_seq: sequential plain server, all requests available at once
        reqs = serve.make_requests(pools, n_requests, rate=1e9, seed=seed, fwhm_mm=fwhm)
        seq = serve.OSEMServer(sens, tof, mode="sequential")
        mu = seq.run(reqs)["frames_per_s"]
        bat = serve.OSEMServer(sens, tof, mode="batched", max_slots=max_slots, use_graphs=use_graphs,
                               hbm_budget=budget)
        bat.reserve(int(2e7), geoms, fwhm_mm=fwhm)
        one = None
        if one_slot_rates:
            one = serve.OSEMServer(sens, tof, mode="batched", max_slots=1, use_graphs=use_graphs)
            one.reserve(int(2e7), geoms, fwhm_mm=fwhm)
        serve.reset(reqs)
        cap = bat.run(reqs)
        out = {"requests": n_requests, "mu_seq_frames_per_s": mu, "batched_capacity_frames_per_s": cap["frames_per_s"],
               "sensitivity_fp64_check": checks, "resolution_fwhm_mm": fwhm, "resolution_model": res_model,
               "max_slots": max_slots, "sweep": []}
        if one is not None:
            serve.reset(reqs)
            out["batched_one_slot_capacity_frames_per_s"] = one.run(reqs)["frames_per_s"]
        for f in sorted(set(arm_rates) | set(one_slot_rates or ())):
            lam = f * mu
            reqs = serve.make_requests(pools, n_requests, rate=lam, seed=seed, fwhm_mm=fwhm)
            row = {"rate_x_mu_seq": f, "rate_frames_per_s": lam}
            if f in arm_rates:
                r_seq = seq.run(reqs)
                row["sequential"] = {k: r_seq[k] for k in ("frames_per_s", "p50_ms", "p99_ms")}
            serve.reset(reqs)
            r_bat = bat.run(reqs)
            row["batched"] = {k: r_bat[k] for k in ("frames_per_s", "p50_ms", "p99_ms", "events_per_s")}
            if one is not None and f in one_slot_rates:
                serve.reset(reqs)
                r_one = one.run(reqs)
                row["batched_one_slot"] = {k: r_one[k] for k in ("frames_per_s", "p50_ms", "p99_ms")}
            out["sweep"].append(row)
        bat.close()
        if one is not None:
            one.close()
        del sens
        torch.cuda.empty_cache()
        return out

    main = arm(fwhm_mm, list(rates), list(control_rates) if extra_arms else [])
    if extra_arms and fwhm_mm > 0:
        main["no_resolution_model"] = arm(0.0, [r for r in control_rates if r <= 1.5], list(control_rates))
    main["setup_s"] = time.perf_counter() - t0
    return main


# ---------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def _oracle_events(W, n):
    xs = W["xs"][:n].cpu().numpy()
    xe = W["xe"][:n].cpu().numpy()
    tb = W["tb"][:n].cpu().numpy() if W["tb"] is not None else None
    img = W["x"][0].detach().cpu().numpy()
    w = W["w"][:n].cpu().numpy()
    return xs, xe, tb, img, w


def oracle_step(xs, xe, tb, img, w, g, tof, b, threads):
    """FP64 oracle fwd + ratio + back of one event sample (non-TOF when tof is None)."""
    import oracle
    mode = "nontof" if tof is None else "tof_lm"
    p = oracle.fwd(xs, xe, img, g, mode, tof, tof_bin=tb, threads=threads)
    q = w / (p + b)
    oracle.back(xs, xe, q, g, mode, tof, tof_bin=tb, threads=threads)


def cpu_baseline(sample, b, g, tof, n_total, target_s=12.0):
    """The FP64 oracle (fwd + back, all host cores) on the first events of
    frame 0, sized to take about ``target_s`` seconds."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    xs, xe, tb, img, w = sample
    n0 = min(100_000, len(xs))
    t = time.perf_counter()
    oracle_step(xs[:n0], xe[:n0], None if tb is None else tb[:n0], img, w[:n0], g, tof, b, threads)
    dt = time.perf_counter() - t
    n = int(min(len(xs), max(n0, n0 * target_s / max(dt, 1e-3))))
    t = time.perf_counter()
    oracle_step(xs[:n], xe[:n], None if tb is None else tb[:n], img, w[:n], g, tof, b, threads)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n} events of frame 0 (of {n_total} in the batch), FP64 fwd+back, {dt:.1f} s"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2212_12519_gb300 import synth
    dev = "cpu"
    # a bounded sample of the same workload, generated on the host
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    ph = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, 4001, device=dev)
    n = args.ref_events
    xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, n, seed=4051, device=dev)
    w = synth.loss_weights(n, 4999, device=dev)
    b = synth.background_level(ph, tof)
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    nontof = args.workload == "nontof_lm"
    a = (xs.numpy(), xe.numpy(), None if nontof else tb.numpy(), ph.numpy(), w.numpy())
    if nontof:
        tof = None
        m = min(n, 20_000)
        b = 0.1 * float(oracle.fwd(a[0][:m], a[1][:m], a[3], g, "nontof", None, threads=threads).mean())
    for _ in range(args.warmup):
        oracle_step(*a, g, tof, b, threads)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(*a, g, tof, b, threads)
    dt = (time.perf_counter() - t) / args.steps
    value = n / dt
    line = {"impl": "reference", "metric": "non-TOF listmode fwd+back events/s" if nontof else METRIC,
            "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{'nontof' if nontof else 'tof'}_lm_batch{N_FRAMES}x"
                                   f"{EVENTS_PER_FRAME // 1_000_000}M_200x200x71",
                       "sample": f"{n} events of frame 0 per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n} events per step, FP64 fwd+back"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=N_FRAMES)
    ap.add_argument("--events", type=int, default=EVENTS_PER_FRAME)
    ap.add_argument("--ref-events", type=int, default=400_000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--det", action="store_true",
                    help="profile_case: bind the events from detector indices and the detector table")
    ap.add_argument("--e2e-buffers", type=int, default=3,
                    help="device input buffer sets of the end-to-end pipeline (>= 2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=200)
    ap.add_argument("--serving-rates", default="0.8,1.0,1.5")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the clinical-sinogram, TOF-sinogram and LM-OSEM-iteration lines of the default run")
    ap.add_argument("--workload", default="tof_lm",
                    choices=["tof_lm", "nontof_lm", "sino_small", "sino_clinical", "tof_sino", "osem",
                             "sino_osem", "layout_study", "lm_osem_iter", "profile_case", "profile_osem",
                             "profile_tof_sino", "profile_sino"])
    ap.add_argument("--cpu-lors", type=int, default=200_000)
    ap.add_argument("--budget-gb", type=float, default=None)
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--fwhm", type=float, default=4.5, help="OSEM resolution model FWHM in mm (0: none)")
    ap.add_argument("--path", default="quads", choices=["quads", "tiles"],
                    help="projection kernels of sorted plans: quad images or shared-memory tiles")
    ap.add_argument("--tile-lors", type=int, default=0, help="plan option: LORs per tile (0 = default)")
    ap.add_argument("--block", type=int, default=0, help="plan option: threads per CTA (0 = default)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="plan option: resident CTAs per SM (0 = default)")
    ap.add_argument("--lors-per-warp", type=int, default=0, help="plan option: LORs per warp (0 = default)")
    ap.add_argument("--lm-mode", default="tof_lm", choices=["tof_lm", "nontof"],
                    help="profile_case: TOF or non-TOF listmode")
    ap.add_argument("--event-sigma", action="store_true",
                    help="listmode workload with per-event TOF sigma (three timing classes)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "profile_case":
        run_profile_case(args)
    elif args.workload == "profile_osem":
        run_profile_osem(args)
    elif args.workload == "profile_tof_sino":
        run_profile_tof_sino(args)
    elif args.workload == "profile_sino":
        run_profile_sino(args)
    elif args.workload in SINO_WORKLOADS:
        run_sino(args)
    elif args.workload == "sino_osem":
        run_sino_osem(args)
    elif args.workload == "layout_study":
        run_layout_study(args)
    elif args.workload == "lm_osem_iter":
        run_lm_osem_iter(args)
    elif args.workload == "osem":
        from paper_2212_12519_gb300 import build as jbuild, ops
        jbuild.build()
        ops.load()
        rates = [float(r) for r in args.serving_rates.split(",")]
        out = run_serving(n_requests=args.serving_requests, rates=rates, max_slots=args.serving_slots,
                          budget_gb=args.budget_gb, use_graphs=not args.no_graphs, fwhm_mm=args.fwhm)
        print(json.dumps({"metric": "served listmode OSEM frames/s; p50/p99 latency", "workload": "osem_stream",
                          **out}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
