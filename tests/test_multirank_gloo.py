"""Two CPU ranks (gloo): the sharded projector arithmetic.  Each rank
projects its contiguous LOR shard with the FP64 oracle; the sum-allreduce of
the partial back projections equals the whole back projection, the gathered
forward shards equal the whole forward projection, and the step time is the
maximum over ranks.  A rank that fails before its collective is reported to
the other by a short process-group timeout, not a hang."""
import datetime
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from paper_2212_12519_gb300 import synth
    g = synth.ImageGeom.centred((12, 10, 8), (2.0, 2.0, 2.0))
    xs, xe = synth.random_lors(3001, g, seed=77)
    y = synth.uniform_values(len(xs), 78)
    img = synth.uniform_values(g.shape, 79)
    return g, xs, xe, y, img


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    import oracle
    from paper_2212_12519_gb300 import dist as jdist
    g, xs, xe, y, img = _problem()
    n = len(xs)
    back = jdist.back_allreduce(lambda s, e: torch.from_numpy(oracle.back(xs[s:e], xe[s:e], y[s:e], g)), n)
    fwd = jdist.fwd_gather(lambda s, e: torch.from_numpy(oracle.fwd(xs[s:e], xe[s:e], img, g)), n)
    t = jdist.max_over_ranks(1.0 + rank)
    if rank == 0:
        q.put((back.numpy(), fwd.numpy(), t))
    dist.destroy_process_group()


def test_two_rank_partition_equals_whole():
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    back, fwd, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g, xs, xe, y, img = _problem()
    whole_b = oracle.back(xs, xe, y, g)
    whole_f = oracle.fwd(xs, xe, img, g)
    assert np.abs(back - whole_b).max() <= 1e-12 * np.abs(whole_b).max()
    assert np.array_equal(fwd, whole_f)
    assert t == 2.0


def test_shard_ranges_cover_exactly():
    from paper_2212_12519_gb300.dist import shard
    for n in (0, 1, 7, 1000, 1001):
        for w in (1, 2, 3, 8):
            rs = [shard(n, r, w) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(w - 1))
            assert max(e - s for s, e in rs) - min(e - s for s, e in rs) <= 1


def _failing_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        # a rank that dies between steps, before its collective
        os._exit(3)
    try:
        t = torch.ones(4)
        dist.all_reduce(t)
        q.put("no error")
    except Exception as e:  # the survivor learns of it through the timeout
        q.put("error: " + type(e).__name__)


def test_lost_rank_is_detected_not_hung():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    msg = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert msg.startswith("error")


def _osem_problem():
    from paper_2212_12519_gb300 import synth
    g = synth.ImageGeom.centred((14, 12, 8), (2.0, 2.0, 2.0))
    ph = synth.ellipsoid_phantom(g, synth.PhantomSpec((10.0, 8.0, 5.0), (3.0,)), 81)
    tof = synth.TOF_CLINICAL
    xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, 2001, seed=82)
    rng = np.random.Generator(np.random.PCG64(83))
    sens = rng.uniform(0.5, 2.0, size=g.shape)
    return g, tof, xs.numpy(), xe.numpy(), tb.numpy(), sens, 0.3


def _osem_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    import oracle
    from paper_2212_12519_gb300 import dist as jdist
    g, tof, xs, xe, tb, sens, b = _osem_problem()
    n_sub = 4
    x = torch.from_numpy((sens > 0).astype(np.float64))
    for m in range(n_sub):
        sx, se, st = xs[m::n_sub], xe[m::n_sub], tb[m::n_sub]
        s, e = jdist.shard(len(sx), rank, world)

        def local_bp(xc, s=s, e=e, sx=sx, se=se, st=st):
            p = oracle.fwd(sx[s:e], se[s:e], xc.numpy(), g, "tof_lm", tof, tof_bin=st[s:e])
            return torch.from_numpy(oracle.back(sx[s:e], se[s:e], 1.0 / (p + b), g, "tof_lm", tof, tof_bin=st[s:e]))

        def update(xc, bp):
            sc = torch.from_numpy(sens / n_sub)
            return torch.where(sc > 0, xc * bp / torch.where(sc > 0, sc, torch.ones_like(sc)), torch.zeros_like(xc))

        x = jdist.osem_subset_allreduce(x, local_bp, update)
    q.put((rank, x.numpy()))
    dist.destroy_process_group()


def test_two_rank_osem_subsets_equal_single_process():
    """LM-OSEM with each subset's events split over two ranks and one image
    allreduce per subset: both replicas equal the single-process oracle
    OSEM."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_osem_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g, tof, xs, xe, tb, sens, b = _osem_problem()
    whole = oracle.lm_osem(xs, xe, tb, g, tof, sens, b, n_iter=1, n_sub=4)
    for r in (0, 1):
        assert np.abs(got[r] - whole).max() <= 1e-11 * np.abs(whole).max()
    assert np.array_equal(got[0], got[1])
