"""Full-size parity in the launch configuration the benchmark times.

For each full workload (clinical non-TOF sinogram, 136.3M LORs; TOF
sinogram, 68.1M LORs x 29 bins; TOF listmode batch, 8 x 40M events) the GPU
projects every LOR through one plan, and the test checks
  * forward: a contiguous block of 4M sinogram LORs / one whole 40M-event
    frame element by element against the FP64 oracle (threaded on the host),
    plus a seeded sample of outputs elsewhere;
  * back: a dense input on that block / frame (zeros elsewhere) through the
    full launch, against the oracle's back projection of the block / frame;
    in the listmode batch also a sparse input in another frame, and every
    other frame's image stays zero;
  * the adjoint identity <A x, y> = <x, A^T y> over the whole workload, with
    FP64 dot products of the FP32 results (FP32 accumulation of ~1e4
    contributions per voxel bounds the gap near 1e-6; the test allows 1e-5).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_12519_gb300 import synth
from _parity import AMB_EPS, BACK_TOL, FWD_TOL, amb_check, fwd_err, rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

THREADS = 16
N_SAMPLE = 12_000
N_SPARSE = 400
N_BLOCK = 4_000_000  # contiguous sinogram LORs checked in full


@pytest.fixture(scope="module")
def ops():
    from paper_2212_12519_gb300 import build, ops as _ops
    build.build()
    _ops.load()
    return _ops


def sample_idx(n, k, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


def adjoint_gap(p, y, x, aty):
    lhs = float(torch.dot(p.reshape(-1).double(), y.reshape(-1).double()))
    rhs = float(torch.dot(x.reshape(-1).double(), aty.reshape(-1).double()))
    return abs(lhs - rhs) / abs(lhs)


@pytest.mark.parametrize("workload", ["sino_clinical", "tof_sino"])
def test_fullsize_sinogram(ops, workload):
    is_tof = workload == "tof_sino"
    spec = synth.SINO_TOF if is_tof else synth.SINO_CLINICAL
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL if is_tof else None
    sb = 3000 if is_tof else 2000
    img = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, sb + 1, device="cuda")
    xs, xe = synth.sinogram_lors(spec, device="cuda")
    n = xs.shape[0]
    assert n == (68_148_864 if is_tof else 136_297_728)
    plan = ops.jp_plan_create(xs, xe, g)
    p = ops.jp_fwd_tof_sino(plan, img, tof) if is_tof else ops.jp_fwd(plan, img)
    mode = "tof_sino" if is_tof else "nontof"
    img_h = img.cpu().numpy()
    # forward, sampled
    idx = sample_idx(n, N_SAMPLE, sb + 7)
    sx, se = xs[idx].cpu().numpy(), xe[idx].cpu().numpy()
    p_or, amb = oracle.fwd(sx, se, img_h, g, mode, tof, threads=THREADS, amb_eps=AMB_EPS, return_amb=True)
    ps = p[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    assert fwd_err(ps, p_or, amb) <= FWD_TOL
    # forward, a contiguous block of LORs in full
    b0 = n // 2 - N_BLOCK // 2
    bx, be = xs[b0:b0 + N_BLOCK].cpu().numpy(), xe[b0:b0 + N_BLOCK].cpu().numpy()
    p_or, amb = oracle.fwd(bx, be, img_h, g, mode, tof, threads=THREADS, amb_eps=AMB_EPS, return_amb=True)
    if is_tof:
        amb_check(amb, bx, be, g, tof, np.abs(img_h).max())
    assert fwd_err(p[b0:b0 + N_BLOCK].cpu().numpy(), p_or, amb) <= FWD_TOL
    del p_or, amb
    # back, a dense input on the block through the full launch
    nb = tof.n_bins if is_tof else 1
    rng = np.random.Generator(np.random.PCG64(sb + 9))
    yb = rng.uniform(0.5, 1.5, size=(N_BLOCK, nb) if is_tof else (N_BLOCK,)).astype(np.float32)
    y = torch.zeros((n, nb) if is_tof else (n,), device="cuda")
    y[b0:b0 + N_BLOCK] = torch.from_numpy(yb).cuda()
    out = torch.zeros(g.shape, device="cuda")
    if is_tof:
        ops.jp_back_tof_sino(plan, y, tof, out)
    else:
        ops.jp_back(plan, y, out)
    b_or = oracle.back(bx, be, yb, g, mode, tof, threads=THREADS)
    assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL
    del bx, be, yb, b_or
    # adjoint identity over the whole workload
    gen = torch.Generator(device="cuda")
    gen.manual_seed(sb + 10)
    xr = torch.rand(g.shape, generator=gen, device="cuda")
    yr = torch.rand(y.shape, generator=gen, device="cuda")
    pr = ops.jp_fwd_tof_sino(plan, xr, tof) if is_tof else ops.jp_fwd(plan, xr)
    aty = torch.zeros(g.shape, device="cuda")
    if is_tof:
        ops.jp_back_tof_sino(plan, yr, tof, aty)
    else:
        ops.jp_back(plan, yr, aty)
    assert adjoint_gap(pr, yr, xr, aty) <= 1e-5
    plan.destroy()


def test_fullsize_tof_listmode_batch(ops):
    """8 frames x 40M events in one batched plan, each frame its own image."""
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    F, E = 8, 40_000_000
    imgs, xs_l, xe_l, tb_l = [], [], [], []
    for f in range(F):
        seed = 4001 + f
        ph = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, seed, device="cuda")
        xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, E, seed=seed + 50, device="cuda")
        imgs.append(ph)
        xs_l.append(xs)
        xe_l.append(xe)
        tb_l.append(tb)
    x = torch.stack(imgs).contiguous()
    xs, xe, tb = torch.cat(xs_l), torch.cat(xe_l), torch.cat(tb_l)
    del xs_l, xe_l, tb_l
    off = [E * f for f in range(F + 1)]
    plan = ops.jp_plan_create_batch(xs, xe, g, off, tof_bin=tb, tof_bin_width=tof.bin_width)
    p = ops.jp_fwd_tof_lm(plan, x, tof)
    # forward: frame 0 in full, frames 3 and 7 sampled
    p_or, amb = oracle.fwd(xs[:E].cpu().numpy(), xe[:E].cpu().numpy(), x[0].cpu().numpy(), g, "tof_lm", tof,
                           tof_bin=tb[:E].cpu().numpy(), threads=THREADS, amb_eps=AMB_EPS, return_amb=True)
    amb_check(amb, xs[:E].cpu().numpy(), xe[:E].cpu().numpy(), g, tof, float(x[0].abs().max()))
    assert fwd_err(p[:E].cpu().numpy(), p_or, amb) <= FWD_TOL
    del p_or, amb
    for f in (3, 7):
        idx = sample_idx(E, N_SAMPLE // 3, 4100 + f) + E * f
        ti = torch.as_tensor(idx, device="cuda")
        p_or, amb = oracle.fwd(xs[ti].cpu().numpy(), xe[ti].cpu().numpy(), x[f].cpu().numpy(), g, "tof_lm", tof,
                               tof_bin=tb[ti].cpu().numpy(), threads=THREADS, amb_eps=AMB_EPS, return_amb=True)
        assert fwd_err(p[ti].cpu().numpy(), p_or, amb) <= FWD_TOL
    # back through the full launch: frame 1 dense (all 40M events), frame 6
    # sparse, every other frame zero
    y = torch.zeros(F * E, device="cuda")
    out = torch.zeros_like(x)
    rng = np.random.Generator(np.random.PCG64(4200))
    y1 = rng.uniform(0.5, 1.5, size=E).astype(np.float32)
    y[E:2 * E] = torch.from_numpy(y1).cuda()
    sp = sample_idx(E, N_SPARSE, 4207) + E * 6
    vals = rng.uniform(0.5, 1.5, size=len(sp)).astype(np.float32)
    y[torch.as_tensor(sp, device="cuda")] = torch.from_numpy(vals).cuda()
    ops.jp_back_tof_lm(plan, y, tof, out)
    b_or = oracle.back(xs[E:2 * E].cpu().numpy(), xe[E:2 * E].cpu().numpy(), y1, g, "tof_lm", tof,
                       tof_bin=tb[E:2 * E].cpu().numpy(), threads=THREADS)
    assert rel_l2(out[1].cpu().numpy(), b_or) <= BACK_TOL
    del b_or, y1
    ts = torch.as_tensor(sp, device="cuda")
    b_or = oracle.back(xs[ts].cpu().numpy(), xe[ts].cpu().numpy(), vals, g, "tof_lm", tof,
                       tof_bin=tb[ts].cpu().numpy(), threads=THREADS)
    assert rel_l2(out[6].cpu().numpy(), b_or) <= BACK_TOL
    for f in (0, 2, 3, 4, 5, 7):
        assert float(out[f].abs().sum()) == 0.0
    # adjoint identity over all 320M events
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4300)
    yr = torch.rand(F * E, generator=gen, device="cuda")
    aty = torch.zeros_like(x)
    ops.jp_back_tof_lm(plan, yr, tof, aty)
    assert adjoint_gap(p, yr, x, aty) <= 1e-5
    plan.destroy()
