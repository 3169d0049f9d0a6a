"""The shared-memory tile kernels (JP_PLAN_TILES: non-TOF and TOF listmode,
sorted plans) against the quad-image kernels and the FP64 oracle.

A forward projection through the tiles splits every LOR's planes over the
lanes of a group exactly as the quad-image group kernels do, and its
samples read the same voxel values, so the two agree bit for bit at the
same lane count.  Back projections agree with the oracle at the back
tolerance (the order of the atomic additions varies)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_12519_gb300 import synth
from _parity import AMB_EPS, BACK_TOL, FWD_TOL, amb_check, fwd_err, rel_l2

pytestmark = pytest.mark.gpu

THREADS = 8


@pytest.fixture(scope="module")
def ops():
    from paper_2212_12519_gb300 import build, ops as _ops
    build.build()
    _ops.load()
    return _ops


def cuda(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


@pytest.fixture(scope="module")
def clinical():
    g = synth.GEOM_CLINICAL
    img = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, 2101).numpy()
    xs, xe, tb = synth.lm_events(torch.from_numpy(img), g, synth.SCANNER_CLINICAL, synth.TOF_CLINICAL,
                                 200_003, seed=4201)
    return g, img, xs.numpy(), xe.numpy(), tb.numpy()


def _project(ops, plan, mode, img, y, tof, g):
    out = torch.zeros(g.shape, device="cuda")
    if mode == "nontof":
        p = ops.jp_fwd(plan, img)
        ops.jp_back(plan, y, out)
    else:
        p = ops.jp_fwd_tof_lm(plan, img, tof)
        ops.jp_back_tof_lm(plan, y, tof, out)
    torch.cuda.synchronize()
    return p, out


@pytest.mark.parametrize("mode,exact", [("nontof", False), ("tof_lm", False), ("tof_lm", True)])
@pytest.mark.parametrize("lpw", [1, 2, 4, 8])
def test_tile_forward_bitwise_equals_quads(ops, clinical, mode, exact, lpw):
    g, img, xs, xe, tb = clinical
    tof = synth.TOF_CLINICAL
    kw = dict(tof_bin=cuda(tb, torch.int16), tof_bin_width=tof.bin_width) if mode == "tof_lm" else {}
    y = cuda(synth.uniform_values(len(xs), 4202, 0.5, 1.5).astype(np.float32))
    pt = ops.jp_plan_create(cuda(xs), cuda(xe), g, lors_per_warp=lpw, tof_exact=exact, tiles=True, **kw)
    pq = ops.jp_plan_create(cuda(xs), cuda(xe), g, lors_per_warp=lpw, tof_exact=exact, **kw)
    ft, bt = _project(ops, pt, mode, cuda(img), y, tof, g)
    fq, bq = _project(ops, pq, mode, cuda(img), y, tof, g)
    assert torch.equal(ft, fq)
    assert rel_l2(bt.cpu().numpy(), bq.cpu().numpy().astype(np.float64)) <= 1e-6
    pt.destroy()
    pq.destroy()


@pytest.mark.parametrize("opts", [dict(tile_lors=32), dict(tile_lors=1024), dict(slope_bins=1, offset_bins=1),
                                  dict(window_bins=1, zoff_bins=1)])
def test_tile_options_vs_oracle(ops, clinical, opts):
    """Tiles of 32 and 1024 LORs (more LORs than threads), one line per
    principal axis (boxes too large for shared memory: the global path) and
    no window / axial-offset keys, TOF listmode, against the oracle."""
    g, img, xs, xe, tb = clinical
    tof = synth.TOF_CLINICAL
    n = 60_000
    xs, xe, tb = xs[:n], xe[:n], tb[:n]
    y = synth.uniform_values(n, 4203, 0.5, 1.5)
    p_or, amb = oracle.fwd(xs, xe, img, g, "tof_lm", tof, tof_bin=tb, threads=THREADS, amb_eps=AMB_EPS,
                           return_amb=True)
    b_or = oracle.back(xs, xe, y, g, "tof_lm", tof, tof_bin=tb, threads=THREADS)
    plan = ops.jp_plan_create(cuda(xs), cuda(xe), g, tof_bin=cuda(tb, torch.int16), tof_bin_width=tof.bin_width,
                              tiles=True, **opts)
    p, out = _project(ops, plan, "tof_lm", cuda(img), cuda(y.astype(np.float32)), tof, g)
    amb_check(amb, xs, xe, g, tof, np.abs(img).max())
    assert fwd_err(p.cpu().numpy(), p_or, amb) <= FWD_TOL
    assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL
    plan.destroy()


@pytest.mark.parametrize("mode", ["nontof", "tof_lm"])
def test_tile_free_axis_b(ops, mode):
    """A grid whose longest in-plane extent is axis c for principal axes 0
    and 1, so the keys' line axis is c and the box columns run along b
    (strided in the image); non-isotropic voxels, an off-centre origin,
    LORs starting inside the image; frames with their own images."""
    g = synth.ImageGeom((22, 26, 41), (-21.0, -20.5, -38.0), (1.9, 1.6, 1.8))
    rng = np.random.Generator(np.random.PCG64(4301))
    imgs = rng.uniform(0, 2, size=(2,) + g.shape).astype(np.float32)
    xs1, xe1 = synth.random_lors(30_000, g, seed=4302)
    xs2, xe2 = synth.random_lors(6_000, g, seed=4303, kind="inside")
    xs, xe = np.concatenate([xs1, xs2]), np.concatenate([xe1, xe2])
    n = len(xs)
    tof = synth.TofParams(bin_width=7.0, sigma=6.0, n_sigmas=3.0, n_bins=15)
    tb = rng.integers(-7, 8, size=n).astype(np.int16)
    cuts = [0, 20_000, n]
    t = tof if mode == "tof_lm" else None
    kw = dict(tof_bin=cuda(tb), tof_bin_width=tof.bin_width) if mode == "tof_lm" else {}
    okw = dict(tof_bin=None) if mode == "nontof" else {}
    y = rng.uniform(0.2, 1.0, size=n).astype(np.float32)
    plan = ops.jp_plan_create_batch(cuda(xs), cuda(xe), g, cuts, lors_per_warp=4, tiles=True, **kw)
    out = torch.zeros((2,) + g.shape, device="cuda")
    if mode == "nontof":
        p = ops.jp_fwd(plan, cuda(imgs))
        ops.jp_back(plan, cuda(y), out)
    else:
        p = ops.jp_fwd_tof_lm(plan, cuda(imgs), tof)
        ops.jp_back_tof_lm(plan, cuda(y), tof, out)
    torch.cuda.synchronize()
    p = p.cpu().numpy()
    out = out.cpu().numpy()
    # the quad-image group kernel with the same 8 lanes per LOR
    pq = ops.jp_plan_create_batch(cuda(xs), cuda(xe), g, cuts, lors_per_warp=4, **kw)
    q = (ops.jp_fwd(pq, cuda(imgs)) if mode == "nontof" else ops.jp_fwd_tof_lm(pq, cuda(imgs), tof)).cpu().numpy()
    assert np.array_equal(p, q)
    for f in range(2):
        a, b = cuts[f], cuts[f + 1]
        lk = dict(tof_bin=tb[a:b]) if mode == "tof_lm" else okw
        p_or, amb = oracle.fwd(xs[a:b], xe[a:b], imgs[f], g, mode, t, threads=THREADS, amb_eps=AMB_EPS,
                               return_amb=True, **lk)
        if t is not None:
            amb_check(amb, xs[a:b], xe[a:b], g, t, np.abs(imgs[f]).max())
        assert fwd_err(p[a:b], p_or, amb) <= FWD_TOL
        b_or = oracle.back(xs[a:b], xe[a:b], y[a:b], g, mode, t, threads=THREADS, **lk)
        assert rel_l2(out[f], b_or) <= BACK_TOL
    plan.destroy()
    pq.destroy()


def test_tile_back_accumulates_and_handles_zero_weights(ops, clinical):
    """The back projection adds into the image (img += A^T y); LORs with
    y = 0 are skipped; repeated calls give the same image up to summation
    order."""
    g, img, xs, xe, tb = clinical
    tof = synth.TOF_CLINICAL
    n = 50_000
    y = synth.uniform_values(n, 4204, 0.5, 1.5).astype(np.float32)
    y[::3] = 0.0
    plan = ops.jp_plan_create(cuda(xs[:n]), cuda(xe[:n]), g, tof_bin=cuda(tb[:n], torch.int16),
                              tof_bin_width=tof.bin_width, tiles=True)
    base = torch.full(g.shape, 0.25, device="cuda")
    out = base.clone()
    ops.jp_back_tof_lm(plan, cuda(y), tof, out)
    ops.jp_back_tof_lm(plan, cuda(y), tof, out)
    torch.cuda.synchronize()
    b_or = oracle.back(xs[:n], xe[:n], y, g, "tof_lm", tof, tof_bin=tb[:n], threads=THREADS)
    assert rel_l2(out.cpu().numpy() - 0.25, 2.0 * b_or) <= BACK_TOL
    plan.destroy()


@pytest.mark.parametrize("mode", ["nontof", "tof_lm"])
def test_tile_back_wide_dynamic_range(ops, clinical, mode):
    """The back projection accumulates each tile in fixed point with a scale
    set by the tile's largest possible cell sum; back-projection inputs
    spanning six decades with both signs (as gradients do) still meet the
    back tolerance against the oracle."""
    g, img, xs, xe, tb = clinical
    tof = synth.TOF_CLINICAL
    n = 80_000
    rng = np.random.Generator(np.random.PCG64(4205))
    y = (10.0 ** rng.uniform(-3, 3, size=n) * rng.choice([-1.0, 1.0], size=n)).astype(np.float32)
    t = tof if mode == "tof_lm" else None
    kw = dict(tof_bin=cuda(tb[:n], torch.int16), tof_bin_width=tof.bin_width) if mode == "tof_lm" else {}
    okw = dict(tof_bin=tb[:n]) if mode == "tof_lm" else {}
    plan = ops.jp_plan_create(cuda(xs[:n]), cuda(xe[:n]), g, tiles=True, **kw)
    out = torch.zeros(g.shape, device="cuda")
    if mode == "nontof":
        ops.jp_back(plan, cuda(y), out)
    else:
        ops.jp_back_tof_lm(plan, cuda(y), tof, out)
    torch.cuda.synchronize()
    b_or = oracle.back(xs[:n], xe[:n], y, g, mode, t, threads=THREADS, **okw)
    assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL
    plan.destroy()
