"""GPU (CUDA, sm_103a) vs FP64 oracle parity, element by element, at sizes
the oracle finishes in seconds (several CTAs and a ragged tail), plus edge
cases.  Forward: max|err| <= 1e-5 max|oracle| (TOF-window decisions inside
the FP32/FP64 rounding band excepted); back: relative L2 <= 1e-4."""
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


# ---------------------------------------------------------------------------
# small sinogram workload (266,240 LORs, 64x64x16), non-TOF
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small():
    g = synth.GEOM_SMALL
    img = synth.ellipsoid_phantom(g, synth.PHANTOM_SMALL, 1001).numpy()
    xs, xe = synth.sinogram_lors(synth.SINO_SMALL)
    xs, xe = xs.numpy(), xe.numpy()
    y = synth.uniform_values(len(xs), 1002)
    p_or = oracle.fwd(xs, xe, img, g, threads=THREADS)
    b_or = oracle.back(xs, xe, y, g, threads=THREADS)
    return g, img, xs, xe, y, p_or, b_or


@pytest.mark.parametrize("planned", [0, 1, 4, 32, False])
def test_small_nontof(ops, small, planned):
    g, img, xs, xe, y, p_or, b_or = small
    dxs, dxe, dimg, dy = cuda(xs), cuda(xe), cuda(img), cuda(y)
    out = torch.zeros(g.shape, device="cuda")
    if planned is not False:
        plan = ops.jp_plan_create(dxs, dxe, g, lors_per_warp=planned)
        p = ops.jp_fwd(plan, dimg)
        ops.jp_back(plan, dy, out)
    else:
        p = ops.jp_fwd_lors(dxs, dxe, dimg, g)
        ops.jp_back_lors(dxs, dxe, dy, g, out)
    torch.cuda.synchronize()
    assert fwd_err(p.cpu().numpy(), p_or) <= FWD_TOL
    assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL


def test_plan_permutation_is_a_permutation(ops, small):
    g, img, xs, xe, *_ = small
    plan = ops.jp_plan_create(cuda(xs), cuda(xe), g)
    perm = plan.perm().cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(len(xs)))
    keep = ops.jp_plan_create(cuda(xs), cuda(xe), g, keep_order=True)
    assert np.array_equal(keep.perm().cpu().numpy(), np.arange(len(xs)))


def test_forward_is_deterministic(ops, small):
    g, img, xs, xe, *_ = small
    plan = ops.jp_plan_create(cuda(xs), cuda(xe), g)
    a = ops.jp_fwd(plan, cuda(img)).cpu()
    plan2 = ops.jp_plan_create(cuda(xs), cuda(xe), g, slope_bins=7, offset_bins=5)
    b = ops.jp_fwd(plan2, cuda(img)).cpu()
    assert torch.equal(a, b)  # bitwise: the sort order does not change a LOR's arithmetic
    c = ops.jp_fwd_lors(cuda(xs), cuda(xe), cuda(img), g).cpu()
    assert fwd_err(c.numpy(), a.numpy()) <= 1e-6  # planless path: scalar gathers, other rounding


# ---------------------------------------------------------------------------
# clinical image, TOF sinogram (a subset of views/planes of the TOF sinogram)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def clinical_img():
    return synth.ellipsoid_phantom(synth.GEOM_CLINICAL, synth.PHANTOM_CLINICAL, 2001).numpy()


def tof_sino_subset(n_planes=24, view_step=16):
    spec = synth.SinoSpec(synth.SCANNER_CLINICAL, 336, 313, view_step=view_step)
    xs, xe = synth.sinogram_lors(spec, plane_range=(0, 1296))
    # a spread of planes (ring pairs), every view_step-th view
    idx = np.linspace(0, 1295, n_planes).astype(np.int64)
    per = len(spec.views) * spec.n_rad
    sel = (idx[:, None] * per + np.arange(per)[None, :]).ravel()
    return xs.numpy()[sel], xe.numpy()[sel]


@pytest.mark.parametrize("planned", ["lut", "exact", "planless"])
def test_tof_sino(ops, clinical_img, planned):
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    xs, xe = tof_sino_subset()
    n = len(xs)
    y = synth.poisson_values((n, tof.n_bins), 3002)
    p_or, amb = oracle.fwd(xs, xe, clinical_img, g, "tof_sino", tof, threads=THREADS,
                           amb_eps=AMB_EPS, return_amb=True)
    b_or = oracle.back(xs, xe, y, g, "tof_sino", tof, threads=THREADS)
    out = torch.zeros(g.shape, device="cuda")
    if planned != "planless":
        plan = ops.jp_plan_create(cuda(xs), cuda(xe), g, tof_exact=(planned == "exact"))
        p = ops.jp_fwd_tof_sino(plan, cuda(clinical_img), tof)
        ops.jp_back_tof_sino(plan, cuda(y), tof, out)
    else:
        p = ops.jp_fwd_lors(cuda(xs), cuda(xe), cuda(clinical_img), g, "tof_sino", tof)
        ops.jp_back_lors(cuda(xs), cuda(xe), cuda(y), g, out, "tof_sino", tof)
    torch.cuda.synchronize()
    amb_check(amb, xs, xe, g, tof, np.abs(clinical_img).max())
    assert fwd_err(p.cpu().numpy(), p_or, amb) <= FWD_TOL
    assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL


def test_tof_sino_forward_block_sizes_agree(ops, clinical_img):
    """The TOF-sinogram forward's default 512-thread CTAs and explicit
    256 / 64-thread ones compute every LOR's bins with the same arithmetic:
    identical output."""
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    xs, xe = tof_sino_subset()
    img = cuda(clinical_img)
    outs = []
    for block in (0, 256, 64):
        plan = ops.jp_plan_create(cuda(xs), cuda(xe), g, block=block)
        outs.append(ops.jp_fwd_tof_sino(plan, img, tof))
        plan.destroy()
    assert float(outs[0].abs().max()) > 0
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


# ---------------------------------------------------------------------------
# TOF listmode
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def lm_events(clinical_img):
    g = synth.GEOM_CLINICAL
    xs, xe, tb = synth.lm_events(torch.from_numpy(clinical_img), g, synth.SCANNER_CLINICAL,
                                 synth.TOF_CLINICAL, 300_001, seed=4101)
    return xs.numpy(), xe.numpy(), tb.numpy()


@pytest.mark.parametrize("planned", ["lut", "exact", "planless", "lpw1", "lpw2", "lpw32"])
def test_tof_lm(ops, clinical_img, lm_events, planned):
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    xs, xe, tb = lm_events
    y = synth.uniform_values(len(xs), 4102, 0.5, 1.5)
    p_or, amb = oracle.fwd(xs, xe, clinical_img, g, "tof_lm", tof, tof_bin=tb, threads=THREADS,
                           amb_eps=AMB_EPS, return_amb=True)
    b_or = oracle.back(xs, xe, y, g, "tof_lm", tof, tof_bin=tb, threads=THREADS)
    out = torch.zeros(g.shape, device="cuda")
    dtb = cuda(tb, torch.int16)
    if planned != "planless":
        lpw = int(planned[3:]) if planned.startswith("lpw") else 0
        plan = ops.jp_plan_create(cuda(xs), cuda(xe), g, tof_bin=dtb, tof_bin_width=tof.bin_width,
                                  tof_exact=(planned == "exact"), lors_per_warp=lpw)
        p = ops.jp_fwd_tof_lm(plan, cuda(clinical_img), tof)
        ops.jp_back_tof_lm(plan, cuda(y), tof, out)
    else:
        p = ops.jp_fwd_lors(cuda(xs), cuda(xe), cuda(clinical_img), g, "tof_lm", tof, tof_bin=dtb)
        ops.jp_back_lors(cuda(xs), cuda(xe), cuda(y), g, out, "tof_lm", tof, tof_bin=dtb)
    torch.cuda.synchronize()
    amb_check(amb, xs, xe, g, tof, np.abs(clinical_img).max())
    assert fwd_err(p.cpu().numpy(), p_or, amb) <= FWD_TOL
    assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL


def test_tof_offsets_and_nonisotropic(ops):
    """Per-LOR TOF centre offsets, non-isotropic voxels, an off-centre origin
    and LORs starting/ending inside the image, all three TOF modes."""
    g = synth.ImageGeom((37, 29, 23), (-40.0, -25.0, -20.5), (2.1, 1.7, 1.9))
    rng = np.random.Generator(np.random.PCG64(5001))
    img = rng.uniform(0, 3, size=g.shape).astype(np.float32)
    xs1, xe1 = synth.random_lors(40_000, g, seed=5002)
    xs2, xe2 = synth.random_lors(9_000, g, seed=5003, kind="inside")
    xs, xe = np.concatenate([xs1, xs2]), np.concatenate([xe1, xe2])
    n = len(xs)
    tof = synth.TofParams(bin_width=9.0, sigma=7.0, n_sigmas=3.0, n_bins=15)
    delta = rng.normal(0, 4, size=n).astype(np.float32)
    tb = rng.integers(-7, 8, size=n).astype(np.int16)
    for mode in ["nontof", "tof_sino", "tof_lm"]:
        t = None if mode == "nontof" else tof
        kw = dict(tof_bin=tb) if mode == "tof_lm" else {}
        p_or, amb = oracle.fwd(xs, xe, img, g, mode, t, delta=delta if mode != "nontof" else None,
                               threads=THREADS, amb_eps=AMB_EPS, return_amb=True, **kw)
        nout = tof.n_bins if mode == "tof_sino" else 1
        y = rng.uniform(0, 1, size=n * nout).astype(np.float32)
        b_or = oracle.back(xs, xe, y, g, mode, t, delta=delta if mode != "nontof" else None,
                           threads=THREADS, **kw)
        plan = ops.jp_plan_create(cuda(xs), cuda(xe), g, tof_bin=cuda(tb),
                                  delta=cuda(delta), tof_bin_width=tof.bin_width, block=128)
        out = torch.zeros(g.shape, device="cuda")
        dy = cuda(y.reshape((n, nout)) if mode == "tof_sino" else y)
        if mode == "nontof":
            p = ops.jp_fwd(plan, cuda(img))
            ops.jp_back(plan, dy, out)
        elif mode == "tof_sino":
            p = ops.jp_fwd_tof_sino(plan, cuda(img), tof)
            ops.jp_back_tof_sino(plan, dy, tof, out)
        else:
            p = ops.jp_fwd_tof_lm(plan, cuda(img), tof)
            ops.jp_back_tof_lm(plan, dy, tof, out)
        torch.cuda.synchronize()
        if t is not None:
            amb_check(amb, xs, xe, g, t, np.abs(img).max())
        assert fwd_err(p.cpu().numpy(), p_or, amb) <= FWD_TOL, mode
        assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL, mode


def test_edge_cases(ops):
    """Empty input, degenerate LORs, misses, axis-aligned rays, exact
    principal-axis ties, every principal axis including axis 2."""
    g = synth.ImageGeom((9, 8, 7), (-4.0, -3.5, -3.0), (1.0, 1.0, 1.0))
    rng = np.random.Generator(np.random.PCG64(6001))
    img = rng.uniform(0, 2, size=g.shape).astype(np.float32)
    xs = [(0.1, 0.2, 0.3), (-20, 30, 5), (-20, 0.0, 0.0), (0.5, -20, 0.5), (0.25, -0.5, -20),
          (-6.0, -6.3, -0.9), (-4.0, 1.0, -4.1), (-3.0, -2.0, -9.0), (-9.0, 0.0, 0.0)]
    xe = [(0.1, 0.2, 0.3), (20, 30, 5), (20, 0.0, 0.0), (0.5, 20, 0.5), (0.25, -0.5, 20),
          (6.0, 5.7, 0.8), (4.0, -0.3, 3.9), (2.0, 2.5, 9.0), (0.0, 0.0, 0.0)]
    xs = np.asarray(xs, np.float32)
    xe = np.asarray(xe, np.float32)
    p_or = oracle.fwd(xs, xe, img, g)
    p = ops.jp_fwd_lors(cuda(xs), cuda(xe), cuda(img), g).cpu().numpy()
    assert p[0] == 0.0 and p[1] == 0.0
    assert fwd_err(p, p_or) <= FWD_TOL
    plan = ops.jp_plan_create(cuda(xs), cuda(xe), g)
    assert fwd_err(ops.jp_fwd(plan, cuda(img)).cpu().numpy(), p_or) <= FWD_TOL
    # empty input
    e = torch.zeros((0, 3), device="cuda")
    assert ops.jp_fwd_lors(e, e, cuda(img), g).numel() == 0
    plan0 = ops.jp_plan_create(e, e, g)
    assert ops.jp_fwd(plan0, cuda(img)).numel() == 0
    out = torch.zeros(g.shape, device="cuda")
    ops.jp_back(plan0, torch.zeros(0, device="cuda"), out)
    assert float(out.abs().sum()) == 0.0


def test_batched_frames(ops, clinical_img, lm_events):
    """Three frames (one of them empty) in one plan and one launch, frame f
    reading image f; each frame equals the oracle on its own events."""
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    xs, xe, tb = lm_events
    cuts = [0, 70_001, 70_001, 130_000]
    imgs = np.stack([clinical_img, 0.5 * clinical_img[::-1].copy(), clinical_img ** 2])
    ys = synth.uniform_values(cuts[-1], 7001)
    plan = ops.jp_plan_create_batch(cuda(xs[:cuts[-1]]), cuda(xe[:cuts[-1]]), g, cuts,
                                    tof_bin=cuda(tb[:cuts[-1]]), tof_bin_width=tof.bin_width)
    p = ops.jp_fwd_tof_lm(plan, cuda(imgs), tof).cpu().numpy()
    out = torch.zeros((3,) + g.shape, device="cuda")
    ops.jp_back_tof_lm(plan, cuda(ys), tof, out)
    out = out.cpu().numpy()
    for f in range(3):
        a, b = cuts[f], cuts[f + 1]
        if a == b:
            assert float(np.abs(out[f]).sum()) == 0.0
            continue
        p_or, amb = oracle.fwd(xs[a:b], xe[a:b], imgs[f], g, "tof_lm", tof, tof_bin=tb[a:b],
                               threads=THREADS, amb_eps=AMB_EPS, return_amb=True)
        amb_check(amb, xs[a:b], xe[a:b], g, tof, np.abs(imgs[f]).max())
        assert fwd_err(p[a:b], p_or, amb) <= FWD_TOL
        b_or = oracle.back(xs[a:b], xe[a:b], ys[a:b], g, "tof_lm", tof, tof_bin=tb[a:b], threads=THREADS)
        assert rel_l2(out[f], b_or) <= BACK_TOL
    # rebind the same plan with a different split (no allocation)
    cuts2 = [0, 10_000, 130_000]
    ops.jp_plan_rebind(plan, cuda(xs[:cuts2[-1]]), cuda(xe[:cuts2[-1]]), cuts2, tof_bin=cuda(tb[:cuts2[-1]]))
    p2 = ops.jp_fwd_tof_lm(plan, cuda(imgs[:2]), tof).cpu().numpy()
    p_or0, amb0 = oracle.fwd(xs[:10_000], xe[:10_000], imgs[0], g, "tof_lm", tof, tof_bin=tb[:10_000],
                             threads=THREADS, amb_eps=AMB_EPS, return_amb=True)
    amb_check(amb0, xs[:10_000], xe[:10_000], g, tof, np.abs(imgs[0]).max())
    assert fwd_err(p2[:10_000], p_or0, amb0) <= FWD_TOL


@pytest.mark.parametrize("lpw", [0, 4, 32])
def test_nontof_lm_batch(ops, clinical_img, lm_events, lpw):
    """Non-TOF listmode: the events of two frames (TOF bins dropped) in one
    batched plan without TOF keys, as the non-TOF listmode benchmark runs
    them; each frame against the oracle on its own image."""
    g = synth.GEOM_CLINICAL
    xs, xe, _ = lm_events
    cuts = [0, 90_001, 200_000]
    imgs = np.stack([clinical_img, 0.25 + clinical_img[:, ::-1].copy()])
    ys = synth.uniform_values(cuts[-1], 7101, 0.5, 1.5)
    plan = ops.jp_plan_create_batch(cuda(xs[:cuts[-1]]), cuda(xe[:cuts[-1]]), g, cuts, lors_per_warp=lpw)
    p = ops.jp_fwd(plan, cuda(imgs)).cpu().numpy()
    out = torch.zeros((2,) + g.shape, device="cuda")
    ops.jp_back(plan, cuda(ys), out)
    out = out.cpu().numpy()
    for f in range(2):
        a, b = cuts[f], cuts[f + 1]
        p_or = oracle.fwd(xs[a:b], xe[a:b], imgs[f], g, "nontof", threads=THREADS)
        assert fwd_err(p[a:b], p_or) <= FWD_TOL
        b_or = oracle.back(xs[a:b], xe[a:b], ys[a:b], g, "nontof", threads=THREADS)
        assert rel_l2(out[f], b_or) <= BACK_TOL


def test_osem_elementwise(ops):
    rng = np.random.Generator(np.random.PCG64(8001))
    p = rng.uniform(0, 5, size=100_003).astype(np.float32)
    b = np.array([0.3, 1.1], np.float32)
    q = ops.jp_osem_ratio(None, cuda(p), cuda(b[:1]), out=torch.empty(len(p), device="cuda"))
    np.testing.assert_allclose(q.cpu().numpy(), 1.0 / (p.astype(np.float64) + 0.3), rtol=1e-6)
    x = rng.uniform(0, 2, size=(2, 1000)).astype(np.float32)
    bp = rng.uniform(0, 2, size=(2, 1000)).astype(np.float32)
    s = rng.uniform(0, 2, size=1000).astype(np.float32)
    s[::7] = 0
    dx = cuda(x)
    ops.jp_osem_update(dx, cuda(bp), cuda(s), 0.125, 1000, n_frames=2, img_stride=1000, s_stride=0)
    ref = np.where(s > 0, x.astype(np.float64) * bp / (s.astype(np.float64) * 0.125), 0.0)
    np.testing.assert_allclose(dx.cpu().numpy(), ref, rtol=2e-6)
    v = rng.uniform(0, 1, size=1_000_001).astype(np.float32)
    assert float(ops.jp_sum_f64(cuda(v))) == pytest.approx(float(v.astype(np.float64).sum()), rel=1e-12)


@pytest.mark.parametrize("shape", [(1, 24, 20), (17, 1, 9), (11, 13, 1), (1, 1, 30)])
def test_degenerate_axes(ops, shape):
    """Images with a single voxel along one or two axes (2D and 1D grids),
    every mode, planned and planless."""
    g = synth.ImageGeom.centred(shape, (2.0, 1.5, 2.5))
    rng = np.random.Generator(np.random.PCG64(6101))
    img = rng.uniform(0, 2, size=shape).astype(np.float32)
    xs, xe = synth.random_lors(5000, g, seed=6102)
    tof = synth.TofParams(bin_width=6.0, sigma=5.0, n_sigmas=3.0, n_bins=9)
    tb = rng.integers(-4, 5, size=len(xs)).astype(np.int16)
    for mode in ["nontof", "tof_sino", "tof_lm"]:
        t = None if mode == "nontof" else tof
        kw = dict(tof_bin=tb) if mode == "tof_lm" else {}
        p_or, amb = oracle.fwd(xs, xe, img, g, mode, t, amb_eps=AMB_EPS, return_amb=True, **kw)
        plan = ops.jp_plan_create(cuda(xs), cuda(xe), g, tof_bin=cuda(tb), tof_bin_width=tof.bin_width)
        if mode == "nontof":
            p = ops.jp_fwd(plan, cuda(img))
        elif mode == "tof_sino":
            p = ops.jp_fwd_tof_sino(plan, cuda(img), tof)
        else:
            p = ops.jp_fwd_tof_lm(plan, cuda(img), tof)
        q = ops.jp_fwd_lors(cuda(xs), cuda(xe), cuda(img), g, mode, t, tof_bin=cuda(tb) if mode == "tof_lm" else None)
        torch.cuda.synchronize()
        if t is not None:
            amb_check(amb, xs, xe, g, t, np.abs(img).max())
        assert fwd_err(p.cpu().numpy(), p_or, amb) <= FWD_TOL, mode
        assert fwd_err(q.cpu().numpy(), p_or, amb) <= FWD_TOL, mode
        nout = tof.n_bins if mode == "tof_sino" else 1
        y = rng.uniform(0, 1, size=len(xs) * nout).astype(np.float32)
        b_or = oracle.back(xs, xe, y, g, mode, t, **kw)
        out = torch.zeros(shape, device="cuda")
        dy = cuda(y.reshape(len(xs), nout) if mode == "tof_sino" else y)
        if mode == "nontof":
            ops.jp_back(plan, dy, out)
        elif mode == "tof_sino":
            ops.jp_back_tof_sino(plan, dy, tof, out)
        else:
            ops.jp_back_tof_lm(plan, dy, tof, out)
        torch.cuda.synchronize()
        if np.abs(b_or).max() > 0:
            assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL, mode


def test_detector_index_plans(ops, clinical_img):
    """Plans from detector-index events equal plans from the gathered
    coordinates: identical forward projections, back projections equal up
    to summation order, and against the oracle; an index outside the
    table gives an empty LOR; rebinding to other events works."""
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    sc = synth.SCANNER_CLINICAL
    xs, xe, tb, ds, de = synth.lm_events(torch.from_numpy(clinical_img), g, sc, tof, 120_001, seed=4601,
                                         return_det=True)
    table = sc.crystal_table("cuda")
    img = cuda(clinical_img)
    ds_c, de_c = ds.cuda(), de.cuda()
    ds_c[::5000] = -1
    de_c[7::5000] = table.shape[0]
    bad = (ds_c < 0) | (de_c >= table.shape[0])
    cuts = [0, 50_000, 120_001]
    pd = ops.jp_plan_create_batch_det(ds_c, de_c, table, g, cuts, tof_bin=tb.cuda(), tof_bin_width=tof.bin_width)
    pc = ops.jp_plan_create_batch(xs.cuda(), xe.cuda(), g, cuts, tof_bin=tb.cuda(), tof_bin_width=tof.bin_width)
    imgs = torch.stack([img, 0.5 * img]).contiguous()
    fd = ops.jp_fwd_tof_lm(pd, imgs, tof)
    fc = ops.jp_fwd_tof_lm(pc, imgs, tof)
    assert torch.equal(fd[~bad], fc[~bad])
    assert float(fd[bad].abs().max()) == 0.0
    y = torch.rand(cuts[-1], device="cuda")
    y[bad] = 0.0
    bd = ops.jp_back_tof_lm(pd, y, tof, torch.zeros_like(imgs))
    bc = ops.jp_back_tof_lm(pc, y, tof, torch.zeros_like(imgs))
    assert rel_l2(bd.cpu().numpy(), bc.cpu().numpy().astype(np.float64)) <= 1e-6
    ok = (~bad).cpu().numpy()
    p_or, amb = oracle.fwd(xs.numpy()[:50_000][ok[:50_000]], xe.numpy()[:50_000][ok[:50_000]], clinical_img, g,
                           "tof_lm", tof, tof_bin=tb.numpy()[:50_000][ok[:50_000]], threads=THREADS,
                           amb_eps=AMB_EPS, return_amb=True)
    amb_check(amb, xs.numpy()[:50_000][ok[:50_000]], xe.numpy()[:50_000][ok[:50_000]], g, tof,
              np.abs(clinical_img).max())
    assert fwd_err(fd[:50_000][~bad[:50_000]].cpu().numpy(), p_or, amb) <= FWD_TOL
    # rebind to the second half of the events as one frame
    ops.jp_plan_rebind_det(pd, ds.cuda()[60_000:], de.cuda()[60_000:], table, tof_bin=tb.cuda()[60_000:])
    f2 = ops.jp_fwd_tof_lm(pd, img, tof).cpu().numpy()
    p_or2, amb2 = oracle.fwd(xs.numpy()[60_000:], xe.numpy()[60_000:], clinical_img, g, "tof_lm", tof,
                             tof_bin=tb.numpy()[60_000:], threads=THREADS, amb_eps=AMB_EPS, return_amb=True)
    amb_check(amb2, xs.numpy()[60_000:], xe.numpy()[60_000:], g, tof, np.abs(clinical_img).max())
    assert fwd_err(f2, p_or2, amb2) <= FWD_TOL
    pd.destroy()
    pc.destroy()


def test_detector_table_read_paths(ops, clinical_img):
    """The plan reads detector coordinates from its 16-byte-padded copy of
    the table when the table fits the copy made at creation, else from the
    caller's [n_det][3] table; both give the coordinate plan's forward bit
    for bit (a plan created from coordinates and rebound to detector input,
    and a detector plan rebound to a larger table, take the second path)."""
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    sc = synth.SCANNER_CLINICAL
    xs, xe, tb, ds, de = synth.lm_events(torch.from_numpy(clinical_img), g, sc, tof, 80_003, seed=4611,
                                         return_det=True)
    table = sc.crystal_table("cuda")
    # the table followed by 100 unused entries: more detectors than a plan
    # created with `table` holds in its padded copy
    big = torch.cat([table, torch.zeros((100, 3), device="cuda")]).contiguous()
    img = cuda(clinical_img)
    ds_c, de_c, tb_c = ds.cuda(), de.cuda(), tb.cuda()
    ref_plan = ops.jp_plan_create(xs.cuda(), xe.cuda(), g, tof_bin=tb_c, tof_bin_width=tof.bin_width)
    ref = ops.jp_fwd_tof_lm(ref_plan, img, tof)
    padded = ops.jp_plan_create_batch_det(ds_c, de_c, table, g, [0, len(xs)], tof_bin=tb_c,
                                          tof_bin_width=tof.bin_width)
    assert torch.equal(ops.jp_fwd_tof_lm(padded, img, tof), ref)
    ops.jp_plan_rebind_det(padded, ds_c, de_c, big, tof_bin=tb_c)  # n_det above the copy: the caller's table
    assert torch.equal(ops.jp_fwd_tof_lm(padded, img, tof), ref)
    ops.jp_plan_rebind_det(padded, ds_c, de_c, table, tof_bin=tb_c)  # back to the copy
    assert torch.equal(ops.jp_fwd_tof_lm(padded, img, tof), ref)
    ops.jp_plan_rebind_det(ref_plan, ds_c, de_c, table, tof_bin=tb_c)  # coordinate plan: no copy
    assert torch.equal(ops.jp_fwd_tof_lm(ref_plan, img, tof), ref)
    padded.destroy()
    ref_plan.destroy()
    # non-TOF plans (no TOF bins) from detector indices, both table paths
    ref_plan = ops.jp_plan_create(xs.cuda(), xe.cuda(), g)
    ref = ops.jp_fwd(ref_plan, img)
    padded = ops.jp_plan_create_batch_det(ds_c, de_c, table, g, [0, len(xs)])
    assert torch.equal(ops.jp_fwd(padded, img), ref)
    ops.jp_plan_rebind_det(padded, ds_c, de_c, big)
    assert torch.equal(ops.jp_fwd(padded, img), ref)
    padded.destroy()
    ref_plan.destroy()
