"""Tabulated (non-Gaussian) TOF kernels and per-event TOF sigma (paper
Sec. 4: a 1D lookup table permits non-Gaussian kernels; listmode events
with their own TOF resolution) against the FP64 oracle: planned (shared-
memory table / exact per-event erf) and planless paths, TOF sinogram and
listmode, forward element by element and back projection."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_12519_gb300 import synth
from _parity import AMB_EPS, BACK_TOL, FWD_TOL, fwd_err, rel_l2

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


GEOM = synth.ImageGeom((37, 29, 23), (-40.0, -25.0, -20.5), (2.1, 1.7, 1.9))


def lors(n=30_000, seed=7401):
    xs1, xe1 = synth.random_lors(n, GEOM, seed=seed)
    xs2, xe2 = synth.random_lors(n // 5, GEOM, seed=seed + 1, kind="inside")
    return np.concatenate([xs1, xs2]), np.concatenate([xe1, xe2])


def skewed_table(nodes, hw):
    """A smooth asymmetric bin response with non-zero values at both ends."""
    d = np.linspace(-hw, hw, nodes)
    return np.exp(-0.5 * ((d - 0.25 * hw) / (0.35 * hw)) ** 2) * (1.0 + 0.4 * d / hw) + 0.01


@pytest.mark.parametrize("mode", ["tof_sino", "tof_lm"])
@pytest.mark.parametrize("path", ["planned", "planned_exact_flag", "planless"])
def test_tabulated_kernel_vs_oracle(ops, mode, path):
    xs, xe = lors()
    n = len(xs)
    rng = np.random.Generator(np.random.PCG64(7402))
    img = rng.uniform(0, 3, size=GEOM.shape).astype(np.float32)
    hw = 22.0
    tof = synth.TofParams.tabulated(9.0, 13, skewed_table(257, hw).tolist(), hw)
    tb = rng.integers(-6, 7, size=n).astype(np.int16) if mode == "tof_lm" else None
    delta = rng.normal(0, 3, size=n).astype(np.float32)
    p_or, amb = oracle.fwd(xs, xe, img, GEOM, mode, tof, tof_bin=tb, delta=delta, threads=THREADS,
                           amb_eps=AMB_EPS, return_amb=True)
    nout = tof.n_bins if mode == "tof_sino" else 1
    y = rng.uniform(0, 1, size=(n, nout) if nout > 1 else n).astype(np.float32)
    b_or = oracle.back(xs, xe, y, GEOM, mode, tof, tof_bin=tb, delta=delta, threads=THREADS)
    out = torch.zeros(GEOM.shape, device="cuda")
    dtb = None if tb is None else cuda(tb)
    if path == "planless":
        p = ops.jp_fwd_lors(cuda(xs), cuda(xe), cuda(img), GEOM, mode, tof, tof_bin=dtb, delta=cuda(delta))
        ops.jp_back_lors(cuda(xs), cuda(xe), cuda(y), GEOM, out, mode, tof, tof_bin=dtb, delta=cuda(delta))
    else:
        plan = ops.jp_plan_create(cuda(xs), cuda(xe), GEOM, tof_bin=dtb, delta=cuda(delta),
                                  tof_bin_width=tof.bin_width, tof_exact=(path == "planned_exact_flag"))
        if mode == "tof_sino":
            p = ops.jp_fwd_tof_sino(plan, cuda(img), tof)
            ops.jp_back_tof_sino(plan, cuda(y), tof, out)
        else:
            p = ops.jp_fwd_tof_lm(plan, cuda(img), tof)
            ops.jp_back_tof_lm(plan, cuda(y), tof, out)
    torch.cuda.synchronize()
    assert fwd_err(p.cpu().numpy(), p_or, amb) <= FWD_TOL
    assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL


def test_tabulated_triangle_partition_of_unity(ops):
    """A triangle of half-width one bin sums to 1 over the bins: the TOF
    sinogram summed over its bins equals the non-TOF projection."""
    xs, xe = lors(8_000, seed=7410)
    rng = np.random.Generator(np.random.PCG64(7411))
    img = cuda(rng.uniform(0, 2, size=GEOM.shape).astype(np.float32))
    tri = synth.TofParams.tabulated(6.0, 41, (0.0, 1.0, 0.0), 6.0)
    plan = ops.jp_plan_create(cuda(xs), cuda(xe), GEOM)
    p_tof = ops.jp_fwd_tof_sino(plan, img, tri).double().sum(dim=1)
    p_non = ops.jp_fwd(plan, img).double()
    assert float((p_tof - p_non).abs().max()) <= 1e-5 * float(p_non.abs().max())


@pytest.mark.parametrize("lpw", [0, 1, 4, 32])
def test_per_event_sigma_vs_oracle(ops, lpw):
    xs, xe = lors(25_000, seed=7420)
    n = len(xs)
    rng = np.random.Generator(np.random.PCG64(7421))
    img = rng.uniform(0, 3, size=GEOM.shape).astype(np.float32)
    tof = synth.TofParams(bin_width=9.0, sigma=7.0, n_sigmas=3.0, n_bins=15)
    tb = rng.integers(-6, 7, size=n).astype(np.int16)
    sig = (7.0 * rng.uniform(0.6, 1.6, size=n)).astype(np.float32)
    sig[::97] = 0.0  # <= 0 keeps the plan's sigma
    sig_or = np.where(sig > 0, sig, tof.sigma).astype(np.float64)
    p_or, amb = oracle.fwd(xs, xe, img, GEOM, "tof_lm", tof, tof_bin=tb, sigma=sig_or, threads=THREADS,
                           amb_eps=AMB_EPS, return_amb=True)
    y = rng.uniform(0, 1, size=n).astype(np.float32)
    b_or = oracle.back(xs, xe, y, GEOM, "tof_lm", tof, tof_bin=tb, sigma=sig_or, threads=THREADS)
    plan = ops.jp_plan_create(cuda(xs), cuda(xe), GEOM, tof_bin=cuda(tb), tof_bin_width=tof.bin_width,
                              lors_per_warp=lpw)
    ops.jp_plan_set_event_sigma(plan, cuda(sig))
    p = ops.jp_fwd_tof_lm(plan, cuda(img), tof)
    out = torch.zeros(GEOM.shape, device="cuda")
    ops.jp_back_tof_lm(plan, cuda(y), tof, out)
    torch.cuda.synchronize()
    assert fwd_err(p.cpu().numpy(), p_or, amb) <= FWD_TOL
    assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL
    # the exact sample count follows each event's own window
    cnt = ops.jp_count_samples(plan, "tof_lm", tof)
    ops.jp_plan_set_event_sigma(plan, None)
    assert ops.jp_count_samples(plan, "tof_lm", tof) != cnt
    # rebinding clears the per-event sigma: the scalar-sigma result comes back
    ops.jp_plan_set_event_sigma(plan, cuda(sig))
    ops.jp_plan_rebind(plan, cuda(xs), cuda(xe), tof_bin=cuda(tb))
    p_scalar = ops.jp_fwd_tof_lm(plan, cuda(img), tof).cpu().numpy()
    p_or0, amb0 = oracle.fwd(xs, xe, img, GEOM, "tof_lm", tof, tof_bin=tb, threads=THREADS, amb_eps=AMB_EPS,
                             return_amb=True)
    assert fwd_err(p_scalar, p_or0, amb0) <= FWD_TOL
    # per-event sigma is a listmode property
    ops.jp_plan_set_event_sigma(plan, cuda(sig))
    with pytest.raises(ops.JosephError):
        ops.jp_fwd_tof_sino(plan, cuda(img), tof)
    plan.destroy()


@pytest.mark.parametrize("path", ["quads", "direct"])
def test_osem_per_event_sigma_vs_oracle(ops, path):
    from paper_2212_12519_gb300 import osem
    g = synth.ImageGeom.centred((64, 64, 24), (3.0, 3.0, 3.0))
    tof = synth.TOF_CLINICAL
    ph = synth.ellipsoid_phantom(g, synth.PhantomSpec((80.0, 60.0, 30.0), (6.0, 9.0)), 7430)
    xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, 40_001, seed=7431)
    rng = np.random.Generator(np.random.PCG64(7432))
    sig = (tof.sigma * rng.choice([0.8, 1.0, 1.3], size=len(xs))).astype(np.float32)
    s = rng.uniform(0.5, 1.5, size=g.shape)
    b = synth.background_level(ph, tof)
    x_or = oracle.lm_osem(xs.numpy(), xe.numpy(), tb.numpy(), g, tof, s, b, n_iter=1, n_sub=4, threads=THREADS,
                          sigma=sig.astype(np.float64))
    spec = osem.FrameSpec(xs.cuda(), xe.cuda(), tb.cuda(), g, b, n_iter=1, n_sub=4, path=path,
                          sigma=cuda(sig))
    x = osem.LMOSEMFrame(spec, cuda(s.astype(np.float32)), tof).run()
    torch.cuda.synchronize()
    assert rel_l2(x.cpu().numpy(), x_or) <= 1e-4


@pytest.mark.parametrize("bin_width,sigma,n_bins", [(9.0, 7.0, 15), (10.0, 9.9667, 9), (4.0, 7.0, 25),
                                                     (9.0, 7.0, 3), (9.0, 7.0, 1), (30.0, 2.0, 7),
                                                     (1.0, 1.0, 128)])
def test_tof_sino_bin_windows(ops, bin_width, sigma, n_bins):
    """Gaussian TOF sinograms whose plane samples reach 1 to 12 bins (2 R / w
    from 1.4 to 11.5, the bin-aligned table), with TOF centre offsets and
    LORs in both directions; few bins (the window clipped at both ends), a
    single bin, and the most bins a sinogram may have (JP_MAX_TOF_BINS, whose
    per-thread accumulators cap the forward's block size)."""
    xs, xe = lors(20_000, seed=7460)
    n = len(xs)
    rng = np.random.Generator(np.random.PCG64(7461))
    img = rng.uniform(0, 3, size=GEOM.shape).astype(np.float32)
    tof = synth.TofParams(bin_width=bin_width, sigma=sigma, n_sigmas=3.0, n_bins=n_bins)
    delta = rng.normal(0, 3, size=n).astype(np.float32)
    p_or, amb = oracle.fwd(xs, xe, img, GEOM, "tof_sino", tof, delta=delta, threads=THREADS, amb_eps=AMB_EPS,
                           return_amb=True)
    y = rng.uniform(0, 1, size=(n, n_bins)).astype(np.float32)
    b_or = oracle.back(xs, xe, y, GEOM, "tof_sino", tof, delta=delta, threads=THREADS)
    plan = ops.jp_plan_create(cuda(xs), cuda(xe), GEOM, delta=cuda(delta))
    p = ops.jp_fwd_tof_sino(plan, cuda(img), tof)
    out = torch.zeros(GEOM.shape, device="cuda")
    ops.jp_back_tof_sino(plan, cuda(y), tof, out)
    torch.cuda.synchronize()
    assert fwd_err(p.cpu().numpy(), p_or, amb) <= FWD_TOL
    assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL
    plan.destroy()


@pytest.mark.parametrize("table", ["box2", "max_nodes"])
def test_tabulated_kernel_extremes(ops, table):
    """The smallest table (2 nodes: a box, value 1 up to the support edge)
    and the largest (JP_TOF_TABLE nodes), listmode and sinogram."""
    xs, xe = lors(6_000, seed=7440)
    n = len(xs)
    rng = np.random.Generator(np.random.PCG64(7441))
    img = rng.uniform(0, 3, size=GEOM.shape).astype(np.float32)
    if table == "box2":
        tof = synth.TofParams.tabulated(9.0, 13, (1.0, 1.0), 4.5)
    else:
        tof = synth.TofParams.tabulated(9.0, 13, skewed_table(2048, 20.0).tolist(), 20.0)
    tb = rng.integers(-6, 7, size=n).astype(np.int16)
    for mode in ("tof_lm", "tof_sino"):
        kw = dict(tof_bin=tb) if mode == "tof_lm" else {}
        p_or, amb = oracle.fwd(xs, xe, img, GEOM, mode, tof, threads=THREADS, amb_eps=AMB_EPS,
                               return_amb=True, **kw)
        plan = ops.jp_plan_create(cuda(xs), cuda(xe), GEOM, tof_bin=cuda(tb), tof_bin_width=tof.bin_width)
        p = (ops.jp_fwd_tof_lm(plan, cuda(img), tof) if mode == "tof_lm"
             else ops.jp_fwd_tof_sino(plan, cuda(img), tof))
        torch.cuda.synchronize()
        assert fwd_err(p.cpu().numpy(), p_or, amb) <= FWD_TOL, mode
        plan.destroy()


def test_tabulated_kernel_argument_checks(ops):
    xs, xe = lors(100, seed=7450)
    plan = ops.jp_plan_create(cuda(xs), cuda(xe), GEOM)
    img = torch.zeros(GEOM.shape, device="cuda")
    bad = [synth.TofParams.tabulated(9.0, 13, [1.0] * 4, 0.0),          # half width 0
           synth.TofParams.tabulated(9.0, 13, [1.0] * 2049, 10.0),      # more nodes than the table holds
           synth.TofParams(bin_width=1.0, sigma=1.0, n_sigmas=3.0, n_bins=129)]  # above JP_MAX_TOF_BINS
    for tof in bad:
        with pytest.raises(ops.JosephError):
            ops.jp_fwd_tof_sino(plan, img, tof)
    plan.destroy()
