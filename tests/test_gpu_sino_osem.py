"""GPU sinogram OSEM (34-style view subsets, emission + contamination
sinograms; paper Sec. 2.6 and 4) against the FP64 oracle update, and the
layout independence of the binned projector (sinogram orders PVR / VRP /
RVP, image symmetry axis 0 / 1 / 2; paper Sec. 2.6)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_12519_gb300 import synth
from _parity import FWD_TOL, fwd_err, rel_l2

pytestmark = pytest.mark.gpu

OSEM_TOL = 1e-4
N_SUB = 8


@pytest.fixture(scope="module")
def ops():
    from paper_2212_12519_gb300 import build, ops as _ops
    build.build()
    _ops.load()
    return _ops


def subset_data(spec, nb, seed):
    """Per-subset emission counts and contamination drawn on the host
    (the update is defined for any y >= 0, c >= 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ys, cs, lors = [], [], []
    for m in range(N_SUB):
        xs, xe = synth.sinogram_lors(spec.subset(m, N_SUB))
        shape = (xs.shape[0], nb) if nb > 1 else (xs.shape[0],)
        ys.append(rng.poisson(2.0, size=shape).astype(np.float32))
        cs.append(np.full(shape, 0.4, dtype=np.float32))
        lors.append((xs.numpy(), xe.numpy()))
    return ys, cs, lors


@pytest.mark.parametrize("mode,fwhm", [("nontof", 0.0), ("tof_sino", 0.0), ("nontof", 4.5)])
def test_sino_osem_vs_oracle(ops, mode, fwhm):
    from paper_2212_12519_gb300 import sino_osem
    g, spec = synth.GEOM_SMALL, synth.SINO_SMALL
    tof = synth.TOF_CLINICAL if mode == "tof_sino" else None
    nb = tof.n_bins if tof else 1
    ys, cs, lors = subset_data(spec, nb, 8100 + nb)
    so = sino_osem.SinoOSEM(spec, g, n_sub=N_SUB, tof=tof, fwhm_mm=fwhm)
    so.set_data([torch.from_numpy(y).cuda() for y in ys], [torch.from_numpy(c).cuda() for c in cs])
    # oracle: per-subset sensitivity (through H^T with the resolution model)
    sens = []
    for xs, xe in lors:
        ones = np.ones((len(xs), nb) if nb > 1 else len(xs))
        s = oracle.back(xs, xe, ones, g, mode, tof, threads=8)
        sens.append(oracle.gauss3d(s, g, fwhm, adjoint=True) if fwhm > 0 else s)
        assert rel_l2(so.sens[len(sens) - 1].cpu().numpy(), sens[-1]) <= 1e-4
    x_or = (sum(sens) > 0).astype(np.float64)
    for m, (xs, xe) in enumerate(lors):
        if fwhm > 0:
            # x <- x / s' * H^T A^T (y / (A H x + c)): the oracle update on H x,
            # then H^T on the back projection
            hx = oracle.gauss3d(x_or, g, fwhm)
            p = oracle.fwd(xs, xe, hx, g, mode, tof, threads=8)
            den = p + cs[m]
            q = np.where(den > 0, ys[m] / np.where(den > 0, den, 1.0), 0.0)
            bp = oracle.gauss3d(oracle.back(xs, xe, q, g, mode, tof, threads=8), g, fwhm, adjoint=True)
            x_or = np.where(sens[m] > 0, x_or * bp / np.where(sens[m] > 0, sens[m], 1.0), 0.0)
        else:
            x_or = oracle.sino_osem_subset_update(x_or, xs, xe, ys[m], cs[m], sens[m], g, mode, tof, threads=8)
    x = so.run(1)
    torch.cuda.synchronize()
    assert rel_l2(x.cpu().numpy(), x_or) <= OSEM_TOL
    so.close()


def test_ratio_sino_edge_cases(ops):
    p = torch.tensor([1.0, 0.0, 2.0, 0.0, 3.0, -1.0, 0.5], device="cuda")
    y = torch.tensor([2.0, 5.0, 0.0, 0.0, 6.0, 1.0, 1.0], device="cuda")
    c = torch.tensor([1.0, 0.0, 0.5, 0.0, 0.0, 0.5, 0.0], device="cuda")
    q = ops.jp_osem_ratio_sino(p, y, c).cpu().numpy()
    assert np.array_equal(q, np.array([1.0, 0.0, 0.0, 0.0, 2.0, 0.0, 2.0], dtype=np.float32))
    # no contamination, in place, unaligned tail through the scalar path
    p2 = torch.arange(1, 12, dtype=torch.float32, device="cuda")
    y2 = torch.full_like(p2, 3.0)
    out = ops.jp_osem_ratio_sino(p2[1:], y2[1:], None, out=p2[1:])
    assert torch.allclose(out, 3.0 / torch.arange(2, 12, dtype=torch.float32, device="cuda"))


@pytest.mark.parametrize("order", ["VRP", "RVP"])
def test_projection_independent_of_sinogram_order(ops, order):
    """The same subset in another memory order gives the same projections
    (permuted) and the same back projection."""
    g, spec = synth.GEOM_SMALL, synth.SINO_SMALL.subset(3, 8)
    img = synth.ellipsoid_phantom(g, synth.PHANTOM_SMALL, 8201).cuda()
    P, V, R = spec.n_planes, len(spec.views), spec.n_rad
    xs0, xe0 = synth.sinogram_lors(spec, device="cuda")
    xs1, xe1 = synth.sinogram_lors(spec, device="cuda", order=order)
    perm = {"VRP": (1, 2, 0), "RVP": (2, 1, 0)}[order]
    assert torch.equal(xs0.view(P, V, R, 3).permute(*perm, 3).reshape(-1, 3), xs1)
    p0 = ops.jp_fwd(ops.jp_plan_create(xs0, xe0, g), img).view(P, V, R).permute(*perm).reshape(-1)
    p1 = ops.jp_fwd(ops.jp_plan_create(xs1, xe1, g), img)
    assert torch.equal(p0, p1)  # per-LOR arithmetic does not depend on the order
    y = torch.rand(P * V * R, device="cuda")
    b0 = ops.jp_back(ops.jp_plan_create(xs0, xe0, g), y, torch.zeros(g.shape, device="cuda"))
    y1 = y.view(P, V, R).permute(*perm).reshape(-1).contiguous()
    b1 = ops.jp_back(ops.jp_plan_create(xs1, xe1, g), y1, torch.zeros(g.shape, device="cuda"))
    assert rel_l2(b1.cpu().numpy(), b0.cpu().numpy().astype(np.float64)) <= 1e-6


@pytest.mark.parametrize("axis", [0, 1])
def test_projection_independent_of_symmetry_axis(ops, axis):
    """Placing the scanner axis on image axis 0 or 1 permutes voxels only:
    forward projections agree with the oracle, back projections with the
    permuted axis-2 result."""
    g, spec = synth.GEOM_SMALL, synth.SINO_SMALL.subset(1, 8)
    img = synth.ellipsoid_phantom(g, synth.PHANTOM_SMALL, 8301)
    xs, xe = synth.sinogram_lors(spec)
    g2, xs2, xe2 = synth.symmetry_axis(g, xs, xe, axis)
    order = {0: (2, 0, 1), 1: (0, 2, 1)}[axis]
    img2 = img.permute(*order).contiguous()
    plan = ops.jp_plan_create(xs2.cuda(), xe2.cuda(), g2)
    p = ops.jp_fwd(plan, img2.cuda()).cpu().numpy()
    sel = np.arange(0, len(xs), 37)
    p_or = oracle.fwd(xs.numpy()[sel], xe.numpy()[sel], img.numpy(), g, threads=8)
    assert fwd_err(p[sel], p_or) <= FWD_TOL
    y = torch.rand(len(xs), device="cuda")
    b2 = ops.jp_back(plan, y, torch.zeros(g2.shape, device="cuda"))
    b = ops.jp_back(ops.jp_plan_create(xs.cuda(), xe.cuda(), g), y, torch.zeros(g.shape, device="cuda"))
    assert rel_l2(b2.cpu().numpy(), b.permute(*order).cpu().numpy().astype(np.float64)) <= 1e-5
