"""GPU image-based resolution model (separable 3D Gaussian, paper Sec. 2.6)
against the FP64 oracle's direct 3D correlation, and listmode OSEM with the
resolution model against the oracle OSEM.

Tolerance: each output voxel is a sum of at most (2R+1)^3 positive terms
accumulated in FP32 over three passes (relative rounding ~1e-6); the test
allows max|err| <= 1e-5 max|oracle|, the forward-projection bound."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_12519_gb300 import synth
from _parity import FWD_TOL, rel_l2

pytestmark = pytest.mark.gpu

OSEM_TOL = 1e-4


@pytest.fixture(scope="module")
def ops():
    from paper_2212_12519_gb300 import build, ops as _ops
    build.build()
    _ops.load()
    return _ops


def max_err(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-30))


CASES = [
    # geometry, FWHM (mm, per axis or isotropic)
    (synth.ImageGeom((37, 29, 23), (-40.0, -25.0, -20.5), (2.1, 1.7, 1.9)), (4.5, 3.0, 6.0)),
    (synth.GEOM_SMALL, 4.5),
    (synth.ImageGeom.centred((96, 96, 40), (2.0, 2.0, 2.0)), 4.5),
    # axes shorter than the kernel radius, an axis of one voxel
    (synth.ImageGeom.centred((3, 40, 1), (2.0, 2.0, 2.0)), (10.0, 4.5, 4.5)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_gauss3d_vs_oracle(ops, case):
    g, fwhm = CASES[case]
    rng = np.random.Generator(np.random.PCG64(7300 + case))
    x = rng.uniform(0.0, 1.0, size=g.shape).astype(np.float32)
    ref = oracle.gauss3d(x, g, fwhm)
    out = ops.jp_gauss3d(torch.from_numpy(x).cuda(), g, fwhm)
    torch.cuda.synchronize()
    assert max_err(out.cpu().numpy(), ref) <= FWD_TOL


def test_gauss3d_stack_identity_and_adjoint(ops):
    from paper_2212_12519_gb300.autograd import GaussianResolution
    g = synth.ImageGeom((21, 18, 13), (-20.0, -17.0, -12.0), (2.0, 2.0, 2.0))
    rng = np.random.Generator(np.random.PCG64(7310))
    xs = rng.uniform(0.0, 1.0, size=(3,) + g.shape).astype(np.float32)
    out = ops.jp_gauss3d(torch.from_numpy(xs).cuda(), g, 4.5).cpu().numpy()
    for i in range(3):
        assert max_err(out[i], oracle.gauss3d(xs[i], g, 4.5)) <= FWD_TOL
    # FWHM 0: every pass is a single tap 1, the image comes back bit for bit
    x0 = torch.from_numpy(xs[0]).cuda()
    assert torch.equal(ops.jp_gauss3d(x0, g, 0.0), x0)
    # no images: no-op
    e = torch.empty((0,) + g.shape, device="cuda")
    assert ops.jp_gauss3d(e, g, 4.5).shape == e.shape
    # autograd: the gradient of <H x, y> is H^T y = H y
    x = torch.from_numpy(xs[1]).cuda().requires_grad_(True)
    y = torch.from_numpy(xs[2]).cuda()
    (GaussianResolution.apply(x, g, 4.5) * y).sum().backward()
    assert max_err(x.grad.cpu().numpy(), oracle.gauss3d(xs[2], g, 4.5, adjoint=True)) <= FWD_TOL
    lhs = float((ops.jp_gauss3d(x.detach(), g, 4.5).double() * y.double()).sum())
    rhs = float((x.detach().double() * ops.jp_gauss3d(y, g, 4.5).double()).sum())
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def res_frame():
    g = synth.ImageGeom.centred((72, 72, 30), (3.0, 3.0, 3.0))
    ph = synth.ellipsoid_phantom(g, synth.PhantomSpec((90.0, 70.0, 40.0), (6.0, 9.0, 12.0)), 7320)
    xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, synth.TOF_CLINICAL, 60_001, seed=7321)
    rng = np.random.Generator(np.random.PCG64(7322))
    s = rng.uniform(0.5, 1.5, size=g.shape)
    s[:, :, :5] = 0.0  # beyond the kernel radius (3 voxels): s' = H^T s is 0 on planes 0 and 1
    return g, ph, xs, xe, tb, s.astype(np.float32), synth.background_level(ph, synth.TOF_CLINICAL)


@pytest.mark.parametrize("path", ["fused", "graph", "plain", "direct", "direct_graph"])
def test_osem_with_resolution_model_vs_oracle(ops, path):
    from paper_2212_12519_gb300 import osem
    g, ph, xs, xe, tb, s, b = res_frame()
    tof = synth.TOF_CLINICAL
    n_iter, n_sub, fwhm = 2, 4, 4.5
    s_eff = oracle.gauss3d(s, g, fwhm, adjoint=True).astype(np.float32)
    x_or = oracle.lm_osem(xs.numpy(), xe.numpy(), tb.numpy(), g, tof, s_eff, b, n_iter=n_iter, n_sub=n_sub,
                          threads=8, fwhm_mm=fwhm)
    # the library's own s' = H^T s agrees with the oracle's
    sens_gpu = osem.resolution_sensitivity(torch.from_numpy(s).cuda(), g, fwhm)
    assert max_err(sens_gpu.cpu().numpy(), s_eff) <= FWD_TOL
    spec = osem.FrameSpec(xs.cuda(), xe.cuda(), tb.cuda(), g, b, n_iter=n_iter, n_sub=n_sub, fwhm_mm=fwhm,
                          path="direct" if path.startswith("direct") else "quads")
    sens = torch.from_numpy(s_eff).cuda()
    if path == "plain":
        x = osem.reconstruct_plain(spec, sens, tof)
    else:
        fr = osem.LMOSEMFrame(spec, sens, tof)
        x = fr.run_graph() if path.endswith("graph") else fr.run()
    torch.cuda.synchronize()
    assert rel_l2(x.cpu().numpy(), x_or) <= OSEM_TOL
    # voxels without sensitivity stay 0
    assert np.all(s_eff[:, :, :2] == 0.0) and np.all(s_eff[:, :, 2] > 0.0)
    assert float(x[:, :, :2].abs().sum()) == 0.0


def test_slot_graph_with_resolution_model(ops):
    """Per-slot graphs captured once with the resolution model serve two
    different frames after rebinding; each equals its own direct run, on
    both subset-update paths."""
    from paper_2212_12519_gb300 import osem, serve
    g, ph, xs, xe, tb, s, b = res_frame()
    tof = synth.TOF_CLINICAL
    sens = osem.resolution_sensitivity(torch.from_numpy(s).cuda(), g, 4.5)
    srv = serve.OSEMServer({g.shape: sens}, tof, mode="batched", max_slots=1, use_graphs=True)
    srv.reserve(60_001, [g], n_sub=4, fwhm_mm=4.5)
    for lo, hi, bb in ((0, 60_001, b), (7, 41_000, 2.0 * b)):
        spec = osem.FrameSpec(xs[lo:hi].cuda(), xe[lo:hi].cuda(), tb[lo:hi].cuda(), g, bb, n_iter=2, n_sub=4,
                              fwhm_mm=4.5)
        x_graph = srv.slot_graphs[(0, g.shape)].run(spec)
        x_direct = osem.LMOSEMFrame(spec, sens, tof).run()
        spec.path = "quads"
        x_graph_q = srv.slot_graphs[(0, g.shape)].run(spec)
        torch.cuda.synchronize()
        assert rel_l2(x_graph.cpu().numpy(), x_direct.cpu().numpy()) <= 1e-5
        assert rel_l2(x_graph_q.cpu().numpy(), x_direct.cpu().numpy()) <= 1e-5
    srv.close()


def test_gauss3d_many_planes_and_large_radius(ops):
    """More image planes than one grid dimension holds (65535) and radii
    above the unrolled kernels' 8: the generic pass and the grid loops."""
    g = synth.ImageGeom((700, 3, 5), (0.0, 0.0, 0.0), (2.0, 2.0, 2.0))
    rng = np.random.Generator(np.random.PCG64(7340))
    xs = rng.uniform(0.0, 1.0, size=(100,) + g.shape).astype(np.float32)
    for fwhm in (4.5, (30.0, 4.5, 4.5)):  # R = 4 on every axis; R = 26 on axis 0 (generic pass)
        out = ops.jp_gauss3d(torch.from_numpy(xs).cuda(), g, fwhm).cpu().numpy()
        for i in (0, 57, 99):
            assert max_err(out[i], oracle.gauss3d(xs[i], g, fwhm)) <= FWD_TOL


@pytest.mark.parametrize("path", ["quads", "direct"])
def test_osem_empty_subsets(ops, path):
    """A frame with fewer events than subsets: the empty subsets back-project
    nothing, so the update zeroes the image, as the oracle's does."""
    from paper_2212_12519_gb300 import osem
    g, ph, xs, xe, tb, s, b = res_frame()
    tof = synth.TOF_CLINICAL
    n = 5
    x_or = oracle.lm_osem(xs[:n].numpy(), xe[:n].numpy(), tb[:n].numpy(), g, tof, s, b, n_iter=1, n_sub=8)
    spec = osem.FrameSpec(xs[:n].cuda(), xe[:n].cuda(), tb[:n].cuda(), g, b, n_iter=1, n_sub=8, path=path)
    x = osem.LMOSEMFrame(spec, torch.from_numpy(s).cuda(), tof).run()
    torch.cuda.synchronize()
    assert np.all(np.isfinite(x.cpu().numpy()))
    assert np.abs(x.cpu().numpy() - x_or).max() <= 1e-6 * max(1.0, np.abs(x_or).max())
