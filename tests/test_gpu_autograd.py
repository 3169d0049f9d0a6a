"""torch.autograd.Function whose backward is the hand-written adjoint: the
gradient of sum(w log(Ax + b)) on a 16x16x8 crop with 20k events against the
FP64 oracle gradient (which is itself pinned against FP64 finite
differences in test_oracle_pins)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_12519_gb300 import synth
from _parity import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    from paper_2212_12519_gb300 import build, ops as _ops
    build.build()
    _ops.load()
    return _ops


def crop_problem(seed=4201, n=20_000):
    g = synth.ImageGeom.centred((16, 16, 8), (2.0, 2.0, 2.0))
    ph = synth.ellipsoid_phantom(g, synth.PhantomSpec((12.0, 10.0, 6.0), (3.0,)), seed)
    xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, synth.TOF_CLINICAL, n, seed=seed + 1)
    w = synth.loss_weights(n, seed + 2)
    return g, ph, xs, xe, tb, w


def test_gradient_vs_oracle(ops):
    from paper_2212_12519_gb300.autograd import JosephTOFLM
    g, ph, xs, xe, tb, w = crop_problem()
    tof = synth.TOF_CLINICAL
    b = 0.3
    x = (ph + 0.1).cuda().requires_grad_(True)
    plan = ops.jp_plan_create(xs.cuda(), xe.cuda(), g, tof_bin=tb.cuda(), tof_bin_width=tof.bin_width)
    p = JosephTOFLM.apply(x, plan, tof)
    loss = (w.cuda() * torch.log(p + b)).sum()
    loss.backward()
    f_or, g_or = oracle.poisson_loglik_grad((ph + 0.1).numpy(), xs.numpy(), xe.numpy(), tb.numpy(), g, tof,
                                            w.numpy(), b)
    assert float(loss) == pytest.approx(f_or, rel=1e-5)
    assert rel_l2(x.grad.cpu().numpy(), g_or) <= 1e-4


def test_batched_frames_autograd(ops):
    """A batch of images [B, n0, n1, n2], one plan holding every frame's
    events: the gradient of each image equals its own frame's gradient."""
    from paper_2212_12519_gb300.autograd import JosephTOFLM
    tof = synth.TOF_CLINICAL
    probs = [crop_problem(seed=4300 + 10 * k, n=5000 + 1000 * k) for k in range(3)]
    g = probs[0][0]
    xs = torch.cat([p[2] for p in probs]).cuda()
    xe = torch.cat([p[3] for p in probs]).cuda()
    tb = torch.cat([p[4] for p in probs]).cuda()
    w = torch.cat([p[5] for p in probs]).cuda()
    off = np.cumsum([0] + [p[2].shape[0] for p in probs]).tolist()
    plan = ops.jp_plan_create_batch(xs, xe, g, off, tof_bin=tb, tof_bin_width=tof.bin_width)
    x = torch.stack([p[1] + 0.1 for p in probs]).cuda().requires_grad_(True)
    p = JosephTOFLM.apply(x, plan, tof)
    loss = (w * torch.log(p + 0.3)).sum()
    loss.backward()
    for k, pr in enumerate(probs):
        _, g_or = oracle.poisson_loglik_grad((pr[1] + 0.1).numpy(), pr[2].numpy(), pr[3].numpy(), pr[4].numpy(),
                                             g, tof, pr[5].numpy(), 0.3)
        assert rel_l2(x.grad[k].cpu().numpy(), g_or) <= 1e-4


def test_torch_gradcheck_double_adjoint(ops):
    """<A x, y> = <x, A^T y> through the autograd path (the VJP of the
    forward is the adjoint) at full FP32 precision."""
    from paper_2212_12519_gb300.autograd import JosephTOFLM
    g, ph, xs, xe, tb, w = crop_problem(seed=4400, n=8000)
    tof = synth.TOF_CLINICAL
    plan = ops.jp_plan_create(xs.cuda(), xe.cuda(), g, tof_bin=tb.cuda(), tof_bin_width=tof.bin_width)
    x = torch.rand(g.shape, device="cuda", requires_grad=True)
    y = torch.rand(xs.shape[0], device="cuda")
    p = JosephTOFLM.apply(x, plan, tof)
    (gx,) = torch.autograd.grad((p * y).sum(), x)
    lhs = float((p.double() * y.double()).sum())
    rhs = float((x.detach().double() * gx.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_fused_poisson_loglik_vs_oracle(ops):
    """The fused log-likelihood Function (value and gradient kernels) with
    the projector: value and image gradient against the FP64 oracle, per
    frame backgrounds from the plan's frames."""
    from paper_2212_12519_gb300.autograd import JosephTOFLM, PoissonLogLik
    tof = synth.TOF_CLINICAL
    probs = [crop_problem(seed=4500 + 10 * k, n=6000 + 500 * k) for k in range(2)]
    g = probs[0][0]
    xs = torch.cat([p[2] for p in probs]).cuda()
    xe = torch.cat([p[3] for p in probs]).cuda()
    tb = torch.cat([p[4] for p in probs]).cuda()
    w = torch.cat([p[5] for p in probs]).cuda()
    off = np.cumsum([0] + [p[2].shape[0] for p in probs]).tolist()
    bvals = [0.3, 0.7]
    plan = ops.jp_plan_create_batch(xs, xe, g, off, tof_bin=tb, tof_bin_width=tof.bin_width)
    x = torch.stack([p[1] + 0.1 for p in probs]).cuda().requires_grad_(True)
    loss = PoissonLogLik.apply(JosephTOFLM.apply(x, plan, tof), plan, w,
                               torch.tensor(bvals, dtype=torch.float32, device="cuda"))
    loss.backward()
    tot = 0.0
    for k, pr in enumerate(probs):
        f_or, g_or = oracle.poisson_loglik_grad((pr[1] + 0.1).numpy(), pr[2].numpy(), pr[3].numpy(), pr[4].numpy(),
                                                g, tof, pr[5].numpy(), bvals[k])
        tot += f_or
        assert rel_l2(x.grad[k].cpu().numpy(), g_or) <= 1e-4
    assert float(loss) == pytest.approx(tot, rel=1e-5)
