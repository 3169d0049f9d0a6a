"""The measurement counters (plane samples, L2 reduction requests of the
quad-image back projection) on inputs whose counts follow from the
geometry alone."""
import numpy as np
import pytest
import torch

from paper_2212_12519_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    from paper_2212_12519_gb300 import build, ops as _ops
    build.build()
    _ops.load()
    return _ops


def test_red_requests_axis_aligned_pairs(ops):
    """LORs along axis 0 through voxel centres cross all 16 planes at one
    (i, j): the lanes of a group start on plane 0, planes 2m and 2m+1 share
    a 32-byte sector of the plane-fastest quads, and LORs at distinct
    (i, j) never share one, so requests = samples / 2 exactly."""
    g = synth.ImageGeom((16, 8, 8), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    jj, kk = np.meshgrid(np.arange(8), np.arange(8), indexing="ij")
    yz = np.stack([jj.ravel(), kk.ravel()], 1).astype(np.float32)
    xs = np.concatenate([np.full((64, 1), -5.0, np.float32), yz], 1)
    xe = np.concatenate([np.full((64, 1), 20.0, np.float32), yz], 1)
    plan = ops.jp_plan_create(torch.from_numpy(xs).cuda(), torch.from_numpy(xe).cuda(), g)
    samples = ops.jp_count_samples(plan, "nontof")
    assert samples == 64 * 16
    assert ops.jp_count_red_requests(plan, "nontof") == samples // 2
    plan.destroy()


def test_red_requests_diagonal_every_sample_its_own_sector(ops):
    """LORs at 45 degrees in the (0, 1) plane, inside the grid along axis 1:
    the quad row changes on every plane, so a LOR's samples never share a
    sector, and with the LORs two rows apart no two LORs' samples do
    either (whatever order the plan gives equal keys): requests = samples."""
    g = synth.ImageGeom((8, 48, 4), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    xs, xe = [], []
    for c in range(12, 30, 2):
        for z in range(4):
            xs.append((-3.0, c - 3.0, float(z)))
            xe.append((11.0, c + 11.0, float(z)))
    xs = torch.tensor(xs, dtype=torch.float32).cuda()
    xe = torch.tensor(xe, dtype=torch.float32).cuda()
    plan = ops.jp_plan_create(xs, xe, g)
    samples = ops.jp_count_samples(plan, "nontof")
    assert samples == len(xs) * 8
    assert ops.jp_count_red_requests(plan, "nontof") == samples
    plan.destroy()


def test_red_requests_bounds_on_listmode(ops):
    """On TOF listmode events: samples / 2 <= requests <= samples (a
    request serves at most two entries' lanes), and the count is stable
    across rebinding the same events."""
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    ph = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, 4401)
    xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, 300_000, seed=4402)
    plan = ops.jp_plan_create(xs.cuda(), xe.cuda(), g, tof_bin=tb.cuda(), tof_bin_width=tof.bin_width)
    s = ops.jp_count_samples(plan, "tof_lm", tof)
    r = ops.jp_count_red_requests(plan, "tof_lm", tof)
    assert s / 2 <= r <= s
    ops.jp_plan_rebind(plan, xs.cuda(), xe.cuda(), tof_bin=tb.cuda())
    r2 = ops.jp_count_red_requests(plan, "tof_lm", tof)
    assert abs(r2 - r) <= 0.01 * r  # only the order of equal keys changes
    plan.destroy()


def test_bench_red_patterns(ops):
    """The reduction ceiling benchmark runs every access pattern and rejects
    an unknown one."""
    for pt in range(5):
        r = ops.jp_bench_red(n_entries=1 << 16, per_thread=4, iters=1, pattern=pt)
        assert r["reductions_per_s"] > 0 and r["sectors_per_s"] > 0
    with pytest.raises(ops.JosephError):
        ops.jp_bench_red(n_entries=1 << 16, per_thread=4, iters=1, pattern=5)
