"""GPU listmode OSEM (fused subset kernel, graphs, serving) against the FP64
oracle OSEM, the sensitivity image against the oracle, and the serving
invariants: a frame's result is the same alone and in a mix."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_12519_gb300 import synth
from _parity import BACK_TOL, rel_l2

pytestmark = pytest.mark.gpu

OSEM_TOL = 1e-4  # relative L2 after 3 iterations x 8 subsets


@pytest.fixture(scope="module")
def ops():
    from paper_2212_12519_gb300 import build, ops as _ops
    build.build()
    _ops.load()
    return _ops


def smooth_sens(geom, seed):
    """A positive sensitivity-like image (zero outside the transaxial FOV
    circle) used as an OSEM input; the OSEM update is defined for any s."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y, Z = [t.numpy() for t in geom.voxel_centres()]
    r = np.sqrt(X ** 2 + Y ** 2)
    rmax = (geom.shape[0] - 1) / 2 * geom.voxsize[0]
    s = (1.0 + 0.3 * np.cos(X / 37.0) * np.sin(Y / 23.0) + 0.2 * rng.uniform(size=geom.shape)) * (1 - (Z / 200) ** 2)
    s[r > 0.95 * rmax] = 0.0
    return s.astype(np.float32)


def frame(geom, ph_spec, n, seed):
    ph = synth.ellipsoid_phantom(geom, ph_spec, seed)
    xs, xe, tb = synth.lm_events(ph, geom, synth.SCANNER_CLINICAL, synth.TOF_CLINICAL, n, seed=seed + 1)
    return ph, xs, xe, tb, synth.background_level(ph, synth.TOF_CLINICAL)


@pytest.mark.parametrize("graph,path", [(False, "quads"), (True, "quads"), (False, "direct"), (True, "direct")])
def test_osem_frame_vs_oracle(ops, graph, path):
    from paper_2212_12519_gb300 import osem
    g = synth.GEOM_OSEM_SMALL
    tof = synth.TOF_CLINICAL
    ph, xs, xe, tb, b = frame(g, synth.PHANTOM_OSEM_SMALL, 120_003, 5101)
    sens = smooth_sens(g, 5102)
    x_or = oracle.lm_osem(xs.numpy(), xe.numpy(), tb.numpy(), g, tof, sens, b, n_iter=3, n_sub=8, threads=8)
    spec = osem.FrameSpec(xs.cuda(), xe.cuda(), tb.cuda(), g, b, path=path)
    fr = osem.LMOSEMFrame(spec, torch.from_numpy(sens).cuda(), tof)
    x = fr.run_graph() if graph else fr.run()
    torch.cuda.synchronize()
    assert rel_l2(x.cpu().numpy(), x_or) <= OSEM_TOL
    # the plain sequential path reaches the same image
    xp = osem.reconstruct_plain(spec, torch.from_numpy(sens).cuda(), tof)
    torch.cuda.synchronize()
    assert rel_l2(xp.cpu().numpy(), x_or) <= OSEM_TOL


def test_sensitivity_vs_oracle(ops):
    from paper_2212_12519_gb300 import osem
    g = synth.GEOM_SMALL
    s, info = osem.sensitivity(g, synth.SINO_SMALL, plane_chunk=24)
    xs, xe = synth.sinogram_lors(synth.SINO_SMALL)
    s_or = oracle.back(xs.numpy(), xe.numpy(), np.ones(len(xs)), g, threads=8)
    assert rel_l2(s.cpu().numpy(), s_or) <= BACK_TOL
    assert info["rel_gap"] <= 1e-5


def test_serving_alone_equals_mix(ops):
    from paper_2212_12519_gb300 import osem, serve
    tof = synth.TOF_CLINICAL
    pools = serve.make_event_pools(tof, pool_events=1_500_000, seed=5200)
    sens = {}
    for shape, pool in pools.items():
        sens[shape] = torch.from_numpy(smooth_sens(pool["geom"], 5201)).cuda()
    reqs = serve.make_requests(pools, 10, rate=1e6, seed=5202, ev_min=2e4, ev_max=1e6)
    mix = serve.OSEMServer(sens, tof, mode="batched", max_slots=4, use_graphs=True)
    mix.reserve(1_000_000, [p["geom"] for p in pools.values()])
    assert len(mix.slot_graphs) == 8
    st = mix.run(reqs)
    assert st["requests"] == 10
    x_mix = [r.x.clone() for r in reqs]
    serve.reset(reqs)
    alone = serve.OSEMServer(sens, tof, mode="batched", max_slots=1, use_graphs=False)
    alone.reserve(1_000_000, [p["geom"] for p in pools.values()])
    for r in reqs:
        r.arrival = 0.0
        alone.run([r])
    for r, xm in zip(reqs, x_mix):
        assert rel_l2(xm.cpu().numpy(), r.x.cpu().numpy()) <= OSEM_TOL
    # the sequential plain server reaches the same images
    serve.reset(reqs)
    seq = serve.OSEMServer(sens, tof, mode="sequential")
    seq.run(reqs)
    for r, xm in zip(reqs, x_mix):
        assert rel_l2(xm.cpu().numpy(), r.x.cpu().numpy()) <= OSEM_TOL
    mix.close()
    alone.close()


def test_serving_admission_budget(ops):
    """A budget that holds only one frame at a time still serves every frame
    (frames wait for memory instead of failing) with identical results."""
    from paper_2212_12519_gb300 import osem, serve
    tof = synth.TOF_CLINICAL
    pools = serve.make_event_pools(tof, pool_events=600_000, seed=5300)
    sens = {shape: torch.from_numpy(smooth_sens(p["geom"], 5301)).cuda() for shape, p in pools.items()}
    reqs = serve.make_requests(pools, 6, rate=1e6, seed=5302, ev_min=1e5, ev_max=5e5)
    big = max(osem.estimate_bytes(r.spec.xs.shape[0], r.spec.geom) for r in reqs)
    srv = serve.OSEMServer(sens, tof, mode="batched", max_slots=4, hbm_budget=big)
    srv.reserve(600_000, [p["geom"] for p in pools.values()])
    st = srv.run(reqs)
    assert st["requests"] == 6 and st["admission_waits"] > 0 and st["peak_bytes"] <= big
    x_budget = [r.x.clone() for r in reqs]
    serve.reset(reqs)
    free_srv = serve.OSEMServer(sens, tof, mode="batched", max_slots=4)
    free_srv.reserve(600_000, [p["geom"] for p in pools.values()])
    free_srv.run(reqs)
    for r, xb in zip(reqs, x_budget):
        assert rel_l2(xb.cpu().numpy(), r.x.cpu().numpy()) <= OSEM_TOL
    srv.close()
    free_srv.close()
