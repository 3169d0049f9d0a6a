"""The allocation-free TOF listmode back projection (for callers that cannot
allocate device memory, e.g. inside a graph capture or under a fixed memory
budget) gives the same image as the allocating planless entry point, on two
calls in a row (its fixed workspace is reused and must be cleared), and
rejects images larger than its fixed workspace."""
import pytest
import torch

from paper_2212_12519_gb300 import synth
from _parity import BACK_TOL, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    from paper_2212_12519_gb300 import build, ops as _ops
    build.build()
    _ops.load()
    return _ops


def test_noalloc_matches_allocating_entry(ops):
    g = synth.GEOM_SMALL  # 64 x 64 x 16: 221,760 workspace entries
    tof = synth.TOF_CLINICAL
    ph = synth.ellipsoid_phantom(g, synth.PHANTOM_SMALL, 9001)
    xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, 200_003, seed=9002)
    dxs, dxe, dtb = xs.cuda(), xe.cuda(), tb.cuda()
    for call in range(2):
        y = torch.from_numpy(synth.uniform_values(len(xs), 9003 + call, 0.5, 1.5)).cuda()
        ref = torch.zeros(g.shape, device="cuda")
        ops.jp_back_lors(dxs, dxe, y, g, ref, "tof_lm", tof, tof_bin=dtb)
        out = torch.zeros(g.shape, device="cuda")
        ops.jp_back_tof_lm_noalloc(dxs, dxe, y, g, out, tof, dtb)
        torch.cuda.synchronize()
        assert float(ref.abs().sum()) > 0
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= BACK_TOL


def test_noalloc_rejects_large_images(ops):
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    xs = torch.zeros((4, 3), device="cuda")
    xe = torch.ones((4, 3), device="cuda")
    tb = torch.zeros(4, dtype=torch.int16, device="cuda")
    y = torch.ones(4, device="cuda")
    out = torch.zeros(g.shape, device="cuda")
    with pytest.raises(ops.JosephError) as e:
        ops.jp_back_tof_lm_noalloc(xs, xe, y, g, out, tof, tb)
    assert e.value.code == -1
