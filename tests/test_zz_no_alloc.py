"""The allocation-free TOF listmode back projection, for callers that cannot
allocate device memory (engines whose device memory is handed out by their
own pool or a fixed budget): against the FP64 oracle and against the
allocating planless entry point, on two calls in a row (its fixed workspace
is reused and must be cleared), with TOF centre offsets and with a
tabulated TOF kernel; images larger than the workspace are rejected."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_12519_gb300 import synth
from _parity import BACK_TOL, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    from paper_2212_12519_gb300 import build, ops as _ops
    build.build()
    _ops.load()
    return _ops


@pytest.mark.parametrize("case", ["gaussian", "offsets", "tabulated"])
def test_noalloc_matches_oracle_and_allocating_entry(ops, case):
    g = synth.GEOM_SMALL  # 64 x 64 x 16: 221,760 workspace entries
    tof = synth.TOF_CLINICAL
    if case == "tabulated":
        # a triangle of half-width 1.5 bin widths as the TOF bin response
        h = 1.5 * tof.bin_width
        tof = synth.TofParams.tabulated(tof.bin_width, tof.n_bins, (0.0, 0.5, 1.0, 0.5, 0.0), h)
    ph = synth.ellipsoid_phantom(g, synth.PHANTOM_SMALL, 9001)
    xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, synth.TOF_CLINICAL, 200_003, seed=9002)
    delta = None
    if case == "offsets":
        delta = np.random.Generator(np.random.PCG64(9004)).normal(0, 6, size=len(xs)).astype(np.float32)
    dxs, dxe, dtb = xs.cuda(), xe.cuda(), tb.cuda()
    ddl = torch.from_numpy(delta).cuda() if delta is not None else None
    for call in range(2):
        yh = synth.uniform_values(len(xs), 9003 + call, 0.5, 1.5)
        y = torch.from_numpy(yh).cuda()
        ref = torch.zeros(g.shape, device="cuda")
        ops.jp_back_lors(dxs, dxe, y, g, ref, "tof_lm", tof, tof_bin=dtb, delta=ddl)
        out = torch.zeros(g.shape, device="cuda")
        ops.jp_back_tof_lm_noalloc(dxs, dxe, y, g, out, tof, dtb, delta=ddl)
        torch.cuda.synchronize()
        b_or = oracle.back(xs.numpy(), xe.numpy(), yh, g, "tof_lm", tof, tof_bin=tb.numpy(), delta=delta,
                           threads=8)
        assert float(np.abs(b_or).sum()) > 0
        assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL
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
