"""Autotuner host logic (CPU, fake timer) and, on the GPU, that the chosen
options keep parity with the oracle."""
import pytest
import torch

from paper_2212_12519_gb300 import autotune, synth


def test_tune_picks_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("JP_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    xs = torch.zeros((1000, 3))
    calls = []

    def fake(opts):
        calls.append(opts)
        return 1.0 + opts["block"] / 1000 + (0 if opts["lors_per_warp"] == 4 else 1) + opts["slope_bins"] / 1e4

    best = autotune.tune(xs, xs, synth.GEOM_SMALL, mode="nontof", timer=fake)
    assert best["block"] == 0 and best["lors_per_warp"] == 4 and best["slope_bins"] == 64 and best["zoff_bins"] == 1
    n = len(calls)
    again = autotune.tune(xs, xs, synth.GEOM_SMALL, mode="nontof", timer=fake)
    assert again == best and len(calls) == n  # served from the cache
    other = autotune.tune(torch.zeros((5000, 3)), xs, synth.GEOM_SMALL, mode="nontof", timer=fake)
    assert len(calls) == 2 * n  # another size bucket is tuned again
    assert other == best


@pytest.mark.gpu
def test_tuned_plan_parity(tmp_path, monkeypatch):
    import oracle
    from paper_2212_12519_gb300 import build, ops
    from _parity import AMB_EPS, BACK_TOL, FWD_TOL, fwd_err, rel_l2
    build.build()
    ops.load()
    monkeypatch.setenv("JP_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    g = synth.GEOM_CLINICAL
    tof = synth.TOF_CLINICAL
    ph = synth.ellipsoid_phantom(g, synth.PHANTOM_CLINICAL, 8101)
    xs, xe, tb = synth.lm_events(ph, g, synth.SCANNER_CLINICAL, tof, 200_000, seed=8102)
    dxs, dxe, dtb = xs.cuda(), xe.cuda(), tb.cuda()
    best = autotune.tune(dxs, dxe, g, mode="tof_lm", tof=tof, tof_bin=dtb, reps=1)
    plan = ops.jp_plan_create(dxs, dxe, g, tof_bin=dtb, tof_bin_width=tof.bin_width, **best)
    p = ops.jp_fwd_tof_lm(plan, ph.cuda(), tof)
    y = torch.from_numpy(synth.uniform_values(len(xs), 8103)).cuda()
    out = torch.zeros(g.shape, device="cuda")
    ops.jp_back_tof_lm(plan, y, tof, out)
    p_or, amb = oracle.fwd(xs.numpy(), xe.numpy(), ph.numpy(), g, "tof_lm", tof, tof_bin=tb.numpy(), threads=8,
                           amb_eps=AMB_EPS, return_amb=True)
    b_or = oracle.back(xs.numpy(), xe.numpy(), y.cpu().numpy(), g, "tof_lm", tof, tof_bin=tb.numpy(), threads=8)
    assert fwd_err(p.cpu().numpy(), p_or, amb) <= FWD_TOL
    assert rel_l2(out.cpu().numpy(), b_or) <= BACK_TOL
