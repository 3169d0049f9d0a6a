"""The C-ABI library builds, loads and exports every symbol of
include/joseph.h; host-side argument checks reject bad input before any
CUDA call (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    with open(os.path.join(ROOT, "include", "joseph.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jp_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_12519_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_host_argument_checks(lib):
    from paper_2212_12519_gb300 import ops
    ops.load()
    g = ops.ImageGeomC()
    for i in range(3):
        g.n[i] = 4
        g.voxsize[i] = 1.0
    P = ctypes.c_void_p
    # negative size
    rc = lib.jp_fwd_lors(P(16), P(16), None, None, ctypes.c_int64(-1), ctypes.byref(g), 0, None,
                         P(16), P(16), None)
    assert rc == -1
    lib.jp_last_error.restype = ctypes.c_char_p
    assert b"n_lor" in lib.jp_last_error()
    # bad voxel size
    g.voxsize[1] = 0.0
    rc = lib.jp_fwd_lors(P(16), P(16), None, None, ctypes.c_int64(5), ctypes.byref(g), 0, None,
                         P(16), P(16), None)
    assert rc == -1
    g.voxsize[1] = 1.0
    # misaligned pointer
    rc = lib.jp_fwd_lors(P(17), P(16), None, None, ctypes.c_int64(5), ctypes.byref(g), 0, None,
                         P(16), P(16), None)
    assert rc == -2
    # TOF listmode without bins
    t = ops.TofC(28.0, 24.5, 3.0, 29)
    rc = lib.jp_fwd_lors(P(16), P(16), None, None, ctypes.c_int64(5), ctypes.byref(g), 2,
                         ctypes.byref(t), P(16), P(16), None)
    assert rc == -1
    # non-positive sigma
    t = ops.TofC(28.0, 0.0, 3.0, 29)
    rc = lib.jp_fwd_lors(P(16), P(16), P(16), None, ctypes.c_int64(5), ctypes.byref(g), 2,
                         ctypes.byref(t), P(16), P(16), None)
    assert rc == -1
    # too many sinogram TOF bins
    t = ops.TofC(28.0, 20.0, 3.0, 100000)
    rc = lib.jp_fwd_lors(P(16), P(16), None, None, ctypes.c_int64(5), ctypes.byref(g), 1,
                         ctypes.byref(t), P(16), P(16), None)
    assert rc == -1
    # plan calls on a NULL plan
    assert lib.jp_fwd(None, P(16), ctypes.c_int64(0), P(16), None) == -1
    assert lib.jp_plan_destroy(None) == 0
    # bad OSEM arguments
    assert lib.jp_osem_update(P(16), P(16), P(16), ctypes.c_float(-1.0), ctypes.c_int64(4), 1,
                              ctypes.c_int64(4), ctypes.c_int64(0), None) == -1


def test_resolution_model_argument_checks(lib):
    """jp_gauss3d / jp_osem_subset_tof_lm_ex reject bad input on the host."""
    from paper_2212_12519_gb300 import ops
    ops.load()
    lib.jp_last_error.restype = ctypes.c_char_p
    g = ops.ImageGeomC()
    for i in range(3):
        g.n[i] = 8
        g.voxsize[i] = 2.0
    P = ctypes.c_void_p
    nb = 8 * 8 * 8 * 4

    def call(r, img=4096, out=4096 + nb, work=4096 + 2 * nb, n=1):
        return lib.jp_gauss3d(P(img), P(out), P(work), n, ctypes.byref(g), ctypes.byref(r), None)

    ok = ops.resolution(4.5)
    assert call(ops.resolution(4.5), n=0) == 0                      # nothing to do, no CUDA call
    assert call(ops.resolution(-1.0)) == -1
    assert call(ops.resolution((4.5, float("nan"), 4.5))) == -1
    assert call(ops.resolution(4.5, truncate=0.0)) == -1
    assert call(ops.resolution(200.0)) == -1                        # radius above 32 voxels
    assert b"radius" in lib.jp_last_error()
    assert call(ok, out=4096 + nb // 2) == -1                       # img and out overlap
    assert b"overlap" in lib.jp_last_error()
    assert call(ok, work=4096 + 4) == -1                            # work overlaps img
    assert call(ok, out=4096 + nb + 2) == -2                        # misaligned
    assert call(ok, n=-1) == -1
    assert lib.jp_gauss3d(P(4096), P(4096 + nb), None, 1, ctypes.byref(g), ctypes.byref(ok), None) == -1
    assert lib.jp_osem_subset_tof_lm_ex(None, 0, 1, P(16), P(16), ctypes.c_float(1.0), ctypes.c_float(0.0),
                                        None, None, None, 0, P(16), None) == -1


def test_binding_constants_match_header():
    """The Python mirrors of the header's #defines hold the same values."""
    import re
    from paper_2212_12519_gb300 import ops
    with open(os.path.join(ROOT, "include", "joseph.h")) as f:
        h = f.read()
    defs = dict(re.findall(r"#define\s+(JP_\w+)\s+(\d+)", h))
    assert int(defs["JP_OSEM_DIRECT_VOXELS_PER_EVENT"]) == ops.OSEM_DIRECT_VOXELS_PER_EVENT
    assert {k: int(defs["JP_OSEM_PATH_" + k.upper()]) for k in ops.OSEM_PATHS} == ops.OSEM_PATHS
    assert int(defs["JP_PLAN_INTERLEAVED"]) == ops.JP_PLAN_INTERLEAVED


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the compiled library every entry point raises: there is no
    CPU or PyTorch fallback behind the binding."""
    import torch
    from paper_2212_12519_gb300 import ops, synth
    monkeypatch.setattr(ops, "_lib", None)
    monkeypatch.setattr(ops, "lib_path", lambda: str(tmp_path / "absent" / "libjoseph.so"))
    with pytest.raises(RuntimeError, match="not built"):
        ops.load()
    g = synth.GEOM_SMALL
    with pytest.raises(RuntimeError, match="not built"):
        ops.jp_gauss3d(torch.zeros(g.shape), g, 4.5)
