"""Pins for the FP64 oracle (CPU only).

Each test checks the oracle against something other than itself: hand-derived
values, closed forms, brute force through an independent formulation,
invariants (adjoint, symmetry, translation, partition of unity) and numerical
quadrature.  ``test_planted_mistakes_are_caught`` rebuilds the oracle with
plausible errors planted in it and shows that the pins catch every one.
"""
import json
import math
import os
from fractions import Fraction
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from paper_2212_12519_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def G(shape, origin, vox):
    return SimpleNamespace(shape=tuple(shape), origin=tuple(origin), voxsize=tuple(vox))


def T(bin_width, sigma, n_sigmas, n_bins):
    return SimpleNamespace(bin_width=bin_width, sigma=sigma, n_sigmas=n_sigmas, n_bins=n_bins)


# ---------------------------------------------------------------------------
# independent formulation (pure Python): tent-function matrix entries
# ---------------------------------------------------------------------------
def _principal_axis_exact(xs, xe):
    d = [abs(Fraction(float(xe[i])) - Fraction(float(xs[i]))) for i in range(3)]
    m = max(d)
    return min(i for i in range(3) if d[i] == m)


def _tent(t):
    return max(0.0, 1.0 - abs(t))


def _gauss_bin(dist, D, s, ns):
    if abs(dist) > ns * s + 0.5 * D:
        return 0.0
    k = 1.0 / (math.sqrt(2.0) * s)
    return 0.5 * (math.erf((dist + 0.5 * D) * k) - math.erf((dist - 0.5 * D) * k))


def dense_tent(xs, xe, geom, mode="nontof", tof=None, tof_bin=None):
    """A[row, voxel] = w0 * sum_k [k == voxel_a] tent(u_k - i_b) tent(w_k - i_c) (* TOF)."""
    n = geom.shape
    o = geom.origin
    v = geom.voxsize
    nrow_per = tof.n_bins if mode == "tof_sino" else 1
    A = np.zeros((len(xs) * nrow_per, int(np.prod(n))))
    for r, (p, q) in enumerate(zip(np.asarray(xs, np.float64), np.asarray(xe, np.float64))):
        d = q - p
        L = math.sqrt(float(np.dot(d, d)))
        if L == 0:
            continue
        a = _principal_axis_exact(p, q)
        b, c = [i for i in range(3) if i != a]
        w0 = v[a] * L / abs(d[a])
        for k in range(n[a]):
            X = o[a] + k * v[a]
            if not (min(p[a], q[a]) <= X <= max(p[a], q[a])):
                continue
            t = (X - p[a]) / d[a]
            Pb = p[b] + t * d[b]
            Pc = p[c] + t * d[c]
            u = (Pb - o[b]) / v[b]
            w = (Pc - o[c]) / v[c]
            tau = (t - 0.5) * L
            for ib in range(n[b]):
                tb = _tent(u - ib)
                if tb == 0.0:
                    continue
                for ic in range(n[c]):
                    tc = _tent(w - ic)
                    if tc == 0.0:
                        continue
                    ijk = [0, 0, 0]
                    ijk[a], ijk[b], ijk[c] = k, ib, ic
                    col = (ijk[0] * n[1] + ijk[1]) * n[2] + ijk[2]
                    base = w0 * tb * tc
                    if mode == "nontof":
                        A[r, col] += base
                    elif mode == "tof_sino":
                        for t_ in range(tof.n_bins):
                            cen = (t_ - (tof.n_bins - 1) / 2.0) * tof.bin_width
                            A[r * nrow_per + t_, col] += base * _gauss_bin(
                                tau - cen, tof.bin_width, tof.sigma, tof.n_sigmas)
                    else:
                        cen = tof_bin[r] * tof.bin_width
                        A[r, col] += base * _gauss_bin(tau - cen, tof.bin_width, tof.sigma,
                                                       tof.n_sigmas)
    return A


def dense_by_fwd(xs, xe, geom, mode="nontof", tof=None, tof_bin=None, mutant=0):
    nvox = int(np.prod(geom.shape))
    cols = []
    for j in range(nvox):
        e = np.zeros(nvox)
        e[j] = 1.0
        cols.append(oracle.fwd(xs, xe, e.reshape(geom.shape), geom, mode=mode, tof=tof,
                               tof_bin=tof_bin, mutant=mutant).reshape(-1))
    return np.stack(cols, 1)


def dense_by_back(xs, xe, geom, mode="nontof", tof=None, tof_bin=None, mutant=0):
    nrow_per = tof.n_bins if mode == "tof_sino" else 1
    nrow = len(xs) * nrow_per
    rows = []
    for i in range(nrow):
        e = np.zeros(nrow)
        e[i] = 1.0
        rows.append(oracle.back(xs, xe, e, geom, mode=mode, tof=tof, tof_bin=tof_bin,
                                mutant=mutant).reshape(-1))
    return np.stack(rows, 0)


# small brute-force geometry: non-isotropic voxels, off-centre origin
BF_GEOM = G((4, 4, 4), (-1.7, -2.2, -1.1), (1.0, 1.5, 0.75))
BF_TOF = T(bin_width=1.3, sigma=1.1, n_sigmas=3.0, n_bins=7)


def bf_rays():
    xs, xe = synth.random_lors(24, synth.ImageGeom(BF_GEOM.shape, BF_GEOM.origin, BF_GEOM.voxsize),
                               seed=11, radius_factor=1.6)
    extra_s, extra_e = [], []
    # axis-aligned through voxel centres and between them, each direction
    extra_s += [(-9.0, -0.7, -0.35), (-0.7, -9.0, 0.4), (0.3, 0.8, -9.0)]
    extra_e += [(9.0, -0.7, -0.35), (-0.7, 9.0, 0.4), (0.3, 0.8, 9.0)]
    # exact principal-axis ties with an out-of-plane slope
    extra_s += [(-6.0, -6.3, -0.9), (-0.2, -5.0, -5.4), (-4.0, 1.0, -4.1)]
    extra_e += [(6.0, 5.7, 0.8), (0.9, 5.0, 4.6), (4.0, -0.3, 3.9)]
    # ray ending exactly on a plane centre, inside the image
    extra_s += [(-9.0, 0.1, 0.2)]
    extra_e += [(-1.7 + 2.0, 0.9, -0.4)]
    # degenerate ray
    extra_s += [(0.1, 0.2, 0.3)]
    extra_e += [(0.1, 0.2, 0.3)]
    xs = np.concatenate([xs, np.asarray(extra_s, np.float32)])
    xe = np.concatenate([xe, np.asarray(extra_e, np.float32)])
    return xs, xe


def bf_tof_bins(n):
    rng = np.random.Generator(np.random.PCG64(12))
    return rng.integers(-3, 4, size=n)


# ---------------------------------------------------------------------------
# hand-derived golden values
# ---------------------------------------------------------------------------
def test_hand_golden():
    with open(os.path.join(GOLDEN, "hand_examples.json")) as f:
        gold = json.load(f)
    im = gold["image"]
    g = G(im["shape"], im["origin"], im["voxsize"])
    i0, i1, i2 = np.meshgrid(*[np.arange(n) for n in g.shape], indexing="ij")
    img = 100.0 * i0 + 10.0 * i1 + i2
    for case in gold["cases"]:
        p = oracle.fwd([case["xs"]], [case["xe"]], img, g)[0]
        assert p == pytest.approx(case["expected"], rel=1e-13, abs=1e-12), case["name"]


# ---------------------------------------------------------------------------
# brute force, three ways
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["nontof", "tof_sino", "tof_lm"])
def test_bruteforce_three_ways(mode):
    xs, xe = bf_rays()
    tof = None if mode == "nontof" else BF_TOF
    tb = bf_tof_bins(len(xs)) if mode == "tof_lm" else None
    A1 = dense_by_fwd(xs, xe, BF_GEOM, mode, tof, tb)
    A2 = dense_by_back(xs, xe, BF_GEOM, mode, tof, tb)
    A3 = dense_tent(xs, xe, BF_GEOM, mode, tof, tb)
    scale = np.abs(A3).max()
    assert scale > 0.1
    assert np.abs(A1 - A2).max() <= 1e-14 * scale
    assert np.abs(A1 - A3).max() <= 1e-13 * scale


def test_principal_axis_ties():
    assert oracle.principal_axis([0, 0, 0], [1, 1, 1]) == 0
    assert oracle.principal_axis([0, 0, 0], [0.5, -1, 1]) == 1
    assert oracle.principal_axis([0, 0, 0], [0.5, -1, 1.0000001]) == 2
    # tie decided on the exact difference, not on a rounded one
    xs = np.array([1e-9, 0.0, 0.0], np.float32)
    xe = np.array([400.0, 400.0 - 1e-9 + 1e-9, 0.0], np.float32)
    assert oracle.principal_axis(xs, xe) == _principal_axis_exact(xs, xe)
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(200):
        p = rng.normal(size=3).astype(np.float32) * 300
        q = p.copy()
        s = rng.normal() * 200
        q[0] += np.float32(s)
        q[1] = np.float32(p[1] + (q[0] - p[0]) * rng.choice([-1, 1]))
        assert oracle.principal_axis(p, q) == _principal_axis_exact(p, q)


# ---------------------------------------------------------------------------
# adjoint identity <Ax, y> = <x, A^T y>
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["nontof", "tof_sino", "tof_lm"])
def test_adjoint(mode):
    geom = G((13, 9, 11), (-7.1, -3.3, -6.0), (1.1, 1.7, 0.9))
    sg = synth.ImageGeom(geom.shape, geom.origin, geom.voxsize)
    xs1, xe1 = synth.random_lors(300, sg, seed=21)
    xs2, xe2 = synth.random_lors(100, sg, seed=22, kind="inside")
    xs, xe = np.concatenate([xs1, xs2]), np.concatenate([xe1, xe2])
    tof = T(2.5, 2.0, 3.0, 11)
    rng = np.random.Generator(np.random.PCG64(23))
    tb = rng.integers(-5, 6, size=len(xs)) if mode == "tof_lm" else None
    delta = rng.normal(size=len(xs)) if mode != "nontof" else None
    x = rng.uniform(0, 1, size=geom.shape)
    nout = tof.n_bins if mode == "tof_sino" else 1
    y = rng.uniform(0, 1, size=(len(xs), nout)).reshape(-1)
    Ax = oracle.fwd(xs, xe, x, geom, mode, tof if mode != "nontof" else None, tb, delta)
    ATy = oracle.back(xs, xe, y, geom, mode, tof if mode != "nontof" else None, tb, delta)
    lhs = float(np.dot(Ax.reshape(-1), y))
    rhs = float(np.sum(x * ATy))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_threaded_equals_single():
    g = synth.GEOM_SMALL
    img = synth.ellipsoid_phantom(g, synth.PHANTOM_SMALL, 1001).numpy()
    xs, xe = synth.random_lors(5000, g, seed=31)
    p1 = oracle.fwd(xs, xe, img, g, threads=1)
    p4 = oracle.fwd(xs, xe, img, g, threads=4)
    assert np.array_equal(p1, p4)
    y = synth.uniform_values(len(xs), 32)
    b1 = oracle.back(xs, xe, y, g, threads=1)
    b4 = oracle.back(xs, xe, y, g, threads=4)
    assert np.abs(b1 - b4).max() <= 1e-12 * np.abs(b1).max()


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
def test_axis_aligned_voxel_sums():
    geom = G((6, 5, 7), (-3.0, 10.0, -2.5), (1.2, 0.8, 2.0))
    rng = np.random.Generator(np.random.PCG64(41))
    img = rng.uniform(0, 5, size=geom.shape)
    for a in range(3):
        b, c = [i for i in range(3) if i != a]
        for _ in range(5):
            ib, ic = rng.integers(0, geom.shape[b]), rng.integers(0, geom.shape[c])
            xs = np.zeros(3)
            xs[b] = geom.origin[b] + ib * geom.voxsize[b]
            xs[c] = geom.origin[c] + ic * geom.voxsize[c]
            xe = xs.copy()
            xs[a] = geom.origin[a] - 10.0
            xe[a] = geom.origin[a] + geom.shape[a] * geom.voxsize[a] + 10.0
            sl = [slice(None)] * 3
            sl[b], sl[c] = ib, ic
            expect = geom.voxsize[a] * img[tuple(sl)].sum()
            p = oracle.fwd([xs], [xe], img, geom)[0]
            assert p == pytest.approx(expect, rel=1e-13)
            p_rev = oracle.fwd([xe], [xs], img, geom)[0]
            assert p_rev == pytest.approx(expect, rel=1e-13)


def test_affine_image_closed_form_and_uniform_cube():
    """Affine image, every sample interior: bilinear interpolation is exact
    and the plane sum is a midpoint rule, p = n_a v_a / cos_a * f(P_mid).
    With f = 1 this is the chord length of the ray through the slab of
    voxel edges, n_a v_a / cos_a (uniform cube)."""
    geom = G((20, 20, 20), (-9.5, -9.5, -9.5), (1.0, 1.0, 1.0))
    X, Y, Z = np.meshgrid(*[np.arange(20) * 1.0 - 9.5] * 3, indexing="ij")
    alpha, beta = 2.0, np.array([0.3, -0.2, 0.15])
    img = alpha + beta[0] * X + beta[1] * Y + beta[2] * Z
    rng = np.random.Generator(np.random.PCG64(42))
    for _ in range(40):
        a = int(rng.integers(0, 3))
        b, c = [i for i in range(3) if i != a]
        d = np.zeros(3)
        d[a] = 1.0
        d[b], d[c] = rng.uniform(-0.3, 0.3, size=2)  # keeps samples interior
        m = np.zeros(3)
        m[b], m[c] = rng.uniform(-2, 2, size=2)
        xs = m - 30 * d
        xe = m + 30 * d
        if rng.uniform() < 0.5:
            xs, xe = xe, xs
        cosa = 1.0 / np.linalg.norm(d)
        Pmid = m  # the sample at the central plane (coordinate 0)
        expect = 20 * 1.0 / cosa * (alpha + beta @ Pmid)
        p = oracle.fwd([xs], [xe], img, geom)[0]
        assert p == pytest.approx(expect, rel=1e-12)
        pu = oracle.fwd([xs], [xe], np.ones(geom.shape), geom)[0]
        assert pu == pytest.approx(20 * 1.0 / cosa, rel=1e-12)


def test_parallel_rays_partition_of_unity():
    """Back-projecting ones along a lattice of parallel rays offset by one
    voxel pitch in (b, c) gives every interior voxel exactly v_a / cos_a."""
    geom = G((8, 10, 9), (-4.0, -5.0, -4.0), (1.0, 1.25, 0.8))
    for a, slopes in [(0, (0.31, -0.17)), (1, (-0.23, 0.41)), (2, (0.12, 0.27))]:
        b, c = [i for i in range(3) if i != a]
        d = np.zeros(3)
        d[a] = 1.0
        d[b], d[c] = slopes
        xs_l, xe_l = [], []
        for ib in range(-6, geom.shape[b] + 6):
            for ic in range(-6, geom.shape[c] + 6):
                p0 = np.zeros(3)
                p0[a] = geom.origin[a]
                p0[b] = geom.origin[b] + (ib + 0.37) * geom.voxsize[b]
                p0[c] = geom.origin[c] + (ic + 0.61) * geom.voxsize[c]
                xs_l.append(p0 - 40 * d)
                xe_l.append(p0 + 40 * d)
        img = oracle.back(xs_l, xe_l, np.ones(len(xs_l)), geom)
        w0 = geom.voxsize[a] * np.linalg.norm(d) / 1.0
        # the lattice spacing is one voxel pitch in b and c at every plane a
        # only if the offsets are in voxel units at each plane: true because
        # all rays are parallel and the lattice is defined on plane 0
        interior = [slice(None)] * 3
        interior[b] = slice(1, geom.shape[b] - 1)
        interior[c] = slice(1, geom.shape[c] - 1)
        vals = img[tuple(interior)]
        assert np.allclose(vals, w0, rtol=1e-12, atol=0)


# ---------------------------------------------------------------------------
# TOF
# ---------------------------------------------------------------------------
def test_tof_weight_vs_quadrature():
    """g = integral over the bin [c - D/2, c + D/2] of the Gaussian pdf of
    width sigma centred on tau (composite Simpson, 4000 panels)."""
    D, s = 28.0, 24.503
    for tau, cen in [(0.0, 0.0), (13.0, 28.0), (-40.0, 28.0), (70.0, 0.0), (-50.0, -28.0)]:
        x = np.linspace(cen - D / 2, cen + D / 2, 8001)
        pdf = np.exp(-0.5 * ((x - tau) / s) ** 2) / (s * math.sqrt(2 * math.pi))
        h = x[1] - x[0]
        simpson = h / 3 * (pdf[0] + pdf[-1] + 4 * pdf[1:-1:2].sum() + 2 * pdf[2:-1:2].sum())
        assert oracle.tof_weight(tau, cen, D, s, 3.0) == pytest.approx(simpson, rel=1e-12)
    # truncation: zero beyond n_sigmas*sigma + D/2
    assert oracle.tof_weight(3 * s + D / 2 + 1e-6, 0.0, D, s, 3.0) == 0.0
    assert oracle.tof_weight(3 * s + D / 2 - 1e-6, 0.0, D, s, 3.0) > 0.0


def _line_geom():
    return G((40, 3, 3), (-39.0, -2.0, -2.0), (2.0, 2.0, 2.0))


def test_tof_sum_equals_nontof():
    geom = G((30, 20, 10), (-29.0, -19.0, -9.0), (2.0, 2.0, 2.0))
    sg = synth.ImageGeom(geom.shape, geom.origin, geom.voxsize)
    rng = np.random.Generator(np.random.PCG64(51))
    img = rng.uniform(0, 2, size=geom.shape)
    xs, xe = synth.random_lors(200, sg, seed=52)
    p = oracle.fwd(xs, xe, img, geom)
    # window covers every ray (N*D >= L + 2 n_sigmas sigma + D) with n_sigmas = 8
    tof8 = T(10.0, 4.0, 8.0, 41)
    pt = oracle.fwd(xs, xe, img, geom, "tof_sino", tof8)
    assert np.allclose(pt.sum(1), p, rtol=1e-12, atol=1e-12 * p.max())
    # n_sigmas = 3: telescoping bound sum_t g_t in [erf(3/sqrt2), 1] per sample
    tof3 = T(10.0, 4.0, 3.0, 41)
    pt3 = oracle.fwd(xs, xe, img, geom, "tof_sino", tof3)
    lo = math.erf(3 / math.sqrt(2))
    assert np.all(pt3.sum(1) >= lo * p - 1e-12 * p.max())
    assert np.all(pt3.sum(1) <= p + 1e-12 * p.max())


def test_mirror_symmetry():
    geom = G((16, 12, 10), (-15.0, -11.0, -9.0), (2.0, 2.0, 2.0))
    sg = synth.ImageGeom(geom.shape, geom.origin, geom.voxsize)
    rng = np.random.Generator(np.random.PCG64(61))
    img = rng.uniform(0, 2, size=geom.shape)
    xs, xe = synth.random_lors(300, sg, seed=62)
    tof = T(7.0, 5.0, 3.0, 9)
    assert np.allclose(oracle.fwd(xs, xe, img, geom), oracle.fwd(xe, xs, img, geom), rtol=1e-12)
    a = oracle.fwd(xs, xe, img, geom, "tof_sino", tof)
    b = oracle.fwd(xe, xs, img, geom, "tof_sino", tof)
    assert np.allclose(a, b[:, ::-1], rtol=1e-12, atol=1e-13 * np.abs(a).max())
    tb = rng.integers(-4, 5, size=len(xs))
    la = oracle.fwd(xs, xe, img, geom, "tof_lm", tof, tof_bin=tb)
    lb = oracle.fwd(xe, xs, img, geom, "tof_lm", tof, tof_bin=-tb)
    assert np.allclose(la, lb, rtol=1e-12, atol=1e-13 * np.abs(la).max())
    # the sign convention itself: bins increase toward xe
    line = _line_geom()
    one = np.zeros(line.shape)
    one[35, 1, 1] = 1.0  # a hot voxel near the xe end
    pt = oracle.fwd([(-100.0, 0.0, 0.0)], [(100.0, 0.0, 0.0)], one, line, "tof_sino",
                    T(10.0, 3.0, 3.0, 21))[0]
    assert int(np.argmax(pt)) > 10


def test_lm_equals_sino():
    geom = G((16, 12, 10), (-15.0, -11.0, -9.0), (2.0, 2.0, 2.0))
    sg = synth.ImageGeom(geom.shape, geom.origin, geom.voxsize)
    rng = np.random.Generator(np.random.PCG64(71))
    img = rng.uniform(0, 2, size=geom.shape)
    xs, xe = synth.random_lors(300, sg, seed=72)
    tof = T(7.0, 5.0, 3.0, 9)
    delta = rng.normal(size=len(xs)) * 3
    ps = oracle.fwd(xs, xe, img, geom, "tof_sino", tof, delta=delta)
    for ts in range(-4, 5):
        pl = oracle.fwd(xs, xe, img, geom, "tof_lm", tof, tof_bin=np.full(len(xs), ts), delta=delta)
        assert np.array_equal(pl, ps[:, ts + 4])
    tbv = rng.integers(-4, 5, size=len(xs))
    y = rng.uniform(size=len(xs))
    ysino = np.zeros((len(xs), 9))
    ysino[np.arange(len(xs)), tbv + 4] = y
    bl = oracle.back(xs, xe, y, geom, "tof_lm", tof, tof_bin=tbv, delta=delta)
    bs = oracle.back(xs, xe, ysino, geom, "tof_sino", tof, delta=delta)
    assert np.allclose(bl, bs, rtol=1e-12, atol=1e-13 * np.abs(bl).max())


def test_translation_invariance():
    geom = G((12, 10, 8), (-11.0, -9.0, -7.0), (2.0, 1.5, 1.0))
    sg = synth.ImageGeom(geom.shape, geom.origin, geom.voxsize)
    rng = np.random.Generator(np.random.PCG64(81))
    img = rng.uniform(0, 2, size=geom.shape)
    xs, xe = synth.random_lors(200, sg, seed=82)
    shift = np.array([3 * 2.0, -2 * 1.5, 5 * 1.0])
    g2 = G(geom.shape, tuple(np.array(geom.origin) + shift), geom.voxsize)
    tof = T(6.0, 4.0, 3.0, 7)
    for mode in ["nontof", "tof_sino"]:
        t = tof if mode != "nontof" else None
        a = oracle.fwd(xs, xe, img, geom, mode, t)
        b = oracle.fwd(xs.astype(np.float64) + shift, xe.astype(np.float64) + shift, img, g2, mode, t)
        assert np.allclose(a, b, rtol=1e-10, atol=1e-11 * np.abs(a).max())


# ---------------------------------------------------------------------------
# OSEM and gradient
# ---------------------------------------------------------------------------
def _small_lm_problem(n_events=3000, seed=91):
    g = synth.ImageGeom.centred((16, 16, 8), (2.0, 2.0, 2.0))
    ph = synth.PhantomSpec((12.0, 10.0, 6.0), (3.0,))
    x = synth.ellipsoid_phantom(g, ph, seed).numpy()
    tof = synth.TOF_CLINICAL
    xs, xe, tb = synth.lm_events(synth.ellipsoid_phantom(g, ph, seed), g, synth.SCANNER_CLINICAL,
                                 tof, n_events, seed)
    return g, tof, x, xs.numpy(), xe.numpy(), tb.numpy()


def test_osem_count_preservation():
    """sum_j (s_j / n_sub) x_new_j = sum_{e in S} (Ax)_e / ((Ax)_e + b), for
    any sensitivity s > 0 (here a random positive image)."""
    g, tof, x, xs, xe, tb = _small_lm_problem()
    rng = np.random.Generator(np.random.PCG64(92))
    sens = rng.uniform(0.5, 2.0, size=g.shape)
    b, n_sub, m = 0.7, 4, 1
    x0 = rng.uniform(0.2, 1.5, size=g.shape)
    x1 = oracle.lm_osem_subset_update(x0, xs, xe, tb, g, tof, sens, b, m, n_sub)
    p = oracle.fwd(xs[m::n_sub], xe[m::n_sub], x0, g, "tof_lm", tof, tof_bin=tb[m::n_sub])
    lhs = float(np.sum(sens / n_sub * x1))
    rhs = float(np.sum(p / (p + b)))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert np.all(x1 >= 0)
    # b = 0: the preserved count is the subset size (events with Ax > 0)
    x1b = oracle.lm_osem_subset_update(x0, xs, xe, tb, g, tof, sens, 0.0, m, n_sub)
    assert float(np.sum(sens / n_sub * x1b)) == pytest.approx(float(np.sum(p > 0)), rel=1e-12)


def test_gradient_vs_finite_differences():
    g, tof, x, xs, xe, tb = _small_lm_problem(n_events=2000, seed=93)
    rng = np.random.Generator(np.random.PCG64(94))
    w = rng.uniform(0.5, 1.5, size=len(xs))
    b = 0.3
    x = x + 0.1
    f0, grad = oracle.poisson_loglik_grad(x, xs, xe, tb, g, tof, w, b)
    h = 1e-6
    idx = rng.choice(x.size, size=40, replace=False)
    for j in idx:
        e = np.zeros(x.size)
        e[j] = h
        e = e.reshape(x.shape)
        # f(x+h e_j) - f(x-h e_j), summed per event as log1p of the relative
        # change so that the O(|f|) rounding of the full sums does not swamp
        # the O(h) difference
        pp = oracle.fwd(xs, xe, x + e, g, "tof_lm", tof, tof_bin=tb)
        pm = oracle.fwd(xs, xe, x - e, g, "tof_lm", tof, tof_bin=tb)
        fd = float(np.sum(w * np.log1p((pp - pm) / (pm + b)))) / (2 * h)
        gj = grad.reshape(-1)[j]
        assert abs(fd - gj) <= 1e-7 * max(abs(gj), 1e-3 * np.abs(grad).max()), (j, fd, gj)


# ---------------------------------------------------------------------------
# planted mistakes must be caught
# ---------------------------------------------------------------------------
def _pins(mutant):
    """Fast versions of the pins above, run against a (possibly mutated)
    oracle build.  Returns the names of the pins that failed."""
    failed = []
    xs, xe = bf_rays()
    for mode in ["nontof", "tof_sino", "tof_lm"]:
        tof = None if mode == "nontof" else BF_TOF
        tb = bf_tof_bins(len(xs)) if mode == "tof_lm" else None
        A1 = dense_by_fwd(xs, xe, BF_GEOM, mode, tof, tb, mutant=mutant)
        A3 = dense_tent(xs, xe, BF_GEOM, mode, tof, tb)
        if np.abs(A1 - A3).max() > 1e-13 * np.abs(A3).max():
            failed.append("bruteforce-" + mode)
    D, s = 28.0, 24.503
    x = np.linspace(-D / 2, D / 2, 8001)
    pdf = np.exp(-0.5 * ((x - 5.0) / s) ** 2) / (s * math.sqrt(2 * math.pi))
    h = x[1] - x[0]
    simpson = h / 3 * (pdf[0] + pdf[-1] + 4 * pdf[1:-1:2].sum() + 2 * pdf[2:-1:2].sum())
    if abs(oracle.tof_weight(5.0, 0.0, D, s, 3.0, mutant=mutant) - simpson) > 1e-12 * simpson:
        failed.append("quadrature")
    with open(os.path.join(GOLDEN, "hand_examples.json")) as f:
        gold = json.load(f)
    im = gold["image"]
    gg = G(im["shape"], im["origin"], im["voxsize"])
    i0, i1, i2 = np.meshgrid(*[np.arange(n) for n in gg.shape], indexing="ij")
    himg = 100.0 * i0 + 10.0 * i1 + i2
    for case in gold["cases"]:
        p = oracle.fwd([case["xs"]], [case["xe"]], himg, gg, mutant=mutant)[0]
        if abs(p - case["expected"]) > 1e-12 * max(1.0, abs(case["expected"])):
            failed.append("golden")
            break
    geom = G((20, 20, 20), (-9.5, -9.5, -9.5), (1.0, 1.0, 1.0))
    pu = oracle.fwd([(-30.0, -3.0, 1.0)], [(30.0, 4.0, -2.0)], np.ones(geom.shape), geom,
                    mutant=mutant)[0]
    if abs(pu - 20 * math.sqrt(60 ** 2 + 7 ** 2 + 3 ** 2) / 60) > 1e-12 * pu:
        failed.append("uniform-cube")
    return failed


def test_planted_mistakes_are_caught():
    assert _pins(0) == []
    for mutant in range(1, 8):
        oracle.joseph.build(mutant)
        assert _pins(mutant), f"planted mistake {mutant} not caught"


# ---------------------------------------------------------------------------
# image-based resolution model (paper Sec. 2.6: 3D Gaussian, 4.5 mm FWHM)
# ---------------------------------------------------------------------------
RES_FWHM = 4.5
# voxels fine enough that the sampled Gaussian keeps the continuous moments
# (Poisson summation: the error is ~exp(-2 pi^2 sigma^2 / d^2) < 1e-19), and
# a grid that holds the whole 7-sigma support around its centre voxel
RES_GEOM = G((23, 29, 25), (-13.75, -14.0, -14.4), (1.25, 1.0, 1.2))
RES_CENTRE = (11, 14, 12)


def _res_pins(mutant=0):
    """Pins of oracle.gauss3d / gauss_taps; returns the names that failed."""
    from oracle import resolution as R
    failed = []
    # (1) defining property of the FWHM: the normalised taps (truncated at
    #     8 sigma, so their moments are the continuous ones) have unit mass,
    #     zero mean, and a variance v with exp(-(FWHM/2)^2 / (2 v)) = 1/2
    for d in (0.25, 0.6):
        w = R.gauss_taps(RES_FWHM, (d, d, d), truncate=8.0, _mutant=mutant)[0]
        r = (len(w) - 1) // 2
        t = np.arange(-r, r + 1) * d
        if abs(w.sum() - 1.0) > 1e-13 or abs(np.dot(w, t)) > 1e-12:
            failed.append("taps-mass-mean")
            break
        v = float(np.dot(w, t * t))
        if abs(math.exp(-0.5 * (RES_FWHM / 2) ** 2 / v) - 0.5) > 1e-10:
            failed.append("taps-fwhm")
            break
    # (2) response to an interior delta, non-isotropic voxels: unit mass,
    #     rank-one (separable) and, along every axis, the marginal's variance
    #     in mm^2 is the same sigma^2 (the FWHM is isotropic in mm)
    delta = np.zeros(RES_GEOM.shape)
    c = RES_CENTRE
    delta[c] = 1.0
    h = R.gauss3d(delta, RES_GEOM, RES_FWHM, truncate=7.0, _mutant=mutant)
    if abs(h.sum() - 1.0) > 1e-12:
        failed.append("delta-mass")
    variances = []
    for a in range(3):
        m = h.sum(axis=tuple(b for b in range(3) if b != a))
        t = (np.arange(RES_GEOM.shape[a]) - c[a]) * RES_GEOM.voxsize[a]
        variances.append(float(np.dot(m, t * t) / m.sum()))
    v_true = (RES_FWHM / 2) ** 2 / (2 * math.log(2.0))  # half maximum at FWHM/2
    if max(abs(v - v_true) for v in variances) > 1e-9 * v_true:
        failed.append("delta-variance")
    m0, m1, m2 = (h.sum(axis=(1, 2)), h.sum(axis=(0, 2)), h.sum(axis=(0, 1)))
    if np.abs(h - np.einsum("i,j,k->ijk", m0, m1, m2)).max() > 1e-15:
        failed.append("delta-separable")
    # (3) special case that reduces to a library routine: the separable
    #     correlation with scipy.ndimage.correlate1d (zero outside the grid)
    import scipy.ndimage as ndi
    rng = np.random.Generator(np.random.PCG64(131))
    g2 = G((9, 12, 7), (-4.0, -6.0, -5.25), (2.0, 1.5, 3.0))
    x = rng.uniform(0.0, 1.0, g2.shape)
    taps = R.gauss_taps(RES_FWHM, g2.voxsize)
    ref = x
    for a in range(3):
        ref = ndi.correlate1d(ref, taps[a], axis=a, mode="constant", cval=0.0)
    if np.abs(R.gauss3d(x, g2, RES_FWHM, _mutant=mutant) - ref).max() > 1e-14:
        failed.append("scipy-separable")
    # (4) zero outside the grid: a corner delta keeps, per axis, the centre
    #     tap and one half of the others, i.e. (1 + w_centre) / 2
    corner = np.zeros(g2.shape)
    corner[0, 0, 0] = 1.0
    kept = np.prod([(1.0 + w[(len(w) - 1) // 2]) / 2.0 for w in taps])
    if abs(R.gauss3d(corner, g2, RES_FWHM, _mutant=mutant).sum() - kept) > 1e-14:
        failed.append("corner-mass")
    return failed


def test_resolution_model_pins():
    assert _res_pins() == []


def test_resolution_model_adjoint_and_identity():
    from oracle import resolution as R
    rng = np.random.Generator(np.random.PCG64(132))
    g2 = G((10, 8, 13), (-3.0, -2.0, -6.0), (2.0, 2.5, 1.5))
    x, y = rng.uniform(size=g2.shape), rng.uniform(size=g2.shape)
    hx = R.gauss3d(x, g2, (4.5, 3.0, 6.0))
    hty = R.gauss3d(y, g2, (4.5, 3.0, 6.0), adjoint=True)
    assert float(np.sum(hx * y)) == pytest.approx(float(np.sum(x * hty)), rel=1e-13)
    # symmetric taps: H^T = H
    assert np.abs(hty - R.gauss3d(y, g2, (4.5, 3.0, 6.0))).max() < 1e-15
    # FWHM 0 is the identity
    assert np.array_equal(R.gauss3d(x, g2, 0.0), x)
    # a stack of images is filtered image by image
    st = R.gauss3d(np.stack([x, y]), g2, 4.5)
    assert np.array_equal(st[1], R.gauss3d(y, g2, 4.5))


def test_resolution_model_planted_mistakes():
    for mutant in (1, 2, 3, 4):
        assert _res_pins(mutant), f"planted resolution-model mistake {mutant} not caught"


def test_osem_with_resolution_model():
    """Count preservation with H: sum_j (s'_j / n_sub) x_new_j equals
    sum_{e in S} p_e / (p_e + b) with p = A_S H x (as H^T is the adjoint);
    FWHM 0 gives the plain update."""
    g, tof, x, xs, xe, tb = _small_lm_problem(n_events=2500, seed=95)
    rng = np.random.Generator(np.random.PCG64(96))
    sens = rng.uniform(0.5, 2.0, size=g.shape)
    b, n_sub, m = 0.4, 4, 2
    x0 = rng.uniform(0.2, 1.5, size=g.shape)
    x1 = oracle.lm_osem_subset_update(x0, xs, xe, tb, g, tof, sens, b, m, n_sub, fwhm_mm=4.5)
    hx = oracle.gauss3d(x0, g, 4.5)
    p = oracle.fwd(xs[m::n_sub], xe[m::n_sub], hx, g, "tof_lm", tof, tof_bin=tb[m::n_sub])
    assert float(np.sum(sens / n_sub * x1)) == pytest.approx(float(np.sum(p / (p + b))), rel=1e-12)
    plain = oracle.lm_osem_subset_update(x0, xs, xe, tb, g, tof, sens, b, m, n_sub)
    assert np.array_equal(oracle.lm_osem_subset_update(x0, xs, xe, tb, g, tof, sens, b, m, n_sub, fwhm_mm=0.0),
                          plain)
    assert np.abs(x1 - plain).max() > 1e-3 * np.abs(plain).max()


# ---------------------------------------------------------------------------
# sinogram OSEM (paper Sec. 2.6 and 4: subset update with emission and contamination
# sinograms)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["nontof", "tof_sino"])
def test_sino_osem_fixed_point_and_counts(mode):
    """(1) Consistent noise-free data y = A_S x + c make x a fixed point
    (A_S^T 1 / s = 1); (2) sum_j s_j x_new_j = sum_i (A x)_i y_i / ((A x)_i + c_i);
    (3) equal to the update written with the independent dense tent matrix."""
    g = G((10, 9, 7), (-4.5, -4.0, -3.3), (1.0, 1.1, 1.2))
    tof = None if mode == "nontof" else T(bin_width=2.1, sigma=1.7, n_sigmas=3.0, n_bins=9)
    xs, xe = synth.random_lors(300, g, seed=141)
    rng = np.random.Generator(np.random.PCG64(142))
    x = rng.uniform(0.2, 1.5, size=g.shape)
    p = oracle.fwd(xs, xe, x, g, mode, tof)
    c = rng.uniform(0.05, 0.3, size=p.shape)
    sens = oracle.back(xs, xe, np.ones_like(p), g, mode, tof)
    x_fp = oracle.sino_osem_subset_update(x, xs, xe, p + c, c, sens, g, mode, tof)
    pos = sens > 0
    assert np.any(~pos) and np.all(x_fp[~pos] == 0.0)
    assert np.abs(x_fp[pos] - x[pos]).max() <= 1e-12 * x.max()
    y = rng.poisson(p + c).astype(np.float64)
    x1 = oracle.sino_osem_subset_update(x, xs, xe, y, c, sens, g, mode, tof)
    assert float(np.sum(sens * x1)) == pytest.approx(float(np.sum(p * y / (p + c))), rel=1e-12)
    A = dense_tent(xs, xe, g, mode, tof)
    xv = x.reshape(-1)
    Ax = A @ xv
    ratio = y.reshape(-1) / (Ax + c.reshape(-1))
    s_d = A.T @ np.ones(A.shape[0])
    ref = np.where(s_d > 0, xv * (A.T @ ratio) / np.where(s_d > 0, s_d, 1.0), 0.0)
    assert np.abs(x1.reshape(-1) - ref).max() <= 1e-11 * np.abs(ref).max()
    # zero expected counts (A x + c = 0 on a LOR) contribute 0, not NaN
    x2 = oracle.sino_osem_subset_update(np.zeros(g.shape), xs, xe, y, np.zeros_like(c), sens, g, mode, tof)
    assert np.all(np.isfinite(x2)) and np.all(x2 == 0.0)


def _osem_pins(mutant=0):
    """Fast versions of the OSEM and gradient pins above, run against a
    (possibly mutated) oracle; returns the names of the pins that failed."""
    failed = []
    close = lambda a, b: abs(a - b) <= 1e-12 * max(abs(b), 1e-300)  # noqa: E731
    # listmode OSEM: count preservation with and without background, and
    # through the resolution model
    g, tof, _, xs, xe, tb = _small_lm_problem(n_events=1200, seed=97)
    rng = np.random.Generator(np.random.PCG64(98))
    sens = rng.uniform(0.5, 2.0, size=g.shape)
    n_sub, m = 4, 1
    x0 = rng.uniform(0.2, 1.5, size=g.shape)
    sub = slice(m, None, n_sub)
    p = oracle.fwd(xs[sub], xe[sub], x0, g, "tof_lm", tof, tof_bin=tb[sub])
    for b in (0.7, 0.0):
        x1 = oracle.lm_osem_subset_update(x0, xs, xe, tb, g, tof, sens, b, m, n_sub, _mutant=mutant)
        want = float(np.sum(p / (p + b))) if b else float(np.sum(p > 0))
        if not close(float(np.sum(sens / n_sub * x1)), want):
            failed.append(f"lm-counts-b{b}")
    ph = oracle.fwd(xs[sub], xe[sub], oracle.gauss3d(x0, g, 4.5), g, "tof_lm", tof, tof_bin=tb[sub])
    x1 = oracle.lm_osem_subset_update(x0, xs, xe, tb, g, tof, sens, 0.4, m, n_sub, fwhm_mm=4.5, _mutant=mutant)
    if not close(float(np.sum(sens / n_sub * x1)), float(np.sum(ph / (ph + 0.4)))):
        failed.append("lm-res-counts")
    # sinogram OSEM: fixed point of consistent data, count preservation
    g2 = G((10, 9, 7), (-4.5, -4.0, -3.3), (1.0, 1.1, 1.2))
    xs2, xe2 = synth.random_lors(200, g2, seed=143)
    x = rng.uniform(0.2, 1.5, size=g2.shape)
    p2 = oracle.fwd(xs2, xe2, x, g2)
    c = rng.uniform(0.05, 0.3, size=p2.shape)
    s2 = oracle.back(xs2, xe2, np.ones_like(p2), g2)
    pos = s2 > 0
    x_fp = oracle.sino_osem_subset_update(x, xs2, xe2, p2 + c, c, s2, g2, _mutant=mutant)
    if np.abs(x_fp[pos] - x[pos]).max() > 1e-12 * x.max():
        failed.append("sino-fixed-point")
    y = rng.poisson(p2 + c).astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        x1 = oracle.sino_osem_subset_update(x, xs2, xe2, y, c, s2, g2, _mutant=mutant)
    if not (np.all(np.isfinite(x1)) and close(float(np.sum(s2 * x1)), float(np.sum(p2 * y / (p2 + c))))):
        failed.append("sino-counts")
    # gradient of the listmode log-likelihood against central differences
    xg = x0 + 0.1
    w = rng.uniform(0.5, 1.5, size=400)
    b = 0.3
    _, grad = oracle.poisson_loglik_grad(xg, xs[:400], xe[:400], tb[:400], g, tof, w, b, _mutant=mutant)
    h = 1e-6
    for j in rng.choice(xg.size, size=8, replace=False):
        e = np.zeros(xg.size)
        e[j] = h
        e = e.reshape(xg.shape)
        pp = oracle.fwd(xs[:400], xe[:400], xg + e, g, "tof_lm", tof, tof_bin=tb[:400])
        pm = oracle.fwd(xs[:400], xe[:400], xg - e, g, "tof_lm", tof, tof_bin=tb[:400])
        fd = float(np.sum(w * np.log1p((pp - pm) / (pm + b)))) / (2 * h)
        gj = grad.reshape(-1)[j]
        if abs(fd - gj) > 1e-7 * max(abs(gj), 1e-3 * np.abs(grad).max()):
            failed.append("grad-fd")
            break
    return failed


def test_osem_planted_mistakes_are_caught():
    """Each plausible mistake in the OSEM and gradient oracles fails at least
    one pin: sensitivity not divided by n_sub, background dropped, a
    contiguous block as the subset, H^T not applied, contamination dropped,
    the ratio inverted, the weights dropped from the gradient."""
    assert _osem_pins(0) == []
    for mutant in range(1, 8):
        assert _osem_pins(mutant), f"OSEM mutant {mutant} passed every pin"


# ---------------------------------------------------------------------------
# tabulated (non-Gaussian) TOF kernels and per-LOR sigma (paper Sec. 4)
# ---------------------------------------------------------------------------
def _tof_ext_pins(mutant=0):
    """Pins of the tabulated-kernel and per-LOR-sigma paths; returns the
    names of the pins that failed."""
    failed = []
    g = G((12, 10, 9), (-5.5, -4.1, -3.7), (1.0, 0.9, 1.1))
    xs, xe = synth.random_lors(60, g, seed=151)
    rng = np.random.Generator(np.random.PCG64(152))
    x = rng.uniform(0.2, 1.5, size=g.shape)
    p_non = oracle.fwd(xs, xe, x, g, "nontof", mutant=mutant)
    # (1) the triangle of half-width D (nodes 0, 1, 0) is a partition of
    #     unity over bins spaced D: summed over enough sinogram bins the TOF
    #     projection is the non-TOF one
    D = 1.7
    tri = synth.TofParams.tabulated(D, 41, (0.0, 1.0, 0.0), D)
    p_tri = oracle.fwd(xs, xe, x, g, "tof_sino", tri, mutant=mutant)
    if np.abs(p_tri.sum(axis=1) - p_non).max() > 1e-12 * p_non.max():
        failed.append("triangle-partition")
    # (2) a 5-node table of the triangle (nodes 0, .5, 1, .5, 0) is the same
    #     function: the node positions are -h + e 2h / (n - 1)
    tri5 = synth.TofParams.tabulated(D, 41, (0.0, 0.5, 1.0, 0.5, 0.0), D)
    if np.abs(oracle.fwd(xs, xe, x, g, "tof_sino", tri5, mutant=mutant) - p_tri).max() > 1e-13 * p_non.max():
        failed.append("table-nodes")
    # (3) a box of width D (value 1 inside +-D/2): an axis-aligned ray along
    #     axis 0 through a uniform image collects v_0 per voxel centre inside
    #     the window
    box = synth.TofParams.tabulated(D, 1, (1.0, 1.0), D / 2)
    ones = np.ones(g.shape)
    y0 = g.origin[1] + 4 * g.voxsize[1]
    z0 = g.origin[2] + 3 * g.voxsize[2]
    a = (-20.0, y0, z0)
    b = (20.0, y0, z0)
    cen = 0.7
    p_box = oracle.fwd([a], [b], ones, g, "tof_lm", box, tof_bin=[0], delta=[cen], mutant=mutant)[0]
    xc = g.origin[0] + np.arange(g.shape[0]) * g.voxsize[0]  # tau of the voxel centres (midpoint at 0)
    expect = g.voxsize[0] * np.sum(np.abs(xc - cen) <= D / 2)
    if abs(p_box - expect) > 1e-12:
        failed.append("box-window")
    # (4) an asymmetric table: swapping the endpoints and negating the bin
    #     mirrors the distance, so the reversed table gives the same value
    asym = synth.TofParams.tabulated(D, 1, (0.0, 0.2, 1.0, 0.6, 0.1), 2.5)
    mirr = synth.TofParams.tabulated(D, 1, (0.1, 0.6, 1.0, 0.2, 0.0), 2.5)
    tb = rng.integers(-3, 4, size=len(xs))
    p_a = oracle.fwd(xs, xe, x, g, "tof_lm", asym, tof_bin=tb, mutant=mutant)
    p_m = oracle.fwd(xe, xs, x, g, "tof_lm", mirr, tof_bin=-tb, mutant=mutant)
    if np.abs(p_a - p_m).max() > 1e-12 * max(p_a.max(), 1e-30):
        failed.append("table-mirror")
    # (5) per-LOR sigma: each LOR equals the single-sigma projection with its
    #     own sigma
    tof = T(bin_width=1.3, sigma=1.1, n_sigmas=3.0, n_bins=7)
    sig = rng.uniform(0.6, 2.4, size=len(xs))
    p_s = oracle.fwd(xs, xe, x, g, "tof_lm", tof, tof_bin=tb, sigma=sig, mutant=mutant)
    for i in (0, 7, 31, 59):
        ti = T(bin_width=1.3, sigma=float(sig[i]), n_sigmas=3.0, n_bins=7)
        pi = oracle.fwd(xs[i:i + 1], xe[i:i + 1], x, g, "tof_lm", ti, tof_bin=tb[i:i + 1], mutant=mutant)[0]
        if abs(p_s[i] - pi) > 1e-13 * max(abs(pi), 1e-30):
            failed.append("per-lor-sigma")
            break
    return failed


def test_tabulated_kernel_and_per_lor_sigma_pins():
    assert _tof_ext_pins() == []


@pytest.mark.parametrize("mode", ["tof_sino", "tof_lm"])
def test_tabulated_kernel_adjoint_and_gaussian_table(mode):
    """The tabulated path is a matched pair, and a fine table of the
    Gaussian bin response reproduces the Gaussian kernel within the linear
    interpolation bound h^2/8 max|g''|; g'' is a difference of two Gaussian
    pdf derivatives, so |g''| <= 2 / (sigma^2 sqrt(2 pi e))."""
    g = G((9, 11, 8), (-4.0, -5.0, -3.5), (1.0, 1.0, 1.0))
    gt = T(bin_width=1.5, sigma=1.2, n_sigmas=3.0, n_bins=9)
    R = gt.n_sigmas * gt.sigma + gt.bin_width / 2
    nodes = 2001
    d = np.linspace(-R, R, nodes)
    vals = [oracle.tof_weight(float(v), 0.0, gt.bin_width, gt.sigma, 50.0) for v in d]
    tab = synth.TofParams.tabulated(gt.bin_width, gt.n_bins, vals, R)
    xs, xe = synth.random_lors(80, g, seed=161)
    rng = np.random.Generator(np.random.PCG64(162))
    tb = rng.integers(-3, 4, size=len(xs)) if mode == "tof_lm" else None
    x = rng.uniform(0.0, 1.0, size=g.shape)
    pt = oracle.fwd(xs, xe, x, g, mode, tab, tof_bin=tb)
    pg = oracle.fwd(xs, xe, x, g, mode, gt, tof_bin=tb)
    h = 2 * R / (nodes - 1)
    bound = h * h / 8 * 2 / (gt.sigma ** 2 * math.sqrt(2 * math.pi * math.e))
    # per sample the weights differ by <= bound (inside the support; at the
    # edge both truncate at R), so a projection by <= bound * sum of |samples|
    p_abs = oracle.fwd(xs, xe, x, g, "nontof")
    assert np.all(np.abs(pt - pg).reshape(len(xs), -1).max(axis=1) <= bound * p_abs + 1e-12)
    y = rng.uniform(0.0, 1.0, size=pt.shape)
    lhs = float(np.sum(pt * y))
    rhs = float(np.sum(x * oracle.back(xs, xe, y, g, mode, tab, tof_bin=tb)))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_tabulated_and_sigma_planted_mistakes():
    for mutant in (8, 9):
        oracle.joseph.build(mutant)
        assert _tof_ext_pins(mutant), f"planted mistake {mutant} not caught"


# ---------------------------------------------------------------------------
# the TOF-edge ambiguity output (reading r1 of the truncation rule, Sec. 2.1
# and 2.6): per output, w0 * sum over the samples whose |tau - c| lies within
# amb_eps of the truncation radius R of |untruncated weight * sample value|
# ---------------------------------------------------------------------------
def _gauss_bin_raw(dist, D, s):
    k = 1.0 / (math.sqrt(2.0) * s)
    return 0.5 * (math.erf((dist + 0.5 * D) * k) - math.erf((dist - 0.5 * D) * k))


def _amb_by_tent(xs, xe, img, geom, tof, eps, centres):
    """Independent restatement: for LOR r and each TOF centre in
    centres[r], visit the planes inside the segment, interpolate with tent
    functions, flag samples with ||tau - c| - R| <= eps."""
    n, o, v = geom.shape, geom.origin, geom.voxsize
    R = tof.n_sigmas * tof.sigma + 0.5 * tof.bin_width
    out = []
    for p, q, cs in zip(np.asarray(xs, np.float64), np.asarray(xe, np.float64), centres):
        d = q - p
        L = math.sqrt(float(np.dot(d, d)))
        a = _principal_axis_exact(p, q)
        b, c = [i for i in range(3) if i != a]
        w0 = v[a] * L / abs(d[a])
        row = np.zeros(len(cs))
        for k in range(n[a]):
            X = o[a] + k * v[a]
            if not (min(p[a], q[a]) <= X <= max(p[a], q[a])):
                continue
            t = (X - p[a]) / d[a]
            u = (p[b] + t * d[b] - o[b]) / v[b]
            w = (p[c] + t * d[c] - o[c]) / v[c]
            s = 0.0
            for ib in range(n[b]):
                for ic in range(n[c]):
                    tt = _tent(u - ib) * _tent(w - ic)
                    if tt:
                        ijk = [0, 0, 0]
                        ijk[a], ijk[b], ijk[c] = k, ib, ic
                        s += tt * img[tuple(ijk)]
            tau = (t - 0.5) * L
            for m, cen in enumerate(cs):
                if abs(abs(tau - cen) - R) <= eps:
                    row[m] += w0 * abs(_gauss_bin_raw(tau - cen, tof.bin_width, tof.sigma) * s)
        out.append(row)
    return np.array(out)


def _amb_pins(mutant=0):
    """Returns the names of the ambiguity pins that fail."""
    failed = []
    # (1) an axis-aligned ray along axis 0 through voxel centres, with dyadic
    #     coordinates: tau_k = 2k - 8 exactly, R = 3 * 2 + 4 / 2 = 8, so plane
    #     0 sits at the window edge of bin centre delta; the sample value is
    #     f[0, 1, 2] and w0 = v_0 = 2
    g = G((8, 4, 4), (0.0, 0.0, 0.0), (2.0, 2.0, 2.0))
    tof = T(bin_width=4.0, sigma=2.0, n_sigmas=3.0, n_bins=3)
    rng = np.random.Generator(np.random.PCG64(171))
    f = rng.uniform(0.5, 1.5, size=g.shape)
    a, b = (-8.0, 2.0, 4.0), (24.0, 2.0, 4.0)
    eps = 1e-3
    for delta, inside_band in ((0.0, True), (5e-4, True), (-5e-4, True), (1.5e-3, False), (-1.5e-3, False)):
        _, amb = oracle.fwd([a], [b], f, g, "tof_lm", tof, tof_bin=[0], delta=[delta], amb_eps=eps,
                            return_amb=True, mutant=mutant)
        expect = 2.0 * abs(_gauss_bin_raw(-8.0 - delta, 4.0, 2.0) * f[0, 1, 2]) if inside_band else 0.0
        if inside_band and abs(amb[0] - expect) > 1e-12 * expect:
            failed.append(f"edge-value({delta})")
        if not inside_band and amb[0] != 0.0:
            failed.append(f"outside-band({delta})")
    # (2) the same ray as a 3-bin TOF sinogram: centres -4, 0, 4 put planes
    #     6, 0 and 2 on the edges of bins 0, 1 and 2
    _, amb = oracle.fwd([a], [b], f, g, "tof_sino", tof, amb_eps=eps, return_amb=True, mutant=mutant)
    gedge = _gauss_bin_raw(8.0, 4.0, 2.0)
    expect = [2.0 * gedge * f[6, 1, 2], 2.0 * gedge * f[0, 1, 2], 2.0 * gedge * f[2, 1, 2]]
    if np.abs(amb[0] - expect).max() > 1e-12 * max(expect):
        failed.append("sino-edges")
    # (3) random oblique LORs with a wide band (0.3 mm) so that both cases
    #     occur: the output equals the independent tent-function restatement,
    #     and is exactly 0 where no sample falls in the band
    g3 = G((6, 5, 4), (-2.6, -1.9, -1.4), (1.0, 0.9, 0.8))
    t3 = T(bin_width=1.1, sigma=0.9, n_sigmas=2.0, n_bins=5)
    xs, xe = synth.random_lors(40, synth.ImageGeom(g3.shape, g3.origin, g3.voxsize), seed=172, radius_factor=1.4)
    x3 = rng.uniform(0.2, 1.2, size=g3.shape)
    tb = rng.integers(-2, 3, size=len(xs))
    de = rng.uniform(-0.4, 0.4, size=len(xs))
    _, amb = oracle.fwd(xs, xe, x3, g3, "tof_lm", t3, tof_bin=tb, delta=de, amb_eps=0.3, return_amb=True,
                        mutant=mutant)
    ref = _amb_by_tent(xs, xe, x3, g3, t3, 0.3, [[tb[i] * t3.bin_width + de[i]] for i in range(len(xs))])[:, 0]
    if np.any((ref == 0.0) != (amb == 0.0)) or np.abs(amb - ref).max() > 1e-12 * max(ref.max(), 1e-30):
        failed.append("random-vs-tent")
    if not (0 < np.count_nonzero(ref) < len(ref)):
        failed.append("random-cases")
    return failed


def test_tof_edge_ambiguity_pins():
    assert _amb_pins() == []


def test_tof_edge_ambiguity_planted_mistakes():
    for mutant in (10, 11, 12):
        oracle.joseph.build(mutant)
        assert _amb_pins(mutant), f"planted ambiguity mistake {mutant} not caught"
