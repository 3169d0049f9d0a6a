"""Seeded synthetic inputs: scanner LORs, phantoms, listmode events.

This module is shared by the CUDA path's tests/benchmarks and by the FP64
oracle's tests.  It holds none of the projector's arithmetic (no plane
stepping, no interpolation, no TOF kernel): it only places detectors, draws
phantoms and simulates emissions.  Seeds follow ``1000 * workload + purpose``.

Workloads (the paper's benchmark shapes, Sec. 2.6, rebuilt on synthetic data):

* ``small``: 8 rings x 128 crystals on R = 150 mm, 64 planes x 64 views x 65
  radial bins (266,240 LORs), image 64x64x16 @ 2 mm.
* ``clinical``: 36 rings x 672 crystals on R = 400 mm, 1296 planes x 336 views
  x 313 radial bins (136,297,728 LORs), image 200x200x71 @ 2 mm.
* ``tof_sino``: the clinical scanner with every 2nd view (168 views), 29 TOF
  bins of 28 mm, FWHM 57.7 mm, truncated at 3 sigma.
* ``tof_lm``: 8 clinical-size phantoms x 40M TOF listmode events each.
* ``osem_stream``: served LM-OSEM frames of log-uniform 1e5..2e7 events.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np
import torch


# --------------------------------------------------------------------------
# geometry containers
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class ImageGeom:
    """Voxel grid: ``shape`` (n0, n1, n2), C order (axis 2 fastest).

    ``origin`` is the world coordinate (mm) of the centre of voxel (0,0,0);
    ``voxsize`` may be non-isotropic (Sec. 2.6 notes non-isotropic support).
    """

    shape: Tuple[int, int, int]
    origin: Tuple[float, float, float]
    voxsize: Tuple[float, float, float]

    @staticmethod
    def centred(shape: Sequence[int], voxsize: Sequence[float]) -> "ImageGeom":
        shape = tuple(int(s) for s in shape)
        vox = tuple(float(v) for v in voxsize)
        origin = tuple(float(-(n - 1) / 2.0 * v) for n, v in zip(shape, vox))
        return ImageGeom(shape, origin, vox)

    @property
    def numel(self) -> int:
        return int(np.prod(self.shape))

    def voxel_centres(self, device="cpu", dtype=torch.float64):
        axes = [torch.arange(n, device=device, dtype=dtype) * v + o
                for n, v, o in zip(self.shape, self.voxsize, self.origin)]
        return torch.meshgrid(*axes, indexing="ij")


@dataclass(frozen=True)
class TofParams:
    """TOF kernel parameters (Sec. 2.1 and 2.6): bin width (mm), Gaussian
    sigma (mm), truncation in sigmas, number of sinogram TOF bins.

    ``kernel`` optionally replaces the Gaussian by a tabulated bin response
    (Sec. 4: a 1D lookup table for non-Gaussian TOF kernels): the values at
    the distances -h + e 2h / (len - 1) from the bin centre, h =
    ``kernel_half_width``, linearly interpolated, 0 beyond h."""

    bin_width: float
    sigma: float
    n_sigmas: float
    n_bins: int
    kernel: Optional[Tuple[float, ...]] = None
    kernel_half_width: float = 0.0

    @staticmethod
    def from_fwhm(bin_width: float, fwhm: float, n_sigmas: float, n_bins: int) -> "TofParams":
        return TofParams(float(bin_width), float(fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))),
                         float(n_sigmas), int(n_bins))

    @staticmethod
    def tabulated(bin_width: float, n_bins: int, values: Sequence[float], half_width: float) -> "TofParams":
        """A non-Gaussian TOF kernel given by its table (sigma, n_sigmas unused)."""
        vals = tuple(float(v) for v in values)
        if len(vals) < 2:
            raise ValueError("a TOF kernel table needs at least 2 nodes")
        return TofParams(float(bin_width), 0.0, 0.0, int(n_bins), vals, float(half_width))


@dataclass(frozen=True)
class Scanner:
    """Cylindrical scanner: crystal c of ring r sits at
    (R cos 2 pi c/n_c, R sin 2 pi c/n_c, (r - (n_r-1)/2) * ring_spacing)."""

    radius: float
    n_crystals: int
    n_rings: int
    ring_spacing: float

    def crystal_xyz(self, device="cpu") -> torch.Tensor:
        c = torch.arange(self.n_crystals, device=device, dtype=torch.float64)
        r = torch.arange(self.n_rings, device=device, dtype=torch.float64)
        phi = 2.0 * math.pi * c / self.n_crystals
        x = (self.radius * torch.cos(phi))[None, :].expand(self.n_rings, -1)
        y = (self.radius * torch.sin(phi))[None, :].expand(self.n_rings, -1)
        z = ((r - (self.n_rings - 1) / 2.0) * self.ring_spacing)[:, None].expand(-1, self.n_crystals)
        return torch.stack([x, y, z], dim=-1)  # [n_rings, n_crystals, 3]

    @property
    def half_axial(self) -> float:
        return (self.n_rings / 2.0) * self.ring_spacing

    def crystal_table(self, device="cpu") -> torch.Tensor:
        """float32 [n_rings * n_crystals, 3] detector coordinates; detector
        index r * n_crystals + c (the listmode events' index form)."""
        return self.crystal_xyz(device).reshape(-1, 3).to(torch.float32).contiguous()


# --------------------------------------------------------------------------
# workload definitions
# --------------------------------------------------------------------------
TOF_CLINICAL = TofParams.from_fwhm(bin_width=28.0, fwhm=57.7, n_sigmas=3.0, n_bins=29)

SCANNER_SMALL = Scanner(radius=150.0, n_crystals=128, n_rings=8, ring_spacing=4.0)
SCANNER_CLINICAL = Scanner(radius=400.0, n_crystals=672, n_rings=36, ring_spacing=4.0)

GEOM_SMALL = ImageGeom.centred((64, 64, 16), (2.0, 2.0, 2.0))
GEOM_CLINICAL = ImageGeom.centred((200, 200, 71), (2.0, 2.0, 2.0))
GEOM_OSEM_SMALL = ImageGeom.centred((128, 128, 71), (2.0, 2.0, 2.0))


@dataclass(frozen=True)
class SinoSpec:
    scanner: Scanner
    n_views: int
    n_rad: int
    view_step: int = 1  # 2 keeps every 2nd view (TOF sinogram workload)
    view_start: int = 0

    @property
    def n_planes(self) -> int:
        return self.scanner.n_rings ** 2

    @property
    def views(self) -> np.ndarray:
        return np.arange(self.view_start, self.n_views, self.view_step)

    def subset(self, m: int, n_sub: int) -> "SinoSpec":
        """Views m, m + n_sub, m + 2 n_sub, ... of this sinogram's views: the
        equally spaced view subsets of sinogram OSEM (paper Sec. 2.6)."""
        return SinoSpec(self.scanner, self.n_views, self.n_rad, self.view_step * n_sub,
                        self.view_start + m * self.view_step)

    @property
    def n_lor(self) -> int:
        return self.n_planes * len(self.views) * self.n_rad


SINO_SMALL = SinoSpec(SCANNER_SMALL, n_views=64, n_rad=65)
SINO_CLINICAL = SinoSpec(SCANNER_CLINICAL, n_views=336, n_rad=313)
SINO_TOF = SinoSpec(SCANNER_CLINICAL, n_views=336, n_rad=313, view_step=2)


# --------------------------------------------------------------------------
# sinogram LORs
# --------------------------------------------------------------------------
SINO_ORDERS = ("PVR", "VRP", "RVP")


def sinogram_lors(spec: SinoSpec, device="cpu", plane_range: Optional[Tuple[int, int]] = None,
                  order: str = "PVR"):
    """Crystal-centre endpoints of every LOR of a span-1 sinogram.

    Mapping (view v, radial index rho in [-(n_rad-1)/2, (n_rad-1)/2]):
    c1 = (v + floor(rho/2)) mod n_c, c2 = (v - ceil(rho/2) + n_c/2) mod n_c;
    plane = r1 * n_rings + r2 over all ring pairs.  ``order`` names the flat
    memory order from the slowest to the fastest axis (paper Sec. 2.6): "PVR"
    (default) is plane-major, then view, then radial (radial fastest); "VRP"
    has the plane fastest and the view slowest; "RVP" the radial slowest and
    the plane fastest.  Returns float32 (xs, xe) [n, 3].  ``plane_range``
    restricts to planes [p0, p1) (for chunked generation).
    """
    sc = spec.scanner
    xyz = sc.crystal_xyz(device)  # [R, C, 3] float64
    nc = sc.n_crystals
    views = torch.as_tensor(spec.views, device=device, dtype=torch.int64)
    rho = torch.arange(spec.n_rad, device=device, dtype=torch.int64) - (spec.n_rad - 1) // 2
    c1 = torch.remainder(views[:, None] + torch.div(rho, 2, rounding_mode="floor")[None, :], nc)
    c2 = torch.remainder(views[:, None] - (-torch.div(-rho, 2, rounding_mode="floor"))[None, :] + nc // 2, nc)
    p0, p1 = (0, spec.n_planes) if plane_range is None else plane_range
    planes = torch.arange(p0, p1, device=device, dtype=torch.int64)
    r1 = torch.div(planes, sc.n_rings, rounding_mode="floor")
    r2 = planes - r1 * sc.n_rings
    xs = xyz[r1[:, None, None], c1[None, :, :]]  # [P, V, R, 3]
    xe = xyz[r2[:, None, None], c2[None, :, :]]
    if order not in SINO_ORDERS:
        raise ValueError(f"order must be one of {SINO_ORDERS}")
    perm = {"PVR": (0, 1, 2, 3), "VRP": (1, 2, 0, 3), "RVP": (2, 1, 0, 3)}[order]
    xs, xe = xs.permute(*perm), xe.permute(*perm)
    return (xs.reshape(-1, 3).to(torch.float32).contiguous(),
            xe.reshape(-1, 3).to(torch.float32).contiguous())


def symmetry_axis(geom: "ImageGeom", xs: torch.Tensor, xe: torch.Tensor, axis: int):
    """Places the scanner's axial direction (z) on image axis ``axis`` (paper
    Sec. 2.6, "symmetry axis" 0/1/2; 2 = axial fastest in memory, the default
    of the other generators): permutes the image geometry and the LOR
    coordinates alike, so projections equal those of axis 2 up to the voxel
    permutation.  Returns (geom, xs, xe)."""
    if axis not in (0, 1, 2):
        raise ValueError("axis must be 0, 1 or 2")
    order = {2: (0, 1, 2), 0: (2, 0, 1), 1: (0, 2, 1)}[axis]
    g = ImageGeom(tuple(geom.shape[i] for i in order), tuple(geom.origin[i] for i in order),
                  tuple(geom.voxsize[i] for i in order))
    return g, xs[:, list(order)].contiguous(), xe[:, list(order)].contiguous()


# --------------------------------------------------------------------------
# phantoms
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class PhantomSpec:
    semi_axes: Tuple[float, float, float]
    radii: Tuple[float, ...]
    background: float = 1.0
    hot: float = 4.0


PHANTOM_SMALL = PhantomSpec((50.0, 40.0, 12.0), (5.0, 5.0, 5.0))
PHANTOM_CLINICAL = PhantomSpec((250.0, 180.0, 65.0), tuple(np.linspace(4.0, 12.0, 8)))
PHANTOM_OSEM_SMALL = PhantomSpec((160.0, 115.0, 65.0), tuple(np.linspace(4.0, 12.0, 8)))


def ellipsoid_phantom(geom: ImageGeom, spec: PhantomSpec, seed: int, device="cpu") -> torch.Tensor:
    """Uniform ellipsoid (value ``background``) sampled at voxel centres, with
    spheres of value ``hot`` replacing the values inside them.  Sphere centres
    are seeded-uniform inside the ellipsoid shrunk by the sphere radius."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ax = np.asarray(spec.semi_axes, dtype=np.float64)
    centres = []
    for r in spec.radii:
        inner = np.maximum(ax - r, 1e-3)
        while True:
            p = rng.uniform(-1.0, 1.0, size=3)
            if np.sum(p * p) <= 1.0:
                centres.append(p * inner)
                break
    X, Y, Z = geom.voxel_centres(device)
    img = torch.zeros(geom.shape, dtype=torch.float64, device=device)
    inside = (X / ax[0]) ** 2 + (Y / ax[1]) ** 2 + (Z / ax[2]) ** 2 <= 1.0
    img[inside] = spec.background
    for c, r in zip(centres, spec.radii):
        m = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r
        img[m] = spec.hot
    return img.to(torch.float32).contiguous()


def background_level(phantom: torch.Tensor, tof: TofParams, fraction: float = 0.1) -> float:
    """Per-frame additive background b used by the LM-OSEM workloads.

    Stands for ``fraction * mean_e (A x)_e`` without running a projector: a
    TOF listmode event inside a uniform region of activity xbar integrates the
    TOF bin kernel (area = bin width) along the LOR, giving xbar * bin_width.
    xbar is the mean phantom value over its support."""
    sup = phantom[phantom > 0]
    xbar = float(sup.double().mean()) if sup.numel() else 0.0
    return float(fraction * xbar * tof.bin_width)


# --------------------------------------------------------------------------
# listmode events (Monte-Carlo emission + detection)
# --------------------------------------------------------------------------
def lm_events(phantom: torch.Tensor, geom: ImageGeom, scanner: Scanner, tof: TofParams,
              n_events: int, seed: int, device="cpu", chunk: int = 1 << 22, return_det: bool = False):
    """TOF listmode events drawn by simulating emissions in the phantom.

    1. emission point: voxel drawn with probability proportional to its value,
       uniform jitter inside the voxel;
    2. isotropic direction (restricted to the band of polar angles that can
       reach the detector), both cylinder intersections must lie within the
       axial extent; endpoints snap to the nearest crystal centres, so a crystal
       pair is detected with probability proportional to the activity along it;
    3. TOF: tau_emit = (E - m) . u along the crystal LOR (m its midpoint, u its
       unit vector), tau_meas = tau_emit + N(0, sigma^2), signed bin
       t = round(tau_meas / bin_width), events with |t| > (n_bins-1)/2 dropped;
    4. the endpoints are swapped with probability 1/2 (negating t).

    Returns float32 xs, xe [n, 3] and int16 signed TOF bins [n] on ``device``;
    with ``return_det`` also the int32 detector indices [n] of the two
    endpoints (r * n_crystals + c, so xs == scanner.crystal_table()[ds]).
    """
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    dev = torch.device(device)
    w = phantom.to(dev).reshape(-1).double()
    cdf = torch.cumsum(w, 0)
    total = float(cdf[-1])
    if total <= 0:
        raise ValueError("phantom has no activity")
    n0, n1, n2 = geom.shape
    vox = torch.tensor(geom.voxsize, dtype=torch.float64, device=dev)
    org = torch.tensor(geom.origin, dtype=torch.float64, device=dev)
    xyz = scanner.crystal_xyz(dev)
    R = scanner.radius
    nc, nr = scanner.n_crystals, scanner.n_rings
    zext = scanner.half_axial
    # max |u_z| of a direction that can hit the detector on both sides from a
    # point inside the image's bounding cylinder
    half = torch.tensor([(n - 1) / 2.0 * v + v / 2.0 for n, v in zip(geom.shape, geom.voxsize)])
    rmax = float(torch.sqrt(half[0] ** 2 + half[1] ** 2))
    chord = 2.0 * math.sqrt(max(R * R - rmax * rmax, 1.0))
    slope = (2.0 * zext) / chord
    cmax = min(1.0, 1.05 * slope / math.sqrt(1.0 + slope * slope))
    hmax = (tof.n_bins - 1) // 2

    outs_s, outs_e, outs_t, outs_ds, outs_de = [], [], [], [], []
    got = 0
    while got < n_events:
        m = chunk
        u0 = torch.rand(m, generator=gen, device=dev, dtype=torch.float64) * total
        idx = torch.searchsorted(cdf, u0, right=True).clamp_(max=w.numel() - 1)
        i0 = torch.div(idx, n1 * n2, rounding_mode="floor")
        rem = idx - i0 * n1 * n2
        i1 = torch.div(rem, n2, rounding_mode="floor")
        i2 = rem - i1 * n2
        ijk = torch.stack([i0, i1, i2], 1).double()
        jit = torch.rand(m, 3, generator=gen, device=dev, dtype=torch.float64) - 0.5
        E = org + (ijk + jit) * vox
        cz = (torch.rand(m, generator=gen, device=dev, dtype=torch.float64) * 2.0 - 1.0) * cmax
        ph = torch.rand(m, generator=gen, device=dev, dtype=torch.float64) * (2.0 * math.pi)
        sz = torch.sqrt(1.0 - cz * cz)
        ux, uy, uz = sz * torch.cos(ph), sz * torch.sin(ph), cz
        a = ux * ux + uy * uy
        bq = 2.0 * (E[:, 0] * ux + E[:, 1] * uy)
        cq = E[:, 0] ** 2 + E[:, 1] ** 2 - R * R
        disc = torch.sqrt(torch.clamp(bq * bq - 4.0 * a * cq, min=0.0))
        tp = (-bq + disc) / (2.0 * a)
        tm = (-bq - disc) / (2.0 * a)
        P1 = E + tp[:, None] * torch.stack([ux, uy, uz], 1)
        P2 = E + tm[:, None] * torch.stack([ux, uy, uz], 1)

        def snap(P):
            phi = torch.atan2(P[:, 1], P[:, 0])
            c = torch.remainder(torch.round(phi * nc / (2.0 * math.pi)).long(), nc)
            r = torch.round(P[:, 2] / scanner.ring_spacing + (nr - 1) / 2.0).long()
            return c, r

        c1, r1 = snap(P1)
        c2, r2 = snap(P2)
        ok = (r1 >= 0) & (r1 < nr) & (r2 >= 0) & (r2 < nr) & (c1 != c2)
        ok &= (P1[:, 2].abs() <= zext) & (P2[:, 2].abs() <= zext)
        r1c, r2c = r1.clamp(0, nr - 1), r2.clamp(0, nr - 1)
        xs = xyz[r1c, c1]
        xe = xyz[r2c, c2]
        d = xe - xs
        L = torch.linalg.norm(d, dim=1).clamp_min(1e-12)
        uu = d / L[:, None]
        mid = 0.5 * (xs + xe)
        tau = ((E - mid) * uu).sum(1)
        tau = tau + tof.sigma * torch.randn(m, generator=gen, device=dev, dtype=torch.float64)
        t = torch.round(tau / tof.bin_width).long()
        ok &= t.abs() <= hmax
        swap = torch.rand(m, generator=gen, device=dev) < 0.5
        xs2 = torch.where(swap[:, None], xe, xs)
        xe2 = torch.where(swap[:, None], xs, xe)
        t2 = torch.where(swap, -t, t)
        d1, d2 = r1c * nc + c1, r2c * nc + c2
        sel = torch.nonzero(ok).squeeze(1)
        take = min(int(sel.numel()), n_events - got)
        sel = sel[:take]
        outs_s.append(xs2[sel].float())
        outs_e.append(xe2[sel].float())
        outs_t.append(t2[sel].to(torch.int16))
        if return_det:
            outs_ds.append(torch.where(swap, d2, d1)[sel].to(torch.int32))
            outs_de.append(torch.where(swap, d1, d2)[sel].to(torch.int32))
        got += take
    out = (torch.cat(outs_s).contiguous(), torch.cat(outs_e).contiguous(), torch.cat(outs_t).contiguous())
    if return_det:
        out = out + (torch.cat(outs_ds).contiguous(), torch.cat(outs_de).contiguous())
    return out


def loss_weights(n: int, seed: int, device="cpu") -> torch.Tensor:
    """Per-event loss weights w ~ U(0.5, 1.5) (float32)."""
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    return (torch.rand(n, generator=gen, device=device) + 0.5).contiguous()


# --------------------------------------------------------------------------
# generic random LORs for tests
# --------------------------------------------------------------------------
def random_lors(n: int, geom: ImageGeom, seed: int, radius_factor: float = 1.3,
                kind: str = "sphere"):
    """Random oblique LORs for tests (numpy float32 [n,3] x 2).

    ``sphere``: both endpoints uniform on a sphere enclosing the image (every
    plane the line crosses inside the image lies between the endpoints).
    ``inside``: endpoints uniform inside the image box (partial rays).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    half = np.array([(n_ - 1) / 2.0 * v + v / 2.0 for n_, v in zip(geom.shape, geom.voxsize)])
    centre = np.array(geom.origin) + np.array([(n_ - 1) / 2.0 * v for n_, v in zip(geom.shape, geom.voxsize)])
    if kind == "sphere":
        R = radius_factor * float(np.linalg.norm(half))
        def pts():
            v = rng.normal(size=(n, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            return centre + R * v
        xs, xe = pts(), pts()
    elif kind == "inside":
        xs = centre + rng.uniform(-1, 1, size=(n, 3)) * half
        xe = centre + rng.uniform(-1, 1, size=(n, 3)) * half
    else:
        raise ValueError(kind)
    return xs.astype(np.float32), xe.astype(np.float32)


def uniform_values(shape, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


def poisson_values(shape, seed: int, lam: float = 2.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.poisson(lam, size=shape).astype(np.float32)
