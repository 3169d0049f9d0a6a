// Joseph forward and back projection kernels (paper Sec. 2.1, 2.2).
//
// One thread follows one LOR plane by plane along its principal axis
// (steps a2-a6 of the hot path):
//   a2  per-LOR setup (exact principal axis, plane range, affine maps in
//       voxel units anchored at the centre plane so every sample is one FMA
//       from a small anchor value, never a long running sum);
//   a3  forward: bilinear interpolation of the 4 nearest voxels through
//       read-only (L1/L2-resident) loads, summed and scaled by v_a / cos_a;
//   a4  TOF weights as differences of erff at the bin edges (a TOF sinogram
//       shares each inner edge between two neighbouring bins, so W bins cost
//       W+1 erff; listmode evaluates only the planes of its TOF window);
//   a5  back projection: the transposed coefficients scattered with
//       fire-and-forget atomic adds (RED) into the image;
//   a6  planned calls read LORs in binned order and scatter/gather the
//       projection values through the plan's permutation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "jp_internal.cuh"

namespace jp {

int make_geom(const jp_image_geom* g, DevGeom* out) {
  if (!g) return fail(JP_ERR_ARG, "geometry is NULL");
  int64_t nv = 1;
  for (int i = 0; i < 3; ++i) {
    if (g->n[i] < 1) return fail(JP_ERR_ARG, "image shape must be >= 1 on every axis");
    if (!(g->voxsize[i] > 0.f) || !isfinite(g->voxsize[i])) return fail(JP_ERR_ARG, "voxel size must be finite and > 0");
    if (!isfinite(g->origin[i])) return fail(JP_ERR_ARG, "origin must be finite");
    nv *= g->n[i];
  }
  if (nv >= (int64_t)INT32_MAX) return fail(JP_ERR_ARG, "image has >= 2^31 voxels");
  for (int i = 0; i < 3; ++i) {
    out->n[i] = g->n[i];
    out->o[i] = g->origin[i];
    out->v[i] = g->voxsize[i];
    out->inv_v[i] = 1.0f / g->voxsize[i];
  }
  out->stride[0] = g->n[1] * g->n[2];
  out->stride[1] = g->n[2];
  out->stride[2] = 1;
  return JP_OK;
}

int make_tof(const jp_tof* t, bool sino, DevTof* out) {
  if (!t) return fail(JP_ERR_ARG, "TOF parameters are NULL");
  if (!(t->bin_width > 0.f) || !isfinite(t->bin_width)) return fail(JP_ERR_ARG, "TOF bin width must be finite and > 0");
  if (!(t->sigma > 0.f) || !isfinite(t->sigma)) return fail(JP_ERR_ARG, "TOF sigma must be finite and > 0");
  if (!(t->n_sigmas > 0.f) || !isfinite(t->n_sigmas)) return fail(JP_ERR_ARG, "TOF n_sigmas must be finite and > 0");
  if (sino && (t->n_bins < 1 || t->n_bins > JP_MAX_TOF_BINS))
    return fail(JP_ERR_ARG, "TOF n_bins must be in 1..JP_MAX_TOF_BINS");
  out->width = t->bin_width;
  out->half = 0.5f * t->bin_width;
  out->k = 1.0f / (1.41421356237309515f * t->sigma);
  out->R = t->n_sigmas * t->sigma + 0.5f * t->bin_width;
  out->R_over_w = out->R / t->bin_width;
  out->inv_w = 1.0f / t->bin_width;
  out->nbins = sino ? t->n_bins : 1;
  out->hbin = 0.5f * (float)(out->nbins - 1);
  return JP_OK;
}

namespace {

constexpr int kMaxBlock = 512;
constexpr int kLut = JP_TOF_TABLE;  // table nodes over [-R, R]

struct ProjParams {
  // planned source
  const float4* lor;
  const int32_t* perm;
  const int64_t* frame_off;
  int n_frames;
  // direct source
  const float* xs;
  const float* xe;
  const int16_t* tof_bin;
  const float* delta;
  int64_t n;
  int64_t img_stride;
  DevGeom g;
  DevTof tof;
  const float* img_in;
  float* proj_out;
  const float* proj_in;
  float* img_out;
  // planned workspace
  float4* quads;
  QuadLayout ql;
  const int32_t* axis_used;
  int shared;  // all frames use one image (img_stride == 0)
};

__device__ __forceinline__ int frame_of(const int64_t* __restrict__ off, int n_frames, int64_t i) {
  int lo = 0, hi = n_frames - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// TOF weight table: node e at dist = -R + e h, h = 2R / (kLut - 1); entry e
// holds (g_e, g_{e+1} - g_e) so a lookup is one 8-byte shared load and an FMA.
// The nodes are exact erf differences; linear interpolation between them is
// the table method of the TOF kernel mentioned in the paper's Sec. 4.
// ---------------------------------------------------------------------------
__device__ void build_lut(float2* lut, const DevTof& T) {
  const float h = 2.f * T.R / (float)(kLut - 1);
  for (int e = threadIdx.x; e < kLut - 1; e += blockDim.x) {
    float g0 = tof_g(fmaf((float)e, h, -T.R), T);
    float g1 = tof_g(fmaf((float)(e + 1), h, -T.R), T);
    lut[e] = make_float2(g0, g1 - g0);
  }
}

__device__ __forceinline__ float lut_g(const float2* lut, float dist, float R, float inv_h) {
  float x = (dist + R) * inv_h;
  x = fminf(fmaxf(x, 0.f), (float)(kLut - 1) - 1e-3f);
  int ix = (int)x;
  float fr = x - (float)ix;
  float2 e = lut[ix];
  return fmaf(fr, e.y, e.x);
}

template <bool LUT>
__device__ __forceinline__ float tof_weight(const float2* lut, float dist, const DevTof& T, float inv_h) {
  if (LUT) return lut_g(lut, dist, T.R, inv_h);
  return tof_g(dist, T);
}

// ---------------------------------------------------------------------------
// planned projection kernel: persistent CTAs over binned LORs, quad images
// ---------------------------------------------------------------------------
template <int MODE, bool BACK, bool LUT>
__global__ void __launch_bounds__(kMaxBlock) planned_kernel(const ProjParams p) {
  extern __shared__ float4 smem4[];
  float2* lut = reinterpret_cast<float2*>(smem4);
  float* accbase = reinterpret_cast<float*>(lut + ((MODE != 0 && LUT) ? kLut : 0));
  float* acc = accbase + threadIdx.x;  // TOF sinogram: acc[t * blockDim.x]
  const DevTof& T = p.tof;
  if (MODE != 0 && LUT) {
    build_lut(lut, T);
    __syncthreads();
  }
  const float inv_h = (MODE != 0) ? (float)(kLut - 1) / (2.f * T.R) : 0.f;
  const int N = T.nbins;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += step) {
    const float4 A = __ldg(p.lor + 2 * i);
    const float4 B = __ldg(p.lor + 2 * i + 1);
    const float xs[3] = {A.x, A.y, A.z};
    const float xe[3] = {B.x, B.y, B.z};
    const float delta = A.w;
    const int tbin = __float_as_int(B.w);
    const int64_t j = __ldg(p.perm + i);
    const int f = (p.n_frames > 1) ? frame_of(p.frame_off, p.n_frames, i) : 0;
    const int slot = p.shared ? 0 : f;
    Ray r;
    bool live = ray_setup(xs, xe, p.g, r);
    float d0 = 0.f;  // tau(kc) - c  (listmode)
    if (MODE == 2 && live) {
      const float c = (float)tbin * T.width + delta;
      d0 = r.tc - c;
      const float t1 = (-T.R - d0) / r.dt, t2 = (T.R - d0) / r.dt;
      const float lo = fmaxf(ceilf(r.kc + fminf(t1, t2)), (float)r.k0);
      const float hi = fminf(floorf(r.kc + fmaxf(t1, t2)), (float)r.k1);
      r.k0 = (int)lo;
      r.k1 = (int)hi;
      live = lo <= hi;
    }
    const int a = r.a;
    const int nc2 = sel3(a, p.ql.nc2[0], p.ql.nc2[1], p.ql.nc2[2]);
    const int plane = (int)sel3(a, p.ql.plane[0], p.ql.plane[1], p.ql.plane[2]);
    const int64_t qoff = (int64_t)slot * p.ql.slot + sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
    const float ub = (float)r.nb, wb = (float)r.nc;

    if (!BACK) {
      // ------------------------------ forward ------------------------------
      const float4* __restrict__ Q = p.quads + qoff;
      if (MODE == 1)
        for (int t = 0; t < N; ++t) acc[t * blockDim.x] = 0.f;
      float sum = 0.f;
      if (live) {
        for (int k = r.k0; k <= r.k1; ++k) {
          const float kk = (float)k - r.kc;
          const float u = fminf(fmaxf(fmaf(kk, r.du, r.uc), -1.f), ub);
          const float w = fminf(fmaxf(fmaf(kk, r.dw, r.wc), -1.f), wb);
          const float fu = floorf(u), fw = floorf(w);
          const float al = u - fu, be = w - fw;
          const float4 v = __ldg(Q + (k * plane + ((int)fu + 1) * nc2 + ((int)fw + 1)));
          const float top = fmaf(be, v.z - v.x, v.x);
          const float bot = fmaf(be, v.w - v.y, v.y);
          const float s = fmaf(al, bot - top, top);
          if (MODE == 0) {
            sum += s;
          } else if (MODE == 2) {
            sum = fmaf(tof_weight<LUT>(lut, fmaf(kk, r.dt, d0), T, inv_h), s, sum);
          } else {
            if (s == 0.f) continue;
            const float tau = fmaf(kk, r.dt, r.tc);
            const float x = (tau - delta) * T.inv_w + T.hbin;
            const int t0 = max(0, (int)ceilf(x - T.R_over_w));
            const int t1 = min(N - 1, (int)floorf(x + T.R_over_w));
            if (t0 > t1) continue;
            const float dlo = (tau - delta) - ((float)t0 - T.hbin) * T.width;
            if (LUT) {
              for (int t = t0; t <= t1; ++t) {
                const float dist = fmaf(-(float)(t - t0), T.width, dlo);
                acc[t * blockDim.x] = fmaf(lut_g(lut, dist, T.R, inv_h), s, acc[t * blockDim.x]);
              }
            } else {
              float e_hi = erff((dlo + T.half) * T.k);
              for (int t = t0; t <= t1; ++t) {
                const float dist = fmaf(-(float)(t - t0), T.width, dlo);
                const float e_lo = erff((dist - T.half) * T.k);
                acc[t * blockDim.x] = fmaf(0.5f * (e_hi - e_lo), s, acc[t * blockDim.x]);
                e_hi = e_lo;
              }
            }
          }
        }
      }
      if (MODE == 1) {
        float* out = p.proj_out + j * (int64_t)N;
        for (int t = 0; t < N; ++t) out[t] = live ? r.w0 * acc[t * blockDim.x] : 0.f;
      } else {
        p.proj_out[j] = live ? r.w0 * sum : 0.f;
      }
    } else {
      // ------------------------------ back --------------------------------
      if (!live) continue;
      float4* Q = p.quads + qoff;
      float val = r.w0;
      if (MODE == 1) {
        const float* yrow = p.proj_in + j * (int64_t)N;
        bool any = false;
        for (int t = 0; t < N; ++t) {
          const float y = __ldg(yrow + t);
          acc[t * blockDim.x] = y;
          any |= (y != 0.f);
        }
        if (!any) continue;
      } else {
        val *= __ldg(p.proj_in + j);
        if (val == 0.f) continue;
      }
      for (int k = r.k0; k <= r.k1; ++k) {
        const float kk = (float)k - r.kc;
        float coef;
        if (MODE == 0) {
          coef = val;
        } else if (MODE == 2) {
          coef = tof_weight<LUT>(lut, fmaf(kk, r.dt, d0), T, inv_h) * val;
        } else {
          const float tau = fmaf(kk, r.dt, r.tc);
          const float x = (tau - delta) * T.inv_w + T.hbin;
          const int t0 = max(0, (int)ceilf(x - T.R_over_w));
          const int t1 = min(N - 1, (int)floorf(x + T.R_over_w));
          if (t0 > t1) continue;
          const float dlo = (tau - delta) - ((float)t0 - T.hbin) * T.width;
          float sy = 0.f;
          if (LUT) {
            for (int t = t0; t <= t1; ++t) {
              const float dist = fmaf(-(float)(t - t0), T.width, dlo);
              sy = fmaf(lut_g(lut, dist, T.R, inv_h), acc[t * blockDim.x], sy);
            }
          } else {
            float e_hi = erff((dlo + T.half) * T.k);
            for (int t = t0; t <= t1; ++t) {
              const float dist = fmaf(-(float)(t - t0), T.width, dlo);
              const float e_lo = erff((dist - T.half) * T.k);
              sy = fmaf(0.5f * (e_hi - e_lo), acc[t * blockDim.x], sy);
              e_hi = e_lo;
            }
          }
          coef = sy * val;
        }
        if (coef == 0.f) continue;
        const float u = fminf(fmaxf(fmaf(kk, r.du, r.uc), -1.f), ub);
        const float w = fminf(fmaxf(fmaf(kk, r.dw, r.wc), -1.f), wb);
        const float fu = floorf(u), fw = floorf(w);
        const float al = u - fu, be = w - fw;
        const float ca = (1.f - al) * coef, cb = al * coef;
        atomicAdd(Q + (k * plane + ((int)fu + 1) * nc2 + ((int)fw + 1)),
                  make_float4(ca * (1.f - be), cb * (1.f - be), ca * be, cb * be));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// quad image build / clear / fold-back
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool slot_axis_used(const int32_t* used, int slot, int a, int shared, int n_frames) {
  if (!shared) return __ldg(used + 3 * slot + a) != 0;
  for (int f = 0; f < n_frames; ++f)
    if (__ldg(used + 3 * f + a)) return true;
  return false;
}

__global__ void quad_build_kernel(const ProjParams p) {
  const int slot = blockIdx.y / 3, a = blockIdx.y - 3 * (blockIdx.y / 3);
  if (!slot_axis_used(p.axis_used, slot, a, p.shared, p.n_frames)) return;
  const int b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
  const DevGeom& g = p.g;
  const int na = sel3(a, g.n[0], g.n[1], g.n[2]);
  const int nb = sel3(b, g.n[0], g.n[1], g.n[2]), nc = sel3(c, g.n[0], g.n[1], g.n[2]);
  const int sa = sel3(a, g.stride[0], g.stride[1], g.stride[2]);
  const int sb = sel3(b, g.stride[0], g.stride[1], g.stride[2]);
  const int sc = sel3(c, g.stride[0], g.stride[1], g.stride[2]);
  const int nc2 = nc + 2;
  const int64_t plane = (int64_t)(nb + 2) * nc2;
  const int64_t total = (int64_t)na * plane;
  const float* __restrict__ im = p.img_in + (int64_t)slot * p.img_stride;
  float4* Q = p.quads + (int64_t)slot * p.ql.slot + sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / plane);
    const int rem = (int)(e - (int64_t)k * plane);
    const int i = rem / nc2 - 1, jj = rem - (rem / nc2) * nc2 - 1;
    const bool i0 = (unsigned)i < (unsigned)nb, i1 = (unsigned)(i + 1) < (unsigned)nb;
    const bool j0 = (unsigned)jj < (unsigned)nc, j1 = (unsigned)(jj + 1) < (unsigned)nc;
    const int64_t base = (int64_t)k * sa + (int64_t)i * sb + (int64_t)jj * sc;
    float4 v;
    v.x = (i0 && j0) ? __ldg(im + base) : 0.f;
    v.y = (i1 && j0) ? __ldg(im + base + sb) : 0.f;
    v.z = (i0 && j1) ? __ldg(im + base + sc) : 0.f;
    v.w = (i1 && j1) ? __ldg(im + base + sb + sc) : 0.f;
    Q[e] = v;
  }
}

__global__ void quad_zero_kernel(const ProjParams p) {
  const int slot = blockIdx.y / 3, a = blockIdx.y - 3 * (blockIdx.y / 3);
  if (!slot_axis_used(p.axis_used, slot, a, p.shared, p.n_frames)) return;
  const int64_t total = (int64_t)sel3(a, p.g.n[0], p.g.n[1], p.g.n[2]) *
                        sel3(a, p.ql.plane[0], p.ql.plane[1], p.ql.plane[2]);
  float4* Q = p.quads + (int64_t)slot * p.ql.slot + sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Q[e] = z;
}

// img[slot] += sum over used axes of the 4 quad slots that hold each voxel
__global__ void quad_reduce_kernel(const ProjParams p) {
  const int slot = blockIdx.y;
  bool used[3];
  for (int a = 0; a < 3; ++a) used[a] = slot_axis_used(p.axis_used, slot, a, p.shared, p.n_frames);
  if (!used[0] && !used[1] && !used[2]) return;
  const DevGeom& g = p.g;
  const int64_t nvox = (int64_t)g.n[0] * g.n[1] * g.n[2];
  const float4* Qs = p.quads + (int64_t)slot * p.ql.slot;
  float* im = p.img_out + (int64_t)slot * p.img_stride;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(v / g.stride[0]);
    const int r0 = (int)(v - (int64_t)i0 * g.stride[0]);
    const int i1 = r0 / g.n[2], i2 = r0 - (r0 / g.n[2]) * g.n[2];
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!used[a]) continue;
      const int k = (a == 0) ? i0 : (a == 1 ? i1 : i2);
      const int I = (a == 0) ? i1 : i0;                 // index along b
      const int J = (a == 2) ? i1 : i2;                 // index along c
      const int nc2 = p.ql.nc2[a];
      const float4* Q = Qs + p.ql.base[a] + (int64_t)k * p.ql.plane[a];
      // padded positions: voxel I sits at I + 1
      s += Q[(I + 1) * nc2 + (J + 1)].x + Q[I * nc2 + (J + 1)].y + Q[(I + 1) * nc2 + J].z + Q[I * nc2 + J].w;
    }
    im[v] += s;
  }
}

// ---------------------------------------------------------------------------
// planless kernel: one thread per LOR in caller order, scalar gathers and
// atomics straight on the caller's image (no workspace)
// ---------------------------------------------------------------------------
template <int MODE, bool BACK>
__global__ void __launch_bounds__(kMaxBlock) direct_kernel(const ProjParams p) {
  extern __shared__ float sbuf[];  // TOF sinogram: [nbins][blockDim]
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  float xs[3], xe[3];
  xs[0] = __ldg(p.xs + 3 * i); xs[1] = __ldg(p.xs + 3 * i + 1); xs[2] = __ldg(p.xs + 3 * i + 2);
  xe[0] = __ldg(p.xe + 3 * i); xe[1] = __ldg(p.xe + 3 * i + 1); xe[2] = __ldg(p.xe + 3 * i + 2);
  const float delta = p.delta ? __ldg(p.delta + i) : 0.f;
  const int tbin = (MODE == 2) ? (int)__ldg(p.tof_bin + i) : 0;
  const DevTof& T = p.tof;
  const int N = T.nbins;
  float* acc = sbuf + threadIdx.x;
  Ray r;
  bool live = ray_setup(xs, xe, p.g, r);
  float d0 = 0.f;
  if (MODE == 2 && live) {
    const float c = (float)tbin * T.width + delta;
    d0 = r.tc - c;
    const float t1 = (-T.R - d0) / r.dt, t2 = (T.R - d0) / r.dt;
    const float lo = fmaxf(ceilf(r.kc + fminf(t1, t2)), (float)r.k0);
    const float hi = fminf(floorf(r.kc + fmaxf(t1, t2)), (float)r.k1);
    r.k0 = (int)lo;
    r.k1 = (int)hi;
    live = lo <= hi;
  }
  if (!BACK) {
    if (MODE == 1)
      for (int t = 0; t < N; ++t) acc[t * blockDim.x] = 0.f;
    float sum = 0.f;
    if (live) {
      for (int k = r.k0; k <= r.k1; ++k) {
        const float kk = (float)k - r.kc;
        Corners q;
        corners(r, k, fmaf(kk, r.du, r.uc), fmaf(kk, r.dw, r.wc), q);
        const float s = interp(p.img_in, r, q);
        if (MODE == 0) {
          sum += s;
        } else if (MODE == 2) {
          sum += tof_g(fmaf(kk, r.dt, d0), T) * s;
        } else {
          if (s == 0.f) continue;
          const float tau = fmaf(kk, r.dt, r.tc);
          const float x = (tau - delta) * T.inv_w + T.hbin;
          const int t0 = max(0, (int)ceilf(x - T.R_over_w));
          const int t1 = min(N - 1, (int)floorf(x + T.R_over_w));
          if (t0 > t1) continue;
          const float dlo = (tau - delta) - ((float)t0 - T.hbin) * T.width;
          float e_hi = erff((dlo + T.half) * T.k);
          for (int t = t0; t <= t1; ++t) {
            const float dist = fmaf(-(float)(t - t0), T.width, dlo);
            const float e_lo = erff((dist - T.half) * T.k);
            acc[t * blockDim.x] += 0.5f * (e_hi - e_lo) * s;
            e_hi = e_lo;
          }
        }
      }
    }
    if (MODE == 1) {
      float* out = p.proj_out + i * (int64_t)N;
      for (int t = 0; t < N; ++t) out[t] = live ? r.w0 * acc[t * blockDim.x] : 0.f;
    } else {
      p.proj_out[i] = live ? r.w0 * sum : 0.f;
    }
  } else {
    if (!live) return;
    float val = r.w0;
    if (MODE == 1) {
      const float* yrow = p.proj_in + i * (int64_t)N;
      bool any = false;
      for (int t = 0; t < N; ++t) {
        const float y = __ldg(yrow + t);
        acc[t * blockDim.x] = y;
        any |= (y != 0.f);
      }
      if (!any) return;
    } else {
      val *= __ldg(p.proj_in + i);
      if (val == 0.f) return;
    }
    for (int k = r.k0; k <= r.k1; ++k) {
      const float kk = (float)k - r.kc;
      float coef;
      if (MODE == 0) {
        coef = val;
      } else if (MODE == 2) {
        coef = tof_g(fmaf(kk, r.dt, d0), T) * val;
      } else {
        const float tau = fmaf(kk, r.dt, r.tc);
        const float x = (tau - delta) * T.inv_w + T.hbin;
        const int t0 = max(0, (int)ceilf(x - T.R_over_w));
        const int t1 = min(N - 1, (int)floorf(x + T.R_over_w));
        if (t0 > t1) continue;
        const float dlo = (tau - delta) - ((float)t0 - T.hbin) * T.width;
        float e_hi = erff((dlo + T.half) * T.k);
        float sy = 0.f;
        for (int t = t0; t <= t1; ++t) {
          const float dist = fmaf(-(float)(t - t0), T.width, dlo);
          const float e_lo = erff((dist - T.half) * T.k);
          sy += 0.5f * (e_hi - e_lo) * acc[t * blockDim.x];
          e_hi = e_lo;
        }
        coef = sy * val;
      }
      if (coef == 0.f) continue;
      Corners q;
      corners(r, k, fmaf(kk, r.du, r.uc), fmaf(kk, r.dw, r.wc), q);
      scatter_add(p.img_out, r, q, coef);
    }
  }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
int pick_block(int block, int mode, const DevTof& t, bool lut) {
  if (block > kMaxBlock) block = kMaxBlock;
  if (mode == 1) {
    int avail = 96 * 1024 - (lut ? kLut * 8 : 0);
    int cap = (avail / (4 * t.nbins)) / 32 * 32;
    if (cap < 32) cap = 32;
    if (block > cap) block = cap;
  }
  return block;
}

template <typename K>
int prepare_smem(K kernel, size_t smem) {
  if (smem > 48 * 1024) {
    JP_TRY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  return JP_OK;
}

template <int MODE, bool BACK, bool LUT>
int launch_planned(const ProjParams& p, int block, cudaStream_t st) {
  auto kern = planned_kernel<MODE, BACK, LUT>;
  const size_t smem = ((MODE != 0 && LUT) ? kLut * sizeof(float2) : 0) +
                      ((MODE == 1) ? (size_t)p.tof.nbins * block * sizeof(float) : 0);
  int rc = prepare_smem(kern, smem);
  if (rc) return rc;
  int per_sm = 0;
  JP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t need = (p.n + block - 1) / block;
  int64_t grid = (int64_t)sm_count() * per_sm;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, block, smem, st>>>(p);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

template <int MODE, bool BACK>
int launch_direct(const ProjParams& p, int block, cudaStream_t st) {
  if (p.n == 0) return JP_OK;
  auto kern = direct_kernel<MODE, BACK>;
  const size_t smem = (MODE == 1) ? (size_t)p.tof.nbins * block * sizeof(float) : 0;
  int rc = prepare_smem(kern, smem);
  if (rc) return rc;
  const int64_t blocks = (p.n + block - 1) / block;
  if (blocks > INT32_MAX) return fail(JP_ERR_ARG, "too many LORs for one launch");
  kern<<<(unsigned)blocks, block, smem, st>>>(p);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

int aux_grid(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  int64_t cap = (int64_t)sm_count() * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

int planned(jp_plan pl, int mode, bool back, const float* in, float* out, int64_t img_stride,
            const jp_tof* t, void* stream) {
  clear_error();
  if (!pl) return fail(JP_ERR_ARG, "plan is NULL");
  if (pl->n > 0 && (!in || !out)) return fail(JP_ERR_ARG, "input/output pointer is NULL");
  if (!aligned(in, 4) || !aligned(out, 4)) return fail(JP_ERR_ALIGN, "arrays must be 4-byte aligned");
  if (img_stride < 0) return fail(JP_ERR_ARG, "img_stride must be >= 0");
  if (mode == 2 && !pl->has_tof_bin) return fail(JP_ERR_STATE, "TOF listmode needs a plan created with tof_bin");
  ProjParams p;
  std::memset(&p, 0, sizeof(p));
  int rc = make_geom(&pl->g, &p.g);
  if (rc) return rc;
  if (img_stride != 0 && pl->n_frames > 1 && img_stride < (int64_t)p.g.n[0] * p.g.n[1] * p.g.n[2])
    return fail(JP_ERR_ARG, "img_stride smaller than one image");
  if (mode != 0) {
    rc = make_tof(t, mode == 1, &p.tof);
    if (rc) return rc;
  } else {
    p.tof.nbins = 1;
  }
  if (pl->n == 0) return JP_OK;
  p.lor = pl->lor;
  p.perm = pl->perm;
  p.frame_off = pl->frame_off_dev;
  p.n_frames = pl->n_frames;
  p.n = pl->n;
  p.img_stride = img_stride;
  p.quads = pl->quads;
  p.ql = pl->ql;
  p.axis_used = pl->axis_used;
  p.shared = (img_stride == 0 || pl->n_frames == 1) ? 1 : 0;
  if (back) { p.proj_in = in; p.img_out = out; } else { p.img_in = in; p.proj_out = out; }
  const int slots = p.shared ? 1 : pl->n_frames;
  if (slots * 3 > 65535) return fail(JP_ERR_ARG, "too many frames with distinct images (max 21845)");
  const bool lut = (mode != 0) && !(pl->opts.flags & JP_PLAN_TOF_EXACT);
  const int block = pick_block(pl->opts.block, mode, p.tof, lut);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t max_quad = std::max(std::max((int64_t)p.g.n[0] * p.ql.plane[0], (int64_t)p.g.n[1] * p.ql.plane[1]),
                                    (int64_t)p.g.n[2] * p.ql.plane[2]);
  dim3 qgrid(aux_grid(max_quad, 256), slots * 3);
  if (!back) {
    quad_build_kernel<<<qgrid, 256, 0, st>>>(p);
  } else {
    quad_zero_kernel<<<qgrid, 256, 0, st>>>(p);
  }
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  switch (mode * 4 + (back ? 2 : 0) + (lut ? 1 : 0)) {
    case 0: rc = launch_planned<0, false, false>(p, block, st); break;
    case 2: rc = launch_planned<0, true, false>(p, block, st); break;
    case 4: rc = launch_planned<1, false, false>(p, block, st); break;
    case 5: rc = launch_planned<1, false, true>(p, block, st); break;
    case 6: rc = launch_planned<1, true, false>(p, block, st); break;
    case 7: rc = launch_planned<1, true, true>(p, block, st); break;
    case 8: rc = launch_planned<2, false, false>(p, block, st); break;
    case 9: rc = launch_planned<2, false, true>(p, block, st); break;
    case 10: rc = launch_planned<2, true, false>(p, block, st); break;
    case 11: rc = launch_planned<2, true, true>(p, block, st); break;
    default: return fail(JP_ERR_ARG, "bad mode");
  }
  if (rc) return rc;
  if (back) {
    const int64_t nvox = (int64_t)p.g.n[0] * p.g.n[1] * p.g.n[2];
    dim3 rgrid(aux_grid(nvox, 256), slots);
    quad_reduce_kernel<<<rgrid, 256, 0, st>>>(p);
    count_launch();
    JP_TRY_CUDA(cudaGetLastError());
  }
  return JP_OK;
}

int direct(int mode, bool back, const float* xs, const float* xe, const int16_t* tof_bin,
           const float* delta, int64_t n, const jp_image_geom* g, const jp_tof* t,
           const float* in, float* out, void* stream) {
  clear_error();
  if (n < 0) return fail(JP_ERR_ARG, "n_lor must be >= 0");
  if (mode < 0 || mode > 2) return fail(JP_ERR_ARG, "tof_mode must be 0, 1 or 2");
  if (n > 0 && (!xs || !xe || !in || !out)) return fail(JP_ERR_ARG, "array pointer is NULL");
  if (mode == 2 && n > 0 && !tof_bin) return fail(JP_ERR_ARG, "tof_bin is NULL in listmode");
  if (!aligned(xs, 4) || !aligned(xe, 4) || !aligned(in, 4) || !aligned(out, 4) ||
      !aligned(delta, 4) || !aligned(tof_bin, 2))
    return fail(JP_ERR_ALIGN, "misaligned array");
  ProjParams p;
  std::memset(&p, 0, sizeof(p));
  int rc = make_geom(g, &p.g);
  if (rc) return rc;
  if (mode != 0) {
    rc = make_tof(t, mode == 1, &p.tof);
    if (rc) return rc;
  } else {
    p.tof.nbins = 1;
  }
  p.xs = xs; p.xe = xe; p.tof_bin = tof_bin; p.delta = delta; p.n = n; p.n_frames = 1;
  if (back) { p.proj_in = in; p.img_out = out; } else { p.img_in = in; p.proj_out = out; }
  const int block = pick_block(256, mode, p.tof, false);
  cudaStream_t st = (cudaStream_t)stream;
  switch (mode * 2 + (back ? 1 : 0)) {
    case 0: return launch_direct<0, false>(p, block, st);
    case 1: return launch_direct<0, true>(p, block, st);
    case 2: return launch_direct<1, false>(p, block, st);
    case 3: return launch_direct<1, true>(p, block, st);
    case 4: return launch_direct<2, false>(p, block, st);
    case 5: return launch_direct<2, true>(p, block, st);
  }
  return fail(JP_ERR_ARG, "bad mode");
}

// per-LOR count of visited plane samples (same setup as the projectors)
template <int MODE>
__global__ void count_kernel(const ProjParams p, unsigned long long* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cnt = 0;
  if (i < p.n) {
    const float4 A = __ldg(p.lor + 2 * i);
    const float4 B = __ldg(p.lor + 2 * i + 1);
    float xs[3] = {A.x, A.y, A.z}, xe[3] = {B.x, B.y, B.z};
    Ray r;
    bool live = ray_setup(xs, xe, p.g, r);
    if (live && MODE == 2) {
      const float c = (float)__float_as_int(B.w) * p.tof.width + A.w;
      const float d0 = r.tc - c;
      const float t1 = (-p.tof.R - d0) / r.dt, t2 = (p.tof.R - d0) / r.dt;
      const float lo = fmaxf(ceilf(r.kc + fminf(t1, t2)), (float)r.k0);
      const float hi = fminf(floorf(r.kc + fmaxf(t1, t2)), (float)r.k1);
      r.k0 = (int)lo;
      r.k1 = (int)hi;
      live = lo <= hi;
    }
    if (live) cnt = (unsigned long long)(r.k1 - r.k0 + 1);
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

}  // namespace
}  // namespace jp

using namespace jp;

extern "C" int jp_count_samples(jp_plan pl, int32_t mode, const jp_tof* t, uint64_t* out, void* stream) {
  clear_error();
  if (!pl || !out) return fail(JP_ERR_ARG, "NULL argument");
  if (mode != 0 && mode != 2) return fail(JP_ERR_ARG, "mode must be 0 or 2");
  if (!aligned(out, 8)) return fail(JP_ERR_ALIGN, "out must be 8-byte aligned");
  if (mode == 2 && !pl->has_tof_bin) return fail(JP_ERR_STATE, "TOF listmode needs a plan created with tof_bin");
  ProjParams p;
  std::memset(&p, 0, sizeof(p));
  int rc = make_geom(&pl->g, &p.g);
  if (rc) return rc;
  if (mode == 2) {
    rc = make_tof(t, false, &p.tof);
    if (rc) return rc;
  }
  p.lor = pl->lor;
  p.n = pl->n;
  cudaStream_t st = (cudaStream_t)stream;
  JP_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
  if (p.n == 0) return JP_OK;
  unsigned blocks = (unsigned)((p.n + 255) / 256);
  if (mode == 0) count_kernel<0><<<blocks, 256, 0, st>>>(p, (unsigned long long*)out);
  else count_kernel<2><<<blocks, 256, 0, st>>>(p, (unsigned long long*)out);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

extern "C" int jp_fwd(jp_plan p, const float* img, int64_t s, float* proj, void* st) {
  return planned(p, 0, false, img, proj, s, nullptr, st);
}
extern "C" int jp_back(jp_plan p, const float* proj, float* img, int64_t s, void* st) {
  return planned(p, 0, true, proj, img, s, nullptr, st);
}
extern "C" int jp_fwd_tof_sino(jp_plan p, const float* img, int64_t s, const jp_tof* t, float* proj, void* st) {
  return planned(p, 1, false, img, proj, s, t, st);
}
extern "C" int jp_back_tof_sino(jp_plan p, const float* proj, const jp_tof* t, float* img, int64_t s, void* st) {
  return planned(p, 1, true, proj, img, s, t, st);
}
extern "C" int jp_fwd_tof_lm(jp_plan p, const float* img, int64_t s, const jp_tof* t, float* proj, void* st) {
  return planned(p, 2, false, img, proj, s, t, st);
}
extern "C" int jp_back_tof_lm(jp_plan p, const float* proj, const jp_tof* t, float* img, int64_t s, void* st) {
  return planned(p, 2, true, proj, img, s, t, st);
}
extern "C" int jp_fwd_lors(const float* xs, const float* xe, const int16_t* tb, const float* dl, int64_t n,
                           const jp_image_geom* g, int32_t mode, const jp_tof* t, const float* img,
                           float* proj, void* st) {
  return direct(mode, false, xs, xe, tb, dl, n, g, t, img, proj, st);
}
extern "C" int jp_back_lors(const float* xs, const float* xe, const int16_t* tb, const float* dl, int64_t n,
                            const jp_image_geom* g, int32_t mode, const jp_tof* t, const float* proj,
                            float* img, void* st) {
  return direct(mode, true, xs, xe, tb, dl, n, g, t, proj, img, st);
}
