// Joseph forward and back projection kernels (paper Sec. 2.1, 2.2).
//
// A thread, or a group of G lanes, follows one LOR plane by plane along its
// principal axis (steps a2-a6 of the hot path; the planless kernels, one
// thread per LOR in caller order, read and add the 4 voxels directly):
//   a2  per-LOR setup (exact principal axis, plane range, affine maps in
//       voxel units anchored at the centre plane so every sample is one FMA
//       from a small anchor value, never a long running sum);
//   a3  forward: bilinear interpolation of the 4 nearest voxels, one
//       16-byte load of a zero-padded quad image per sample (L2-resident),
//       summed and scaled by v_a / cos_a;
//   a4  TOF weights, the difference of erff at the bin edges, by default
//       read from a shared-memory table of exact erf differences with
//       linear interpolation (a caller's table of a non-Gaussian kernel the
//       same way), or with erff itself (a TOF sinogram then shares each
//       inner edge between two neighbouring bins, so W bins cost W+1 erff);
//       listmode evaluates only the planes of its TOF window;
//   a5  back projection: the transposed coefficients scattered with
//       fire-and-forget reductions (RED): one 16-byte vector reduction per
//       sample into the quad images, folded into the image afterwards;
//   a6  planned calls read LORs in binned order and scatter/gather the
//       projection values through the plan's permutation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "jp_internal.cuh"
#include "jp_proj.cuh"

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
  if (t->kernel) {
    if (t->kernel_nodes < 2 || t->kernel_nodes > JP_TOF_TABLE)
      return fail(JP_ERR_ARG, "TOF kernel_nodes must be in 2..JP_TOF_TABLE");
    if (!(t->kernel_half_width > 0.f) || !isfinite(t->kernel_half_width))
      return fail(JP_ERR_ARG, "TOF kernel_half_width must be finite and > 0");
    if (!aligned(t->kernel, 4)) return fail(JP_ERR_ALIGN, "TOF kernel table must be 4-byte aligned");
  } else {
    if (!(t->sigma > 0.f) || !isfinite(t->sigma)) return fail(JP_ERR_ARG, "TOF sigma must be finite and > 0");
    if (!(t->n_sigmas > 0.f) || !isfinite(t->n_sigmas)) return fail(JP_ERR_ARG, "TOF n_sigmas must be finite and > 0");
  }
  if (sino && (t->n_bins < 1 || t->n_bins > JP_MAX_TOF_BINS))
    return fail(JP_ERR_ARG, "TOF n_bins must be in 1..JP_MAX_TOF_BINS");
  out->width = t->bin_width;
  out->half = 0.5f * t->bin_width;
  out->user = t->kernel;
  if (t->kernel) {
    out->k = 0.f;
    out->ns = 0.f;
    out->R = t->kernel_half_width;
    out->nodes = t->kernel_nodes;
  } else {
    out->k = 1.0f / (1.41421356237309515f * t->sigma);
    out->R = t->n_sigmas * t->sigma + 0.5f * t->bin_width;
    out->ns = t->n_sigmas;
    out->nodes = JP_TOF_TABLE;
  }
  out->inv_h = (float)(out->nodes - 1) / (2.f * out->R);
  // bin-aligned sinogram table: the largest m with 2 ceil(R m / w) + 1 <=
  // JP_TOF_TABLE nodes (at least 4 nodes per bin, else not used)
  out->m = 0;
  out->nodes_a = 0;
  out->Rp = 0.f;
  out->inv_hp = 0.f;
  if (!t->kernel) {
    const double cmax = (double)((JP_TOF_TABLE - 1) / 2);
    const double ratio = (double)out->R / (double)t->bin_width;
    const int m = (int)floor(cmax / ratio);
    if (m >= 4) {
      const double h = (double)t->bin_width / m;
      int c = (int)ceil((double)out->R / h);
      if (2 * c + 1 > JP_TOF_TABLE) c = (JP_TOF_TABLE - 1) / 2;
      if ((double)c * h >= (double)out->R) {
        out->m = m;
        out->nodes_a = 2 * c + 1;
        out->Rp = (float)(c * h);
        out->inv_hp = (float)(1.0 / h);
      }
    }
  }
  out->R_over_w = out->R / t->bin_width;
  out->inv_w = 1.0f / t->bin_width;
  out->nbins = sino ? t->n_bins : 1;
  out->hbin = 0.5f * (float)(out->nbins - 1);
  return JP_OK;
}

namespace {

// plane alignment of a back projection's lane group of G lanes: min(G, 8)
template <int G>
constexpr int kGroupAlign = G < 8 ? G : 8;

// Two consecutive plane-fastest quad entries (planes 2m, 2m+1 of one quad
// row, 32-byte aligned) in one 32-byte read-only load.
__device__ __forceinline__ void ld_quad_pair(const float4* q, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(q));
}

// ---------------------------------------------------------------------------
// planned projection kernel: persistent CTAs over binned LORs, quad images
// ---------------------------------------------------------------------------
// The TOF-sinogram forward is compiled for three resident CTAs of 512 (40
// registers); the other instances keep the compiler's own register choice
// (a minimum of 0 CTAs states none: 1 would let the TOF-listmode forward
// grow from 48 to 54 registers and lose a fifth of its resident warps).
template <int MODE, bool BACK, bool LUT>
__global__ void __launch_bounds__(kMaxBlock, (MODE == 1 && !BACK) ? 3 : 0) planned_kernel(const ProjParams p) {
  extern __shared__ float4 smem4[];
  float2* lut = reinterpret_cast<float2*>(smem4);
  float* accbase = reinterpret_cast<float*>(lut + ((MODE != 0 && LUT) ? kLut : 0));
  float* acc = accbase + threadIdx.x;  // TOF sinogram: acc[t * blockDim.x]
  const DevTof& T = p.tof;
  if (MODE != 0 && LUT) {
    if (MODE == 1 && T.m > 0)
      build_lut_aligned(lut, T);
    else
      build_lut(lut, T);
    __syncthreads();
  }
  const int N = T.nbins;
  __shared__ unsigned int tile_s;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) tile_s = atomicAdd(p.counter, 1u);
    __syncthreads();
    const int64_t i = (int64_t)tile_s * blockDim.x + threadIdx.x;
    if ((int64_t)tile_s * blockDim.x >= p.n) break;
    if (i >= p.n) continue;
    const float4 A = __ldcs(p.lor + 2 * i);
    const float4 B = __ldcs(p.lor + 2 * i + 1);
    const float xs[3] = {A.x, A.y, A.z};
    const float xe[3] = {B.x, B.y, B.z};
    const float delta = p.perm_in_rec ? 0.f : A.w;
    const int tbin = __float_as_int(B.w);
    const int64_t j = p.perm_in_rec ? (int64_t)__float_as_int(A.w) : (int64_t)__ldcs(p.perm + i);
    const int f = (p.n_frames > 1) ? frame_of(p.frame_off, p.n_frames, i) : 0;
    const int slot = p.shared ? 0 : f;
    Ray r;
    bool live = ray_setup(xs, xe, p.g, r);
    float d0 = 0.f;  // tau(kc) - c  (listmode)
    float ke = T.k;
    if (MODE == 2 && live) {
      float Re;
      event_tof(p, i, ke, Re);
      const float c = (float)tbin * T.width + delta;
      d0 = r.tc - c;
      const float t1 = (-Re - d0) / r.dt, t2 = (Re - d0) / r.dt;
      const float lo = fmaxf(ceilf(r.kc + fminf(t1, t2)), (float)r.k0);
      const float hi = fminf(floorf(r.kc + fmaxf(t1, t2)), (float)r.k1);
      r.k0 = (int)lo;
      r.k1 = (int)hi;
      live = lo <= hi;
    }
    const int a = r.a;
    const int nc2 = sel3(a, p.ql.nc2[0], p.ql.nc2[1], p.ql.nc2[2]);
    const int nb2 = sel3(a, p.ql.nb2[0], p.ql.nb2[1], p.ql.nb2[2]);
    const int na = sel3(a, p.ql.nap[0], p.ql.nap[1], p.ql.nap[2]);  // k-stride of plane-fastest quads
    const int64_t qoff = (int64_t)slot * p.ql.slot + sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
    const float ub = (float)r.nb, wb = (float)r.nc;

    if (!BACK) {
      // ------------------------------ forward ------------------------------
      const float4* __restrict__ Q = p.quads + qoff;
      if (MODE == 1)
        for (int t = 0; t < N; ++t) acc[t * blockDim.x] = 0.f;
      float sum = 0.f;
      if (MODE == 0 && live && p.kfast) {
        // plane-fastest quads: planes 2m and 2m+1 of a quad row share one
        // 32-byte sector, so two samples that stay in their quad row take a
        // single 32-byte load (the sum keeps the plane order).  Non-TOF
        // only: in TOF listmode the extra registers cost a fifth of the
        // resident warps and the forward gets slower (5.27 vs 5.18 ms on a
        // 40M-event frame; non-TOF 8.18 vs 8.40 ms)
        auto coords = [&](int kq, float& kk, float& al, float& be, int& ip, int& jq) {
          kk = (float)kq - r.kc;
          const float u = fminf(fmaxf(fmaf(kk, r.du, r.uc), -1.f), ub);
          const float w = fminf(fmaxf(fmaf(kk, r.dw, r.wc), -1.f), wb);
          const float fu = floorf(u), fw = floorf(w);
          al = u - fu;
          be = w - fw;
          ip = (int)fu + 1;
          jq = (int)fw + 1;
        };
        auto add = [&](float al, float be, float4 v) {
          const float top = fmaf(be, v.z - v.x, v.x);
          const float bot = fmaf(be, v.w - v.y, v.y);
          sum += fmaf(al, bot - top, top);
        };
        auto load1 = [&](int kq, int ip, int jq) { return __ldg(Q + quad_index(true, kq, ip, jq, na, nb2, nc2)); };
        int k = r.k0;
        float kk0, al0, be0, kk1, al1, be1;
        int ip0, jq0, ip1, jq1;
        if (k & 1) {
          coords(k, kk0, al0, be0, ip0, jq0);
          add(al0, be0, load1(k, ip0, jq0));
          ++k;
        }
        for (; k < r.k1; k += 2) {
          coords(k, kk0, al0, be0, ip0, jq0);
          coords(k + 1, kk1, al1, be1, ip1, jq1);
          float4 v0, v1;
          ld_quad_pair(Q + quad_index(true, k, ip0, jq0, na, nb2, nc2), v0, v1);
          if (ip1 != ip0 || jq1 != jq0) v1 = load1(k + 1, ip1, jq1);
          add(al0, be0, v0);
          add(al1, be1, v1);
        }
        if (k == r.k1) {
          coords(k, kk0, al0, be0, ip0, jq0);
          add(al0, be0, load1(k, ip0, jq0));
        }
      } else if (live) {
        for (int k = r.k0; k <= r.k1; ++k) {
          const float kk = (float)k - r.kc;
          const float u = fminf(fmaxf(fmaf(kk, r.du, r.uc), -1.f), ub);
          const float w = fminf(fmaxf(fmaf(kk, r.dw, r.wc), -1.f), wb);
          const float fu = floorf(u), fw = floorf(w);
          const float al = u - fu, be = w - fw;
          // TOF listmode: the lanes' windows start on different planes, so
          // the quads rarely hit L1 (10%); loads cached in L2 only skip the
          // L1 fills (forward 5.18 vs 5.26 ms on a 40M-event frame)
          const float4* qa = Q + quad_index(p.kfast, k, (int)fu + 1, (int)fw + 1, na, nb2, nc2);
          const float4 v = (MODE == 2) ? __ldcg(qa) : __ldg(qa);
          const float top = fmaf(be, v.z - v.x, v.x);
          const float bot = fmaf(be, v.w - v.y, v.y);
          const float s = fmaf(al, bot - top, top);
          if (MODE == 0) {
            sum += s;
          } else if (MODE == 2) {
            sum = fmaf(tof_weight<LUT>(lut, fmaf(kk, r.dt, d0), T, ke), s, sum);
          } else {
            if (s == 0.f) continue;
            const float tau = fmaf(kk, r.dt, r.tc);
            const float x = (tau - delta) * T.inv_w + T.hbin;
            const int t0 = max(0, (int)ceilf(x - T.R_over_w));
            const int t1 = min(N - 1, (int)floorf(x + T.R_over_w));
            if (t0 > t1) continue;
            const float dlo = (tau - delta) - ((float)t0 - T.hbin) * T.width;
            if (LUT && T.m > 0) {
              // bin-aligned table: one fraction for all of the sample's bins,
              // the node index steps down by m per bin
              const float xl0 = (dlo + T.Rp) * T.inv_hp;
              const int ix0 = min(max((int)xl0, 0), T.nodes_a - 1);
              const float fr = xl0 - (float)ix0;
              float* a = acc + t0 * blockDim.x;
              for (int t = 0, ix = ix0; t <= t1 - t0; ++t, ix -= T.m, a += blockDim.x) {
                const float2 e = lut[max(ix, 0)];
                *a = fmaf(fmaf(fr, e.y, e.x), s, *a);
              }
            } else if (LUT) {
              // table coordinate of bin t0, stepping down by w / h per bin
              const float xl0 = (dlo + T.R) * T.inv_h, step = T.width * T.inv_h;
              float* a = acc + t0 * blockDim.x;
              for (int t = 0; t <= t1 - t0; ++t, a += blockDim.x)
                *a = fmaf(lut_at(lut, fmaf(-(float)t, step, xl0), T.nodes - 1), s, *a);
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
        __stcs(p.proj_out + j, live ? r.w0 * sum : 0.f);
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
        val *= __ldcs(p.proj_in + j);
        if (val == 0.f) continue;
      }
      for (int k = r.k0; k <= r.k1; ++k) {
        const float kk = (float)k - r.kc;
        float coef;
        if (MODE == 0) {
          coef = val;
        } else if (MODE == 2) {
          coef = tof_weight<LUT>(lut, fmaf(kk, r.dt, d0), T, ke) * val;
        } else {
          const float tau = fmaf(kk, r.dt, r.tc);
          const float x = (tau - delta) * T.inv_w + T.hbin;
          const int t0 = max(0, (int)ceilf(x - T.R_over_w));
          const int t1 = min(N - 1, (int)floorf(x + T.R_over_w));
          if (t0 > t1) continue;
          const float dlo = (tau - delta) - ((float)t0 - T.hbin) * T.width;
          float sy = 0.f;
          if (LUT && T.m > 0) {
            const float xl0 = (dlo + T.Rp) * T.inv_hp;
            const int ix0 = min(max((int)xl0, 0), T.nodes_a - 1);
            const float fr = xl0 - (float)ix0;
            const float* a = acc + t0 * blockDim.x;
            for (int t = 0, ix = ix0; t <= t1 - t0; ++t, ix -= T.m, a += blockDim.x) {
              const float2 e = lut[max(ix, 0)];
              sy = fmaf(fmaf(fr, e.y, e.x), *a, sy);
            }
          } else if (LUT) {
            const float xl0 = (dlo + T.R) * T.inv_h, step = T.width * T.inv_h;
            const float* a = acc + t0 * blockDim.x;
            for (int t = 0; t <= t1 - t0; ++t, a += blockDim.x)
              sy = fmaf(lut_at(lut, fmaf(-(float)t, step, xl0), T.nodes - 1), *a, sy);
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
        atomicAdd(Q + quad_index(p.kfast, k, (int)fu + 1, (int)fw + 1, na, nb2, nc2),
                  make_float4(ca * (1.f - be), cb * (1.f - be), ca * be, cb * be));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// planned projection, G lanes per LOR (non-TOF and TOF listmode).  Each warp
// takes 32 binned LORs; every lane sets up one of them, then the warp walks
// them 32/G at a time: the setup is broadcast by shuffles and the G lanes of
// a group step through consecutive planes (k = k0 + lane, k0 + lane + G, ...),
// so their quad loads / reductions touch consecutive 16-byte entries.
// ---------------------------------------------------------------------------

template <int MODE, bool BACK, bool LUT, int G>
__global__ void __launch_bounds__(kMaxBlock) group_kernel(const ProjParams p) {
  static_assert(MODE == 0 || MODE == 2 || (MODE == 1 && BACK),
                "group kernel: non-TOF, TOF listmode, or TOF-sinogram back projection");
  constexpr int E = 32 / G;  // LORs walked at once per warp
  extern __shared__ float4 smem4[];
  float2* lut = reinterpret_cast<float2*>(smem4);
  const DevTof& T = p.tof;
  if (MODE != 0 && LUT) {
    if (MODE == 1 && T.m > 0)
      build_lut_aligned(lut, T);
    else
      build_lut(lut, T);
    __syncthreads();
  }
  const int N = T.nbins;
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, gl = lane - grp * G;
  for (;;) {
    unsigned int chunk = 0;
    if (lane == 0) chunk = atomicAdd(p.counter, 1u);
    const int64_t base = (int64_t)__shfl_sync(0xffffffffu, chunk, 0) * 32;
    if (base >= p.n) break;
    // ---- per-lane setup of LOR base + lane ----
    const int64_t i = base + lane;
    Ray r;
    r.k0 = 1; r.k1 = 0;
    float d0 = 0.f, val = 0.f, delta = 0.f, ke = T.k;
    int slot = 0;
    int32_t j = 0;
    if (i < p.n) {
      const float4 A = __ldcs(p.lor + 2 * i);
      const float4 B = __ldcs(p.lor + 2 * i + 1);
      const float xs[3] = {A.x, A.y, A.z};
      const float xe[3] = {B.x, B.y, B.z};
      j = p.perm_in_rec ? __float_as_int(A.w) : __ldcs(p.perm + i);
      delta = p.perm_in_rec ? 0.f : A.w;
      const int f = (p.n_frames > 1) ? frame_of(p.frame_off, p.n_frames, i) : 0;
      slot = p.shared ? 0 : f;
      bool live = ray_setup(xs, xe, p.g, r);
      if (MODE == 2 && live) {
        float Re;
        event_tof(p, i, ke, Re);
        const float c = (float)__float_as_int(B.w) * T.width + delta;
        d0 = r.tc - c;
        const float t1 = (-Re - d0) / r.dt, t2 = (Re - d0) / r.dt;
        const float lo = fmaxf(ceilf(r.kc + fminf(t1, t2)), (float)r.k0);
        const float hi = fminf(floorf(r.kc + fmaxf(t1, t2)), (float)r.k1);
        r.k0 = (int)lo;
        r.k1 = (int)hi;
        live = lo <= hi;
      }
      if (BACK && live) {
        val = (MODE == 1) ? r.w0 : r.w0 * __ldcs(p.proj_in + j);
        live = val != 0.f;
      }
      if (!live) { r.k0 = 1; r.k1 = 0; r.w0 = 0.f; val = 0.f; }
    } else {
      r.a = 0; r.kc = 0.f; r.uc = r.du = r.wc = r.dw = r.tc = r.dt = r.w0 = 0.f;
    }
    // ---- walk the 32 LORs, E at a time ----
#pragma unroll 1
    for (int pass = 0; pass < G; ++pass) {
      const int src = pass * E + grp;
      const int k0 = __shfl_sync(0xffffffffu, r.k0, src);
      const int k1 = __shfl_sync(0xffffffffu, r.k1, src);
      const int a = __shfl_sync(0xffffffffu, r.a, src);
      const int sl = __shfl_sync(0xffffffffu, slot, src);
      const int32_t jj = __shfl_sync(0xffffffffu, j, src);
      const float uc = __shfl_sync(0xffffffffu, r.uc, src);
      const float du = __shfl_sync(0xffffffffu, r.du, src);
      const float wc = __shfl_sync(0xffffffffu, r.wc, src);
      const float dw = __shfl_sync(0xffffffffu, r.dw, src);
      const float w0 = __shfl_sync(0xffffffffu, BACK ? val : r.w0, src);
      float dd0 = 0.f, ddt = 0.f, dtc = 0.f, ddl = 0.f, dke = 0.f;
      if (MODE == 2) {
        dd0 = __shfl_sync(0xffffffffu, d0, src);
        ddt = __shfl_sync(0xffffffffu, r.dt, src);
        dke = __shfl_sync(0xffffffffu, ke, src);
      }
      if (MODE == 1) {
        ddt = __shfl_sync(0xffffffffu, r.dt, src);
        dtc = __shfl_sync(0xffffffffu, r.tc, src);
        ddl = __shfl_sync(0xffffffffu, delta, src);
      }
      const int na = sel3(a, p.g.n[0], p.g.n[1], p.g.n[2]);
      const int nap = sel3(a, p.ql.nap[0], p.ql.nap[1], p.ql.nap[2]);
      const int nb = (a == 0) ? p.g.n[1] : p.g.n[0];
      const int nc = (a == 2) ? p.g.n[1] : p.g.n[2];
      const int nc2 = nc + 2;
      const float kc = 0.5f * (float)(na - 1);
      const float ub = (float)nb, wb = (float)nc;
      const int64_t qoff = (int64_t)sl * p.ql.slot + sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
      float sum = 0.f;
      if (!BACK) {
        const float4* __restrict__ Qa = p.quads + qoff;
        for (int k = k0 + gl; k <= k1; k += G) {
          const float kk = (float)k - kc;
          const float u = fminf(fmaxf(fmaf(kk, du, uc), -1.f), ub);
          const float w = fminf(fmaxf(fmaf(kk, dw, wc), -1.f), wb);
          const float fu = floorf(u), fw = floorf(w);
          const float al = u - fu, be = w - fw;
          const float4 v = __ldg(Qa + (((int)fu + 1) * nc2 + ((int)fw + 1)) * nap + k);
          const float top = fmaf(be, v.z - v.x, v.x);
          const float bot = fmaf(be, v.w - v.y, v.y);
          const float s = fmaf(al, bot - top, top);
          if (MODE == 0) sum += s;
          else sum = fmaf(tof_weight<LUT>(lut, fmaf(kk, ddt, dd0), T, dke), s, sum);
        }
      }
      // start the group on a plane that is a multiple of min(G, 8): the lanes
      // then cover the (2m, 2m+1) plane pairs that share a 32-byte sector and
      // the 8-plane runs of one 128-byte line of the plane-fastest quads (a
      // reduction costs less when more of its warp's lanes share lines:
      // TOF-LM back 9.50 vs 9.79 ms per 40M-event frame against even planes)
      for (int k = (k0 & ~(kGroupAlign<G> - 1)) + gl; BACK && k <= k1; k += G) {
        if (k < k0) continue;
        const float kk = (float)k - kc;
        const float u = fminf(fmaxf(fmaf(kk, du, uc), -1.f), ub);
        const float w = fminf(fmaxf(fmaf(kk, dw, wc), -1.f), wb);
        const float fu = floorf(u), fw = floorf(w);
        const float al = u - fu, be = w - fw;
        const int q = (((int)fu + 1) * nc2 + ((int)fw + 1)) * nap + k;
        {
          float coef = w0;
          if (MODE == 2) coef *= tof_weight<LUT>(lut, fmaf(kk, ddt, dd0), T, dke);
          if (MODE == 1) {
            // sum over the bins in the window of weight x sinogram value
            const float* yrow = p.proj_in + (int64_t)jj * N;
            const float tau = fmaf(kk, ddt, dtc);
            const float x = (tau - ddl) * T.inv_w + T.hbin;
            const int t0 = max(0, (int)ceilf(x - T.R_over_w));
            const int t1 = min(N - 1, (int)floorf(x + T.R_over_w));
            const float dlo = (tau - ddl) - ((float)t0 - T.hbin) * T.width;
            float sy = 0.f;
            if (LUT && T.m > 0) {
              const float xl0 = (dlo + T.Rp) * T.inv_hp;
              const int ix0 = min(max((int)xl0, 0), T.nodes_a - 1);
              const float fr = xl0 - (float)ix0;
              for (int t = t0, ix = ix0; t <= t1; ++t, ix -= T.m) {
                const float2 e = lut[max(ix, 0)];
                sy = fmaf(fmaf(fr, e.y, e.x), __ldg(yrow + t), sy);
              }
            } else if (LUT) {
              const float xl0 = (dlo + T.R) * T.inv_h, step = T.width * T.inv_h;
              for (int t = t0; t <= t1; ++t)
                sy = fmaf(lut_at(lut, fmaf(-(float)(t - t0), step, xl0), T.nodes - 1), __ldg(yrow + t), sy);
            } else {
              float e_hi = erff((dlo + T.half) * T.k);
              for (int t = t0; t <= t1; ++t) {
                const float e_lo = erff((fmaf(-(float)(t - t0), T.width, dlo) - T.half) * T.k);
                sy = fmaf(0.5f * (e_hi - e_lo), __ldg(yrow + t), sy);
                e_hi = e_lo;
              }
            }
            coef *= sy;
            if (coef == 0.f) continue;
          }
          const float ca = (1.f - al) * coef, cb = al * coef;
          atomicAdd(p.quads + qoff + q, make_float4(ca * (1.f - be), cb * (1.f - be), ca * be, cb * be));
        }
      }
      if (!BACK) {
        sum = group_sum<G>(sum);
        if (gl == 0 && base + src < p.n) __stcs(p.proj_out + jj, w0 * sum);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// listmode OSEM subset kernel: per event, forward projection of x (quads in
// p.quads), ratio 1 / (p + b), back projection of the ratio into p.quads_bp.
// G lanes per event as in group_kernel; both quad sets are plane-fastest.
// ---------------------------------------------------------------------------
// a[0] += v0, a[1] += v1: one 8-byte vector reduction when a is 8-byte
// aligned, else two scalar ones
__device__ __forceinline__ void red_pair(float* a, float v0, float v1) {
  if ((reinterpret_cast<uintptr_t>(a) & 7u) == 0) {
    atomicAdd(reinterpret_cast<float2*>(a), make_float2(v0, v1));
  } else {
    atomicAdd(a, v0);
    atomicAdd(a + 1, v1);
  }
}

// DIRECT = false: forward from the plane-fastest quads of p.img_in (p.quads),
// back projection into the back-projection quads (p.quads_bp), one 16-byte
// load / reduction per sample.  DIRECT = true: forward from the image
// p.img_in itself (4 bounded loads per sample) and back projection with 4
// scalar atomics per sample into the image p.img_out (zeroed by the caller):
// no image-sized quad build, clear and fold, which is the cheaper trade for
// small subsets.  Both compute the same samples with the same arithmetic.
template <bool LUT, int G, bool DIRECT>
__global__ void __launch_bounds__(kMaxBlock) osem_kernel(const ProjParams p) {
  constexpr int E = 32 / G;
  extern __shared__ float4 smem4[];
  float2* lut = reinterpret_cast<float2*>(smem4);
  const DevTof& T = p.tof;
  if (LUT) {
    build_lut(lut, T);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, gl = lane - grp * G;
  const int64_t start = __ldg(p.frame_off + p.f0), end = __ldg(p.frame_off + p.f1);
  const float bg = p.bg_ptr ? __ldg(p.bg_ptr) : p.bg;
  // A warp takes chunks of cp passes x E events.  A small subset gets
  // cp < G, so that its events spread over every warp of the grid instead
  // of queueing G passes deep on a few warps (the passes of a chunk run one
  // after the other); large subsets use full 32-event chunks.
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t per = (end - start + warps * E - 1) / (warps * E);
  const int cp = (int)(per < 1 ? 1 : (per > G ? G : per));
  const int chunk_ev = cp * E;
  for (;;) {
    unsigned int chunk = 0;
    if (lane == 0) chunk = atomicAdd(p.counter, 1u);
    const int64_t base = start + (int64_t)__shfl_sync(0xffffffffu, chunk, 0) * chunk_ev;
    if (base >= end) break;
    const int64_t i = base + lane;
    Ray r;
    r.k0 = 1; r.k1 = 0;
    float d0 = 0.f, ke = T.k;
    if (lane < chunk_ev && i < end) {
      const float4 A = __ldcs(p.lor + 2 * i);
      const float4 B = __ldcs(p.lor + 2 * i + 1);
      const float xs[3] = {A.x, A.y, A.z};
      const float xe[3] = {B.x, B.y, B.z};
      bool live = ray_setup(xs, xe, p.g, r);
      if (live) {
        float Re;
        event_tof(p, i, ke, Re);
        const float c = (float)__float_as_int(B.w) * T.width + (p.perm_in_rec ? 0.f : A.w);
        d0 = r.tc - c;
        const float t1 = (-Re - d0) / r.dt, t2 = (Re - d0) / r.dt;
        const float lo = fmaxf(ceilf(r.kc + fminf(t1, t2)), (float)r.k0);
        const float hi = fminf(floorf(r.kc + fmaxf(t1, t2)), (float)r.k1);
        r.k0 = (int)lo;
        r.k1 = (int)hi;
        live = lo <= hi;
      }
      if (!live) { r.k0 = 1; r.k1 = 0; r.w0 = 0.f; }
    } else {
      r.a = 0; r.uc = r.du = r.wc = r.dw = r.tc = r.dt = r.w0 = 0.f;
    }
#pragma unroll 1
    for (int pass = 0; pass < cp; ++pass) {
      const int src = pass * E + grp;
      const int k0 = __shfl_sync(0xffffffffu, r.k0, src);
      const int k1 = __shfl_sync(0xffffffffu, r.k1, src);
      const int a = __shfl_sync(0xffffffffu, r.a, src);
      const float uc = __shfl_sync(0xffffffffu, r.uc, src);
      const float du = __shfl_sync(0xffffffffu, r.du, src);
      const float wc = __shfl_sync(0xffffffffu, r.wc, src);
      const float dw = __shfl_sync(0xffffffffu, r.dw, src);
      const float w0 = __shfl_sync(0xffffffffu, r.w0, src);
      const float dd0 = __shfl_sync(0xffffffffu, d0, src);
      const float ddt = __shfl_sync(0xffffffffu, r.dt, src);
      const float dke = __shfl_sync(0xffffffffu, ke, src);
      const int na = sel3(a, p.g.n[0], p.g.n[1], p.g.n[2]);
      const int nap = sel3(a, p.ql.nap[0], p.ql.nap[1], p.ql.nap[2]);
      const int nb = (a == 0) ? p.g.n[1] : p.g.n[0];
      const int nc = (a == 2) ? p.g.n[1] : p.g.n[2];
      const int nc2 = nc + 2;
      const float kc = 0.5f * (float)(na - 1);
      const float ub = (float)nb, wb = (float)nc;
      const int64_t qoff = sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
      // image strides along the plane axis a and the in-plane axes b, c
      const int sa = sel3(a, p.g.stride[0], p.g.stride[1], p.g.stride[2]);
      const int sb = (a == 0) ? p.g.stride[1] : p.g.stride[0];
      const int sc = (a == 2) ? p.g.stride[1] : p.g.stride[2];
      // forward
      float sum = 0.f;
      for (int k = k0 + gl; k <= k1; k += G) {
        const float kk = (float)k - kc;
        const float u = fminf(fmaxf(fmaf(kk, du, uc), -1.f), ub);
        const float w = fminf(fmaxf(fmaf(kk, dw, wc), -1.f), wb);
        const float fu = floorf(u), fw = floorf(w);
        const float al = u - fu, be = w - fw;
        float4 v;
        if (DIRECT) {
          const int i = (int)fu, j = (int)fw;
          const bool i0 = (unsigned)i < (unsigned)nb, i1 = (unsigned)(i + 1) < (unsigned)nb;
          const bool j0 = (unsigned)j < (unsigned)nc, j1 = (unsigned)(j + 1) < (unsigned)nc;
          const int64_t idx = (int64_t)k * sa + (int64_t)i * sb + (int64_t)j * sc;
          v.x = (i0 && j0) ? __ldg(p.img_in + idx) : 0.f;
          v.y = (i1 && j0) ? __ldg(p.img_in + idx + sb) : 0.f;
          v.z = (i0 && j1) ? __ldg(p.img_in + idx + sc) : 0.f;
          v.w = (i1 && j1) ? __ldg(p.img_in + idx + sb + sc) : 0.f;
        } else {
          v = __ldg(p.quads + qoff + (((int)fu + 1) * nc2 + ((int)fw + 1)) * nap + k);
        }
        const float top = fmaf(be, v.z - v.x, v.x);
        const float bot = fmaf(be, v.w - v.y, v.y);
        sum = fmaf(tof_weight<LUT>(lut, fmaf(kk, ddt, dd0), T, dke), fmaf(al, bot - top, top), sum);
      }
      sum = group_sum<G>(sum);
      // ratio and back projection of it
      const float coef0 = (k0 <= k1) ? w0 / fmaf(w0, sum, bg) : 0.f;
      for (int k = (k0 & ~(kGroupAlign<G> - 1)) + gl; k <= k1 && coef0 != 0.f; k += G) {
        if (k < k0) continue;
        const float kk = (float)k - kc;
        const float u = fminf(fmaxf(fmaf(kk, du, uc), -1.f), ub);
        const float w = fminf(fmaxf(fmaf(kk, dw, wc), -1.f), wb);
        const float fu = floorf(u), fw = floorf(w);
        const float al = u - fu, be = w - fw;
        const float coef = coef0 * tof_weight<LUT>(lut, fmaf(kk, ddt, dd0), T, dke);
        const float ca = (1.f - al) * coef, cb = al * coef;
        if (DIRECT) {
          const int i = (int)fu, j = (int)fw;
          const bool i0 = (unsigned)i < (unsigned)nb, i1 = (unsigned)(i + 1) < (unsigned)nb;
          const bool j0 = (unsigned)j < (unsigned)nc, j1 = (unsigned)(j + 1) < (unsigned)nc;
          const int64_t idx = (int64_t)k * sa + (int64_t)i * sb + (int64_t)j * sc;
          if (sc == 1 && j0 && j1) {
            // (j, j+1) are adjacent floats: an 8-byte-aligned pair takes one
            // vector reduction instead of two
            if (i0) red_pair(p.img_out + idx, ca * (1.f - be), ca * be);
            if (i1) red_pair(p.img_out + idx + sb, cb * (1.f - be), cb * be);
          } else {
            if (i0 && j0) atomicAdd(p.img_out + idx, ca * (1.f - be));
            if (i1 && j0) atomicAdd(p.img_out + idx + sb, cb * (1.f - be));
            if (i0 && j1) atomicAdd(p.img_out + idx + sc, ca * be);
            if (i1 && j1) atomicAdd(p.img_out + idx + sb + sc, cb * be);
          }
        } else {
          atomicAdd(p.quads_bp + qoff + (((int)fu + 1) * nc2 + ((int)fw + 1)) * nap + k,
                    make_float4(ca * (1.f - be), cb * (1.f - be), ca * be, cb * be));
        }
      }
    }
  }
}

// bp[v] folded from the back-projection quads (p.quads_bp, plane-fastest):
// the 4 quad slots that hold voxel v, over the axes the subset used
__device__ __forceinline__ float fold_bp(const ProjParams& p, const bool use[3], int64_t v) {
  const DevGeom& g = p.g;
  const int i0 = (int)(v / g.stride[0]);
  const int r0 = (int)(v - (int64_t)i0 * g.stride[0]);
  const int i1 = r0 / g.n[2], i2 = r0 - (r0 / g.n[2]) * g.n[2];
  float bp = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!use[a]) continue;
    const int k = (a == 0) ? i0 : (a == 1 ? i1 : i2);
    const int I = (a == 0) ? i1 : i0;
    const int J = (a == 2) ? i1 : i2;
    const int nc2 = p.ql.nc2[a], nb2 = p.ql.nb2[a];
    const int na = p.ql.nap[a];
    const float4* Q = p.quads_bp + p.ql.base[a];
    bp += Q[quad_index(true, k, I + 1, J + 1, na, nb2, nc2)].x + Q[quad_index(true, k, I, J + 1, na, nb2, nc2)].y +
          Q[quad_index(true, k, I + 1, J, na, nb2, nc2)].z + Q[quad_index(true, k, I, J, na, nb2, nc2)].w;
  }
  return bp;
}

// x[v] <- s[v] > 0 ? x[v] * bp[v] / (s[v] * scale) : 0
__global__ void osem_update_kernel(const ProjParams p, float* __restrict__ x) {
  bool use[3];
  for (int a = 0; a < 3; ++a) use[a] = slot_axis_used(p.axis_used, 0, a, 1, p.n_frames);
  const int64_t nvox = (int64_t)p.g.n[0] * p.g.n[1] * p.g.n[2];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (int64_t)gridDim.x * blockDim.x) {
    const float bp = fold_bp(p, use, v);
    const float sv = p.sens[v] * p.sens_scale;
    x[v] = sv > 0.f ? x[v] * bp / sv : 0.f;
  }
}

// z[v] = bp[v] (resolution-model path: H^T is applied to bp before the update)
__global__ void osem_fold_kernel(const ProjParams p, float* __restrict__ z) {
  bool use[3];
  for (int a = 0; a < 3; ++a) use[a] = slot_axis_used(p.axis_used, 0, a, 1, p.n_frames);
  const int64_t nvox = (int64_t)p.g.n[0] * p.g.n[1] * p.g.n[2];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (int64_t)gridDim.x * blockDim.x)
    z[v] = fold_bp(p, use, v);
}

// ---------------------------------------------------------------------------
// quad image build / clear / fold-back
// ---------------------------------------------------------------------------

__global__ void quad_build_kernel(const ProjParams p) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && p.counter) *p.counter = 0u;
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
  const int64_t total = sel3(a, p.ql.size[0], p.ql.size[1], p.ql.size[2]);
  const float* __restrict__ im = p.img_in + (int64_t)slot * p.img_stride;
  float4* Q = p.quads + (int64_t)slot * p.ql.slot + sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
  const int nb2 = nb + 2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int k, i, jj;
    if (p.kfast) {
      const int nap = sel3(a, p.ql.nap[0], p.ql.nap[1], p.ql.nap[2]);
      const int t = (int)(e / nap);
      k = (int)(e - (int64_t)t * nap);
      i = t / nc2 - 1;
      jj = t - (t / nc2) * nc2 - 1;
    } else {
      const int t = (int)(e / nc2);
      jj = (int)(e - (int64_t)t * nc2) - 1;
      k = t / nb2;
      i = t - k * nb2 - 1;
    }
    if (k >= na) {  // padding plane of an odd plane count
      Q[e] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
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

// Plane-fastest quads (p.kfast) of axes 0 and 1 are stored with k fastest
// while the image has its axis 2 (the quads' j) fastest, so a thread per
// quad entry reads the image with a large stride and a thread per voxel
// reads the quads with one.  The tiled kernels below stage a kT x kT
// (k, j) tile of one quad row through shared memory instead: both global
// sides are then read and written in their own fastest order.  (Axis 2 has
// k fastest on both sides; the same kernels handle it with k-fastest loops.)
constexpr int kT = 32;

// Builds plane-fastest quads from p.img_in: grid x over (j, k) tiles, y over
// quad rows i = -1 .. nb, z over (slot, axis); sized for the largest axis.
__global__ void __launch_bounds__(256) quad_build_tile_kernel(const ProjParams p) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && p.counter) *p.counter = 0u;
  const int slot = blockIdx.z / 3, a = blockIdx.z - 3 * (blockIdx.z / 3);
  if (!slot_axis_used(p.axis_used, slot, a, p.shared, p.n_frames)) return;
  const int b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
  const DevGeom& g = p.g;
  const int na = sel3(a, g.n[0], g.n[1], g.n[2]);
  const int nb = sel3(b, g.n[0], g.n[1], g.n[2]), nc = sel3(c, g.n[0], g.n[1], g.n[2]);
  const int sa = sel3(a, g.stride[0], g.stride[1], g.stride[2]);
  const int sb = sel3(b, g.stride[0], g.stride[1], g.stride[2]);
  const int sc = sel3(c, g.stride[0], g.stride[1], g.stride[2]);
  const int nap = sel3(a, p.ql.nap[0], p.ql.nap[1], p.ql.nap[2]);
  const int nc2 = nc + 2;
  const int i = (int)blockIdx.y - 1;  // quad base row
  if (i > nb) return;
  const int ktiles = (nap + kT - 1) / kT, jtiles = (nc2 + kT - 1) / kT;
  if ((int)blockIdx.x >= ktiles * jtiles) return;
  const int jt = blockIdx.x / ktiles, kt = blockIdx.x - jt * ktiles;
  const int j0 = jt * kT - 1, k0 = kt * kT;
  __shared__ float s[2][kT][kT + 1];  // [row i + r][k - k0][j - j0], j - j0 in 0..kT
  const float* __restrict__ im = p.img_in + (int64_t)slot * p.img_stride;
  for (int t = threadIdx.x; t < 2 * kT * (kT + 1); t += blockDim.x) {
    int r, kk, jj;
    if (a == 2) {  // image fastest along k
      kk = t % kT;
      const int u = t / kT;
      jj = u % (kT + 1);
      r = u / (kT + 1);
    } else {       // image fastest along j
      jj = t % (kT + 1);
      const int u = t / (kT + 1);
      kk = u % kT;
      r = u / kT;
    }
    const int k = k0 + kk, ii = i + r, j = j0 + jj;
    float v = 0.f;
    if (k < na && (unsigned)ii < (unsigned)nb && (unsigned)j < (unsigned)nc)
      v = __ldg(im + (int64_t)k * sa + (int64_t)ii * sb + (int64_t)j * sc);
    s[r][kk][jj] = v;
  }
  __syncthreads();
  float4* Q = p.quads + (int64_t)slot * p.ql.slot + sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
  for (int t = threadIdx.x; t < kT * kT; t += blockDim.x) {
    const int kk = t % kT, jj = t / kT;
    const int k = k0 + kk, j = j0 + jj;
    if (k >= nap || j > nc) continue;
    Q[((int64_t)(i + 1) * nc2 + (j + 1)) * nap + k] =
        make_float4(s[0][kk][jj], s[1][kk][jj], s[0][kk][jj + 1], s[1][kk][jj + 1]);
  }
}

// out[slot] (=|+=) the fold of axis a's plane-fastest quads (base quads_base,
// slot stride ql.slot): voxel (k, I, J) of the axis collects the four quad
// slots that hold it.  ADD = false writes every voxel (0 where the axis is
// unused), so a sequence "axis 0 write, axes 1 and 2 add" needs no zeroing.
// Grid x over (J, k) tiles, y over I = 0 .. nb - 1, z over slots.
template <bool ADD>
__global__ void __launch_bounds__(256) quad_fold_tile_kernel(const ProjParams p, const float4* __restrict__ quads_base,
                                                             float* __restrict__ out_base, int a) {
  const int slot = blockIdx.z;
  const bool used = slot_axis_used(p.axis_used, slot, a, p.shared, p.n_frames);
  if (ADD && !used) return;
  const int b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
  const DevGeom& g = p.g;
  const int na = sel3(a, g.n[0], g.n[1], g.n[2]);
  const int nc = sel3(c, g.n[0], g.n[1], g.n[2]);
  const int sa = sel3(a, g.stride[0], g.stride[1], g.stride[2]);
  const int sb = sel3(b, g.stride[0], g.stride[1], g.stride[2]);
  const int sc = sel3(c, g.stride[0], g.stride[1], g.stride[2]);
  const int nap = sel3(a, p.ql.nap[0], p.ql.nap[1], p.ql.nap[2]);
  const int nc2 = nc + 2;
  const int I = blockIdx.y;
  const int ktiles = (na + kT - 1) / kT;
  const int jt = blockIdx.x / ktiles, kt = blockIdx.x - jt * ktiles;
  const int J0 = jt * kT, k0 = kt * kT;
  // component planes: 0 = x and 1 = z of padded row I + 1, 2 = y and 3 = w
  // of padded row I; [plane][padded col - J0][k - k0]
  __shared__ float s[4][kT + 1][kT + 1];
  if (used) {
    const float4* Q = quads_base + (int64_t)slot * p.ql.slot + sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
    for (int t = threadIdx.x; t < 2 * (kT + 1) * kT; t += blockDim.x) {
      const int kk = t % kT;
      const int u = t / kT;
      const int pjj = u % (kT + 1), r = u / (kT + 1);
      const int k = k0 + kk, pj = J0 + pjj;
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < na && pj <= nc + 1) q = Q[((int64_t)(I + r) * nc2 + pj) * nap + k];
      if (r) {
        s[0][pjj][kk] = q.x;
        s[1][pjj][kk] = q.z;
      } else {
        s[2][pjj][kk] = q.y;
        s[3][pjj][kk] = q.w;
      }
    }
  }
  __syncthreads();
  float* out = out_base + (int64_t)slot * p.img_stride;
  for (int t = threadIdx.x; t < kT * kT; t += blockDim.x) {
    int kk, jj;
    if (a == 2) {
      kk = t % kT;
      jj = t / kT;
    } else {
      jj = t % kT;
      kk = t / kT;
    }
    const int k = k0 + kk, J = J0 + jj;
    if (k >= na || J >= nc) continue;
    const float val = used ? s[0][jj + 1][kk] + s[2][jj + 1][kk] + s[1][jj][kk] + s[3][jj][kk] : 0.f;
    const int64_t v = (int64_t)k * sa + (int64_t)I * sb + (int64_t)J * sc;
    out[v] = ADD ? out[v] + val : val;
  }
}

// x[v] <- s[v] * scale > 0 ? x[v] * bp[v] / (s[v] * scale) : 0
__global__ void img_update_kernel(float* __restrict__ x, const float* __restrict__ bp, const float* __restrict__ sens,
                                  float scale, int64_t nvox) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (int64_t)gridDim.x * blockDim.x) {
    const float sv = __ldg(sens + v) * scale;
    x[v] = sv > 0.f ? x[v] * __ldg(bp + v) / sv : 0.f;
  }
}

__global__ void quad_zero_kernel(const ProjParams p) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && p.counter) *p.counter = 0u;
  const int slot = blockIdx.y / 3, a = blockIdx.y - 3 * (blockIdx.y / 3);
  if (!slot_axis_used(p.axis_used, slot, a, p.shared, p.n_frames)) return;
  const int64_t total = sel3(a, p.ql.size[0], p.ql.size[1], p.ql.size[2]);
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
      const int nc2 = p.ql.nc2[a], nb2 = p.ql.nb2[a];
      const int na = p.ql.nap[a];
      const float4* Q = Qs + p.ql.base[a];
      const bool kf = p.kfast;
      // padded positions: voxel I sits at I + 1
      s += Q[quad_index(kf, k, I + 1, J + 1, na, nb2, nc2)].x + Q[quad_index(kf, k, I, J + 1, na, nb2, nc2)].y +
           Q[quad_index(kf, k, I + 1, J, na, nb2, nc2)].z + Q[quad_index(kf, k, I, J, na, nb2, nc2)].w;
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
          if (T.user) {
            for (int t = t0; t <= t1; ++t)
              acc[t * blockDim.x] += user_g(fmaf(-(float)(t - t0), T.width, dlo), T) * s;
            continue;
          }
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
        float sy = 0.f;
        if (T.user) {
          for (int t = t0; t <= t1; ++t)
            sy += user_g(fmaf(-(float)(t - t0), T.width, dlo), T) * acc[t * blockDim.x];
        } else {
          float e_hi = erff((dlo + T.half) * T.k);
          for (int t = t0; t <= t1; ++t) {
            const float dist = fmaf(-(float)(t - t0), T.width, dlo);
            const float e_lo = erff((dist - T.half) * T.k);
            sy += 0.5f * (e_hi - e_lo) * acc[t * blockDim.x];
            e_hi = e_lo;
          }
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
  if (p.max_per_sm > 0 && per_sm > p.max_per_sm) per_sm = p.max_per_sm;
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

template <int MODE, bool BACK, bool LUT, int G>
int launch_group(const ProjParams& p, int block, cudaStream_t st) {
  auto kern = group_kernel<MODE, BACK, LUT, G>;
  const size_t smem = (MODE != 0 && LUT) ? kLut * sizeof(float2) : 0;
  int per_sm = 0;
  JP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem));
  if (p.max_per_sm > 0 && per_sm > p.max_per_sm) per_sm = p.max_per_sm;
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

template <int MODE, bool BACK, bool LUT>
int launch_group_lpw(const ProjParams& p, int block, int lpw, cudaStream_t st) {
  switch (lpw) {
    case 1: return launch_group<MODE, BACK, LUT, 32>(p, block, st);
    case 2: return launch_group<MODE, BACK, LUT, 16>(p, block, st);
    case 4: return launch_group<MODE, BACK, LUT, 8>(p, block, st);
    case 8: return launch_group<MODE, BACK, LUT, 4>(p, block, st);
    case 16: return launch_group<MODE, BACK, LUT, 2>(p, block, st);
    default: return launch_planned<MODE, BACK, LUT>(p, block, st);
  }
}

template <bool LUT>
int launch_sino_back(const ProjParams& p, int block, int lpw, cudaStream_t st) {
  switch (lpw) {
    case 1: return launch_group<1, true, LUT, 32>(p, block, st);
    case 2: return launch_group<1, true, LUT, 16>(p, block, st);
    case 4: return launch_group<1, true, LUT, 8>(p, block, st);
    default: return launch_planned<1, true, LUT>(p, block, st);
  }
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

// per-axis extents (n_a, n_b, n_c) of the quad images
void axis_dims(const DevGeom& g, int a, int* na, int* nb, int* nc) {
  *na = g.n[a];
  *nb = (a == 0) ? g.n[1] : g.n[0];
  *nc = (a == 2) ? g.n[1] : g.n[2];
}

// the tiled kernels index rows through gridDim.y
bool tiles_fit(const DevGeom& g) {
  for (int a = 0; a < 3; ++a) {
    int na, nb, nc;
    axis_dims(g, a, &na, &nb, &nc);
    if (nb + 2 > 65535) return false;
  }
  return true;
}

// plane-fastest quads of every (slot, axis) from p.img_in
int launch_quad_build_tile(const ProjParams& p, int slots, cudaStream_t st) {
  int gx = 1, gy = 1;
  for (int a = 0; a < 3; ++a) {
    int na, nb, nc;
    axis_dims(p.g, a, &na, &nb, &nc);
    const int nap = p.ql.nap[a];
    gx = std::max(gx, ((nap + kT - 1) / kT) * ((nc + 2 + kT - 1) / kT));
    gy = std::max(gy, nb + 2);
  }
  quad_build_tile_kernel<<<dim3(gx, gy, slots * 3), 256, 0, st>>>(p);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

// out[slot] (+)= fold of the plane-fastest quads at `quads` over all axes;
// add_all = false overwrites out with the fold (axis 0 writes, 1 and 2 add)
int launch_quad_fold_tile(const ProjParams& p, const float4* quads, float* out, int slots, bool add_all,
                          cudaStream_t st) {
  for (int a = 0; a < 3; ++a) {
    int na, nb, nc;
    axis_dims(p.g, a, &na, &nb, &nc);
    const dim3 grid(((nc + kT - 1) / kT) * ((na + kT - 1) / kT), nb, slots);
    if (a == 0 && !add_all)
      quad_fold_tile_kernel<false><<<grid, 256, 0, st>>>(p, quads, out, a);
    else
      quad_fold_tile_kernel<true><<<grid, 256, 0, st>>>(p, quads, out, a);
    count_launch();
    JP_TRY_CUDA(cudaGetLastError());
  }
  return JP_OK;
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
  if ((pl->opts.flags & JP_PLAN_INTERLEAVED) && img_stride != 0)
    return fail(JP_ERR_ARG, "frames of an interleaved plan share one image (img_stride must be 0)");
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
  p.counter = pl->work_counter;
  p.perm_in_rec = pl->has_delta ? 0 : 1;
  p.max_per_sm = pl->opts.max_ctas_per_sm;
  if (back) { p.proj_in = in; p.img_out = out; } else { p.img_in = in; p.proj_out = out; }
  const int slots = p.shared ? 1 : pl->n_frames;
  if (slots * 3 > 65535) return fail(JP_ERR_ARG, "too many frames with distinct images (max 21845)");
  if (pl->has_sigma && mode == 2) p.sig = pl->sig_binned;
  if (pl->has_sigma && mode == 1) return fail(JP_ERR_STATE, "per-event sigma applies to TOF listmode only");
  // a tabulated kernel always goes through the shared-memory table; a
  // per-event sigma takes the exact path (the table holds one sigma)
  const bool lut = (mode != 0) && ((!(pl->opts.flags & JP_PLAN_TOF_EXACT) && !p.sig) || p.tof.user);
  // default CTA sizes of the forwards: 512 threads for the TOF sinogram
  // (three CTAs of 512 keep 48 warps resident, its shared-memory accumulators
  // allow no more), 128 for non-TOF and TOF listmode (a persistent CTA's
  // chunk of binned LORs is then narrower: TOF-LM 5.14 vs 5.18 ms, non-TOF
  // 8.24 vs 8.38 ms per 40M-event frame against 256)
  const int want_block = (pl->auto_block && !back) ? (mode == 1 ? kMaxBlock : 128) : pl->opts.block;
  const int block = pick_block(want_block, mode, p.tof, lut);
  cudaStream_t st = (cudaStream_t)stream;
  int lpw = pl->opts.lors_per_warp;
  const bool sorted = !(pl->opts.flags & (JP_PLAN_KEEP_ORDER | JP_PLAN_INTERLEAVED));
  if (sorted && mode != 1 && (pl->opts.flags & JP_PLAN_TILES) &&
      (lpw == 0 || lpw == 1 || lpw == 2 || lpw == 4 || lpw == 8)) {
    // shared-memory tiles over the plan's lines (frame, axis, slope, offset)
    p.line_end = pl->hist;
    p.lines_per_axis = pl->dims.slope_bins * pl->dims.offset_bins;
    p.lines_per_frame = 3 * p.lines_per_axis;
    p.keys_per_line = pl->dims.window_bins * pl->dims.zoff_bins;
    p.n_lines = (int64_t)pl->n_frames * p.lines_per_frame;
    for (int a = 0; a < 3; ++a) p.kb[a] = pl->kb[a];
    p.tile_T = pl->opts.tile_lors;
    p.line_batch = 4;
    p.vec4_out = back && aligned(out, 16) && (p.shared || (img_stride % 4) == 0);
    const int lanes = (lpw == 1) ? 32 : (lpw == 2) ? 16 : (lpw == 8) ? 4 : 8;
    return launch_tile(p, mode, back, lut, lanes, std::min(pl->opts.block, kMaxBlock), st);
  }
  const int64_t max_quad = std::max(std::max(p.ql.size[0], p.ql.size[1]), p.ql.size[2]);
  if (lpw == 0) lpw = (!back || mode == 1) ? 32 : 4;
  if (mode == 1 && !back) lpw = 32;
  p.kfast = (lpw == 32) ? 0 : 1;
  dim3 qgrid(aux_grid(max_quad, 256), slots * 3);
  const bool tiled = p.kfast && tiles_fit(p.g);
  if (!back && tiled) {
    rc = launch_quad_build_tile(p, slots, st);
    if (rc) return rc;
  } else {
    if (!back)
      quad_build_kernel<<<qgrid, 256, 0, st>>>(p);
    else
      quad_zero_kernel<<<qgrid, 256, 0, st>>>(p);
    count_launch();
    JP_TRY_CUDA(cudaGetLastError());
  }
  switch (mode * 4 + (back ? 2 : 0) + (lut ? 1 : 0)) {
    case 0: rc = launch_group_lpw<0, false, false>(p, block, lpw, st); break;
    case 2: rc = launch_group_lpw<0, true, false>(p, block, lpw, st); break;
    case 4: rc = launch_planned<1, false, false>(p, block, st); break;
    case 5: rc = launch_planned<1, false, true>(p, block, st); break;
    case 6: rc = launch_sino_back<false>(p, block, lpw, st); break;
    case 7: rc = launch_sino_back<true>(p, block, lpw, st); break;
    case 8: rc = launch_group_lpw<2, false, false>(p, block, lpw, st); break;
    case 9: rc = launch_group_lpw<2, false, true>(p, block, lpw, st); break;
    case 10: rc = launch_group_lpw<2, true, false>(p, block, lpw, st); break;
    case 11: rc = launch_group_lpw<2, true, true>(p, block, lpw, st); break;
    default: return fail(JP_ERR_ARG, "bad mode");
  }
  if (rc) return rc;
  if (back && tiled) return launch_quad_fold_tile(p, p.quads, p.img_out, slots, true, st);
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

// per-LOR count of visited plane samples (same setup as the projectors);
// MODE 1: TOF-sinogram bin evaluations, the bins of every visited sample's
// window (the sinogram kernels' per-bin work)
template <int MODE>
__global__ void count_kernel(const ProjParams p, unsigned long long* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cnt = 0;
  if (i < p.n) {
    const float4 A = __ldcs(p.lor + 2 * i);
    const float4 B = __ldcs(p.lor + 2 * i + 1);
    float xs[3] = {A.x, A.y, A.z}, xe[3] = {B.x, B.y, B.z};
    Ray r;
    bool live = ray_setup(xs, xe, p.g, r);
    if (live && MODE == 2) {
      float ke, Re;
      event_tof(p, i, ke, Re);
      const float c = (float)__float_as_int(B.w) * p.tof.width + (p.perm_in_rec ? 0.f : A.w);
      const float d0 = r.tc - c;
      const float t1 = (-Re - d0) / r.dt, t2 = (Re - d0) / r.dt;
      const float lo = fmaxf(ceilf(r.kc + fminf(t1, t2)), (float)r.k0);
      const float hi = fminf(floorf(r.kc + fmaxf(t1, t2)), (float)r.k1);
      r.k0 = (int)lo;
      r.k1 = (int)hi;
      live = lo <= hi;
    }
    if (live && MODE != 1) cnt = (unsigned long long)(r.k1 - r.k0 + 1);
    if (live && MODE == 1) {
      const DevTof& T = p.tof;
      const float delta = p.perm_in_rec ? 0.f : A.w;
      for (int k = r.k0; k <= r.k1; ++k) {
        const float tau = fmaf((float)k - r.kc, r.dt, r.tc);
        const float x = (tau - delta) * T.inv_w + T.hbin;
        const int t0 = max(0, (int)ceilf(x - T.R_over_w));
        const int t1 = min(T.nbins - 1, (int)floorf(x + T.R_over_w));
        if (t0 <= t1) cnt += (unsigned long long)(t1 - t0 + 1);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

// Throughput ceiling of the TOF-sinogram kernels' per-bin work, on
// synthetic sample positions: the bins of each window through the
// bin-aligned table (one shared-memory table read and an interpolation per
// bin), accumulated into the thread's shared-memory bins (DIR 0, the
// forward's operation) or multiplied with the thread's shared-memory values
// and summed (DIR 1, the back projection's); *bins counts the bins done.
template <int DIR>
__global__ void bench_tof_bins_kernel(const DevTof T, int per_thread, unsigned long long* bins, float* sink) {
  extern __shared__ float4 smem4[];
  float2* lut = reinterpret_cast<float2*>(smem4);
  float* acc = reinterpret_cast<float*>(lut + kLut) + threadIdx.x;
  build_lut_aligned(lut, T);
  const int N = T.nbins;
  for (int t = 0; t < N; ++t) acc[t * blockDim.x] = DIR ? 1.f : 0.f;
  __syncthreads();
  uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
  unsigned long long nb = 0;
  float sy = 0.f;
  for (int it = 0; it < per_thread; ++it) {
    h = h * 1664525u + 1013904223u;
    const float x = (float)(h >> 8) * (1.0f / 16777216.0f) * (float)N - 0.5f;  // position in bins
    const int t0 = max(0, (int)ceilf(x - T.R_over_w));
    const int t1 = min(N - 1, (int)floorf(x + T.R_over_w));
    const float dlo = (x - T.hbin) * T.width - ((float)t0 - T.hbin) * T.width;
    const float xl0 = (dlo + T.Rp) * T.inv_hp;
    const int ix0 = min(max((int)xl0, 0), T.nodes_a - 1);
    const float fr = xl0 - (float)ix0;
    const float sv = 1.f + 1e-3f * x;
    float* a = acc + t0 * blockDim.x;
    for (int t = 0, ix = ix0; t <= t1 - t0; ++t, ix -= T.m, a += blockDim.x) {
      const float2 e = lut[max(ix, 0)];
      if (DIR == 0) *a = fmaf(fmaf(fr, e.y, e.x), sv, *a);
      else sy = fmaf(fmaf(fr, e.y, e.x), *a, sy);
    }
    nb += (unsigned long long)max(t1 - t0 + 1, 0);
  }
  if (DIR == 0)
    for (int t = 0; t < N; ++t) sy += acc[t * blockDim.x];
  if (sy == 1234.5f) sink[blockIdx.x] = sy;  // keeps the work
  for (int o = 16; o > 0; o >>= 1) nb += __shfl_down_sync(0xffffffffu, nb, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(bins, nb);
}

// L2 reduction requests of the quad-image group back projection
// (group_kernel<MODE, true, *, G>), counted by replaying its schedule: the
// same 32-LOR warp chunks, the same lane -> (LOR, plane) map and the same
// quad entries, with every LOR live (a back-projection input without
// zeros).  A warp's 16-byte vector reductions coalesce per instruction into
// one request per 32-byte sector and lane slot: a sector holds two quad
// entries (planes 2m, 2m+1), so it costs max(lanes on the even entry, lanes
// on the odd one) requests.
template <int MODE, int G>
__global__ void red_count_kernel(const ProjParams p, unsigned long long* out) {
  constexpr int E = 32 / G;
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, gl = lane - grp * G;
  const DevTof& T = p.tof;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long cnt = 0;
  for (int64_t chunk = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); chunk * 32 < p.n;
       chunk += warps) {
    const int64_t base = chunk * 32;
    const int64_t i = base + lane;
    Ray r;
    r.k0 = 1; r.k1 = 0;
    int slot = 0;
    if (i < p.n) {
      const float4 A = __ldcs(p.lor + 2 * i);
      const float4 B = __ldcs(p.lor + 2 * i + 1);
      const float xs[3] = {A.x, A.y, A.z};
      const float xe[3] = {B.x, B.y, B.z};
      const float delta = p.perm_in_rec ? 0.f : A.w;
      const int f = (p.n_frames > 1) ? frame_of(p.frame_off, p.n_frames, i) : 0;
      slot = p.shared ? 0 : f;
      bool live = ray_setup(xs, xe, p.g, r);
      if (MODE == 2 && live) {
        float ke, Re;
        event_tof(p, i, ke, Re);
        const float d0 = r.tc - ((float)__float_as_int(B.w) * T.width + delta);
        const float t1 = (-Re - d0) / r.dt, t2 = (Re - d0) / r.dt;
        const float lo = fmaxf(ceilf(r.kc + fminf(t1, t2)), (float)r.k0);
        const float hi = fminf(floorf(r.kc + fmaxf(t1, t2)), (float)r.k1);
        r.k0 = (int)lo;
        r.k1 = (int)hi;
        live = lo <= hi;
      }
      if (!live) { r.k0 = 1; r.k1 = 0; }
    } else {
      r.a = 0; r.uc = r.du = r.wc = r.dw = 0.f;
    }
#pragma unroll 1
    for (int pass = 0; pass < G; ++pass) {
      const int src = pass * E + grp;
      const int k0 = __shfl_sync(0xffffffffu, r.k0, src);
      const int k1 = __shfl_sync(0xffffffffu, r.k1, src);
      const int a = __shfl_sync(0xffffffffu, r.a, src);
      const int sl = __shfl_sync(0xffffffffu, slot, src);
      const float uc = __shfl_sync(0xffffffffu, r.uc, src);
      const float du = __shfl_sync(0xffffffffu, r.du, src);
      const float wc = __shfl_sync(0xffffffffu, r.wc, src);
      const float dw = __shfl_sync(0xffffffffu, r.dw, src);
      const int na = sel3(a, p.g.n[0], p.g.n[1], p.g.n[2]);
      const int nap = sel3(a, p.ql.nap[0], p.ql.nap[1], p.ql.nap[2]);
      const int nb = (a == 0) ? p.g.n[1] : p.g.n[0];
      const int nc = (a == 2) ? p.g.n[1] : p.g.n[2];
      const int nc2 = nc + 2;
      const float kc = 0.5f * (float)(na - 1);
      const float ub = (float)nb, wb = (float)nc;
      const int64_t qoff = (int64_t)sl * p.ql.slot + sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
      // iterations of the group's plane loop, k = (k0 & ~(A - 1)) + gl + G s,
      // A = kGroupAlign<G>
      const int kfirst = (k0 & ~(kGroupAlign<G> - 1)) + gl;
      const int nit = (k0 <= k1 && kfirst <= k1) ? (k1 - kfirst) / G + 1 : 0;
      const int maxit = __reduce_max_sync(0xffffffffu, nit);
      for (int s = 0; s < maxit; ++s) {
        const int k = kfirst + G * s;
        const bool active = s < nit && k >= k0;
        int64_t entry = 0;
        if (active) {
          const float kk = (float)k - kc;
          const float u = fminf(fmaxf(fmaf(kk, du, uc), -1.f), ub);
          const float w = fminf(fmaxf(fmaf(kk, dw, wc), -1.f), wb);
          entry = qoff + (((int)floorf(u) + 1) * nc2 + ((int)floorf(w) + 1)) * nap + k;
        }
        const unsigned am = __ballot_sync(0xffffffffu, active);
        const unsigned odd = __ballot_sync(0xffffffffu, active && (entry & 1));
        if (active) {
          const unsigned ms = __match_any_sync(am, (unsigned long long)(entry >> 1));
          if (lane == __ffs(ms) - 1) {
            const int no = __popc(ms & odd), ne = __popc(ms) - no;
            cnt += (unsigned long long)max(no, ne);
          }
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if (lane == 0 && cnt) atomicAdd(out, cnt);
}

template <int MODE>
int launch_red_count(const ProjParams& p, int lpw, unsigned long long* out, cudaStream_t st) {
  const int grid = aux_grid((p.n + 31) / 32 * 32, 256);
  switch (lpw) {
    case 1: red_count_kernel<MODE, 32><<<grid, 256, 0, st>>>(p, out); break;
    case 2: red_count_kernel<MODE, 16><<<grid, 256, 0, st>>>(p, out); break;
    case 8: red_count_kernel<MODE, 4><<<grid, 256, 0, st>>>(p, out); break;
    case 16: red_count_kernel<MODE, 2><<<grid, 256, 0, st>>>(p, out); break;
    default: red_count_kernel<MODE, 8><<<grid, 256, 0, st>>>(p, out); break;
  }
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

}  // namespace
}  // namespace jp

using namespace jp;

extern "C" int jp_count_red_requests(jp_plan pl, int32_t mode, const jp_tof* t, uint64_t* out, void* stream) {
  clear_error();
  if (!pl || !out) return fail(JP_ERR_ARG, "NULL argument");
  if (mode != 0 && mode != 2) return fail(JP_ERR_ARG, "mode must be 0 or 2");
  if (!aligned(out, 8)) return fail(JP_ERR_ALIGN, "out must be 8-byte aligned");
  if (mode == 2 && !pl->has_tof_bin) return fail(JP_ERR_STATE, "TOF listmode needs a plan created with tof_bin");
  int lpw = pl->opts.lors_per_warp;
  if (lpw == 0) lpw = 4;
  if (lpw == 32 || (pl->opts.flags & (JP_PLAN_TILES | JP_PLAN_INTERLEAVED)))
    return fail(JP_ERR_STATE, "the plan's back projection does not run the quad-image group kernel");
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
  p.frame_off = pl->frame_off_dev;
  p.n_frames = pl->n_frames;
  p.ql = pl->ql;
  p.shared = 0;  // frames with their own image slots: the launch with the largest footprint
  p.perm_in_rec = pl->has_delta ? 0 : 1;
  if (mode == 2 && pl->has_sigma) p.sig = pl->sig_binned;
  cudaStream_t st = (cudaStream_t)stream;
  JP_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
  if (p.n == 0) return JP_OK;
  return mode == 0 ? launch_red_count<0>(p, lpw, (unsigned long long*)out, st)
                   : launch_red_count<2>(p, lpw, (unsigned long long*)out, st);
}

extern "C" int jp_count_samples(jp_plan pl, int32_t mode, const jp_tof* t, uint64_t* out, void* stream) {
  clear_error();
  if (!pl || !out) return fail(JP_ERR_ARG, "NULL argument");
  if (mode < 0 || mode > 2) return fail(JP_ERR_ARG, "mode must be 0, 1 or 2");
  if (!aligned(out, 8)) return fail(JP_ERR_ALIGN, "out must be 8-byte aligned");
  if (mode == 2 && !pl->has_tof_bin) return fail(JP_ERR_STATE, "TOF listmode needs a plan created with tof_bin");
  ProjParams p;
  std::memset(&p, 0, sizeof(p));
  int rc = make_geom(&pl->g, &p.g);
  if (rc) return rc;
  if (mode != 0) {
    rc = make_tof(t, mode == 1, &p.tof);
    if (rc) return rc;
  }
  p.lor = pl->lor;
  p.n = pl->n;
  p.perm_in_rec = pl->has_delta ? 0 : 1;
  if (mode == 2 && pl->has_sigma) p.sig = pl->sig_binned;
  cudaStream_t st = (cudaStream_t)stream;
  JP_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
  if (p.n == 0) return JP_OK;
  unsigned blocks = (unsigned)((p.n + 255) / 256);
  if (mode == 0) count_kernel<0><<<blocks, 256, 0, st>>>(p, (unsigned long long*)out);
  else if (mode == 1) count_kernel<1><<<blocks, 256, 0, st>>>(p, (unsigned long long*)out);
  else count_kernel<2><<<blocks, 256, 0, st>>>(p, (unsigned long long*)out);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

extern "C" int jp_bench_tof_bins(const jp_tof* t, int32_t direction, int32_t per_thread, float* ms_out,
                                 uint64_t* bins_out, void* stream) {
  clear_error();
  if (!ms_out || !bins_out || per_thread < 1 || (direction != 0 && direction != 1))
    return fail(JP_ERR_ARG, "bad arguments");
  if (!aligned(bins_out, 8)) return fail(JP_ERR_ALIGN, "bins_out must be 8-byte aligned");
  DevTof T;
  int rc = make_tof(t, true, &T);
  if (rc) return rc;
  if (T.user || T.m <= 0) return fail(JP_ERR_ARG, "needs a Gaussian kernel with a bin-aligned table");
  // the CTA size of the projection it stands for: 512 threads for the
  // forward, 256 for the back projection, and 256 when 512 threads' bins
  // would not fit in shared memory
  int block = direction ? 256 : kMaxBlock;
  if ((size_t)kLut * sizeof(float2) + (size_t)T.nbins * block * sizeof(float) > 96 * 1024) block = 256;
  const size_t smem = (size_t)kLut * sizeof(float2) + (size_t)T.nbins * block * sizeof(float);
  cudaStream_t st = (cudaStream_t)stream;
  auto k0 = bench_tof_bins_kernel<0>;
  auto k1 = bench_tof_bins_kernel<1>;
  rc = prepare_smem(k0, smem);
  if (rc) return rc;
  rc = prepare_smem(k1, smem);
  if (rc) return rc;
  int per_sm = 0;
  JP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, direction ? k1 : k0, block, smem));
  const int grid = sm_count() * (per_sm < 1 ? 1 : per_sm);
  float* sink = nullptr;
  JP_TRY_CUDA(cudaMemsetAsync(bins_out, 0, sizeof(uint64_t), st));
  // warm-up launch (its bins are counted, then cleared)
  if (direction) k1<<<grid, block, smem, st>>>(T, per_thread, (unsigned long long*)bins_out, sink);
  else k0<<<grid, block, smem, st>>>(T, per_thread, (unsigned long long*)bins_out, sink);
  count_launch();
  JP_TRY_CUDA(cudaMemsetAsync(bins_out, 0, sizeof(uint64_t), st));
  cudaEvent_t a, b;
  JP_TRY_CUDA(cudaEventCreate(&a));
  JP_TRY_CUDA(cudaEventCreate(&b));
  JP_TRY_CUDA(cudaEventRecord(a, st));
  if (direction) k1<<<grid, block, smem, st>>>(T, per_thread, (unsigned long long*)bins_out, sink);
  else k0<<<grid, block, smem, st>>>(T, per_thread, (unsigned long long*)bins_out, sink);
  count_launch();
  JP_TRY_CUDA(cudaEventRecord(b, st));
  JP_TRY_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  JP_TRY_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms_out = ms;
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

namespace jp {
namespace {
// One listmode-OSEM subset update; with res non-NULL the resolution model H
// wraps the projections (x -> H x before the forward projection, H^T on the
// back projection before the update), using work[0 .. 2 nvox).  path: one of
// JP_OSEM_PATH_* (AUTO takes the direct path for subsets of fewer than
// nvox / JP_OSEM_DIRECT_VOXELS_PER_EVENT events when their count is known on
// the host: below that the quad path's image-sized build, clear and fold
// cost more than the direct path's scalar atomics).

int osem_subset(jp_plan pl, int32_t f0, int32_t f1, float* x, const float* sens, float sens_scale, float b,
                const float* b_dev, const jp_tof* t, const jp_resolution* res, int32_t path, float* work,
                void* stream) {
  clear_error();
  if (!pl) return fail(JP_ERR_ARG, "plan is NULL");
  if (!(pl->opts.flags & JP_PLAN_INTERLEAVED)) return fail(JP_ERR_STATE, "OSEM subsets need a JP_PLAN_INTERLEAVED plan");
  if (!pl->has_tof_bin) return fail(JP_ERR_STATE, "TOF listmode needs a plan created with tof_bin");
  if (f0 < 0 || f1 > pl->n_frames || f0 > f1) return fail(JP_ERR_ARG, "frame range outside the plan");
  if (!x || !sens) return fail(JP_ERR_ARG, "x / sens is NULL");
  if (!aligned(x, 4) || !aligned(sens, 4) || !aligned(b_dev, 4)) return fail(JP_ERR_ALIGN, "arrays must be 4-byte aligned");
  if (!(sens_scale > 0.f) || !isfinite(sens_scale)) return fail(JP_ERR_ARG, "sens_scale must be finite and > 0");
  if (!b_dev && (!(b >= 0.f) || !isfinite(b))) return fail(JP_ERR_ARG, "b must be finite and >= 0");
  if (path != JP_OSEM_PATH_AUTO && path != JP_OSEM_PATH_QUADS && path != JP_OSEM_PATH_DIRECT)
    return fail(JP_ERR_ARG, "path must be JP_OSEM_PATH_AUTO, _QUADS or _DIRECT");
  ProjParams p;
  std::memset(&p, 0, sizeof(p));
  int rc = make_geom(&pl->g, &p.g);
  if (rc) return rc;
  rc = make_tof(t, false, &p.tof);
  if (rc) return rc;
  const int64_t nvox = (int64_t)p.g.n[0] * p.g.n[1] * p.g.n[2];
  GaussTaps taps;
  float *wy = nullptr, *wt = nullptr;
  if (res) {
    rc = make_taps(&pl->g, res, &taps);
    if (rc) return rc;
    if (!work) return fail(JP_ERR_ARG, "work is NULL");
    if (!aligned(work, 4)) return fail(JP_ERR_ALIGN, "work must be 4-byte aligned");
    const uintptr_t w0 = reinterpret_cast<uintptr_t>(work), w1 = w0 + 2 * nvox * sizeof(float);
    const uintptr_t xa = reinterpret_cast<uintptr_t>(x), sa = reinterpret_cast<uintptr_t>(sens);
    const uintptr_t nb = nvox * sizeof(float);
    if ((xa < w1 && w0 < xa + nb) || (sa < w1 && w0 < sa + nb))
      return fail(JP_ERR_ARG, "work must not overlap x or sens");
    wy = work;
    wt = work + nvox;
  }
  // the event count is known only on the device when b is read there (a
  // captured graph serves every frame bound later): size the grid by the
  // host-side count when it is current, else fill the GPU
  const int64_t host_n = b_dev ? pl->capacity : pl->frame_off_host[f1] - pl->frame_off_host[f0];
  const bool tiled = tiles_fit(p.g);
  bool direct = path == JP_OSEM_PATH_DIRECT;
  if (path == JP_OSEM_PATH_AUTO) direct = !b_dev && host_n < nvox / JP_OSEM_DIRECT_VOXELS_PER_EVENT;
  if (direct && !pl->fold_img) return fail(JP_ERR_STATE, "plan has no fold image");
  p.lor = pl->lor;
  p.perm = pl->perm;
  p.frame_off = pl->frame_off_dev;
  p.n_frames = pl->n_frames;
  p.f0 = f0;
  p.f1 = f1;
  p.n = pl->capacity;  // upper bound only; the kernel reads its range on the device
  p.ql = pl->ql;
  p.axis_used = pl->axis_used;
  p.shared = 1;
  p.kfast = 1;
  p.img_in = x;
  cudaStream_t st = (cudaStream_t)stream;
  if (res) {
    // y = H x (passes x -> y -> t -> y); the forward projection reads y
    rc = gauss_passes(x, wy, wt, wy, 1, p.g, taps, nullptr, 0.f, st);
    if (rc) return rc;
    p.img_in = wy;
  }
  p.quads = pl->quads;
  p.quads_bp = pl->quads + pl->ql.slot;
  p.bg = b;
  p.bg_ptr = b_dev;
  p.sens = sens;
  p.sens_scale = sens_scale;
  p.counter = pl->work_counter;
  p.perm_in_rec = pl->has_delta ? 0 : 1;
  p.sig = pl->has_sigma ? pl->sig_binned : nullptr;
  // back-projection image of the direct path (and of the quads path's fold)
  float* bp_img = res ? wt : pl->fold_img;
  const int64_t max_quad = std::max(std::max(p.ql.size[0], p.ql.size[1]), p.ql.size[2]);
  dim3 qgrid(aux_grid(max_quad, 256), 3);
  if (direct) {
    p.img_out = bp_img;
    JP_TRY_CUDA(cudaMemsetAsync(bp_img, 0, sizeof(float) * nvox, st));
    JP_TRY_CUDA(cudaMemsetAsync(p.counter, 0, sizeof(uint32_t), st));
  } else {
    if (tiled) {
      rc = launch_quad_build_tile(p, 1, st);
      if (rc) return rc;
    } else {
      quad_build_kernel<<<qgrid, 256, 0, st>>>(p);
      count_launch();
    }
    ProjParams z = p;
    z.quads = p.quads_bp;
    quad_zero_kernel<<<qgrid, 256, 0, st>>>(z);
    count_launch();
    JP_TRY_CUDA(cudaGetLastError());
  }
  if (pl->capacity > 0) {
    const bool lut = (!(pl->opts.flags & JP_PLAN_TOF_EXACT) && !p.sig) || p.tof.user;
    int lpw = pl->opts.lors_per_warp;
    if (lpw != 1 && lpw != 2) lpw = 4;
    const int block = std::min(pl->opts.block, kMaxBlock);
    const size_t smem = lut ? kLut * sizeof(float2) : 0;
    // events one warp pass handles: 32 / G
    const int64_t ev_per_block = (int64_t)(lpw == 1 ? 1 : (lpw == 2 ? 2 : 4)) * (block / 32);
    auto pick = [&](auto kern) -> int {
      int per_sm = 0;
      JP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem));
      int64_t grid = (int64_t)sm_count() * (per_sm < 1 ? 1 : per_sm);
      const int64_t need = (host_n + ev_per_block - 1) / ev_per_block;
      if (grid > need) grid = need;
      kern<<<(unsigned)(grid < 1 ? 1 : grid), block, smem, st>>>(p);
      count_launch();
      JP_TRY_CUDA(cudaGetLastError());
      return JP_OK;
    };
    const int sel = (lut ? 6 : 0) + (direct ? 3 : 0) + (lpw == 1 ? 0 : (lpw == 2 ? 1 : 2));
    switch (sel) {
      case 0: rc = pick(osem_kernel<false, 32, false>); break;
      case 1: rc = pick(osem_kernel<false, 16, false>); break;
      case 2: rc = pick(osem_kernel<false, 8, false>); break;
      case 3: rc = pick(osem_kernel<false, 32, true>); break;
      case 4: rc = pick(osem_kernel<false, 16, true>); break;
      case 5: rc = pick(osem_kernel<false, 8, true>); break;
      case 6: rc = pick(osem_kernel<true, 32, false>); break;
      case 7: rc = pick(osem_kernel<true, 16, false>); break;
      case 8: rc = pick(osem_kernel<true, 8, false>); break;
      case 9: rc = pick(osem_kernel<true, 32, true>); break;
      case 10: rc = pick(osem_kernel<true, 16, true>); break;
      default: rc = pick(osem_kernel<true, 8, true>); break;
    }
    if (rc) return rc;
  }
  if (!direct) {
    // fold the back-projection quads into the back-projection image
    if (tiled) {
      rc = launch_quad_fold_tile(p, p.quads_bp, bp_img, 1, false, st);
      if (rc) return rc;
    } else if (res) {
      osem_fold_kernel<<<aux_grid(nvox, 256), 256, 0, st>>>(p, wt);
      count_launch();
      JP_TRY_CUDA(cudaGetLastError());
    } else {
      osem_update_kernel<<<aux_grid(nvox, 256), 256, 0, st>>>(p, x);
      count_launch();
      JP_TRY_CUDA(cudaGetLastError());
      return JP_OK;
    }
  }
  if (res) {
    // x <- x * (H^T bp) / (s scale) on the last pass (passes t -> y -> t ->
    // x, bp in t; H^T = H for the symmetric taps)
    return gauss_passes(wt, wy, wt, x, 1, p.g, taps, sens, sens_scale, st);
  }
  img_update_kernel<<<aux_grid(nvox, 256), 256, 0, st>>>(x, bp_img, sens, sens_scale, nvox);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}
}  // namespace
}  // namespace jp

extern "C" int jp_osem_subset_tof_lm(jp_plan pl, int32_t f0, int32_t f1, float* x, const float* sens,
                                     float sens_scale, float b, const jp_tof* t, void* stream) {
  return osem_subset(pl, f0, f1, x, sens, sens_scale, b, nullptr, t, nullptr, JP_OSEM_PATH_AUTO, nullptr, stream);
}

extern "C" int jp_osem_subset_tof_lm_dev(jp_plan pl, int32_t f0, int32_t f1, float* x, const float* sens,
                                         float sens_scale, const float* b_dev, const jp_tof* t, void* stream) {
  if (!b_dev) {
    clear_error();
    return fail(JP_ERR_ARG, "b_dev is NULL");
  }
  return osem_subset(pl, f0, f1, x, sens, sens_scale, 0.f, b_dev, t, nullptr, JP_OSEM_PATH_AUTO, nullptr, stream);
}

extern "C" int jp_osem_subset_tof_lm_ex(jp_plan pl, int32_t f0, int32_t f1, float* x, const float* sens,
                                        float sens_scale, float b, const float* b_dev, const jp_tof* t,
                                        const jp_resolution* r, int32_t path, float* work, void* stream) {
  return osem_subset(pl, f0, f1, x, sens, sens_scale, b, b_dev, t, r, path, work, stream);
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
