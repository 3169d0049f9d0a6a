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
};

__device__ __forceinline__ int frame_of(const int64_t* __restrict__ off, int n_frames, int64_t i) {
  int lo = 0, hi = n_frames - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// MODE: 0 non-TOF, 1 TOF sinogram, 2 TOF listmode
template <int MODE, bool BACK, bool PLANNED>
__global__ void __launch_bounds__(kMaxBlock) proj_kernel(const ProjParams p) {
  extern __shared__ float sbuf[];  // TOF sinogram: [nbins][blockDim]
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  float xs[3], xe[3], delta;
  int tbin;
  int64_t j;  // caller index
  int64_t foff = 0;
  if (PLANNED) {
    const float4 A = __ldg(p.lor + 2 * i);
    const float4 B = __ldg(p.lor + 2 * i + 1);
    xs[0] = A.x; xs[1] = A.y; xs[2] = A.z; delta = A.w;
    xe[0] = B.x; xe[1] = B.y; xe[2] = B.z; tbin = __float_as_int(B.w);
    j = __ldg(p.perm + i);
    if (p.n_frames > 1) foff = (int64_t)frame_of(p.frame_off, p.n_frames, i) * p.img_stride;
  } else {
    j = i;
    xs[0] = __ldg(p.xs + 3 * i); xs[1] = __ldg(p.xs + 3 * i + 1); xs[2] = __ldg(p.xs + 3 * i + 2);
    xe[0] = __ldg(p.xe + 3 * i); xe[1] = __ldg(p.xe + 3 * i + 1); xe[2] = __ldg(p.xe + 3 * i + 2);
    delta = p.delta ? __ldg(p.delta + i) : 0.f;
    tbin = (MODE == 2) ? (int)__ldg(p.tof_bin + i) : 0;
  }
  const DevGeom& g = p.g;
  const DevTof& T = p.tof;
  const int N = T.nbins;
  float* acc = sbuf + threadIdx.x;  // acc[t * blockDim.x]

  Ray r;
  bool live = ray_setup(xs, xe, g, r);

  // -------- TOF listmode window --------------------------------------
  float d0 = 0.f;  // tau(kc) - c
  if (MODE == 2 && live) {
    float c = (float)tbin * T.width + delta;
    d0 = r.tc - c;
    // planes with |tau(k) - c| <= R:  kc + (-R - d0)/dt .. kc + (R - d0)/dt
    float t1 = (-T.R - d0) / r.dt, t2 = (T.R - d0) / r.dt;
    float lo = ceilf(r.kc + fminf(t1, t2)), hi = floorf(r.kc + fmaxf(t1, t2));
    lo = fmaxf(lo, (float)r.k0);
    hi = fminf(hi, (float)r.k1);
    r.k0 = (int)lo;
    r.k1 = (int)hi;
    live = lo <= hi;
  }

  if (!BACK) {
    // ------------------------------ forward ------------------------------
    if (MODE == 1) {
      for (int t = 0; t < N; ++t) acc[t * blockDim.x] = 0.f;
    }
    float sum = 0.f;
    if (live) {
      const float* __restrict__ img = p.img_in + foff;
      for (int k = r.k0; k <= r.k1; ++k) {
        float kk = (float)k - r.kc;
        float u = fmaf(kk, r.du, r.uc);
        float w = fmaf(kk, r.dw, r.wc);
        Corners q;
        corners(r, k, u, w, q);
        float s = interp(img, r, q);
        if (MODE == 0) {
          sum += s;
        } else if (MODE == 2) {
          float dist = fmaf(kk, r.dt, d0);
          sum += tof_g(dist, T) * s;
        } else {
          if (s == 0.f) continue;
          float tau = fmaf(kk, r.dt, r.tc);
          float x = (tau - delta) * T.inv_w + T.hbin;  // continuous bin coordinate
          int t0 = max(0, (int)ceilf(x - T.R_over_w));
          int t1 = min(N - 1, (int)floorf(x + T.R_over_w));
          if (t0 > t1) continue;
          // dist_t = tau - c_t, c_t = (t - hbin) w + delta
          float dlo = (tau - delta) - ((float)t0 - T.hbin) * T.width;
          float e_hi = erff((dlo + T.half) * T.k);
          for (int t = t0; t <= t1; ++t) {
            float dist = fmaf(-(float)(t - t0), T.width, dlo);
            float e_lo = erff((dist - T.half) * T.k);
            acc[t * blockDim.x] += 0.5f * (e_hi - e_lo) * s;
            e_hi = e_lo;
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
    if (!live) return;
    float* img = p.img_out + foff;
    if (MODE == 1) {
      const float* yrow = p.proj_in + j * (int64_t)N;
      bool any = false;
      for (int t = 0; t < N; ++t) {
        float y = __ldg(yrow + t);
        acc[t * blockDim.x] = y;
        any |= (y != 0.f);
      }
      if (!any) return;
    }
    float val = r.w0;
    if (MODE != 1) {
      val *= __ldg(p.proj_in + j);
      if (val == 0.f) return;
    }
    for (int k = r.k0; k <= r.k1; ++k) {
      float kk = (float)k - r.kc;
      float coef;
      if (MODE == 0) {
        coef = val;
      } else if (MODE == 2) {
        float dist = fmaf(kk, r.dt, d0);
        coef = tof_g(dist, T) * val;
      } else {
        float tau = fmaf(kk, r.dt, r.tc);
        float x = (tau - delta) * T.inv_w + T.hbin;
        int t0 = max(0, (int)ceilf(x - T.R_over_w));
        int t1 = min(N - 1, (int)floorf(x + T.R_over_w));
        if (t0 > t1) continue;
        float dlo = (tau - delta) - ((float)t0 - T.hbin) * T.width;
        float e_hi = erff((dlo + T.half) * T.k);
        float sy = 0.f;
        for (int t = t0; t <= t1; ++t) {
          float dist = fmaf(-(float)(t - t0), T.width, dlo);
          float e_lo = erff((dist - T.half) * T.k);
          sy += 0.5f * (e_hi - e_lo) * acc[t * blockDim.x];
          e_hi = e_lo;
        }
        coef = sy * val;
      }
      if (coef == 0.f) continue;
      float u = fmaf(kk, r.du, r.uc);
      float w = fmaf(kk, r.dw, r.wc);
      Corners q;
      corners(r, k, u, w, q);
      scatter_add(img, r, q, coef);
    }
  }
}

template <int MODE, bool BACK, bool PLANNED>
int launch(const ProjParams& p, int block, cudaStream_t st) {
  if (p.n == 0) return JP_OK;
  size_t smem = (MODE == 1) ? (size_t)p.tof.nbins * block * sizeof(float) : 0;
  if (smem > 48 * 1024) {
    JP_TRY_CUDA(cudaFuncSetAttribute(proj_kernel<MODE, BACK, PLANNED>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  int64_t blocks = (p.n + block - 1) / block;
  if (blocks > INT32_MAX) return fail(JP_ERR_ARG, "too many LORs for one launch");
  proj_kernel<MODE, BACK, PLANNED><<<(unsigned)blocks, block, smem, st>>>(p);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

int pick_block(int block, int mode, const DevTof& t) {
  if (block > kMaxBlock) block = kMaxBlock;
  if (mode == 1) {
    int cap = (96 * 1024) / (4 * t.nbins);
    cap = (cap / 32) * 32;
    if (cap < 32) cap = 32;
    if (block > cap) block = cap;
  }
  return block;
}

template <bool PLANNED>
int dispatch(int mode, bool back, const ProjParams& p, int block, cudaStream_t st) {
  block = pick_block(block, mode, p.tof);
  switch (mode * 2 + (back ? 1 : 0)) {
    case 0: return launch<0, false, PLANNED>(p, block, st);
    case 1: return launch<0, true, PLANNED>(p, block, st);
    case 2: return launch<1, false, PLANNED>(p, block, st);
    case 3: return launch<1, true, PLANNED>(p, block, st);
    case 4: return launch<2, false, PLANNED>(p, block, st);
    case 5: return launch<2, true, PLANNED>(p, block, st);
  }
  return fail(JP_ERR_ARG, "bad mode");
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
  if (mode != 0) {
    rc = make_tof(t, mode == 1, &p.tof);
    if (rc) return rc;
  } else {
    p.tof.nbins = 1;
  }
  p.lor = pl->lor;
  p.perm = pl->perm;
  p.frame_off = pl->frame_off_dev;
  p.n_frames = pl->n_frames;
  p.n = pl->n;
  p.img_stride = img_stride;
  if (back) { p.proj_in = in; p.img_out = out; } else { p.img_in = in; p.proj_out = out; }
  return dispatch<true>(mode, back, p, pl->opts.block, (cudaStream_t)stream);
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
  return dispatch<false>(mode, back, p, 256, (cudaStream_t)stream);
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
      float c = (float)__float_as_int(B.w) * p.tof.width + A.w;
      float d0 = r.tc - c;
      float t1 = (-p.tof.R - d0) / r.dt, t2 = (p.tof.R - d0) / r.dt;
      float lo = fmaxf(ceilf(r.kc + fminf(t1, t2)), (float)r.k0);
      float hi = fminf(floorf(r.kc + fmaxf(t1, t2)), (float)r.k1);
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
