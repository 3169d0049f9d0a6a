// Image-based resolution model (paper Sec. 2.6: a shift-invariant isotropic 3D
// Gaussian of 4.5 mm FWHM applied in image space in every listmode OSEM
// reconstruction; Sec. 4: two convolutions per subset became the bottleneck
// once the projectors were fast).
//
// The Gaussian is separable, so H is three 1D correlations, one kernel per
// axis.  A 200x200x71 image is 11 MB and stays in the 129 MB L2 across the
// three passes.  The taps sit in shared memory; zero outside the grid: the
// tap range is clipped per voxel.
// Every pass gives a thread one segment of kSeg consecutive outputs along
// the pass axis, computed from a register window of kSeg + 2R inputs whose
// loads are all in flight together: each input is fetched (kSeg + 2R) / kSeg
// times instead of 2R + 1 times (along a strided axis the neighbours live in
// other CTAs, out of L1's reach), and a thread has 2R + kSeg independent
// loads instead of one latency chain per voxel.
//  * axes 0 and 1 (strided): threads over columns, consecutive threads
//    consecutive in memory; grid y over (segment, image);
//  * axis 2 (contiguous): threads over (row, segment), segment fastest, so a
//    warp covers a contiguous stretch of rows.
// Radii above kMaxUnrolledR use a generic one-voxel-per-thread kernel.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "jp_internal.cuh"

namespace jp {

int make_taps(const jp_image_geom* g, const jp_resolution* r, GaussTaps* out) {
  if (!g) return fail(JP_ERR_ARG, "geometry is NULL");
  if (!r) return fail(JP_ERR_ARG, "resolution parameters are NULL");
  if (!(r->truncate > 0.f) || !isfinite(r->truncate)) return fail(JP_ERR_ARG, "truncate must be finite and > 0");
  // FWHM = sqrt(8 ln 2) sigma
  const double fwhm_per_sigma = sqrt(8.0 * log(2.0));
  for (int a = 0; a < 3; ++a) {
    const float f = r->fwhm_mm[a];
    if (!(f >= 0.f) || !isfinite(f)) return fail(JP_ERR_ARG, "FWHM must be finite and >= 0");
    if (!(g->voxsize[a] > 0.f) || !isfinite(g->voxsize[a])) return fail(JP_ERR_ARG, "voxel size must be finite and > 0");
    for (int t = 0; t < kMaxResTaps; ++t) out->w[a][t] = 0.f;
    if (f == 0.f) {
      out->r[a] = 0;
      out->w[a][0] = 1.f;
      continue;
    }
    const double sigma = (double)f / fwhm_per_sigma;
    const double d = (double)g->voxsize[a];
    const double rr = ceil((double)r->truncate * sigma / d);
    if (!(rr <= (double)JP_MAX_RES_RADIUS))
      return fail(JP_ERR_ARG, "resolution kernel radius exceeds JP_MAX_RES_RADIUS voxels");
    const int R = (int)rr;
    double w[kMaxResTaps];
    double sum = 0.0;
    for (int t = -R; t <= R; ++t) {
      const double u = t * d / sigma;
      w[t + R] = exp(-0.5 * u * u);
      sum += w[t + R];
    }
    out->r[a] = R;
    for (int t = 0; t <= 2 * R; ++t) out->w[a][t] = (float)(w[t] / sum);
  }
  return JP_OK;
}

namespace {

struct GaussPass {
  int n0, n1, n2;      // image shape
  int planes;          // n0 * number of images
  int axis;            // pass axis
  int stride;          // element stride of the pass axis
  int r;               // radius
  float scale;         // OSEM update: sensitivity scale
  const float* sens;   // OSEM update: sensitivity image (shared by all images)
  float w[kMaxResTaps];
};

constexpr int kPassBlock = 256;
constexpr int kMaxUnrolledR = 8;  // launch_pass instantiates the unrolled kernels for R = 0..8
static_assert(kMaxUnrolledR == 8, "launch_pass dispatch covers radii 0..kMaxUnrolledR");

// Generic pass for radii above kMaxUnrolledR: one output voxel per thread,
// runtime tap loop.  Grid: x over the (i1, i2) plane, y over the i0 planes
// of all images.
template <bool UPD>
__global__ void __launch_bounds__(kPassBlock) gauss_pass_kernel(const float* __restrict__ in,
                                                                float* __restrict__ out, const GaussPass gp) {
  __shared__ float sw[kMaxResTaps];
  for (int i = threadIdx.x; i <= 2 * gp.r; i += blockDim.x) sw[i] = gp.w[i];
  __syncthreads();
  const int plane = gp.n1 * gp.n2;
  const int rr = blockIdx.x * kPassBlock + threadIdx.x;  // index in the (i1, i2) plane
  if (rr >= plane) return;
  const int i1 = rr / gp.n2;
  const int c12 = gp.axis == 1 ? i1 : rr - i1 * gp.n2;
  const int n = gp.axis == 0 ? gp.n0 : (gp.axis == 1 ? gp.n1 : gp.n2);
  for (int z = blockIdx.y; z < gp.planes; z += gridDim.y) {
    const int i0 = z % gp.n0;
    const int c = gp.axis == 0 ? i0 : c12;
    const int lo = max(-gp.r, -c), hi = min(gp.r, n - 1 - c);
    const int64_t v = (int64_t)z * plane + rr;
    const float* src = in + v;
    float acc = 0.f;
    for (int t = lo; t <= hi; ++t) acc = fmaf(sw[t + gp.r], __ldg(src + (int64_t)t * gp.stride), acc);
    if (UPD) {
      const float sv = __ldg(gp.sens + (int64_t)i0 * plane + rr) * gp.scale;
      out[v] = sv > 0.f ? out[v] * acc / sv : 0.f;
    } else {
      out[v] = acc;
    }
  }
}

constexpr int kSeg = 8;

// The segment [c0, c0 + kSeg) of the line starting at element base with
// element stride `stride` and n elements; sens_base: the line's offset in the
// (shared) sensitivity image for the OSEM update.
template <bool UPD, int RC>
__device__ __forceinline__ void line_segment(const float* __restrict__ in, float* __restrict__ out,
                                             const GaussPass& gp, const float (&w)[2 * RC + 1], int64_t base,
                                             int64_t stride, int n, int c0, int64_t sens_base) {
  float win[kSeg + 2 * RC];
#pragma unroll
  for (int j = 0; j < kSeg + 2 * RC; ++j) {
    const int pos = c0 - RC + j;
    win[j] = (pos >= 0 && pos < n) ? __ldg(in + base + pos * stride) : 0.f;
  }
#pragma unroll
  for (int k = 0; k < kSeg; ++k) {
    const int pos = c0 + k;
    if (pos >= n) break;
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t <= 2 * RC; ++t) acc = fmaf(w[t], win[k + t], acc);
    const int64_t v = base + pos * stride;
    if (UPD) {
      const float sv = __ldg(gp.sens + sens_base + pos * stride) * gp.scale;
      out[v] = sv > 0.f ? out[v] * acc / sv : 0.f;
    } else {
      out[v] = acc;
    }
  }
}

// Pass along axis 2 (contiguous), radius RC: thread g -> row g / nseg,
// segment g % nseg; rows of all images are consecutive.
template <bool UPD, int RC>
__global__ void __launch_bounds__(kPassBlock) gauss_row_kernel(const float* __restrict__ in,
                                                               float* __restrict__ out, const GaussPass gp) {
  __shared__ float sw[2 * RC + 1];
  for (int i = threadIdx.x; i <= 2 * RC; i += blockDim.x) sw[i] = gp.w[i];
  __syncthreads();
  const int n = gp.n2;
  const int nseg = (n + kSeg - 1) / kSeg;
  const int64_t rows = (int64_t)gp.planes * gp.n1;
  const int64_t g = (int64_t)blockIdx.x * kPassBlock + threadIdx.x;
  if (g >= rows * nseg) return;
  const int64_t row = g / nseg;
  const int seg = (int)(g - row * nseg);
  float w[2 * RC + 1];
#pragma unroll
  for (int t = 0; t <= 2 * RC; ++t) w[t] = sw[t];
  const int64_t rows_img = (int64_t)gp.n0 * gp.n1;
  line_segment<UPD, RC>(in, out, gp, w, row * n, 1, n, seg * kSeg, (row % rows_img) * n);
}

// Pass along axis 0 or 1 (gp.axis), radius RC.  Columns: axis 0 -> (i1, i2)
// [n1*n2 of them], axis 1 -> (i0, i2) [n0*n2]; grid x over columns, y over
// (segment, image) pairs.
template <bool UPD, int RC>
__global__ void __launch_bounds__(kPassBlock) gauss_line_kernel(const float* __restrict__ in,
                                                                float* __restrict__ out, const GaussPass gp) {
  __shared__ float sw[2 * RC + 1];
  for (int i = threadIdx.x; i <= 2 * RC; i += blockDim.x) sw[i] = gp.w[i];
  __syncthreads();
  const int plane = gp.n1 * gp.n2;
  const int ax0 = gp.axis == 0;
  const int ncol = ax0 ? plane : gp.n0 * gp.n2;
  const int n = ax0 ? gp.n0 : gp.n1;
  const int col = blockIdx.x * kPassBlock + threadIdx.x;
  if (col >= ncol) return;
  // offset of the column's first element within one image
  int64_t cbase;
  if (ax0) {
    cbase = col;
  } else {
    const int i0 = col / gp.n2;
    cbase = (int64_t)i0 * plane + (col - i0 * gp.n2);
  }
  const int64_t stride = gp.stride;
  const int nseg = (n + kSeg - 1) / kSeg;
  const int64_t nvox = (int64_t)plane * gp.n0;
  const int n_img = gp.planes / gp.n0;
  float w[2 * RC + 1];
#pragma unroll
  for (int t = 0; t <= 2 * RC; ++t) w[t] = sw[t];
  for (int y = blockIdx.y; y < nseg * n_img; y += gridDim.y) {
    const int img = y / nseg, c0 = (y - img * nseg) * kSeg;
    line_segment<UPD, RC>(in, out, gp, w, (int64_t)img * nvox + cbase, stride, n, c0, cbase);
  }
}

template <bool UPD, int R>
void launch_unrolled(cudaStream_t st, const float* in, float* out, const GaussPass& gp) {
  if (gp.axis == 2) {
    const int64_t threads = (int64_t)gp.planes * gp.n1 * ((gp.n2 + kSeg - 1) / kSeg);
    gauss_row_kernel<UPD, R><<<(unsigned)((threads + kPassBlock - 1) / kPassBlock), kPassBlock, 0, st>>>(in, out, gp);
  } else {
    const int ncol = gp.axis == 0 ? gp.n1 * gp.n2 : gp.n0 * gp.n2;
    const int n = gp.axis == 0 ? gp.n0 : gp.n1;
    const int64_t ny = (int64_t)((n + kSeg - 1) / kSeg) * (gp.planes / gp.n0);
    const dim3 lg((ncol + kPassBlock - 1) / kPassBlock, (unsigned)std::min<int64_t>(ny, 65535));
    gauss_line_kernel<UPD, R><<<lg, kPassBlock, 0, st>>>(in, out, gp);
  }
}

template <bool UPD>
void launch_pass(cudaStream_t st, const float* in, float* out, const GaussPass& gp) {
  switch (gp.r) {
    case 0: return launch_unrolled<UPD, 0>(st, in, out, gp);
    case 1: return launch_unrolled<UPD, 1>(st, in, out, gp);
    case 2: return launch_unrolled<UPD, 2>(st, in, out, gp);
    case 3: return launch_unrolled<UPD, 3>(st, in, out, gp);
    case 4: return launch_unrolled<UPD, 4>(st, in, out, gp);
    case 5: return launch_unrolled<UPD, 5>(st, in, out, gp);
    case 6: return launch_unrolled<UPD, 6>(st, in, out, gp);
    case 7: return launch_unrolled<UPD, 7>(st, in, out, gp);
    case 8: return launch_unrolled<UPD, 8>(st, in, out, gp);
    default: {
      const int plane = gp.n1 * gp.n2;
      const dim3 grid((plane + kPassBlock - 1) / kPassBlock, (unsigned)std::min(gp.planes, 65535));
      gauss_pass_kernel<UPD><<<grid, kPassBlock, 0, st>>>(in, out, gp);
    }
  }
}

bool overlap(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}

}  // namespace

int gauss_passes(const float* in, float* b1, float* b2, float* dst, int n_img, const DevGeom& g,
                 const GaussTaps& t, const float* upd_sens, float scale, cudaStream_t st) {
  const int64_t nvox = (int64_t)g.n[0] * g.n[1] * g.n[2];
  const int64_t total = nvox * n_img;
  if (total == 0) return JP_OK;
  const float* src[3] = {in, b1, b2};
  float* dsts[3] = {b1, b2, dst};
  const int axes[3] = {2, 1, 0};
  const int64_t planes = (int64_t)g.n[0] * n_img;
  if (planes > INT32_MAX) return fail(JP_ERR_ARG, "too many image planes");
  for (int k = 0; k < 3; ++k) {
    const int a = axes[k];
    GaussPass gp;
    gp.n0 = g.n[0];
    gp.n1 = g.n[1];
    gp.n2 = g.n[2];
    gp.planes = (int)planes;
    gp.axis = a;
    gp.stride = g.stride[a];
    gp.r = t.r[a];
    gp.scale = scale;
    gp.sens = upd_sens;
    for (int i = 0; i < kMaxResTaps; ++i) gp.w[i] = t.w[a][i];
    const bool upd = (k == 2) && upd_sens != nullptr;
    if (upd)
      launch_pass<true>(st, src[k], dsts[k], gp);
    else
      launch_pass<false>(st, src[k], dsts[k], gp);
    count_launch();
    JP_TRY_CUDA(cudaGetLastError());
  }
  return JP_OK;
}

}  // namespace jp

extern "C" int jp_gauss3d(const float* img, float* out, float* work, int32_t n_images, const jp_image_geom* g,
                          const jp_resolution* r, void* stream) {
  using namespace jp;
  clear_error();
  if (n_images < 0) return fail(JP_ERR_ARG, "n_images must be >= 0");
  DevGeom dg;
  int rc = make_geom(g, &dg);
  if (rc) return rc;
  GaussTaps taps;
  rc = make_taps(g, r, &taps);
  if (rc) return rc;
  if (n_images == 0) return JP_OK;
  if (!img || !out || !work) return fail(JP_ERR_ARG, "img / out / work is NULL");
  if (!aligned(img, 4) || !aligned(out, 4) || !aligned(work, 4)) return fail(JP_ERR_ALIGN, "arrays must be 4-byte aligned");
  const size_t bytes = (size_t)n_images * dg.n[0] * dg.n[1] * dg.n[2] * sizeof(float);
  if (overlap(img, out, bytes) || overlap(img, work, bytes) || overlap(out, work, bytes))
    return fail(JP_ERR_ARG, "img, out and work must not overlap");
  return gauss_passes(img, out, work, out, n_images, dg, taps, nullptr, 0.f, (cudaStream_t)stream);
}
