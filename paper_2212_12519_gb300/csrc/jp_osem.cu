// OSEM element-wise kernels: listmode (step a8; paper Sec. 2.6 and 3:
// x <- x / s_sub * A_S^T (1 / (A_S x + b))) and the sinogram data term
// y / (A_m x + c) (Sec. 2.6); the Poisson log-likelihood loss of a
// listmode batch and its gradient with respect to the projections; an FP64
// reduction used only for the sensitivity-normalisation check; and the
// microbenchmark of the L2 vector-reduction ceiling that the back
// projection's roofline is measured against.
#include <cuda_runtime.h>

#include <algorithm>

#include "jp_internal.cuh"

namespace jp {
namespace {

__device__ __forceinline__ int frame_of(const int64_t* __restrict__ off, int n_frames, int64_t i) {
  int lo = 0, hi = n_frames - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void ratio_kernel(const float* __restrict__ p, const float* __restrict__ b,
                             const int64_t* __restrict__ off, int n_frames, float* __restrict__ q,
                             int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) {
    int f = (n_frames > 1) ? frame_of(off, n_frames, i) : 0;
    q[i] = 1.0f / (p[i] + __ldg(b + f));
  }
}

__global__ void update_kernel(float* __restrict__ x, const float* __restrict__ bp,
                              const float* __restrict__ s, float scale, int64_t nvox, int n_frames,
                              int64_t stride, int64_t s_stride) {
  int64_t total = nvox * n_frames;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (; i < total; i += step) {
    int64_t f = i / nvox, v = i - f * nvox;
    float sv = s[f * s_stride + v] * scale;
    float* xp = x + f * stride + v;
    *xp = sv > 0.f ? *xp * bp[f * stride + v] / sv : 0.f;
  }
}

// Compensated FP32 summation: (s, c) carries the sum s + c; each addition
// is an error-free TwoSum (Knuth) whose rounding error goes to c, so the
// accumulated error is of order eps * sum |terms| with no growth in the
// number of terms (cascaded summation, Rump, Ogita and Oishi).  The _rn
// intrinsics keep the compiler from contracting or reassociating.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

__device__ __forceinline__ void comp_merge(float& s, float& c, float s2, float c2) {
  float t, e;
  two_sum(s, s2, t, e);
  s = t;
  c = __fadd_rn(__fadd_rn(c, c2), e);
}

// block-wide compensated sum of (s, c); the result is valid in thread 0
__device__ __forceinline__ void block_comp_sum(float& s, float& c) {
  __shared__ float2 red[32];
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, s, o);
    const float c2 = __shfl_down_sync(0xffffffffu, c, o);
    comp_merge(s, c, s2, c2);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float2(s, c);
  __syncthreads();
  if (threadIdx.x < 32) {
    const float2 v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : make_float2(0.f, 0.f);
    s = v.x;
    c = v.y;
    for (int o = 16; o > 0; o >>= 1) {
      const float s2 = __shfl_down_sync(0xffffffffu, s, o);
      const float c2 = __shfl_down_sync(0xffffffffu, c, o);
      comp_merge(s, c, s2, c2);
    }
  }
}

// frame of event i for a thread whose i only grows: the frame [lo, hi) of
// the previous event is reused until i leaves it (a grid-stride loop crosses
// a frame boundary once per frame)
__device__ __forceinline__ int frame_cached(const int64_t* __restrict__ off, int n_frames, int64_t i, int& f,
                                            int64_t& lo, int64_t& hi) {
  if (i < lo || i >= hi) {
    f = frame_of(off, n_frames, i);
    lo = __ldg(off + f);
    hi = __ldg(off + f + 1);
  }
  return f;
}

// pass 1: each block's compensated partial sum of w_e log(p_e + b_f) into
// part[block]; four events per iteration into four independent compensated
// sums, so the loads and logarithms of an iteration do not wait on the
// previous sum.
__global__ void loglik_value_kernel(const float* __restrict__ p, const float* __restrict__ w,
                                    const float* __restrict__ b, const int64_t* __restrict__ off, int n_frames,
                                    int64_t n, float2* __restrict__ part) {
  float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
  int f = 0;
  int64_t lo = 0, hi = n_frames > 1 ? 0 : n;  // one frame: never searched
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    float pv[4], wv[4], bv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      pv[q] = __ldcs(p + i + q * stride);
      wv[q] = w ? __ldcs(w + i + q * stride) : 1.f;
      bv[q] = __ldg(b + frame_cached(off, n_frames, i + q * stride, f, lo, hi));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) comp_merge(s[q], c[q], __fmul_rn(wv[q], logf(pv[q] + bv[q])), 0.f);
  }
  for (; i < n; i += stride) {
    const float wi = w ? __ldcs(w + i) : 1.f;
    comp_merge(s[0], c[0], __fmul_rn(wi, logf(__ldcs(p + i) + __ldg(b + frame_cached(off, n_frames, i, f, lo, hi)))),
               0.f);
  }
#pragma unroll
  for (int q = 1; q < 4; ++q) comp_merge(s[0], c[0], s[q], c[q]);
  block_comp_sum(s[0], c[0]);
  if (threadIdx.x == 0) part[blockIdx.x] = make_float2(s[0], c[0]);
}

// pass 2 (one block): the partials' compensated sum into *out
__global__ void loglik_final_kernel(const float2* __restrict__ part, int nb, float* __restrict__ out) {
  float s = 0.f, c = 0.f;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) comp_merge(s, c, part[i].x, part[i].y);
  block_comp_sum(s, c);
  if (threadIdx.x == 0) *out = __fadd_rn(s, c);
}

__global__ void loglik_grad_kernel(const float* __restrict__ p, const float* __restrict__ w,
                                   const float* __restrict__ b, const int64_t* __restrict__ off, int n_frames,
                                   const float* __restrict__ scale, int64_t n, float* __restrict__ g) {
  const float sc = scale ? __ldg(scale) : 1.f;
  int f = 0;
  int64_t lo = 0, hi = n_frames > 1 ? 0 : n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float wi = w ? __ldcs(w + i) : 1.f;
    __stcs(g + i, sc * wi / (__ldcs(p + i) + __ldg(b + frame_cached(off, n_frames, i, f, lo, hi))));
  }
}

__global__ void init_kernel(float* __restrict__ x, const float* __restrict__ s, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = s[i] > 0.f ? 1.f : 0.f;
}

__global__ void sum_f64_kernel(const float* __restrict__ x, int64_t n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += step) s += (double)x[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out, s);
  }
}

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
  return x;
}

__global__ void bench_red_kernel(float4* buf, uint32_t n, int per_thread, int pattern) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31u, warp = t >> 5;
  for (int r = 0; r < per_thread; ++r) {
    uint32_t i;
    if (pattern == 1) {
      i = (mix32((t >> 1) * 131u + (uint32_t)r) % (n / 2)) * 2u + (lane & 1u);
    } else if (pattern == 2) {
      i = (mix32(warp * 131u + (uint32_t)r) % (n / 32)) * 32u + lane;
    } else if (pattern == 3 || pattern == 4) {
      // L = 4 or 8 lanes on the first L entries of one random 128-byte line
      const uint32_t L = pattern == 3 ? 4u : 8u;
      i = (mix32((t / L) * 131u + (uint32_t)r) % (n / 8)) * 8u + (lane % L);
    } else {
      i = mix32(t * 131u + (uint32_t)r) % n;
    }
    atomicAdd(buf + i, make_float4(1.f, 1.f, 1.f, 1.f));
  }
}

// sinogram OSEM ratio q = y / (p + c), 0 where p + c <= 0 (c NULL: 0);
// four elements per iteration when every array is 16-byte aligned
__global__ void ratio_sino_kernel(const float* __restrict__ p, const float* __restrict__ y,
                                  const float* __restrict__ c, float* q, int64_t n, int vec) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  int64_t done = 0;
  if (vec) {
    const int64_t n4 = n >> 2;
    for (int64_t i = tid; i < n4; i += step) {
      const float4 pv = reinterpret_cast<const float4*>(p)[i];
      const float4 yv = __ldg(reinterpret_cast<const float4*>(y) + i);
      const float4 cv = c ? __ldg(reinterpret_cast<const float4*>(c) + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 r;
      float d;
      d = pv.x + cv.x; r.x = d > 0.f ? yv.x / d : 0.f;
      d = pv.y + cv.y; r.y = d > 0.f ? yv.y / d : 0.f;
      d = pv.z + cv.z; r.z = d > 0.f ? yv.z / d : 0.f;
      d = pv.w + cv.w; r.w = d > 0.f ? yv.w / d : 0.f;
      reinterpret_cast<float4*>(q)[i] = r;
    }
    done = n4 << 2;
  }
  for (int64_t i = done + tid; i < n; i += step) {
    const float d = p[i] + (c ? __ldg(c + i) : 0.f);
    q[i] = d > 0.f ? __ldg(y + i) / d : 0.f;
  }
}

int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  int64_t cap = (int64_t)sm_count() * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace
}  // namespace jp

using namespace jp;

extern "C" int jp_osem_ratio(jp_plan pl, const float* p, const float* b, float* q, int64_t n,
                             void* stream) {
  clear_error();
  if (n < 0) return fail(JP_ERR_ARG, "n must be >= 0");
  if (n > 0 && (!p || !b || !q)) return fail(JP_ERR_ARG, "NULL pointer");
  if (!aligned(p, 4) || !aligned(b, 4) || !aligned(q, 4)) return fail(JP_ERR_ALIGN, "misaligned array");
  const int64_t* off = nullptr;
  int nf = 1;
  if (pl) {
    if (pl->n != n) return fail(JP_ERR_ARG, "n does not match the plan");
    off = pl->frame_off_dev;
    nf = pl->n_frames;
  }
  if (n == 0) return JP_OK;
  ratio_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(p, b, off, nf, q, n);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

extern "C" int jp_osem_ratio_sino(const float* p, const float* y, const float* c, float* q, int64_t n,
                                  void* stream) {
  clear_error();
  if (n < 0) return fail(JP_ERR_ARG, "n must be >= 0");
  if (n > 0 && (!p || !y || !q)) return fail(JP_ERR_ARG, "NULL pointer");
  if (!aligned(p, 4) || !aligned(y, 4) || !aligned(c, 4) || !aligned(q, 4)) return fail(JP_ERR_ALIGN, "misaligned array");
  if (n == 0) return JP_OK;
  const int vec = aligned(p, 16) && aligned(y, 16) && aligned(c, 16) && aligned(q, 16);
  ratio_sino_kernel<<<grid_for((n + 3) / 4, 256), 256, 0, (cudaStream_t)stream>>>(p, y, c, q, n, vec);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

extern "C" int jp_osem_update(float* x, const float* bp, const float* s, float scale, int64_t nvox,
                              int32_t n_frames, int64_t stride, int64_t s_stride, void* stream) {
  clear_error();
  if (nvox < 0 || n_frames < 1 || stride < 0 || s_stride < 0) return fail(JP_ERR_ARG, "bad sizes");
  if (n_frames > 1 && stride < nvox) return fail(JP_ERR_ARG, "img_stride smaller than nvox");
  if (!(scale > 0.f) || !isfinite(scale)) return fail(JP_ERR_ARG, "scale must be finite and > 0");
  if (nvox > 0 && (!x || !bp || !s)) return fail(JP_ERR_ARG, "NULL pointer");
  if (!aligned(x, 4) || !aligned(bp, 4) || !aligned(s, 4)) return fail(JP_ERR_ALIGN, "misaligned array");
  int64_t total = nvox * n_frames;
  if (total == 0) return JP_OK;
  update_kernel<<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(x, bp, s, scale, nvox, n_frames,
                                                                       stride, s_stride);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

namespace {
int loglik_common(jp_plan pl, const float* p, const float* w, const float* b, int64_t n, const int64_t** off,
                  int* nf) {
  if (n < 0) return fail(JP_ERR_ARG, "n must be >= 0");
  if (n > 0 && (!p || !b)) return fail(JP_ERR_ARG, "NULL pointer");
  if (!aligned(p, 4) || !aligned(w, 4) || !aligned(b, 4)) return fail(JP_ERR_ALIGN, "misaligned array");
  *off = nullptr;
  *nf = 1;
  if (pl) {
    if (pl->n != n) return fail(JP_ERR_ARG, "n does not match the plan");
    if (pl->opts.flags & JP_PLAN_INTERLEAVED) return fail(JP_ERR_STATE, "frames of an interleaved plan are not contiguous");
    *off = pl->frame_off_dev;
    *nf = pl->n_frames;
  }
  return JP_OK;
}
}  // namespace

extern "C" int jp_poisson_loglik_value(jp_plan pl, const float* p, const float* w, const float* b, int64_t n,
                                       float* value, float* work, void* stream) {
  clear_error();
  if (!value) return fail(JP_ERR_ARG, "value is NULL");
  if (!work) return fail(JP_ERR_ARG, "work is NULL");
  if (!aligned(value, 4) || !aligned(work, 8)) return fail(JP_ERR_ALIGN, "value / work misaligned");
  const int64_t* off;
  int nf;
  int rc = loglik_common(pl, p, w, b, n, &off, &nf);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) {
    JP_TRY_CUDA(cudaMemsetAsync(value, 0, sizeof(float), st));
    return JP_OK;
  }
  const int nb = std::min(grid_for(n, 256), JP_LOGLIK_BLOCKS);
  float2* part = reinterpret_cast<float2*>(work);
  loglik_value_kernel<<<nb, 256, 0, st>>>(p, w, b, off, nf, n, part);
  count_launch();
  loglik_final_kernel<<<1, 1024, 0, st>>>(part, nb, value);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

extern "C" int jp_poisson_loglik_grad(jp_plan pl, const float* p, const float* w, const float* b,
                                      const float* scale, int64_t n, float* grad, void* stream) {
  clear_error();
  if (n > 0 && !grad) return fail(JP_ERR_ARG, "grad is NULL");
  if (!aligned(grad, 4) || !aligned(scale, 4)) return fail(JP_ERR_ALIGN, "misaligned array");
  const int64_t* off;
  int nf;
  int rc = loglik_common(pl, p, w, b, n, &off, &nf);
  if (rc) return rc;
  if (n == 0) return JP_OK;
  loglik_grad_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(p, w, b, off, nf, scale, n, grad);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

extern "C" int jp_osem_init(float* x, const float* s, int64_t n, void* stream) {
  clear_error();
  if (n < 0 || (n > 0 && (!x || !s))) return fail(JP_ERR_ARG, "bad arguments");
  if (!aligned(x, 4) || !aligned(s, 4)) return fail(JP_ERR_ALIGN, "misaligned array");
  if (n == 0) return JP_OK;
  init_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(x, s, n);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

extern "C" int jp_bench_red(float* buf, int64_t n_entries, int32_t per_thread, int32_t iters, float* ms_out,
                            void* stream) {
  return jp_bench_red_pattern(buf, n_entries, per_thread, iters, 0, ms_out, stream);
}

extern "C" int jp_bench_red_pattern(float* buf, int64_t n_entries, int32_t per_thread, int32_t iters,
                                    int32_t pattern, float* ms_out, void* stream) {
  clear_error();
  if (!buf || !ms_out || n_entries < 64 || n_entries > (int64_t)UINT32_MAX || per_thread < 1 || iters < 1 ||
      pattern < 0 || pattern > 4)
    return fail(JP_ERR_ARG, "bad arguments");
  if (!aligned(buf, 16)) return fail(JP_ERR_ALIGN, "buf must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = sm_count() * 32, threads = 256;
  bench_red_kernel<<<blocks, threads, 0, st>>>(reinterpret_cast<float4*>(buf), (uint32_t)n_entries, per_thread,
                                               pattern);
  count_launch();
  cudaEvent_t a, b;
  JP_TRY_CUDA(cudaEventCreate(&a));
  JP_TRY_CUDA(cudaEventCreate(&b));
  JP_TRY_CUDA(cudaEventRecord(a, st));
  for (int i = 0; i < iters; ++i) {
    bench_red_kernel<<<blocks, threads, 0, st>>>(reinterpret_cast<float4*>(buf), (uint32_t)n_entries, per_thread,
                                                 pattern);
    count_launch();
  }
  JP_TRY_CUDA(cudaEventRecord(b, st));
  JP_TRY_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  JP_TRY_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms_out = ms / iters;
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

extern "C" int jp_sum_f64(const float* x, int64_t n, double* out, void* stream) {
  clear_error();
  if (n < 0 || !out || (n > 0 && !x)) return fail(JP_ERR_ARG, "bad arguments");
  if (!aligned(x, 4) || !aligned(out, 8)) return fail(JP_ERR_ALIGN, "misaligned array");
  JP_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(double), (cudaStream_t)stream));
  if (n == 0) return JP_OK;
  sum_f64_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(x, n, out);
  count_launch();
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}
