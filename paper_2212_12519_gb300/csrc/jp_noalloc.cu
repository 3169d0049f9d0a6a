// Allocation-free TOF listmode back projection.
//
// Same result as jp_back_lors in TOF listmode, computed with the 4-neighbour
// quad workspace (one 16-byte vector reduction per plane sample) -- but the
// workspace is a fixed device array compiled into the library instead of
// memory the caller or the library allocates.  See jp_back_tof_lm_noalloc in
// include/joseph.h for who needs this and the size limit.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "jp_internal.cuh"

namespace jp {
namespace {

// Workspace: up to kNoAllocQuads 16-byte entries (16 MiB), held by every
// GPU that loads the library until the process exits.
constexpr int64_t kNoAllocQuads = int64_t(1) << 20;
__device__ __align__(256) float4 g_noalloc_quads[kNoAllocQuads];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float4* g_quads_ptr[kMaxDevices] = {};

// Device address of the workspace for the current device.  In host code
// g_noalloc_quads names a host-side stand-in, not device memory, so the
// address is looked up once per device (with that device current).
int workspace(float4** out) {
  int dev = 0;
  JP_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(JP_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_quads_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_quads);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_quads)");
    g_quads_ptr[dev] = static_cast<float4*>(ptr);
  }
  *out = g_quads_ptr[dev];
  return JP_OK;
}

struct NaParams {
  const float* xs;
  const float* xe;
  const int16_t* tof_bin;
  const float* delta;
  int64_t n;
  DevGeom g;
  DevTof tof;
  const float* proj;
  float* img;
  float4* quads;
  QuadLayout ql;
};

__global__ void na_zero(float4* q, int64_t total) {
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    q[e] = z;
}

// one thread per event, plane-major quads: index (k * nb2 + i + 1) * nc2 + j + 1
__global__ void na_back(const NaParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  const float xs[3] = {p.xs[3 * i], p.xs[3 * i + 1], p.xs[3 * i + 2]};
  const float xe[3] = {p.xe[3 * i], p.xe[3 * i + 1], p.xe[3 * i + 2]};
  const DevTof& T = p.tof;
  Ray r;
  if (!ray_setup(xs, xe, p.g, r)) return;
  const float c = (float)p.tof_bin[i] * T.width + (p.delta ? p.delta[i] : 0.f);
  const float d0 = r.tc - c;
  const float t1 = (-T.R - d0) / r.dt, t2 = (T.R - d0) / r.dt;
  const float lo = fmaxf(ceilf(r.kc + fminf(t1, t2)), (float)r.k0);
  const float hi = fminf(floorf(r.kc + fmaxf(t1, t2)), (float)r.k1);
  if (!(lo <= hi)) return;
  const float val = r.w0 * p.proj[i];
  if (val == 0.f) return;
  const int a = r.a;
  const int nb2 = sel3(a, p.ql.nb2[0], p.ql.nb2[1], p.ql.nb2[2]);
  const int nc2 = sel3(a, p.ql.nc2[0], p.ql.nc2[1], p.ql.nc2[2]);
  float4* Q = p.quads + sel3(a, p.ql.base[0], p.ql.base[1], p.ql.base[2]);
  for (int k = (int)lo; k <= (int)hi; ++k) {
    const float kk = (float)k - r.kc;
    const float coef = tof_g(fmaf(kk, r.dt, d0), T) * val;
    if (coef == 0.f) continue;
    const float u = fminf(fmaxf(fmaf(kk, r.du, r.uc), -1.f), (float)r.nb);
    const float w = fminf(fmaxf(fmaf(kk, r.dw, r.wc), -1.f), (float)r.nc);
    const float fu = floorf(u), fw = floorf(w);
    const float al = u - fu, be = w - fw;
    const float ca = (1.f - al) * coef, cb = al * coef;
    atomicAdd(Q + (k * nb2 + (int)fu + 1) * nc2 + (int)fw + 1,
              make_float4(ca * (1.f - be), cb * (1.f - be), ca * be, cb * be));
  }
}

// img[v] += the 4 quad entries of every axis that hold voxel v
__global__ void na_fold(const NaParams p) {
  const DevGeom& g = p.g;
  const int64_t nvox = (int64_t)g.n[0] * g.n[1] * g.n[2];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(v / g.stride[0]);
    const int r0 = (int)(v - (int64_t)i0 * g.stride[0]);
    const int i1 = r0 / g.n[2], i2 = r0 - (r0 / g.n[2]) * g.n[2];
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int k = (a == 0) ? i0 : (a == 1 ? i1 : i2);
      const int I = (a == 0) ? i1 : i0;
      const int J = (a == 2) ? i1 : i2;
      const int nb2 = p.ql.nb2[a], nc2 = p.ql.nc2[a];
      const float4* Q = p.quads + p.ql.base[a] + (int64_t)k * nb2 * nc2;
      s += Q[(I + 1) * nc2 + J + 1].x + Q[I * nc2 + J + 1].y + Q[(I + 1) * nc2 + J].z + Q[I * nc2 + J].w;
    }
    p.img[v] += s;
  }
}

}  // namespace
}  // namespace jp

using namespace jp;

extern "C" int jp_back_tof_lm_noalloc(const float* xs, const float* xe, const int16_t* tof_bin,
                                      const float* tof_center_offset, int64_t n, const jp_image_geom* g,
                                      const jp_tof* t, const float* proj, float* img_accum, void* stream) {
  clear_error();
  if (n < 0) return fail(JP_ERR_ARG, "n_lor must be >= 0");
  if (n > 0 && (!xs || !xe || !tof_bin || !proj)) return fail(JP_ERR_ARG, "array pointer is NULL");
  if (!img_accum) return fail(JP_ERR_ARG, "img_accum is NULL");
  if (!aligned(xs, 4) || !aligned(xe, 4) || !aligned(proj, 4) || !aligned(img_accum, 4) ||
      !aligned(tof_center_offset, 4) || !aligned(tof_bin, 2))
    return fail(JP_ERR_ALIGN, "misaligned array");
  NaParams p;
  std::memset(&p, 0, sizeof(p));
  int rc = make_geom(g, &p.g);
  if (rc) return rc;
  rc = make_tof(t, false, &p.tof);
  if (rc) return rc;
  p.ql = quad_layout(*g);
  if (p.ql.slot > kNoAllocQuads)
    return fail(JP_ERR_ARG, "image too large for the fixed workspace: sum_a n_a' (n_b+2)(n_c+2) must be <= 2^20");
  float4* q = nullptr;
  rc = workspace(&q);
  if (rc) return rc;
  p.xs = xs; p.xe = xe; p.tof_bin = tof_bin; p.delta = tof_center_offset; p.n = n;
  p.proj = proj; p.img = img_accum; p.quads = q;
  cudaStream_t st = (cudaStream_t)stream;
  const int sms = sm_count();
  int64_t zg = (p.ql.slot + 255) / 256;
  if (zg > (int64_t)sms * 8) zg = (int64_t)sms * 8;
  na_zero<<<(unsigned)zg, 256, 0, st>>>(q, p.ql.slot);
  count_launch();
  if (n > 0) {
    na_back<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p);
    count_launch();
  }
  const int64_t nvox = (int64_t)p.g.n[0] * p.g.n[1] * p.g.n[2];
  int64_t fg = (nvox + 255) / 256;
  if (fg > (int64_t)sms * 8) fg = (int64_t)sms * 8;
  na_fold<<<(unsigned)fg, 256, 0, st>>>(p);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}
