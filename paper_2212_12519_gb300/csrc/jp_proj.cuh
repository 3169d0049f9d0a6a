// Internal: the launch parameters and device helpers shared by the
// projection kernels (quad-image kernels in jp_project.cu, shared-memory
// tile kernels in jp_tile.cu).
#pragma once

#include <cuda_runtime.h>

#include "jp_internal.cuh"

namespace jp {
constexpr int kMaxBlock = 512;
constexpr int kLut = JP_TOF_TABLE;  // table nodes over [-R, R]

struct ProjParams {
  // per-event TOF sigma in binned order (listmode), or nullptr
  const float* sig;
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
  int kfast;   // quad order: 1 plane-fastest, 0 plane-major
  // listmode OSEM subset update
  float4* quads_bp;   // back-projection quads (plane-fastest)
  float bg;           // additive background b
  const float* bg_ptr;  // or read from device memory when set
  int f0, f1;         // OSEM: subset frames [f0, f1), range read from frame_off on the device
  const float* sens;  // sensitivity image
  float sens_scale;
  int perm_in_rec;    // caller index in the first record's .w (no TOF centre offsets)
  int max_per_sm;     // host side: cap on resident CTAs per SM for persistent launches (0 = occupancy)
  // persistent kernels take chunks of LORs from this counter (reset by the
  // workspace kernel launched just before them), so the chunks in flight
  // stay a contiguous window of the binned order (one frame's image at a time)
  unsigned int* counter;
  // tile kernels: a line is the run of bins sharing (frame, axis, slope,
  // offset); line_end[key] is the binned end offset of bin key
  const uint32_t* line_end;
  int64_t n_lines;      // n_frames * lines_per_frame
  int lines_per_frame;  // 3 * slope * offset bins
  int lines_per_axis;   // slope * offset bins
  int keys_per_line;    // window * zoff bins
  int kb[3];            // per principal axis a: the key's in-plane (line) axis
  int tile_T;           // LORs per tile
  int box_floats;       // shared-memory image box capacity (floats)
  int line_batch;       // lines claimed per counter increment
  int vec4_out;         // back: image rows take aligned 16-byte reductions
};

namespace {
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
// With a tabulated kernel (T.user) the table holds the caller's T.nodes
// nodes instead.  Entry nodes - 1 holds (g_last, 0), so a coordinate that
// rounds to a hair above the last node needs no clamp of the fraction.
__device__ void build_lut(float2* lut, const DevTof& T) {
  if (T.user) {
    for (int e = threadIdx.x; e < T.nodes - 1; e += blockDim.x) {
      const float g0 = __ldg(T.user + e);
      lut[e] = make_float2(g0, __ldg(T.user + e + 1) - g0);
    }
    if (threadIdx.x == 0) lut[T.nodes - 1] = make_float2(__ldg(T.user + T.nodes - 1), 0.f);
    return;
  }
  const float h = 2.f * T.R / (float)(T.nodes - 1);
  for (int e = threadIdx.x; e < T.nodes - 1; e += blockDim.x) {
    float g0 = tof_g(fmaf((float)e, h, -T.R), T);
    float g1 = tof_g(fmaf((float)(e + 1), h, -T.R), T);
    lut[e] = make_float2(g0, g1 - g0);
  }
  if (threadIdx.x == 0) lut[T.nodes - 1] = make_float2(tof_g(T.R, T), 0.f);
}

// bin-aligned table (T.m > 0): node e at -Rp + e h, h = w / m, untruncated
// erf differences (the bin selection applies the truncation), last entry
// (g_last, 0)
__device__ void build_lut_aligned(float2* lut, const DevTof& T) {
  const float h = T.width / (float)T.m;
  for (int e = threadIdx.x; e < T.nodes_a - 1; e += blockDim.x) {
    const float g0 = tof_g(fmaf((float)e, h, -T.Rp), T);
    const float g1 = tof_g(fmaf((float)(e + 1), h, -T.Rp), T);
    lut[e] = make_float2(g0, g1 - g0);
  }
  if (threadIdx.x == 0) lut[T.nodes_a - 1] = make_float2(tof_g(T.Rp, T), 0.f);
}

// table value at the table coordinate xl = (dist + R) / h of a bin inside
// the support (so xl is in [0, nodes - 1] up to rounding); the index clamp
// only keeps the shared-memory read in bounds for any input
__device__ __forceinline__ float lut_at(const float2* lut, float xl, int last) {
  const int ix = min(max((int)xl, 0), last);
  const float2 e = lut[ix];
  return fmaf(xl - (float)ix, e.y, e.x);
}

// x is clamped to [0, nodes - 1] and the last interval also serves x =
// nodes - 1 (fraction 1), so the end nodes are reproduced exactly
__device__ __forceinline__ float lut_g(const float2* lut, float dist, const DevTof& T) {
  float x = (dist + T.R) * T.inv_h;
  x = fminf(fmaxf(x, 0.f), (float)(T.nodes - 1));
  const int ix = min((int)x, T.nodes - 2);
  float fr = x - (float)ix;
  float2 e = lut[ix];
  return fmaf(fr, e.y, e.x);
}

// k_e: 1 / (sqrt2 sigma) of the LOR (its own sigma with per-event TOF
// resolution, else T.k); the shared-memory table holds T's sigma only, so a
// per-event sigma takes the exact path
template <bool LUT>
__device__ __forceinline__ float tof_weight(const float2* lut, float dist, const DevTof& T, float k_e) {
  if (LUT) return lut_g(lut, dist, T);
  if (T.user) return user_g(dist, T);
  return 0.5f * (erff((dist + T.half) * k_e) - erff((dist - T.half) * k_e));
}

__device__ __forceinline__ bool slot_axis_used(const int32_t* used, int slot, int a, int shared, int n_frames) {
  if (!shared) return __ldg(used + 3 * slot + a) != 0;
  for (int f = 0; f < n_frames; ++f)
    if (__ldg(used + 3 * f + a)) return true;
  return false;
}

// TOF resolution of binned listmode LOR i: k = 1 / (sqrt2 sigma) and the
// support half-width R, from its own sigma when the plan has per-event sigma
// (a value <= 0 keeps the scalar one; a tabulated kernel ignores sigma)
__device__ __forceinline__ void event_tof(const ProjParams& p, int64_t i, float& k, float& R) {
  k = p.tof.k;
  R = p.tof.R;
  if (p.sig && !p.tof.user) {
    const float s = __ldg(p.sig + i);
    if (s > 0.f) {
      k = 1.0f / (1.41421356237309515f * s);
      R = fmaf(p.tof.ns, s, p.tof.half);
    }
  }
}

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace

// Tile kernels (jp_tile.cu): planned non-TOF (mode 0) and TOF-listmode
// (mode 2) projections through shared-memory image boxes; lanes = lanes
// per LOR (4, 8, 16 or 32), block = threads per CTA (64..512).
int launch_tile(const ProjParams& p, int mode, bool back, bool lut, int lanes, int block, cudaStream_t st);

}  // namespace jp
