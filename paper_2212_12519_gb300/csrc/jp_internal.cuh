// Internal declarations of libjoseph: device geometry helpers shared by the
// binning and projection kernels, the plan object and host error helpers.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "joseph.h"

namespace jp {

// ---------------------------------------------------------------------------
// host-side error reporting (thread-local message, see jp_last_error)
// ---------------------------------------------------------------------------
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
void clear_error();
int sm_count();
void count_launch(int n = 1);

#define JP_TRY_CUDA(expr)                              \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) return jp::cuda_fail(_e, #expr); \
  } while (0)

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ---------------------------------------------------------------------------
// geometry passed to kernels
// ---------------------------------------------------------------------------
struct DevGeom {
  int n[3];
  float o[3];
  float v[3];
  float inv_v[3];
  int stride[3];  // n1*n2, n2, 1
};

struct DevTof {
  const float* user;  // tabulated kernel (device) or nullptr for the Gaussian
  int nodes;       // table nodes over [-R, R]: the shared-memory table or `user`
  float inv_h;     // (nodes - 1) / (2 R)
  float width;     // TOF bin width w
  float half;      // w / 2
  float k;         // 1 / (sqrt2 sigma)
  float ns;        // n_sigmas (per-event sigma: R_e = ns sigma_e + w / 2)
  float R;         // support half-width: n_sigmas * sigma + w / 2, or the table's
  float R_over_w;  // R / w
  float inv_w;     // 1 / w
  float hbin;      // (N - 1) / 2
  int nbins;       // N
  // bin-aligned table of the sinogram kernels (Gaussian only): node spacing
  // h = w / m, nodes at -Rp + e h with Rp = c h >= R, so the coordinates of
  // one sample's bins differ by exactly m nodes (m = 0: not used)
  int m;
  int nodes_a;     // 2 c + 1
  float Rp;        // c h
  float inv_hp;    // 1 / h
};

int make_geom(const jp_image_geom* g, DevGeom* out);
int make_tof(const jp_tof* t, bool sino, DevTof* out);

// ---------------------------------------------------------------------------
// image-based resolution model (separable Gaussian, jp_res.cu)
// ---------------------------------------------------------------------------
constexpr int kMaxResTaps = 2 * JP_MAX_RES_RADIUS + 1;

struct GaussTaps {
  int r[3];                    // radius R_a per axis
  float w[3][kMaxResTaps];     // normalised taps, index t + R_a
};

int make_taps(const jp_image_geom* g, const jp_resolution* r, GaussTaps* out);

// Three passes in -> b1 (axis 2) -> b2 (axis 1) -> dst (axis 0) over n_img
// images; in != b1, b1 != b2, b2 != dst (in == b2 is allowed: pass 1 has
// consumed it).  With upd_sens non-NULL the last pass is the OSEM update
// dst[j] <- upd_sens[j]*scale > 0 ? dst[j] * (H in)[j] / (upd_sens[j]*scale) : 0
// (one sensitivity image shared by the n_img images).
int gauss_passes(const float* in, float* b1, float* b2, float* dst, int n_img, const DevGeom& g,
                 const GaussTaps& t, const float* upd_sens, float scale, cudaStream_t st);

// ---------------------------------------------------------------------------
// per-LOR setup (paper Sec. 2.1): principal axis, plane range, affine maps
// ---------------------------------------------------------------------------
struct Ray {
  int k0, k1;      // visited planes k0..k1 (empty when k0 > k1)
  float kc;        // anchor plane index (centre plane of axis a)
  float uc, du;    // u(k) = uc + (k - kc) du   (continuous index along b)
  float wc, dw;    // w(k) = wc + (k - kc) dw   (continuous index along c)
  float tc, dt;    // tau(k) = tc + (k - kc) dt (mm from the LOR midpoint)
  float w0;        // v_a / cos_a
  int sa, sb, sc;  // flat-index strides of axes a, b, c
  int nb, nc;      // grid sizes along b, c
  int a;
};

// a - b as hi + lo exactly (two-sum with -b)
__device__ __forceinline__ void two_diff(float a, float b, float& hi, float& lo) {
  float s = __fsub_rn(a, b);
  float bv = __fsub_rn(s, a);
  float av = __fsub_rn(s, bv);
  hi = s;
  lo = __fadd_rn(__fsub_rn(a, av), __fsub_rn(-b, bv));
}

// exact |d_i| > |d_j| for d = hi + lo
__device__ __forceinline__ bool abs_greater(float hi_i, float lo_i, float hi_j, float lo_j) {
  float ai = fabsf(hi_i), aj = fabsf(hi_j);
  if (ai != aj) return ai > aj;
  float ri = hi_i > 0.f ? lo_i : -lo_i;
  float rj = hi_j > 0.f ? lo_j : -lo_j;
  if (hi_i == 0.f) ri = 0.f;
  if (hi_j == 0.f) rj = 0.f;
  return ri > rj;
}

// principal axis: argmax |xe_i - xs_i| decided exactly, lowest index on ties
__device__ __forceinline__ int principal_axis(float xs0, float xs1, float xs2, float xe0, float xe1,
                                              float xe2) {
  float h0, l0, h1, l1, h2, l2;
  two_diff(xe0, xs0, h0, l0);
  two_diff(xe1, xs1, h1, l1);
  two_diff(xe2, xs2, h2, l2);
  int a = 0;
  float ha = h0, la = l0;
  if (abs_greater(h1, l1, ha, la)) { a = 1; ha = h1; la = l1; }
  if (abs_greater(h2, l2, ha, la)) a = 2;
  return a;
}

__device__ __forceinline__ int principal_axis(const float xs[3], const float xe[3]) {
  return principal_axis(xs[0], xs[1], xs[2], xe[0], xe[1], xe[2]);
}

template <typename T>
__device__ __forceinline__ T sel3(int i, T x0, T x1, T x2) {
  return i == 0 ? x0 : (i == 1 ? x1 : x2);
}

// Restricts [kmin, kmax] to planes where t(k) = tcen + (k - kc) * dt can lie
// in the open interval (lo, hi), with one plane of margin on each side (the
// per-sample arithmetic decides exactly; trimmed samples contribute zero).
__device__ __forceinline__ void trim_range(float tcen, float dt, float lo, float hi, float kc,
                                           float& kmin, float& kmax) {
  if (dt == 0.f) {
    if (!(tcen > lo && tcen < hi)) { kmin = 1.f; kmax = 0.f; }
    return;
  }
  float t1 = (lo - tcen) / dt, t2 = (hi - tcen) / dt;
  float a = fminf(t1, t2), b = fmaxf(t1, t2);
  kmin = fmaxf(kmin, floorf(kc + a) - 1.f);
  kmax = fminf(kmax, ceilf(kc + b) + 1.f);
}

// Sets up the ray; returns false for a degenerate LOR or an empty plane range.
__device__ __forceinline__ bool ray_setup(const float xs[3], const float xe[3],
                                          const DevGeom& g, Ray& r) {
  const float d0 = xe[0] - xs[0], d1 = xe[1] - xs[1], d2 = xe[2] - xs[2];
  const float L = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  r.k0 = 1; r.k1 = 0;
  r.a = 0; r.w0 = 0.f; r.kc = 0.f;
  r.uc = r.du = r.wc = r.dw = r.tc = r.dt = 0.f;
  r.sa = r.sb = r.sc = 0; r.nb = r.nc = 1;
  if (!(L > 0.f)) return false;
  const int a = principal_axis(xs, xe);
  const int b = (a == 0) ? 1 : 0;
  const int c = (a == 2) ? 1 : 2;
  r.a = a;
  // gather the per-axis quantities with selects (no dynamic indexing)
  const float da = sel3(a, d0, d1, d2), db = sel3(b, d0, d1, d2), dc = sel3(c, d0, d1, d2);
  const float xsa = sel3(a, xs[0], xs[1], xs[2]), xea = sel3(a, xe[0], xe[1], xe[2]);
  const float xsb = sel3(b, xs[0], xs[1], xs[2]), xeb = sel3(b, xe[0], xe[1], xe[2]);
  const float xsc = sel3(c, xs[0], xs[1], xs[2]), xec = sel3(c, xe[0], xe[1], xe[2]);
  const float oa = sel3(a, g.o[0], g.o[1], g.o[2]), ob = sel3(b, g.o[0], g.o[1], g.o[2]),
              oc = sel3(c, g.o[0], g.o[1], g.o[2]);
  const float va = sel3(a, g.v[0], g.v[1], g.v[2]);
  const float ivb = sel3(b, g.inv_v[0], g.inv_v[1], g.inv_v[2]);
  const float ivc = sel3(c, g.inv_v[0], g.inv_v[1], g.inv_v[2]);
  const int na = sel3(a, g.n[0], g.n[1], g.n[2]);
  r.nb = sel3(b, g.n[0], g.n[1], g.n[2]);
  r.nc = sel3(c, g.n[0], g.n[1], g.n[2]);
  r.sa = sel3(a, g.stride[0], g.stride[1], g.stride[2]);
  r.sb = sel3(b, g.stride[0], g.stride[1], g.stride[2]);
  r.sc = sel3(c, g.stride[0], g.stride[1], g.stride[2]);
  const float inv_da = 1.0f / da;
  r.w0 = va * L * fabsf(inv_da);
  // planes whose centre lies in the closed segment [min, max] along a
  const float lo = fminf(xsa, xea), hi = fmaxf(xsa, xea);
  float kmin = ceilf((lo - oa) / va);
  float kmax = floorf((hi - oa) / va);
  kmin = fmaxf(kmin, 0.f);
  kmax = fminf(kmax, (float)(na - 1));
  // affine maps anchored at the centre plane, from the LOR midpoint
  const float kc = 0.5f * (float)(na - 1);
  const float Xc = oa + kc * va;
  const float ma = 0.5f * (xsa + xea), mb = 0.5f * (xsb + xeb), mc = 0.5f * (xsc + xec);
  const float t = (Xc - ma) * inv_da;  // lambda(kc) - 1/2
  r.kc = kc;
  r.uc = (fmaf(t, db, mb) - ob) * ivb;
  r.wc = (fmaf(t, dc, mc) - oc) * ivc;
  const float step = va * inv_da;  // lambda per plane
  r.du = step * db * ivb;
  r.dw = step * dc * ivc;
  r.tc = t * L;
  r.dt = step * L;
  // planes where the bilinear support can touch the grid
  trim_range(r.uc, r.du, -1.f, (float)r.nb, kc, kmin, kmax);
  trim_range(r.wc, r.dw, -1.f, (float)r.nc, kc, kmin, kmax);
  if (!(kmin <= kmax)) return false;
  r.k0 = (int)kmin;
  r.k1 = (int)kmax;
  return true;
}

// Bilinear sample of plane k with zero padding (paper Fig. 1: the 4 nearest
// voxels of the ray/plane intersection).
struct Corners {
  int idx;                   // flat index of (i, j)
  float w00, w10, w01, w11;  // weights of (i,j), (i+1,j), (i,j+1), (i+1,j+1)
  bool m00, m10, m01, m11;   // inside the grid
};

__device__ __forceinline__ void corners(const Ray& r, int k, float u, float w, Corners& q) {
  u = fminf(fmaxf(u, -2.f), (float)r.nb + 1.f);
  w = fminf(fmaxf(w, -2.f), (float)r.nc + 1.f);
  const float fu = floorf(u), fw = floorf(w);
  const float al = u - fu, be = w - fw;
  const int i = (int)fu, j = (int)fw;
  const bool i0 = (unsigned)i < (unsigned)r.nb, i1 = (unsigned)(i + 1) < (unsigned)r.nb;
  const bool j0 = (unsigned)j < (unsigned)r.nc, j1 = (unsigned)(j + 1) < (unsigned)r.nc;
  q.idx = k * r.sa + i * r.sb + j * r.sc;
  q.m00 = i0 && j0; q.m10 = i1 && j0; q.m01 = i0 && j1; q.m11 = i1 && j1;
  const float ab = 1.f - al, bb = 1.f - be;
  q.w00 = ab * bb; q.w10 = al * bb; q.w01 = ab * be; q.w11 = al * be;
}

__device__ __forceinline__ float interp(const float* __restrict__ img, const Ray& r, const Corners& q) {
  const float v00 = q.m00 ? __ldg(img + q.idx) : 0.f;
  const float v10 = q.m10 ? __ldg(img + q.idx + r.sb) : 0.f;
  const float v01 = q.m01 ? __ldg(img + q.idx + r.sc) : 0.f;
  const float v11 = q.m11 ? __ldg(img + q.idx + r.sb + r.sc) : 0.f;
  return q.w00 * v00 + q.w10 * v10 + q.w01 * v01 + q.w11 * v11;
}

__device__ __forceinline__ void scatter_add(float* img, const Ray& r, const Corners& q, float val) {
  if (q.m00) atomicAdd(img + q.idx, q.w00 * val);
  if (q.m10) atomicAdd(img + q.idx + r.sb, q.w10 * val);
  if (q.m01) atomicAdd(img + q.idx + r.sc, q.w01 * val);
  if (q.m11) atomicAdd(img + q.idx + r.sb + r.sc, q.w11 * val);
}

// tabulated kernel at dist, linear interpolation between the nodes (the
// same formula as the shared-memory table lookup)
__device__ __forceinline__ float user_g(float dist, const DevTof& t) {
  float x = (dist + t.R) * t.inv_h;
  x = fminf(fmaxf(x, 0.f), (float)(t.nodes - 1));
  const int ix = min((int)x, t.nodes - 2);
  const float fr = x - (float)ix;
  const float g0 = __ldg(t.user + ix);
  return fmaf(fr, __ldg(t.user + ix + 1) - g0, g0);
}

// TOF weight of one bin, no truncation test (the caller decides the window)
__device__ __forceinline__ float tof_g(float dist, const DevTof& t) {
  if (t.user) return user_g(dist, t);
  return 0.5f * (erff((dist + t.half) * t.k) - erff((dist - t.half) * t.k));
}

// ---------------------------------------------------------------------------
// quad images: for principal axis a, entry (i, j, k) -- k the plane along a,
// i along b and j along c, i and j from -1 to n_b / n_c -- holds the 4
// bilinear neighbours (f(k,i,j), f(k,i+1,j), f(k,i,j+1), f(k,i+1,j+1)) with
// zeros outside the grid, so a plane sample is one 16-byte load (forward) or
// one 16-byte vector reduction (back projection) with no bounds tests.  Two
// orders are used:
//   plane-major   index = (k * nb2 + (i + 1)) * nc2 + (j + 1): the lanes of a
//                 warp following 32 neighbouring LORs (one per thread) read
//                 nearby entries of the same plane rows;
//   plane-fastest index = ((i + 1) * nc2 + (j + 1)) * nap + k: the lanes of a
//                 group walking consecutive planes of one LOR touch
//                 consecutive 16-byte entries (coalesced reductions).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int quad_index(bool kfast, int k, int ip, int jp, int na, int nb2, int nc2) {
  return kfast ? (ip * nc2 + jp) * na + k : (k * nb2 + ip) * nc2 + jp;
}

struct QuadLayout {
  int nb2[3], nc2[3];  // n_b + 2, n_c + 2 for axis a
  int nap[3];          // n_a rounded up to even: in plane-fastest order the two
                       // entries of a 32-byte sector are always planes 2m, 2m+1
  int64_t size[3];     // nap * nb2 * nc2 entries of Q_a
  int64_t base[3];     // float4 offset of Q_a inside one slot
  int64_t slot;        // float4 per slot (one image)
};

inline QuadLayout quad_layout(const jp_image_geom& g) {
  QuadLayout q;
  int64_t off = 0;
  for (int a = 0; a < 3; ++a) {
    int b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
    q.nb2[a] = g.n[b] + 2;
    q.nc2[a] = g.n[c] + 2;
    q.nap[a] = g.n[a] + (g.n[a] & 1);
    q.size[a] = (int64_t)q.nap[a] * q.nb2[a] * q.nc2[a];
    q.base[a] = off;
    off += q.size[a];
  }
  q.slot = off;
  return q;
}

struct PlanDims {
  int slope_bins, offset_bins, window_bins, zoff_bins;
  int keys_per_frame;
  int keys_per_axis;
};

}  // namespace jp

struct jp_plan_s {
  int64_t capacity;       // LORs allocated
  int32_t frame_capacity;
  int64_t n;              // LORs bound
  int32_t n_frames;
  jp_image_geom g;
  jp_plan_opts opts;
  bool auto_block;        // opts.block was 0: each kernel takes its own default
  jp::PlanDims dims;
  bool has_tof_bin, has_delta;
  int kb[3];              // per principal axis: the in-plane axis of the slope / offset keys
  float4* lor;            // [2*capacity]: (xs, delta or caller index bits), (xe, tof_bin bits)
  int32_t* perm;          // [capacity] binned position -> caller index (used when delta is given;
                          // otherwise the caller index rides in the record's first .w)
  uint32_t* keys;         // [capacity]
  uint32_t* hist;         // [frame_capacity * keys_per_frame + 1]
  uint32_t* block_sums;   // scan scratch
  float4* det4;           // [det4_cap] detector table padded to 16 bytes (detector-index plans)
  int32_t det4_cap;
  int64_t* frame_off_dev; // [frame_capacity + 1]
  int64_t* frame_off_host;// pinned [frame_capacity + 1]
  int64_t hist_len;
  int64_t scan_blocks_cap;
  // projection workspace
  jp::QuadLayout ql;
  float4* quads;          // [quad_slots * ql.slot]
  int32_t quad_slots;     // frames with their own image, or 2 (image + back projection) when interleaved
  int32_t* axis_used;     // [frame_capacity * 3]: frame f has LORs with principal axis a
  uint32_t* work_counter; // chunk counter of the persistent projection kernels
  float* fold_img;        // [nvox] folded back projection of an OSEM subset (interleaved plans only)
  float* sig_binned;      // [capacity] per-event TOF sigma in binned order (allocated on first use)
  bool has_sigma;         // sig_binned is current for the bound LORs
};
