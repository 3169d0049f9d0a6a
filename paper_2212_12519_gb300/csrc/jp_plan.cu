// LOR plan: sorting LORs into coherent bins and packing them.
//
// Step a1 of the hot path.  The paper's kernels walk rays in input order and
// report up to 7.6x run-time spread across memory orders (Sec. 3), traced to
// races and cache behaviour (Sec. 4), and suggest pre-sorting events (Sec. 4).
// Here each LOR gets a key
//     frame | principal axis a | slope d_b/d_a | offset along b at the
//     centre plane | (listmode) TOF window centre along a | offset along c
//     at the centre plane
// (b the longer in-plane axis of a, c the other one) and a counting sort
// (histogram, exclusive scan, scatter) reorders the LORs so that the 32
// lanes of a warp follow nearly parallel, nearby rays.  The sorted LORs are
// packed as two float4, (xs, delta or the caller index) and (xe, tof_bin),
// for 16-byte coalesced loads; with TOF centre offsets perm maps back to
// caller order, otherwise the caller index in the record does.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "jp_internal.cuh"

namespace jp {

namespace {

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanBlock * kScanItems;

__device__ __forceinline__ int frame_of(const int64_t* __restrict__ off, int n_frames, int64_t i) {
  int lo = 0, hi = n_frames - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct KeyParams {
  const float* xs;
  const float* xe;
  // detector-index input (xs / xe NULL): endpoints are det_xyz[ds[j]], det_xyz[de[j]]
  const int32_t* ds;
  const int32_t* de;
  const float* dxyz;
  const float4* det4;  // the plan's 16-byte-padded copy of dxyz, or NULL
  int32_t n_det;
  const int16_t* tof_bin;
  const float* delta;
  int64_t n;
  const int64_t* frame_off;
  int n_frames;
  DevGeom g;
  // per principal axis a: the in-plane axis b of the slope / offset keys (the
  // longer of the two others, so that slope and offset follow the image's
  // wide in-plane direction whichever axis holds the scanner's axial one);
  // the axial-offset key takes the remaining axis c = 3 - a - b
  int kb[3];
  // per image axis: the centre plane's coordinate, and key cells per
  // (padded) index unit of the offset, window and axial-offset keys
  float xc[3], inv_cell_u[3], inv_cell_w[3], inv_cell_z[3];
  int slope_bins, offset_bins, window_bins, zoff_bins, keys_per_frame;
  float tof_width;  // > 0: listmode window binning
  int keep_order;
  int interleaved;  // frame of LOR j is j mod n_frames
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Where the endpoints come from: the coordinate arrays, the caller's
// [n_det][3] detector table, or the plan's 16-byte-padded copy of it.
enum { kSrcXyz = 0, kSrcDet = 1, kSrcDet4 = 2 };

// detector coordinates of index d; an index outside [0, n_det) gives the
// origin (so a LOR with one gives the empty LOR xs = xe = 0)
template <int SRC>
__device__ __forceinline__ void det_xyz(const KeyParams& p, int32_t d, bool ok, float x[3]) {
  if (SRC == kSrcDet4) {
    // the index is clamped too, so no form of the load leaves the table
    const float4 v = __ldg(p.det4 + (ok ? d : 0));
    x[0] = ok ? v.x : 0.f;
    x[1] = ok ? v.y : 0.f;
    x[2] = ok ? v.z : 0.f;
  } else {
    const float* q = p.dxyz + 3 * (int64_t)(ok ? d : 0);
    for (int i = 0; i < 3; ++i) x[i] = ok ? __ldg(q + i) : 0.f;
  }
}

// endpoints of caller LOR j, from the coordinate arrays or from the detector
// table; an index outside [0, n_det) gives the empty LOR xs = xe = 0
template <int SRC>
__device__ __forceinline__ void lor_endpoints(const KeyParams& p, int64_t j, float xs[3], float xe[3]) {
  if (SRC != kSrcXyz) {
    const int32_t a = __ldg(p.ds + j), b = __ldg(p.de + j);
    const bool ok = (unsigned)a < (unsigned)p.n_det && (unsigned)b < (unsigned)p.n_det;
    det_xyz<SRC>(p, a, ok, xs);
    det_xyz<SRC>(p, b, ok, xe);
  } else {
    for (int i = 0; i < 3; ++i) {
      xs[i] = __ldg(p.xs + 3 * j + i);
      xe[i] = __ldg(p.xe + 3 * j + i);
    }
  }
}

// The packed records of PER LORs j[q] (entries with j[q] >= n are zero):
// (xs, w), (xe, tof_bin bits), w = delta[j] when with_delta, else the
// caller index j.  Every load is issued before the caller's stores (the
// detector-table reads after the index reads), so a thread keeps all of its
// LORs' loads in flight at once.
template <int SRC, int PER>
__device__ __forceinline__ void load_records(const KeyParams& p, const int64_t (&j)[PER], bool with_delta,
                                             float4 (&ra)[PER], float4 (&rb)[PER]) {
  int32_t da[PER], db[PER];
  float w[PER];
  int tb[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const bool in = j[q] < p.n;
    da[q] = (in && SRC != kSrcXyz) ? __ldg(p.ds + j[q]) : 0;
    db[q] = (in && SRC != kSrcXyz) ? __ldg(p.de + j[q]) : 0;
    w[q] = (in && with_delta) ? __ldg(p.delta + j[q]) : __int_as_float((int)j[q]);
    tb[q] = (in && p.tof_bin) ? (int)__ldg(p.tof_bin + j[q]) : 0;
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const bool in = j[q] < p.n;
    float xs[3] = {0.f, 0.f, 0.f}, xe[3] = {0.f, 0.f, 0.f};
    if (SRC != kSrcXyz) {
      const bool ok = in && (unsigned)da[q] < (unsigned)p.n_det && (unsigned)db[q] < (unsigned)p.n_det;
      det_xyz<SRC>(p, da[q], ok, xs);
      det_xyz<SRC>(p, db[q], ok, xe);
    } else if (in) {
      for (int i = 0; i < 3; ++i) {
        xs[i] = __ldg(p.xs + 3 * j[q] + i);
        xe[i] = __ldg(p.xe + 3 * j[q] + i);
      }
    }
    ra[q] = make_float4(xs[0], xs[1], xs[2], w[q]);
    rb[q] = make_float4(xe[0], xe[1], xe[2], __int_as_float(tb[q]));
  }
}

// one 32-byte store: a record fills its sector in a single request
__device__ __forceinline__ void st_record(float4* dst, float4 a, float4 b) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "f"(a.x), "f"(a.y), "f"(a.z),
               "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
               : "memory");
}

template <int SRC>
__global__ void key_kernel(KeyParams p, uint32_t* __restrict__ keys, uint32_t* __restrict__ hist) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.n) return;
  int f = p.interleaved ? (int)(j % p.n_frames) : frame_of(p.frame_off, p.n_frames, j);
  uint32_t key = 0;
  if (!p.keep_order) {
    float xs[3], xe[3];
    lor_endpoints<SRC>(p, j, xs, xe);
    const float d0 = xe[0] - xs[0], d1 = xe[1] - xs[1], d2 = xe[2] - xs[2];
    const int a = principal_axis(xs, xe);
    const int b = sel3(a, p.kb[0], p.kb[1], p.kb[2]);
    const DevGeom& g = p.g;
    const float da = sel3(a, d0, d1, d2), db = sel3(b, d0, d1, d2);
    // the keys only order the LORs, so reciprocals stand in for divisions
    const float rda = (da != 0.f) ? __frcp_rn(da) : 0.f;
    const float sb = db * rda;  // in [-1, 1]
    const int qs = clampi((int)floorf((sb + 1.f) * 0.5f * (float)p.slope_bins), 0, p.slope_bins - 1);
    // in-plane offset (continuous index along b) where the line crosses the centre plane
    const float oa = sel3(a, g.o[0], g.o[1], g.o[2]), ob = sel3(b, g.o[0], g.o[1], g.o[2]);
    const float ivb = sel3(b, g.inv_v[0], g.inv_v[1], g.inv_v[2]);
    const float ma = 0.5f * (sel3(a, xs[0], xs[1], xs[2]) + sel3(a, xe[0], xe[1], xe[2]));
    const float mb = 0.5f * (sel3(b, xs[0], xs[1], xs[2]) + sel3(b, xe[0], xe[1], xe[2]));
    const float t = (sel3(a, p.xc[0], p.xc[1], p.xc[2]) - ma) * rda;
    const float u = (fmaf(t, db, mb) - ob) * ivb;
    const int qu = clampi((int)floorf((u + 1.f) * sel3(b, p.inv_cell_u[0], p.inv_cell_u[1], p.inv_cell_u[2])), 0,
                          p.offset_bins - 1);
    int qw = 0;
    if (p.window_bins > 1 && p.tof_width > 0.f && p.tof_bin != nullptr) {
      const float L2 = d0 * d0 + d1 * d1 + d2 * d2;
      const float cen = (float)p.tof_bin[j] * p.tof_width + (p.delta ? p.delta[j] : 0.f);
      const float ca = (L2 > 0.f) ? fmaf(cen * da, rsqrtf(L2), ma) : ma;  // window centre along a
      const float ka = (ca - oa) * sel3(a, g.inv_v[0], g.inv_v[1], g.inv_v[2]);
      qw = clampi((int)floorf((ka + 1.f) * sel3(a, p.inv_cell_w[0], p.inv_cell_w[1], p.inv_cell_w[2])), 0,
                  p.window_bins - 1);
    }
    int qz = 0;
    if (p.zoff_bins > 1) {
      const int c = 3 - a - b;
      const float oc = sel3(c, g.o[0], g.o[1], g.o[2]), ivc = sel3(c, g.inv_v[0], g.inv_v[1], g.inv_v[2]);
      const float mc = 0.5f * (sel3(c, xs[0], xs[1], xs[2]) + sel3(c, xe[0], xe[1], xe[2]));
      const float w = (fmaf(t, sel3(c, d0, d1, d2), mc) - oc) * ivc;
      qz = clampi((int)floorf((w + 1.f) * sel3(c, p.inv_cell_z[0], p.inv_cell_z[1], p.inv_cell_z[2])), 0,
                  p.zoff_bins - 1);
    }
    key = (uint32_t)((((a * p.slope_bins + qs) * p.offset_bins + qu) * p.window_bins + qw) * p.zoff_bins + qz);
  }
  key += (uint32_t)f * (uint32_t)p.keys_per_frame;
  keys[j] = key;
  if (!p.keep_order) atomicAdd(hist + key, 1u);
}

// exclusive scan, three passes: tile sums, scan of tile sums, tile scan
__global__ void scan_tile_sums(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
  __shared__ uint32_t red[kScanBlock / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    int64_t i = base + (int64_t)q * kScanBlock + threadIdx.x;
    if (i < n) s += in[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = red[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = s;
  }
}

// block-wide exclusive scan of kScanTile values held kScanItems per thread
// (thread t holds items t*kScanItems .. t*kScanItems + kScanItems - 1)
__device__ void block_exclusive_scan(uint32_t (&v)[kScanItems], uint32_t carry_in, uint32_t* total) {
  __shared__ uint32_t warp_tot[kScanBlock / 32];
  uint32_t local = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) { uint32_t x = v[q]; v[q] = local; local += x; }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = (lane < kScanBlock / 32) ? warp_tot[lane] : 0;
    uint32_t wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < kScanBlock / 32) warp_tot[lane] = wi - w;  // exclusive
    if (lane == 31 && total) *total = wi;
  }
  __syncthreads();
  uint32_t off = carry_in + warp_tot[wid] + (incl - local);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) v[q] += off;
  __syncthreads();
}

// single CTA: exclusive scan of the tile sums (nt <= kScanTile)
__global__ void scan_sums_kernel(uint32_t* __restrict__ sums, int64_t nt) {
  uint32_t v[kScanItems];
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    int64_t i = (int64_t)threadIdx.x * kScanItems + q;
    v[q] = i < nt ? sums[i] : 0u;
  }
  block_exclusive_scan(v, 0u, nullptr);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    int64_t i = (int64_t)threadIdx.x * kScanItems + q;
    if (i < nt) sums[i] = v[q];
  }
}

__global__ void scan_apply_kernel(uint32_t* __restrict__ data, int64_t n, const uint32_t* __restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t v[kScanItems];
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + q;
    v[q] = i < n ? data[i] : 0u;
  }
  block_exclusive_scan(v, sums[blockIdx.x], nullptr);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + q;
    if (i < n) data[i] = v[q];
  }
}

// Each thread places kScatterPer LORs: it issues all their input loads,
// then their slot claims (independent returning atomics), then one 32-byte
// record store each, so every thread keeps several LORs in flight.
constexpr int kScatterPer = 2;  // 13.10 vs 13.23 ms (4) and 13.9 ms (6) per 8 x 40M batch

template <int SRC>
__global__ void scatter_kernel(KeyParams p, const uint32_t* __restrict__ keys, uint32_t* __restrict__ cursor,
                               float4* __restrict__ lor, int32_t* __restrict__ perm) {
  const int64_t base = ((int64_t)blockIdx.x * blockDim.x) * kScatterPer + threadIdx.x;
  int64_t j[kScatterPer];
  uint32_t key[kScatterPer], pos[kScatterPer];
#pragma unroll
  for (int q = 0; q < kScatterPer; ++q) {
    j[q] = base + (int64_t)q * blockDim.x;
    key[q] = (!p.keep_order && j[q] < p.n) ? __ldg(keys + j[q]) : 0u;
  }
  // without TOF centre offsets the caller index rides in the record, so a
  // LOR costs one scattered 32-byte sector instead of two
  float4 ra[kScatterPer], rb[kScatterPer];
  load_records<SRC, kScatterPer>(p, j, p.delta != nullptr, ra, rb);
#pragma unroll
  for (int q = 0; q < kScatterPer; ++q)
    pos[q] = (j[q] < p.n) ? (p.keep_order ? (uint32_t)j[q] : atomicAdd(cursor + key[q], 1u)) : 0u;
#pragma unroll
  for (int q = 0; q < kScatterPer; ++q) {
    if (j[q] >= p.n) continue;
    st_record(lor + 2 * (int64_t)pos[q], ra[q], rb[q]);
    if (p.delta) perm[pos[q]] = (int32_t)j[q];
  }
}

// padded copy of the detector table: one 16-byte load per endpoint
__global__ void det4_fill_kernel(const float* __restrict__ xyz, int32_t n_det, float4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_det) out[i] = make_float4(xyz[3 * (int64_t)i], xyz[3 * (int64_t)i + 1], xyz[3 * (int64_t)i + 2], 0.f);
}

// Frame offsets reach the device as kernel arguments (copied at launch), so
// the host array may be reused as soon as the call returns.
constexpr int kOffChunk = 256;
struct OffChunk {
  int64_t v[kOffChunk];
};

__global__ void set_offsets_kernel(int64_t* __restrict__ dst, OffChunk c, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = c.v[i];
}

// Frame f has LORs with principal axis a iff its keys of axis a hold any LOR.
// After the scatter, cursor[key] is the end offset of bin `key`.
__global__ void axis_flags_kernel(const uint32_t* __restrict__ cursor, int n_frames, int keys_per_frame,
                                  int keys_per_axis, int keep_order, int32_t* __restrict__ used) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_frames * 3) return;
  if (keep_order) { used[t] = 1; return; }
  int f = t / 3, a = t - 3 * f;
  int64_t first = (int64_t)f * keys_per_frame + (int64_t)a * keys_per_axis;
  int64_t last = first + keys_per_axis - 1;
  uint32_t start = first > 0 ? cursor[first - 1] : 0u;
  used[t] = cursor[last] > start ? 1 : 0;
}

int validate_offsets(const int64_t* off, int32_t n_frames, int64_t* n_total) {
  if (!off) return fail(JP_ERR_ARG, "frame_offsets is NULL");
  if (n_frames < 1) return fail(JP_ERR_ARG, "n_frames must be >= 1");
  if (off[0] != 0) return fail(JP_ERR_ARG, "frame_offsets[0] must be 0");
  for (int32_t f = 0; f < n_frames; ++f)
    if (off[f + 1] < off[f]) return fail(JP_ERR_ARG, "frame_offsets must be non-decreasing");
  *n_total = off[n_frames];
  if (*n_total >= (int64_t)INT32_MAX) return fail(JP_ERR_ARG, "n_total must be < 2^31");
  return JP_OK;
}

// The LORs come either as coordinate arrays (xs, xe) or as detector
// indices into a detector coordinate table (det != nullptr).
struct DetInput {
  const int32_t* ds;
  const int32_t* de;
  const float* xyz;
  int32_t n_det;
};

int bind(jp_plan p, const float* xs, const float* xe, const int16_t* tof_bin, const float* delta,
         const int64_t* off, int32_t n_frames, cudaStream_t st, const DetInput* det = nullptr) {
  int64_t n = 0;
  const bool interleaved = (p->opts.flags & JP_PLAN_INTERLEAVED) != 0;
  if (interleaved) {
    if (!off || n_frames < 1) return fail(JP_ERR_ARG, "frame_offsets / n_frames");
    n = off[n_frames];
    if (n < 0 || n >= (int64_t)INT32_MAX) return fail(JP_ERR_ARG, "n_total must be in [0, 2^31)");
  } else {
    int rc0 = validate_offsets(off, n_frames, &n);
    if (rc0) return rc0;
  }
  int rc = JP_OK;
  if (n > p->capacity || n_frames > p->frame_capacity)
    return fail(JP_ERR_ARG, "rebind exceeds the plan's capacity");
  if (det) {
    if (n > 0 && (!det->ds || !det->de || !det->xyz)) return fail(JP_ERR_ARG, "det_start/det_end/det_xyz is NULL");
    if (det->n_det < 1) return fail(JP_ERR_ARG, "n_det must be >= 1");
    if (!aligned(det->ds, 4) || !aligned(det->de, 4) || !aligned(det->xyz, 4))
      return fail(JP_ERR_ALIGN, "misaligned detector arrays");
  } else if (n > 0 && (!xs || !xe)) {
    return fail(JP_ERR_ARG, "xstart/xend is NULL");
  }
  // a new binding invalidates the per-event sigma gathered for the old one
  p->has_sigma = false;
  if (!aligned(xs, 4) || !aligned(xe, 4) || !aligned(tof_bin, 2) || !aligned(delta, 4))
    return fail(JP_ERR_ALIGN, "misaligned LOR arrays");
  p->has_tof_bin = tof_bin != nullptr;
  p->has_delta = delta != nullptr;
  DevGeom g;
  rc = make_geom(&p->g, &g);
  if (rc) return rc;
  if (interleaved) {
    // frame f holds LORs f, f + n_frames, ...: its count is known up front
    p->frame_off_host[0] = 0;
    for (int32_t f = 0; f < n_frames; ++f)
      p->frame_off_host[f + 1] = p->frame_off_host[f] + n / n_frames + (f < n % n_frames ? 1 : 0);
  } else {
    std::memcpy(p->frame_off_host, off, sizeof(int64_t) * (n_frames + 1));
  }
  for (int32_t c0 = 0; c0 <= n_frames; c0 += kOffChunk) {
    OffChunk chunk;
    const int cnt = std::min<int32_t>(kOffChunk, n_frames + 1 - c0);
    std::memcpy(chunk.v, p->frame_off_host + c0, sizeof(int64_t) * cnt);
    set_offsets_kernel<<<1, 256, 0, st>>>(p->frame_off_dev + c0, chunk, cnt);
    count_launch();
  }
  JP_TRY_CUDA(cudaGetLastError());
  p->n = n;
  p->n_frames = n_frames;
  if (n == 0) {
    JP_TRY_CUDA(cudaMemsetAsync(p->axis_used, 0, sizeof(int32_t) * 3 * n_frames, st));
    return JP_OK;
  }
  KeyParams kp;
  kp.xs = det ? nullptr : xs; kp.xe = det ? nullptr : xe;
  kp.ds = det ? det->ds : nullptr; kp.de = det ? det->de : nullptr;
  kp.dxyz = det ? det->xyz : nullptr; kp.n_det = det ? det->n_det : 0;
  kp.det4 = nullptr;
  if (det && p->det4 && det->n_det <= p->det4_cap) {
    det4_fill_kernel<<<(det->n_det + 255) / 256, 256, 0, st>>>(det->xyz, det->n_det, p->det4);
    count_launch();
    kp.det4 = p->det4;
  }
  kp.tof_bin = tof_bin; kp.delta = delta; kp.n = n;
  kp.frame_off = p->frame_off_dev; kp.n_frames = n_frames; kp.g = g;
  for (int a = 0; a < 3; ++a) {
    const int b0 = (a == 0) ? 1 : 0, b1 = (a == 2) ? 1 : 2;
    const double e0 = (double)g.n[b0] * g.v[b0], e1 = (double)g.n[b1] * g.v[b1];
    kp.kb[a] = (e1 > e0) ? b1 : b0;
    p->kb[a] = kp.kb[a];
  }
  for (int a = 0; a < 3; ++a) {
    const float cells = (float)(g.n[a] + 2);
    kp.xc[a] = g.o[a] + 0.5f * (float)(g.n[a] - 1) * g.v[a];
    kp.inv_cell_u[a] = (float)p->dims.offset_bins / cells;
    kp.inv_cell_w[a] = (float)p->dims.window_bins / cells;
    kp.inv_cell_z[a] = (float)p->dims.zoff_bins / cells;
  }
  kp.slope_bins = p->dims.slope_bins; kp.offset_bins = p->dims.offset_bins;
  kp.window_bins = p->dims.window_bins; kp.zoff_bins = p->dims.zoff_bins;
  kp.keys_per_frame = p->dims.keys_per_frame;
  kp.tof_width = p->opts.tof_bin_width;
  kp.keep_order = (p->opts.flags & JP_PLAN_KEEP_ORDER) ? 1 : 0;
  kp.interleaved = interleaved ? 1 : 0;
  if (interleaved && kp.keep_order) return fail(JP_ERR_ARG, "JP_PLAN_INTERLEAVED needs sorting (not KEEP_ORDER)");
  int64_t hist_len = (int64_t)n_frames * p->dims.keys_per_frame;
  int blocks = (int)((n + 255) / 256);
  if (!kp.keep_order) {
    JP_TRY_CUDA(cudaMemsetAsync(p->hist, 0, sizeof(uint32_t) * hist_len, st));
  }
  const int src = kp.det4 ? kSrcDet4 : (kp.dxyz ? kSrcDet : kSrcXyz);
  auto key_k = src == kSrcDet4 ? key_kernel<kSrcDet4> : (src == kSrcDet ? key_kernel<kSrcDet> : key_kernel<kSrcXyz>);
  key_k<<<blocks, 256, 0, st>>>(kp, p->keys, p->hist);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  if (!kp.keep_order) {
    int64_t nt = (hist_len + kScanTile - 1) / kScanTile;
    scan_tile_sums<<<(unsigned)nt, kScanBlock, 0, st>>>(p->hist, hist_len, p->block_sums);
    count_launch();
    scan_sums_kernel<<<1, kScanBlock, 0, st>>>(p->block_sums, nt);
    count_launch();
    scan_apply_kernel<<<(unsigned)nt, kScanBlock, 0, st>>>(p->hist, hist_len, p->block_sums);
    count_launch();
    JP_TRY_CUDA(cudaGetLastError());
  }
  auto scatter_k = src == kSrcDet4 ? scatter_kernel<kSrcDet4>
                                   : (src == kSrcDet ? scatter_kernel<kSrcDet> : scatter_kernel<kSrcXyz>);
  scatter_k<<<(unsigned)((n + 256 * kScatterPer - 1) / (256 * kScatterPer)), 256, 0, st>>>(
      kp, p->keys, p->hist, p->lor, p->perm);
  count_launch();
  axis_flags_kernel<<<(n_frames * 3 + 127) / 128, 128, 0, st>>>(p->hist, n_frames, p->dims.keys_per_frame,
                                                               p->dims.keys_per_axis, kp.keep_order,
                                                               p->axis_used);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

void free_plan(jp_plan p) {
  if (!p) return;
  cudaFree(p->lor);
  cudaFree(p->perm);
  cudaFree(p->keys);
  cudaFree(p->hist);
  cudaFree(p->block_sums);
  cudaFree(p->det4);
  cudaFree(p->frame_off_dev);
  cudaFreeHost(p->frame_off_host);
  cudaFree(p->quads);
  cudaFree(p->axis_used);
  cudaFree(p->work_counter);
  cudaFree(p->fold_img);
  cudaFree(p->sig_binned);
  delete p;
}

}  // namespace

}  // namespace jp

using namespace jp;

static int create_batch(jp_plan* out, const float* xs, const float* xe, const int16_t* tof_bin, const float* delta,
                        const int64_t* off, int32_t n_frames, const jp_image_geom* g, const jp_plan_opts* opts,
                        void* stream, const DetInput* det) {
  clear_error();
  if (!out) return fail(JP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!g) return fail(JP_ERR_ARG, "geometry is NULL");
  DevGeom dg;
  int rc = make_geom(g, &dg);
  if (rc) return rc;
  int64_t n = 0;
  const bool interleaved = opts && (opts->flags & JP_PLAN_INTERLEAVED);
  if (interleaved) {
    if (!off || n_frames < 1) return fail(JP_ERR_ARG, "frame_offsets / n_frames");
    n = off[n_frames];
    if (n < 0 || n >= (int64_t)INT32_MAX) return fail(JP_ERR_ARG, "n_total must be in [0, 2^31)");
  } else {
    rc = validate_offsets(off, n_frames, &n);
    if (rc) return rc;
  }
  jp_plan_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  const bool auto_block = (o.block == 0);
  if (o.block == 0) o.block = 256;
  if (o.block < 64 || o.block > 512 || (o.block % 32) != 0) return fail(JP_ERR_ARG, "opts.block must be 64..512, multiple of 32");
  if (o.slope_bins == 0) o.slope_bins = 128;
  if (o.offset_bins == 0) o.offset_bins = 256;
  if (o.window_bins == 0) o.window_bins = 16;
  if (o.zoff_bins == 0) o.zoff_bins = 8;
  if (o.slope_bins < 1 || o.offset_bins < 1 || o.window_bins < 1 || o.zoff_bins < 1)
    return fail(JP_ERR_ARG, "bin counts must be >= 1");
  if (o.lors_per_warp != 0 && o.lors_per_warp != 1 && o.lors_per_warp != 2 && o.lors_per_warp != 4 &&
      o.lors_per_warp != 8 && o.lors_per_warp != 16 && o.lors_per_warp != 32)
    return fail(JP_ERR_ARG, "opts.lors_per_warp must be 0, 1, 2, 4, 8, 16 or 32");
  if (!(o.tof_bin_width >= 0.f) || !isfinite(o.tof_bin_width)) return fail(JP_ERR_ARG, "opts.tof_bin_width must be finite and >= 0");
  if (o.tile_lors == 0) o.tile_lors = 256;
  if (o.tile_lors < 32 || o.tile_lors > 1024) return fail(JP_ERR_ARG, "opts.tile_lors must be 0 or 32..1024");
  int window_bins = (o.tof_bin_width > 0.f && tof_bin) ? o.window_bins : 1;
  int64_t kpf = 3LL * o.slope_bins * o.offset_bins * window_bins * o.zoff_bins;
  if (o.flags & JP_PLAN_KEEP_ORDER) kpf = 1;
  if (kpf * (int64_t)n_frames >= (int64_t)kScanTile * kScanTile)
    return fail(JP_ERR_ARG, "too many bins (n_frames * 3 * slope * offset * window >= 2^28)");
  jp_plan p = new (std::nothrow) jp_plan_s();
  if (!p) return fail(JP_ERR_NOMEM, "host allocation failed");
  std::memset(p, 0, sizeof(*p));
  p->capacity = n;
  p->frame_capacity = n_frames;
  p->g = *g;
  p->opts = o;
  p->auto_block = auto_block;
  p->dims.slope_bins = o.slope_bins;
  p->dims.offset_bins = o.offset_bins;
  p->dims.window_bins = window_bins;
  p->dims.keys_per_frame = (int)kpf;
  p->dims.zoff_bins = o.zoff_bins;
  p->dims.keys_per_axis = (o.flags & JP_PLAN_KEEP_ORDER) ? 1 : o.slope_bins * o.offset_bins * window_bins * o.zoff_bins;
  p->ql = quad_layout(*g);
  for (int a = 0; a < 3; ++a)
    if (p->ql.size[a] >= (int64_t)INT32_MAX) {
      delete p;
      return fail(JP_ERR_ARG, "padded image too large (>= 2^31 entries per axis)");
    }
  p->has_tof_bin = tof_bin != nullptr;
  p->has_delta = delta != nullptr;
  p->hist_len = kpf * n_frames;
  p->scan_blocks_cap = (p->hist_len + kScanTile - 1) / kScanTile;
  p->n = 0;
  size_t nn = (size_t)std::max<int64_t>(n, 1);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&p->lor, sizeof(float4) * 2 * nn);
  if (e == cudaSuccess) e = cudaMalloc(&p->perm, sizeof(int32_t) * nn);
  if (e == cudaSuccess) e = cudaMalloc(&p->keys, sizeof(uint32_t) * nn);
  if (e == cudaSuccess) e = cudaMalloc(&p->hist, sizeof(uint32_t) * (p->hist_len + 1));
  if (e == cudaSuccess) e = cudaMalloc(&p->block_sums, sizeof(uint32_t) * (p->scan_blocks_cap + 1));
  if (e == cudaSuccess && det && det->n_det > 0) {
    e = cudaMalloc(&p->det4, sizeof(float4) * (size_t)det->n_det);
    p->det4_cap = det->n_det;
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->frame_off_dev, sizeof(int64_t) * (n_frames + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&p->frame_off_host, sizeof(int64_t) * (n_frames + 1));
  p->quad_slots = interleaved ? 2 : std::max<int32_t>(n_frames, 1);
  if (e == cudaSuccess) e = cudaMalloc(&p->quads, sizeof(float4) * (size_t)p->ql.slot * (size_t)p->quad_slots);
  if (e == cudaSuccess) e = cudaMalloc(&p->axis_used, sizeof(int32_t) * 3 * (size_t)n_frames);
  if (e == cudaSuccess) e = cudaMalloc(&p->work_counter, 256);
  if (e == cudaSuccess && interleaved)
    e = cudaMalloc(&p->fold_img, sizeof(float) * (size_t)g->n[0] * g->n[1] * g->n[2]);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_plan(p);
    return fail(e == cudaErrorMemoryAllocation ? JP_ERR_NOMEM : JP_ERR_CUDA,
                std::string("plan allocation: ") + cudaGetErrorString(e));
  }
  rc = bind(p, xs, xe, tof_bin, delta, off, n_frames, (cudaStream_t)stream, det);
  if (rc) {
    free_plan(p);
    return rc;
  }
  *out = p;
  return JP_OK;
}

extern "C" int jp_plan_create_batch(jp_plan* out, const float* xs, const float* xe,
                                    const int16_t* tof_bin, const float* delta,
                                    const int64_t* off, int32_t n_frames, const jp_image_geom* g,
                                    const jp_plan_opts* opts, void* stream) {
  return create_batch(out, xs, xe, tof_bin, delta, off, n_frames, g, opts, stream, nullptr);
}

extern "C" int jp_plan_create_batch_det(jp_plan* out, const int32_t* det_start, const int32_t* det_end,
                                        const float* det_xyz, int32_t n_det, const int16_t* tof_bin,
                                        const float* delta, const int64_t* off, int32_t n_frames,
                                        const jp_image_geom* g, const jp_plan_opts* opts, void* stream) {
  const DetInput det{det_start, det_end, det_xyz, n_det};
  return create_batch(out, nullptr, nullptr, tof_bin, delta, off, n_frames, g, opts, stream, &det);
}

extern "C" int jp_plan_create(jp_plan* out, const float* xs, const float* xe,
                              const int16_t* tof_bin, const float* delta, int64_t n_lor,
                              const jp_image_geom* g, const jp_plan_opts* opts, void* stream) {
  if (n_lor < 0) {
    clear_error();
    return fail(JP_ERR_ARG, "n_lor must be >= 0");
  }
  int64_t off[2] = {0, n_lor};
  return jp_plan_create_batch(out, xs, xe, tof_bin, delta, off, 1, g, opts, stream);
}

namespace jp {
namespace {
// sig_binned[i] = sigma[caller index of binned LOR i]
__global__ void sigma_gather_kernel(const float4* __restrict__ lor, const int32_t* __restrict__ perm, int perm_in_rec,
                                    const float* __restrict__ sigma, float* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = perm_in_rec ? (int64_t)__float_as_int(lor[2 * i].w) : (int64_t)perm[i];
    out[i] = __ldg(sigma + j);
  }
}
}  // namespace
}  // namespace jp

extern "C" int jp_plan_set_event_sigma(jp_plan p, const float* sigma, void* stream) {
  using namespace jp;
  clear_error();
  if (!p) return fail(JP_ERR_ARG, "plan is NULL");
  if (!sigma) {
    p->has_sigma = false;
    return JP_OK;
  }
  if (!aligned(sigma, 4)) return fail(JP_ERR_ALIGN, "sigma must be 4-byte aligned");
  if (!p->sig_binned) {
    cudaError_t e = cudaMalloc(&p->sig_binned, sizeof(float) * (size_t)std::max<int64_t>(p->capacity, 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      p->sig_binned = nullptr;
      return fail(e == cudaErrorMemoryAllocation ? JP_ERR_NOMEM : JP_ERR_CUDA,
                  std::string("per-event sigma allocation: ") + cudaGetErrorString(e));
    }
  }
  if (p->n > 0) {
    const int64_t blocks = std::min<int64_t>((p->n + 255) / 256, (int64_t)sm_count() * 8);
    sigma_gather_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p->lor, p->perm, p->has_delta ? 0 : 1,
                                                                           sigma, p->sig_binned, p->n);
    count_launch();
    JP_TRY_CUDA(cudaGetLastError());
  }
  p->has_sigma = true;
  return JP_OK;
}

extern "C" int jp_plan_rebind(jp_plan p, const float* xs, const float* xe, const int16_t* tof_bin,
                              const float* delta, const int64_t* off, int32_t n_frames,
                              void* stream) {
  clear_error();
  if (!p) return fail(JP_ERR_ARG, "plan is NULL");
  return bind(p, xs, xe, tof_bin, delta, off, n_frames, (cudaStream_t)stream);
}

extern "C" int jp_plan_rebind_det(jp_plan p, const int32_t* det_start, const int32_t* det_end, const float* det_xyz,
                                  int32_t n_det, const int16_t* tof_bin, const float* delta, const int64_t* off,
                                  int32_t n_frames, void* stream) {
  clear_error();
  if (!p) return fail(JP_ERR_ARG, "plan is NULL");
  const DetInput det{det_start, det_end, det_xyz, n_det};
  return bind(p, nullptr, nullptr, tof_bin, delta, off, n_frames, (cudaStream_t)stream, &det);
}

extern "C" int jp_plan_destroy(jp_plan p) {
  clear_error();
  if (!p) return JP_OK;
  cudaDeviceSynchronize();
  free_plan(p);
  return JP_OK;
}

namespace jp {
namespace {
__global__ void perm_from_records(const float4* __restrict__ lor, int64_t n, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float_as_int(lor[2 * i].w);
}
}  // namespace
}  // namespace jp

extern "C" int jp_plan_info(jp_plan p, int64_t* n_lor, int32_t* n_frames, int32_t* perm_out,
                            void* stream) {
  clear_error();
  if (!p) return fail(JP_ERR_ARG, "plan is NULL");
  if (n_lor) *n_lor = p->n;
  if (n_frames) *n_frames = p->n_frames;
  if (perm_out && p->n > 0) {
    if (!aligned(perm_out, 4)) return fail(JP_ERR_ALIGN, "perm_out must be 4-byte aligned");
    if (p->has_delta) {
      JP_TRY_CUDA(cudaMemcpyAsync(perm_out, p->perm, sizeof(int32_t) * p->n, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream));
    } else {
      int64_t g = (p->n + 255) / 256;
      if (g > (int64_t)sm_count() * 8) g = (int64_t)sm_count() * 8;
      perm_from_records<<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(p->lor, p->n, perm_out);
      count_launch();
      JP_TRY_CUDA(cudaGetLastError());
    }
  }
  return JP_OK;
}
