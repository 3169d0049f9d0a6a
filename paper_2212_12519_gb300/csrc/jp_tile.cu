// Shared-memory tile kernels of the planned non-TOF and TOF-listmode
// projections (paper Sec. 2.1 and 2.2; Sec. 4 on the atomic adds of the back
// projection, their races and the suggested pre-sorting of events).
//
// A plan's sort key starts with (frame, principal axis a, in-plane slope,
// in-plane offset): the LORs of one such "line" cross the image close to one
// transaxial line.  A CTA claims lines from a counter and works on tiles of
// up to T consecutive binned LORs of a line.  For a tile it keeps a box of
// the image in shared memory:
//   planes   k in [kmin, kmax], the union of the tile's plane ranges;
//   rows     along the line axis l (the key's in-plane axis): r = i_l -
//            floor(ref(k)), ref(k) the line coordinate of the tile's first
//            live LOR on plane k, so nearly parallel LORs share a few rows;
//   columns  along the free axis (the other in-plane axis): the voxels the
//            tile's LORs reach, plus one on each side.
// Back projection: each plane sample adds its 4 bilinear terms into the box
// with shared-memory atomics, and the box is then added into the image,
// coalesced along the image rows, once per voxel that received anything:
// the L2 reductions per plane sample drop from one 16-byte reduction (0.73
// sectors) into zero-padded quad images to a fraction of a sector.
// Forward: the box is loaded from the image with coalesced loads and the
// samples read their 4 voxels from shared memory.
// A box larger than the shared-memory budget is processed in slabs of
// planes.  The box bounds come from the ends of each LOR's plane range, so
// rounding can put a sample's voxels one row outside; such a sample reads or
// adds them in global memory instead, and every sample stays exact.
//
// The sample coordinates are clamped to [-1, n] as in the quad kernels (a
// clamped sample has zero weight on every voxel inside the grid), the box
// holds zeros outside the grid (forward) or drops what lands there (back),
// and the G lanes of a group step through one LOR's planes k = k0 + lane
// (mod G) in increasing order: a forward projection equals the quad-image
// group kernel's with the same G bit for bit, whatever the tiling.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "jp_proj.cuh"

namespace jp {
namespace {

constexpr int kMaxSlabs = 16;  // a tile needing more slabs takes the global path

__device__ __forceinline__ int clamp_to_int(float x) {
  return (int)fminf(fmaxf(x, -1048576.f), 1048576.f);
}

// shared-memory layout of one CTA
struct TileSmem {
  float2* lut;
  float *lc, *ld, *fc, *fd, *d0, *dt, *ke, *w;  // per LOR of the tile
  int *k0, *k1, *j;
  float* lsum;  // forward: [T][G] lane partial sums
  float* box;
};

// per-tile box geometry (identical in every thread)
struct TileBox {
  int kmin, kmax, rlo, qa, qb, Rn, Jq, kstride, Ks, nslab;
  int rlim;        // Rn - 1 with the box, 0 without (no sample is then inside)
  float rc, rd;    // reference line coordinate at the centre plane, per plane
  float scale;     // back: fixed-point scale of the box (a power of two)
  float inv_scale;
};

// per-line constants
struct LineGeo {
  int nb, nc, sa, sb, sc, nl, nf, sl, sf;
  float kc;
};

// One slab's walk, box load and flush for a tile whose line axis is b (LU)
// or c (!LU).
template <int MODE, bool BACK, bool LUT, int G, bool LU>
__device__ __forceinline__ void tile_slabs(const ProjParams& p, const TileSmem& S, const TileBox& B,
                                           const LineGeo& L, int nt, const float* __restrict__ img_in,
                                           float* img_out) {
  const DevTof& TT = p.tof;
  const int NG = blockDim.x / G;
  const int grp = threadIdx.x / G, gl = threadIdx.x - grp * G;
  const int rounds = (nt + NG - 1) / NG;
  const int Jq = B.Jq, Rn = B.Rn;
  const float inv_Jq = 1.0f / (float)Jq, inv_Rn = 1.0f / (float)Rn;
  constexpr bool lu = LU;
  const float ubf = (float)L.nb, wbf = (float)L.nc;
  for (int s = 0; s < B.nslab; ++s) {
    const int ks0 = B.kmin + s * B.Ks, ks1 = min(B.kmax, ks0 + B.Ks - 1);
    const int cells = (ks1 - ks0 + 1) * Rn * Jq;
    if (!BACK && B.rlim > 0) {
      // ---- load the slab of the image box (row-major: coalesced along the free axis) ----
      for (int e = threadIdx.x; e < cells; e += blockDim.x) {
        const int row = (int)(((float)e + 0.5f) * inv_Jq), col = e - row * Jq;
        const int kq = (int)(((float)row + 0.5f) * inv_Rn), rr = row - kq * Rn;
        const int k = ks0 + kq;
        const int il = (int)floorf(fmaf((float)k - L.kc, B.rd, B.rc)) + B.rlo + rr;
        const int iq = B.qa - 1 + col;
        float v = 0.f;
        if ((unsigned)il < (unsigned)L.nl && (unsigned)iq < (unsigned)L.nf)
          v = __ldg(img_in + (int64_t)k * L.sa + (int64_t)il * L.sl + (int64_t)iq * L.sf);
        S.box[kq * B.kstride + rr * Jq + col] = v;
      }
      __syncthreads();
    }
    // ---- walk: the G lanes of a group step through one LOR's planes ----
    for (int m = 0; m < rounds; ++m) {
      const int e = grp + m * NG;
      if (e >= nt) break;
      const int k0 = S.k0[e], k1 = S.k1[e];
      const int kb = max(k0, ks0), ke = min(k1, ks1);
      if (kb > ke) continue;
      // the b and c coordinate maps of the LOR (stored as line / free)
      const float uc = LU ? S.lc[e] : S.fc[e], du = LU ? S.ld[e] : S.fd[e];
      const float wc = LU ? S.fc[e] : S.lc[e], dw = LU ? S.fd[e] : S.ld[e];
      const float d0 = (MODE == 2) ? S.d0[e] : 0.f;
      const float dt = (MODE == 2) ? S.dt[e] : 0.f;
      const float kev = (MODE == 2) ? S.ke[e] : 0.f;
      const float w = S.w[e];
      float sum = BACK ? 0.f : S.lsum[e * G + gl];
      for (int k = kb + ((gl - (kb - k0)) & (G - 1)); k <= ke; k += G) {
        const float kk = (float)k - L.kc;
        const float u = fminf(fmaxf(fmaf(kk, du, uc), -1.f), ubf);
        const float v = fminf(fmaxf(fmaf(kk, dw, wc), -1.f), wbf);
        const float fu = floorf(u), fv = floorf(v);
        const float al = u - fu, be = v - fv;
        const int i = (int)fu, j = (int)fv;
        const int il = lu ? i : j, iq = lu ? j : i;
        const int rr = il - (int)floorf(fmaf(kk, B.rd, B.rc)) - B.rlo;
        const int cc = iq - (B.qa - 1);
        const bool inbox = (unsigned)rr < (unsigned)B.rlim && (unsigned)cc < (unsigned)(Jq - 1);
        const int bi = (k - ks0) * B.kstride + rr * Jq + cc;
        constexpr int unit = 1;
        const int sbb = lu ? Jq : unit, scb = lu ? unit : Jq;  // box offsets of i+1 and j+1
        if (!BACK) {
          float4 q;
          if (inbox) {
            q.x = S.box[bi];
            q.y = S.box[bi + sbb];
            q.z = S.box[bi + scb];
            q.w = S.box[bi + sbb + scb];
          } else {
            const bool i0 = (unsigned)i < (unsigned)L.nb, i1 = (unsigned)(i + 1) < (unsigned)L.nb;
            const bool j0 = (unsigned)j < (unsigned)L.nc, j1 = (unsigned)(j + 1) < (unsigned)L.nc;
            const int64_t gi = (int64_t)k * L.sa + (int64_t)i * L.sb + (int64_t)j * L.sc;
            q.x = (i0 && j0) ? __ldg(img_in + gi) : 0.f;
            q.y = (i1 && j0) ? __ldg(img_in + gi + L.sb) : 0.f;
            q.z = (i0 && j1) ? __ldg(img_in + gi + L.sc) : 0.f;
            q.w = (i1 && j1) ? __ldg(img_in + gi + L.sb + L.sc) : 0.f;
          }
          const float top = fmaf(be, q.z - q.x, q.x);
          const float bot = fmaf(be, q.w - q.y, q.y);
          const float sv = fmaf(al, bot - top, top);
          if (MODE == 0) sum += sv;
          else sum = fmaf(tof_weight<LUT>(S.lut, fmaf(kk, dt, d0), TT, kev), sv, sum);
        } else {
          float coef = w;
          if (MODE == 2) coef *= tof_weight<LUT>(S.lut, fmaf(kk, dt, d0), TT, kev);
          const float ca = (1.f - al) * coef, cb = al * coef;
          if (inbox) {
            // fixed point: integer shared-memory atomics; positions outside
            // the grid land in box cells the flush drops
            int* bx = reinterpret_cast<int*>(S.box) + bi;
            const float s = B.scale;
            atomicAdd(bx, __float2int_rn(ca * (1.f - be) * s));
            atomicAdd(bx + sbb, __float2int_rn(cb * (1.f - be) * s));
            atomicAdd(bx + scb, __float2int_rn(ca * be * s));
            atomicAdd(bx + sbb + scb, __float2int_rn(cb * be * s));
          } else {
            const bool i0 = (unsigned)i < (unsigned)L.nb, i1 = (unsigned)(i + 1) < (unsigned)L.nb;
            const bool j0 = (unsigned)j < (unsigned)L.nc, j1 = (unsigned)(j + 1) < (unsigned)L.nc;
            const int64_t gi = (int64_t)k * L.sa + (int64_t)i * L.sb + (int64_t)j * L.sc;
            if (i0 && j0) atomicAdd(img_out + gi, ca * (1.f - be));
            if (i1 && j0) atomicAdd(img_out + gi + L.sb, cb * (1.f - be));
            if (i0 && j1) atomicAdd(img_out + gi + L.sc, ca * be);
            if (i1 && j1) atomicAdd(img_out + gi + L.sb + L.sc, cb * be);
          }
        }
      }
      if (!BACK) S.lsum[e * G + gl] = sum;
    }
    __syncthreads();
    if (BACK && B.rlim > 0) {
      // ---- add the slab into the image (coalesced along the free axis) and clear it ----
      for (int e = threadIdx.x; e < cells; e += blockDim.x) {
        const int row = (int)(((float)e + 0.5f) * inv_Jq), col = e - row * Jq;
        const int kq = (int)(((float)row + 0.5f) * inv_Rn), rr = row - kq * Rn;
        int* c = reinterpret_cast<int*>(S.box) + kq * B.kstride + rr * Jq + col;
        const int qv = *c;
        if (qv == 0) continue;
        *c = 0;
        const float v = (float)qv * B.inv_scale;
        const int k = ks0 + kq;
        const int il = (int)floorf(fmaf((float)k - L.kc, B.rd, B.rc)) + B.rlo + rr;
        const int iq = B.qa - 1 + col;
        if ((unsigned)il < (unsigned)L.nl && (unsigned)iq < (unsigned)L.nf)
          atomicAdd(img_out + (int64_t)k * L.sa + (int64_t)il * L.sl + (int64_t)iq * L.sf, v);
      }
      __syncthreads();
    }
  }
}

template <int MODE, bool BACK, bool LUT, int G>
__global__ void __launch_bounds__(512) tile_kernel(const ProjParams p) {
  static_assert(MODE == 0 || MODE == 2, "tile kernel: non-TOF or TOF listmode");
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const DevTof& TT = p.tof;
  const int T = p.tile_T;
  TileSmem S;
  S.lut = reinterpret_cast<float2*>(sm);
  float* ev = sm + ((MODE == 2 && LUT) ? 2 * kLut : 0);
  S.lc = ev;          // line-axis coordinate at the centre plane
  S.ld = ev + T;      //   ... change per plane
  S.fc = ev + 2 * T;  // free-axis coordinate at the centre plane
  S.fd = ev + 3 * T;
  S.d0 = ev + 4 * T;  // tau(kc) - TOF bin centre
  S.dt = ev + 5 * T;  // tau per plane
  S.ke = ev + 6 * T;  // 1 / (sqrt2 sigma) of the LOR
  S.w = ev + 7 * T;   // back: w0 * y; forward: w0 (0 when not live)
  S.k0 = reinterpret_cast<int*>(ev + 8 * T);
  S.k1 = S.k0 + T;
  S.j = S.k1 + T;     // caller index
  S.lsum = reinterpret_cast<float*>(S.j + T);
  S.box = S.lsum + (BACK ? 0 : T * G);
  __shared__ unsigned int s_line;
  __shared__ int s_ref, s_kmin, s_kmax, s_rlo, s_rhi, s_qlo, s_qhi;
  __shared__ float s_wsum, s_gmax;

  if (MODE == 2 && LUT) build_lut(S.lut, TT);
  if (BACK) {
    for (int e = threadIdx.x; e < p.box_floats; e += blockDim.x) S.box[e] = 0.f;
    // bound of a sample's TOF weight: the Gaussian bin weight (an erf
    // difference) is <= 1, a tabulated kernel its largest |node|
    if (threadIdx.x == 0) s_gmax = 1.f;
    __syncthreads();
    if (MODE == 2 && TT.user) {
      float m = 0.f;
      for (int e = threadIdx.x; e < TT.nodes; e += blockDim.x) m = fmaxf(m, fabsf(__ldg(TT.user + e)));
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(&s_gmax), __float_as_int(m));
    }
  }
  __syncthreads();

  const int NG = blockDim.x / G;
  const int grp = threadIdx.x / G, gl = threadIdx.x - grp * G;
  const int lane = threadIdx.x & 31;
  const DevGeom& g = p.g;

  for (;;) {
    if (threadIdx.x == 0) s_line = atomicAdd(p.counter, (unsigned)p.line_batch);
    __syncthreads();
    const int64_t L0 = s_line;
    __syncthreads();
    if (L0 >= p.n_lines) break;
    const int64_t L1 = min(L0 + (int64_t)p.line_batch, p.n_lines);
    for (int64_t Li = L0; Li < L1; ++Li) {
      const int64_t key0 = Li * p.keys_per_line;
      const int64_t lo = key0 > 0 ? (int64_t)__ldg(p.line_end + key0 - 1) : 0;
      const int64_t hi = (int64_t)__ldg(p.line_end + key0 + p.keys_per_line - 1);
      if (lo >= hi) continue;
      // per-line constants: frame, principal axis, line and free axes
      const int f = (int)(Li / p.lines_per_frame);
      const int a = (int)((Li - (int64_t)f * p.lines_per_frame) / p.lines_per_axis);
      const int b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
      const bool lu = sel3(a, p.kb[0], p.kb[1], p.kb[2]) == b;  // line axis is b (else c)
      LineGeo LG;
      const int na = sel3(a, g.n[0], g.n[1], g.n[2]);
      LG.nb = sel3(b, g.n[0], g.n[1], g.n[2]);
      LG.nc = sel3(c, g.n[0], g.n[1], g.n[2]);
      LG.sa = sel3(a, g.stride[0], g.stride[1], g.stride[2]);
      LG.sb = sel3(b, g.stride[0], g.stride[1], g.stride[2]);
      LG.sc = sel3(c, g.stride[0], g.stride[1], g.stride[2]);
      LG.nl = lu ? LG.nb : LG.nc;
      LG.nf = lu ? LG.nc : LG.nb;
      LG.sl = lu ? LG.sb : LG.sc;
      LG.sf = lu ? LG.sc : LG.sb;
      LG.kc = 0.5f * (float)(na - 1);
      const int slot = p.shared ? 0 : f;
      const float* __restrict__ img_in = BACK ? nullptr : p.img_in + (int64_t)slot * p.img_stride;
      float* img_out = BACK ? p.img_out + (int64_t)slot * p.img_stride : nullptr;

      for (int64_t t0 = lo; t0 < hi; t0 += T) {
        const int nt = (int)min((int64_t)T, hi - t0);
        if (threadIdx.x == 0) {
          s_ref = INT_MAX; s_kmin = INT_MAX; s_kmax = INT_MIN;
          s_rlo = INT_MAX; s_rhi = INT_MIN; s_qlo = INT_MAX; s_qhi = INT_MIN;
          s_wsum = 0.f;
        }
        __syncthreads();
        // ---- (1) per-LOR setup (steps a2, a4 window, a6 caller index) ----
        {
          int ref = INT_MAX, kmn = INT_MAX, kmx = INT_MIN;
          float wabs = 0.f;
          for (int t = threadIdx.x; t < nt; t += blockDim.x) {
            const int64_t i = t0 + t;
            const float4 A = __ldcs(p.lor + 2 * i);
            const float4 Bv = __ldcs(p.lor + 2 * i + 1);
            const float xs[3] = {A.x, A.y, A.z};
            const float xe[3] = {Bv.x, Bv.y, Bv.z};
            const int32_t j = p.perm_in_rec ? __float_as_int(A.w) : __ldcs(p.perm + i);
            const float delta = p.perm_in_rec ? 0.f : A.w;
            Ray r;
            bool live = ray_setup(xs, xe, p.g, r);
            float d0 = 0.f, ke = TT.k;
            if (MODE == 2 && live) {
              float Re;
              event_tof(p, i, ke, Re);
              const float cen = (float)__float_as_int(Bv.w) * TT.width + delta;
              d0 = r.tc - cen;
              const float u1 = (-Re - d0) / r.dt, u2 = (Re - d0) / r.dt;
              const float klo = fmaxf(ceilf(r.kc + fminf(u1, u2)), (float)r.k0);
              const float khi = fminf(floorf(r.kc + fmaxf(u1, u2)), (float)r.k1);
              r.k0 = (int)klo;
              r.k1 = (int)khi;
              live = klo <= khi;
            }
            float w = r.w0;
            if (BACK && live) {
              w = r.w0 * __ldcs(p.proj_in + j);
              live = w != 0.f;
            }
            S.lc[t] = lu ? r.uc : r.wc;
            S.ld[t] = lu ? r.du : r.dw;
            S.fc[t] = lu ? r.wc : r.uc;
            S.fd[t] = lu ? r.dw : r.du;
            S.d0[t] = d0;
            S.dt[t] = r.dt;
            S.ke[t] = ke;
            S.w[t] = live ? w : 0.f;
            S.k0[t] = live ? r.k0 : 1;
            S.k1[t] = live ? r.k1 : 0;
            S.j[t] = j;
            if (!BACK)
              for (int q = 0; q < G; ++q) S.lsum[t * G + q] = 0.f;
            if (live) {
              ref = min(ref, t);
              kmn = min(kmn, r.k0);
              kmx = max(kmx, r.k1);
              wabs += fabsf(w);
            }
          }
          ref = __reduce_min_sync(0xffffffffu, ref);
          kmn = __reduce_min_sync(0xffffffffu, kmn);
          kmx = __reduce_max_sync(0xffffffffu, kmx);
          if (BACK)
            for (int o = 16; o > 0; o >>= 1) wabs += __shfl_xor_sync(0xffffffffu, wabs, o);
          if (lane == 0) {
            atomicMin(&s_ref, ref);
            atomicMin(&s_kmin, kmn);
            atomicMax(&s_kmax, kmx);
            if (BACK) atomicAdd(&s_wsum, wabs);
          }
        }
        __syncthreads();
        // ---- (2) box bounds relative to the reference LOR ----
        TileBox B;
        const int ref = s_ref;
        B.rc = ref != INT_MAX ? S.lc[ref] : 0.f;
        B.rd = ref != INT_MAX ? S.ld[ref] : 0.f;
        {
          int rl = INT_MAX, rh = INT_MIN, ql = INT_MAX, qh = INT_MIN;
          for (int t = threadIdx.x; t < nt; t += blockDim.x) {
            const int k0 = S.k0[t], k1 = S.k1[t];
            if (k0 > k1) continue;
            const float kk0 = (float)k0 - LG.kc, kk1 = (float)k1 - LG.kc;
            const float lc = S.lc[t], ld = S.ld[t], fc = S.fc[t], fd = S.fd[t];
            const float dA = fmaf(kk0, ld, lc) - fmaf(kk0, B.rd, B.rc);
            const float dB = fmaf(kk1, ld, lc) - fmaf(kk1, B.rd, B.rc);
            const float fA = fmaf(kk0, fd, fc), fB = fmaf(kk1, fd, fc);
            rl = min(rl, clamp_to_int(floorf(fminf(dA, dB))));
            rh = max(rh, clamp_to_int(ceilf(fmaxf(dA, dB))) + 1);
            ql = min(ql, clamp_to_int(floorf(fminf(fA, fB))));
            qh = max(qh, clamp_to_int(floorf(fmaxf(fA, fB))) + 1);
          }
          rl = __reduce_min_sync(0xffffffffu, rl);
          rh = __reduce_max_sync(0xffffffffu, rh);
          ql = __reduce_min_sync(0xffffffffu, ql);
          qh = __reduce_max_sync(0xffffffffu, qh);
          if (lane == 0 && rl != INT_MAX) {
            atomicMin(&s_rlo, rl);
            atomicMax(&s_rhi, rh);
            atomicMin(&s_qlo, ql);
            atomicMax(&s_qhi, qh);
          }
        }
        __syncthreads();
        // ---- (3) box geometry ----
        B.kmin = s_kmin;
        B.kmax = s_kmax;
        const bool any = B.kmin <= B.kmax;  // the tile has a live LOR (then every bound is set)
        B.rlo = any ? s_rlo : 0;
        B.qa = any ? max(s_qlo, 0) : 0;
        B.qb = any ? min(s_qhi, LG.nf - 1) : -1;
        B.Rn = any ? s_rhi - s_rlo + 1 : 1;  // rows, the +1 neighbour included
        B.Jq = B.qb - B.qa + 3;              // columns qa - 1 .. qb + 1
        const int64_t cells = (int64_t)B.Rn * B.Jq;
        bool use_box = any && B.qa <= B.qb && B.Rn > 1 && cells < (int64_t)p.box_floats;
        // odd plane stride: lanes on consecutive planes hit distinct banks
        B.kstride = use_box ? (int)cells + (((int)cells & 1) ^ 1) : 1;
        const int K = any ? B.kmax - B.kmin + 1 : 0;
        use_box = use_box && B.kstride <= p.box_floats;
        B.Ks = use_box ? p.box_floats / B.kstride : max(K, 1);
        if (use_box && (K + B.Ks - 1) / B.Ks > kMaxSlabs) {
          use_box = false;
          B.Ks = K;
        }
        if (!use_box) {
          B.Rn = 1;
          B.Jq = 1;
        }
        // Back projection: the box accumulates integers c * scale.  Every
        // cell receives at most one sample per LOR (its plane), with weight
        // <= 1 x |coef| <= |w0 y| gmax, so |sum| <= bound * scale with bound =
        // sum over the tile of |w0 y| gmax; scale = 2^e <= 2^30 / bound keeps
        // every cell, rounding included, inside int32.  Each contribution
        // rounds by at most 0.5 / scale <= bound / 2^31.  A bound that is
        // not finite sends the tile to the global path.
        B.scale = 1.f;
        if (BACK && use_box) {
          const float bound = s_wsum * s_gmax;
          if (bound > 0.f && isfinite(bound)) {
            int ex;
            frexpf(bound, &ex);                // bound < 2^ex
            B.scale = ldexpf(1.f, 30 - ex);
            use_box = isfinite(B.scale) && B.scale > 0.f;
          } else {
            use_box = false;
          }
          if (!use_box) {
            B.Ks = K;
            B.Rn = 1;
            B.Jq = 1;
          }
        }
        B.inv_scale = 1.f / B.scale;
        B.rlim = use_box ? B.Rn - 1 : 0;
        B.nslab = any ? (K + B.Ks - 1) / B.Ks : 0;
        if (lu)
          tile_slabs<MODE, BACK, LUT, G, true>(p, S, B, LG, nt, img_in, img_out);
        else
          tile_slabs<MODE, BACK, LUT, G, false>(p, S, B, LG, nt, img_in, img_out);
        if (!BACK) {
          // ---- (4) outputs in caller order: the group sums of the lane partials ----
          const int rounds = (nt + NG - 1) / NG;
          for (int m = 0; m < rounds; ++m) {
            const int e = grp + m * NG;
            float v = e < nt ? S.lsum[e * G + gl] : 0.f;
            v = group_sum<G>(v);
            if (gl == 0 && e < nt) __stcs(p.proj_out + S.j[e], S.w[e] * v);
          }
        }
        __syncthreads();  // the next tile resets the bounds and overwrites the parameters
      }
    }
  }
}

size_t tile_smem(int mode, bool back, bool lut, int G, int T, int box_floats) {
  size_t b = (mode == 2 && lut) ? (size_t)kLut * sizeof(float2) : 0;
  b += (size_t)T * 11 * sizeof(float);
  if (!back) b += (size_t)T * G * sizeof(float);
  return b + (size_t)box_floats * sizeof(float);
}

template <int MODE, bool BACK, bool LUT, int G>
int launch_tile_t(ProjParams p, int block, cudaStream_t st) {
  auto kern = tile_kernel<MODE, BACK, LUT, G>;
  int dev = 0;
  JP_TRY_CUDA(cudaGetDevice(&dev));
  int sm_bytes = 0, optin = 0, reserved = 0;
  JP_TRY_CUDA(cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  JP_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  JP_TRY_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  cudaFuncAttributes fa;
  JP_TRY_CUDA(cudaFuncGetAttributes(&fa, kern));
  // resident CTAs per SM the box is sized for (default two: one loads or
  // flushes its box while the other walks)
  const int target = p.max_per_sm > 0 ? p.max_per_sm : 2;
  int per_cta = sm_bytes / target - reserved - (int)fa.sharedSizeBytes;
  if (per_cta > optin - (int)fa.sharedSizeBytes) per_cta = optin - (int)fa.sharedSizeBytes;
  const int fixed = (int)tile_smem(MODE, BACK, LUT, G, p.tile_T, 0);
  p.box_floats = (per_cta - fixed) / (int)sizeof(float);
  if (p.box_floats < 64) return fail(JP_ERR_ARG, "tile does not fit in shared memory (reduce tile_lors)");
  const size_t smem = tile_smem(MODE, BACK, LUT, G, p.tile_T, p.box_floats);
  JP_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  JP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem));
  if (per_sm > target) per_sm = target;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)sm_count() * per_sm;
  const int64_t need = (p.n_lines + p.line_batch - 1) / p.line_batch;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  JP_TRY_CUDA(cudaMemsetAsync(p.counter, 0, sizeof(unsigned int), st));
  kern<<<(unsigned)grid, block, smem, st>>>(p);
  count_launch();
  JP_TRY_CUDA(cudaGetLastError());
  return JP_OK;
}

template <int MODE, bool BACK, bool LUT>
int launch_tile_g(const ProjParams& p, int lanes, int block, cudaStream_t st) {
  switch (lanes) {
    case 4: return launch_tile_t<MODE, BACK, LUT, 4>(p, block, st);
    case 16: return launch_tile_t<MODE, BACK, LUT, 16>(p, block, st);
    case 32: return launch_tile_t<MODE, BACK, LUT, 32>(p, block, st);
    default: return launch_tile_t<MODE, BACK, LUT, 8>(p, block, st);
  }
}

}  // namespace

int launch_tile(const ProjParams& p, int mode, bool back, bool lut, int lanes, int block, cudaStream_t st) {
  if (p.n == 0) return JP_OK;
  if (p.tile_T < 32 || p.tile_T > 1024) return fail(JP_ERR_ARG, "tile LOR count must be in 32..1024");
  if (block < 64 || block > 512 || block % 32) return fail(JP_ERR_ARG, "tile block must be 64..512, multiple of 32");
  switch (mode * 4 + (back ? 2 : 0) + (lut ? 1 : 0)) {
    case 0: case 1: return launch_tile_g<0, false, false>(p, lanes, block, st);
    case 2: case 3: return launch_tile_g<0, true, false>(p, lanes, block, st);
    case 8: return launch_tile_g<2, false, false>(p, lanes, block, st);
    case 9: return launch_tile_g<2, false, true>(p, lanes, block, st);
    case 10: return launch_tile_g<2, true, false>(p, lanes, block, st);
    case 11: return launch_tile_g<2, true, true>(p, lanes, block, st);
  }
  return fail(JP_ERR_ARG, "tile kernels cover non-TOF and TOF listmode only");
}

}  // namespace jp
