/*
 * joseph.h -- C ABI of libjoseph, a GB300 (sm_103a) Joseph projector.
 *
 * The library computes Joseph's ray-driven forward projection and its exact
 * adjoint (back projection) of a 3D voxel image along lines of response
 * (LORs) given by their start and end points (paper Sec. 2.1, Fig. 1; the
 * generic "list of start and end points" interface of Sec. 2.2), in three
 * forms (Sec. 2.2): non-TOF, TOF sinogram (all TOF bins of a LOR in one
 * traversal) and TOF listmode (the single TOF bin of each event).  The TOF
 * kernel is a Gaussian of width sigma integrated over a TOF bin, i.e. a
 * difference of two error functions, truncated at n_sigmas (Sec. 2.1, 2.6).
 *
 * Conventions (the same for every call):
 *   image     float32, C order [n0][n1][n2] (axis 2 fastest); `origin` is the
 *             world coordinate (mm) of the CENTRE of voxel (0,0,0); voxel
 *             sizes may differ per axis.
 *   LOR       start xs and end xe, float32 [n][3] (mm).  The principal axis
 *             a = argmax_i |xe_i - xs_i| (lowest index on exact ties) is
 *             decided exactly; every plane k of axis a whose centre
 *             o_a + k v_a lies in [min(xs_a,xe_a), max(xs_a,xe_a)] contributes
 *             a bilinear interpolation of the 4 nearest voxels (zero outside
 *             the grid); the sum is scaled by v_a / cos_a.  xs == xe projects
 *             to 0; a LOR missing the image projects to 0.
 *   TOF       tau = signed distance of a plane sample from the LOR midpoint,
 *             positive toward xe.  Sinogram bin t of N has centre
 *             (t - (N-1)/2) * bin_width + delta; a listmode event with signed
 *             bin t_s has centre t_s * bin_width + delta (delta = optional
 *             per-LOR TOF centre offset, default 0).  Weight
 *             g = 1/2 [erf((tau-c+w/2)/(sqrt2 s)) - erf((tau-c-w/2)/(sqrt2 s))]
 *             if |tau - c| <= n_sigmas*s + w/2, else 0.  TOF sinograms are
 *             float32 [n_lor][N] (TOF fastest).
 *   pointers  every array argument is a DEVICE pointer owned by the caller
 *             (the library never frees it) unless stated otherwise; `stream`
 *             is a cudaStream_t (NULL = legacy default stream).  All
 *             projection calls are asynchronous on `stream` and allocate
 *             nothing.  Forward calls overwrite their output; back
 *             projections ACCUMULATE into the image (the caller zeroes it).
 *   errors    every call returns JP_OK (0) or a negative JP_ERR_* code;
 *             jp_last_error() gives a message for the calling thread.
 *             Argument checks run on the host before anything is launched.
 *   threads   distinct plans may be used from distinct host threads; one plan
 *             must not be rebound while a call using it is in flight, and two
 *             back projections into the same image must not overlap on
 *             different streams.
 */
#ifndef JOSEPH_H
#define JOSEPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define JP_OK 0
#define JP_ERR_ARG (-1)     /* null pointer, size <= 0, non-finite or non-positive parameter */
#define JP_ERR_ALIGN (-2)   /* pointer not aligned to its element type */
#define JP_ERR_CUDA (-3)    /* CUDA runtime error (message in jp_last_error) */
#define JP_ERR_TIMEOUT (-4) /* a bounded device-side wait gave up */
#define JP_ERR_NOMEM (-5)   /* device allocation failed (plan creation only) */
#define JP_ERR_STATE (-6)   /* plan lacks what the call needs (e.g. TOF bins) */

#define JP_MAX_TOF_BINS 128

typedef struct jp_plan_s* jp_plan;

/* image grid: shape, centre of voxel (0,0,0) in mm, voxel size in mm */
typedef struct {
  int32_t n[3];
  float origin[3];
  float voxsize[3];
} jp_image_geom;

/* TOF kernel: bin width (mm), Gaussian sigma (mm, = FWHM / 2.35482),
 * truncation in sigmas, number of sinogram TOF bins (unused in listmode).
 *
 * Optional tabulated kernel (paper Sec. 4: a 1D lookup table allows
 * non-Gaussian TOF kernels): when `kernel` is non-NULL it is a device array
 * of `kernel_nodes` float32 values (2 .. JP_TOF_TABLE) of the bin response
 * at the signed distances d_e = -h + e * 2h / (kernel_nodes - 1) from the bin
 * centre (h = kernel_half_width > 0).  A sample at distance d then weighs
 * the linear interpolation of the table, and 0 where |d| > h; sigma and
 * n_sigmas are ignored.  The table must stay valid while calls that use it
 * run. */
typedef struct {
  float bin_width;
  float sigma;
  float n_sigmas;
  int32_t n_bins;
  const float* kernel;
  int32_t kernel_nodes;
  float kernel_half_width;
} jp_tof;

/* Plan options (zero-initialise for defaults).  A plan sorts its LORs into
 * bins by principal axis, in-plane direction and position so that the 32
 * LORs of a warp walk nearly the same voxels (paper Sec. 4 suggests event
 * pre-sorting; Sec. 2.6 and 3 show the memory-order sensitivity it removes). */
typedef struct {
  int32_t block;          /* threads per CTA for projections (64..512, multiple of 32; 0 = 256,
                             except 512 for the TOF-sinogram forward and 128 for the
                             non-TOF and TOF-listmode forwards) */
  int32_t slope_bins;     /* bins over the in-plane slope d_b/d_a in [-1,1] (0 = 128) */
  int32_t offset_bins;    /* bins over the in-plane offset at the central plane (0 = 256) */
  int32_t window_bins;    /* bins over the TOF-window centre along the principal
                             axis, listmode plans only (0 = 16); n_frames * 3 * slope *
                             offset * window * zoff must stay below 2^28 */
  float tof_bin_width;    /* mm; > 0 with tof_bin given: bin listmode events by
                             their TOF window centre; 0 = ignore */
  int32_t lors_per_warp;  /* LORs a warp walks at once: 32 = one LOR per thread;
                             1, 2, 4, 8 or 16 = 32, 16, 8, 4 or 2 lanes step through
                             consecutive planes of one LOR (coalesced); 0 = per-mode
                             default */
  int32_t flags;          /* JP_PLAN_KEEP_ORDER: no sorting (identity order);
                             JP_PLAN_TOF_EXACT: evaluate every TOF weight with erff
                             instead of the interpolated table (see below) */
  int32_t zoff_bins;      /* bins over the offset along axis c (the fastest image
                             axis for principal axes 0 and 1) at the central plane,
                             the last (fastest) key field (0 = 8; 1 = not binned) */
  int32_t max_ctas_per_sm;/* cap on the resident CTAs per SM of the persistent
                             projection kernels, leaving room for work on other
                             streams (0 = as many as fit) */
  int32_t tile_lors;      /* LORs per tile of the shared-memory tile kernels
                             (JP_PLAN_TILES; 0 = 256; 32..1024) */
} jp_plan_opts;

#define JP_PLAN_KEEP_ORDER 1
#define JP_PLAN_TOF_EXACT 2
#define JP_PLAN_INTERLEAVED 4  /* frame of caller LOR j is j mod n_frames (listmode
                                  OSEM subsets); frame_offsets then only give
                                  offsets[n_frames] = n_total and all frames share
                                  one image */
#define JP_PLAN_TILES 8        /* project through the shared-memory tiles (below)
                                  instead of the quad images */

/* Projection paths of a sorted plan (neither KEEP_ORDER nor INTERLEAVED).
 * By default every call goes through zero-padded quad images, one per
 * principal axis, holding the 4 bilinear neighbours of every sample
 * position: a sample is one 16-byte load (forward) or one 16-byte vector
 * reduction into L2 (back projection).
 * JP_PLAN_TILES sends non-TOF and TOF-listmode calls with lors_per_warp 0, 1,
 * 2, 4 or 8 through shared-memory tiles instead: a CTA takes up to
 * tile_lors consecutive sorted LORs that share (frame, principal axis, slope
 * bin, offset bin), i.e. cross the image close to one line, and holds the
 * image voxels they reach in shared memory.  The back projection adds its
 * samples there (fixed-point integer atomics, scaled per tile so that no
 * cell can overflow; absolute error per sample <= sum over the tile of
 * |w0 y g_max| / 2^31) and then adds the box into the image (the race-prone
 * scatter of Sec. 2.2 privatised per CTA); the forward projection reads its
 * samples from the box and equals the quad path's with the same lanes per
 * LOR bit for bit.  32/lors_per_warp lanes (at least 4) walk one LOR.  On
 * the clinical workloads this path cuts the L2 reductions per sample from
 * ~0.73 sectors to ~0.23 but executes more instructions than it saves, and
 * is slower; TOF-sinogram calls always use the quad images. */

/* TOF weights in planned calls come by default from a table of the exact
 * erf difference at JP_TOF_TABLE nodes over [-R, R] (R = n_sigmas*sigma +
 * w/2) with linear interpolation (max relative deviation ~1e-6 of the peak
 * weight for the clinical parameters); JP_PLAN_TOF_EXACT selects erff. */
#define JP_TOF_TABLE 2048

/*
 * jp_plan_create_batch -- sort and pack the LORs of n_frames frames.
 *   xstart, xend       device float32 [n_total][3] (mm), caller order
 *   tof_bin            device int16 [n_total] signed listmode TOF bins, or NULL
 *   tof_center_offset  device float32 [n_total] TOF centre offsets delta (mm), or NULL
 *   frame_offsets      HOST int64 [n_frames+1], frame f owns LORs
 *                      [frame_offsets[f], frame_offsets[f+1]); offsets[0] = 0,
 *                      non-decreasing; n_total = offsets[n_frames] < 2^31
 *   g, opts            image grid (all frames share it); opts may be NULL
 * The plan allocates device memory for exactly n_total LORs and n_frames
 * frames (its capacity) and copies what it needs: the input arrays may be
 * freed once the stream has passed this call.  It also holds the projection
 * workspace (per frame, a zero-padded 4-neighbour copy of the image for each
 * principal axis: 16 * sum_a n_a (n_b+2)(n_c+2) bytes), so the projection
 * calls allocate nothing.  Frame f of a batched call
 * reads/writes image f at `image + f * img_stride`.
 * Errors: JP_ERR_ARG, JP_ERR_ALIGN, JP_ERR_NOMEM, JP_ERR_CUDA.
 */
int jp_plan_create_batch(jp_plan* out, const float* xstart, const float* xend,
                         const int16_t* tof_bin, const float* tof_center_offset,
                         const int64_t* frame_offsets, int32_t n_frames,
                         const jp_image_geom* g, const jp_plan_opts* opts, void* stream);

/* single-frame form: frame_offsets = {0, n_lor} */
int jp_plan_create(jp_plan* out, const float* xstart, const float* xend,
                   const int16_t* tof_bin, const float* tof_center_offset, int64_t n_lor,
                   const jp_image_geom* g, const jp_plan_opts* opts, void* stream);

/*
 * jp_plan_rebind -- re-sort new LORs into an existing plan without allocating
 * (same arguments as jp_plan_create_batch; n_total and n_frames must not
 * exceed the plan's capacity).  Asynchronous on `stream`.
 */
int jp_plan_rebind(jp_plan p, const float* xstart, const float* xend, const int16_t* tof_bin,
                   const float* tof_center_offset, const int64_t* frame_offsets,
                   int32_t n_frames, void* stream);

/*
 * Detector-index input (listmode data as recorded: a pair of detector
 * indices per event).  det_start / det_end are device int32 [n_total]
 * indices into det_xyz, a device float32 [n_det][3] table of detector
 * coordinates (mm); LOR j runs from det_xyz[det_start[j]] to
 * det_xyz[det_end[j]].  The endpoints are read through the table while the
 * LORs are binned, so the plan is the one jp_plan_create_batch /
 * jp_plan_rebind would build from the gathered coordinates, bit for bit.
 * An index outside [0, n_det) gives the empty LOR (xs = xe = 0: no samples).
 * The plan keeps a copy of the table padded to 16 bytes per detector (16 *
 * n_det bytes for the creating call's n_det), refilled on every bind so that
 * each endpoint costs one 16-byte read; a rebind with more detectors than
 * that reads det_xyz itself (the same plan, a slower bind).
 * Other arguments and errors as jp_plan_create_batch / jp_plan_rebind; also
 * JP_ERR_ARG for n_det < 1 or NULL detector arrays with n_total > 0.
 */
int jp_plan_create_batch_det(jp_plan* out, const int32_t* det_start, const int32_t* det_end,
                             const float* det_xyz, int32_t n_det, const int16_t* tof_bin,
                             const float* tof_center_offset, const int64_t* frame_offsets,
                             int32_t n_frames, const jp_image_geom* g, const jp_plan_opts* opts,
                             void* stream);
int jp_plan_rebind_det(jp_plan p, const int32_t* det_start, const int32_t* det_end, const float* det_xyz,
                       int32_t n_det, const int16_t* tof_bin, const float* tof_center_offset,
                       const int64_t* frame_offsets, int32_t n_frames, void* stream);

/*
 * jp_plan_set_event_sigma -- per-event TOF resolution for a TOF-listmode
 * plan: sigma is a device float32 array of the bound LORs' Gaussian sigmas
 * (mm) in caller order (n_total entries); it is gathered into the plan's
 * binned order (storage allocated on the first call, `capacity` floats).
 * Listmode projections and OSEM updates of the plan then use, per event,
 * k = 1/(sqrt2 sigma_e) and the window n_sigmas sigma_e + bin_width / 2
 * (values <= 0 keep the jp_tof sigma), on the exact erf path (the TOF table
 * holds a single sigma); a tabulated kernel ignores sigma.  Rebinding the
 * plan clears it; sigma = NULL clears it.  TOF-sinogram projections of a
 * plan with per-event sigma fail with JP_ERR_STATE.
 * Errors: JP_ERR_ARG, JP_ERR_ALIGN, JP_ERR_NOMEM, JP_ERR_CUDA.
 */
int jp_plan_set_event_sigma(jp_plan p, const float* sigma, void* stream);

/* releases the plan's device memory (synchronises the device first) */
int jp_plan_destroy(jp_plan p);

/* number of LORs / frames currently bound (host pointers, may be NULL);
 * perm_out (device int32 [n_lor] or NULL) receives a copy of the plan's
 * permutation, binned position -> caller index, asynchronously on stream */
int jp_plan_info(jp_plan p, int64_t* n_lor, int32_t* n_frames, int32_t* perm_out, void* stream);

/*
 * Planned projections (paper Sec. 2.1-2.2): forward proj = A img, back
 * img_accum += A^T proj, non-TOF, TOF sinogram (all N bins of a LOR in one
 * traversal) or TOF listmode (the event's bin only, over its TOF window).
 *   img / img_accum  device float32 images, frame f at offset f*img_stride
 *                    elements (img_stride = 0: every frame uses the same
 *                    image); the back projection accumulates (the caller
 *                    zeroes img_accum)
 *   proj             device float32 in caller order, [n_total] or
 *                    [n_total][N] (TOF sinogram, bin fastest); the forward
 *                    overwrites it
 *   t                TOF parameters (host struct; a tabulated kernel's table
 *                    is a device pointer)
 * TOF listmode calls need a plan created with tof_bin; delta comes from the
 * plan (0 if it was created without tof_center_offset).  All pointers are
 * the caller's; the calls allocate nothing and run asynchronously on
 * `stream`.  One plan must not run two calls at once (its workspace is
 * shared).
 * Errors: JP_ERR_ARG (NULL plan or arrays, img_stride < 0 or smaller than
 * one image with per-frame images, invalid TOF parameters), JP_ERR_ALIGN
 * (arrays not 4-byte aligned), JP_ERR_STATE (TOF listmode without tof_bin,
 * per-event sigma with a TOF sinogram), JP_ERR_CUDA.
 */
int jp_fwd(jp_plan p, const float* img, int64_t img_stride, float* proj, void* stream);
int jp_back(jp_plan p, const float* proj, float* img_accum, int64_t img_stride, void* stream);
int jp_fwd_tof_sino(jp_plan p, const float* img, int64_t img_stride, const jp_tof* t,
                    float* proj, void* stream);
int jp_back_tof_sino(jp_plan p, const float* proj, const jp_tof* t, float* img_accum,
                     int64_t img_stride, void* stream);
int jp_fwd_tof_lm(jp_plan p, const float* img, int64_t img_stride, const jp_tof* t,
                  float* proj, void* stream);
int jp_back_tof_lm(jp_plan p, const float* proj, const jp_tof* t, float* img_accum,
                   int64_t img_stride, void* stream);

/*
 * Planless projections: one thread per LOR in caller order, reading the
 * endpoint arrays directly (the paper's own parallelisation, Sec. 2.2).
 *   tof_mode  0 non-TOF, 1 TOF sinogram, 2 TOF listmode
 *   t         TOF parameters (NULL for tof_mode 0)
 *   tof_bin   int16 [n] (tof_mode 2), else ignored; tof_center_offset may be NULL
 * Same output conventions as the planned calls.  Allocates nothing.
 */
int jp_fwd_lors(const float* xstart, const float* xend, const int16_t* tof_bin,
                const float* tof_center_offset, int64_t n_lor, const jp_image_geom* g,
                int32_t tof_mode, const jp_tof* t, const float* img, float* proj, void* stream);
int jp_back_lors(const float* xstart, const float* xend, const int16_t* tof_bin,
                 const float* tof_center_offset, int64_t n_lor, const jp_image_geom* g,
                 int32_t tof_mode, const jp_tof* t, const float* proj, float* img_accum,
                 void* stream);

/*
 * Listmode OSEM element-wise steps (paper Sec. 2.6 and 3, listmode OSEM:
 * x <- x / s_sub * A_S^T (1 / (A_S x + b))).
 *   jp_osem_ratio   q[e] = 1 / (p[e] + b[frame(e)])   (q may alias p)
 *                   b: device float32 [n_frames]; frame of e from the plan's
 *                   frame offsets (plan may be NULL: one frame, b[0])
 *   jp_osem_update  x[f][j] = s[f][j] > 0 ? x[f][j] * bp[f][j] / (s[f][j]*scale) : 0
 *                   for n_frames images of nvox voxels, strides img_stride
 *                   (x, bp, s); s_stride = 0 shares one sensitivity image.
 * Errors: JP_ERR_ARG, JP_ERR_ALIGN, JP_ERR_CUDA.
 */
int jp_osem_ratio(jp_plan p, const float* proj, const float* b, float* q, int64_t n,
                  void* stream);
int jp_osem_update(float* x, const float* bp, const float* sens, float scale, int64_t nvox,
                   int32_t n_frames, int64_t img_stride, int64_t s_stride, void* stream);

/*
 * jp_osem_ratio_sino -- the data term of a sinogram OSEM subset update
 * (paper Sec. 2.6: OSEM subset update of a span-1 subset sinogram; Sec. 4:
 * emission and contamination sinograms), elementwise over n sinogram
 * entries (LORs x TOF bins, any order shared by the arrays):
 *     q[i] = p[i] + c[i] > 0 ? y[i] / (p[i] + c[i]) : 0
 *   p  forward projection A_S x (device float32), may alias q
 *   y  emission counts (device float32)
 *   c  additive contamination (device float32), NULL for none
 * Errors: JP_ERR_ARG (n < 0, NULL p / y / q with n > 0), JP_ERR_ALIGN,
 * JP_ERR_CUDA.
 */
int jp_osem_ratio_sino(const float* proj, const float* y, const float* c, float* q, int64_t n, void* stream);

/*
 * jp_osem_subset_tof_lm -- the projection work of one listmode-OSEM subset
 * update (paper Sec. 2.6 and 3, x <- x / s_sub * A_S^T (1 / (A_S x + b))),
 * fused per event: forward projection of x, ratio 1/(p + b) and back
 * projection of the ratio, for the events of frames [f0, f1) of a
 * JP_PLAN_INTERLEAVED plan; then, per voxel,
 *     x[j] <- sens[j] > 0 ? x[j] * bp[j] / (sens[j] * sens_scale) : 0
 * where bp = A_S^T (1/(A_S x + b)) is held in the plan's workspace.
 *   x          device float32 image (updated in place)
 *   sens       device float32 sensitivity image A^T 1
 *   sens_scale 1 / n_subsets in the paper's update
 *   b          additive background (> = 0) of every event
 * Errors: JP_ERR_ARG, JP_ERR_STATE (plan not interleaved or without TOF bins),
 * JP_ERR_CUDA.
 */
int jp_osem_subset_tof_lm(jp_plan p, int32_t f0, int32_t f1, float* x, const float* sens,
                          float sens_scale, float b, const jp_tof* t, void* stream);

/*
 * jp_osem_subset_tof_lm_dev -- the same subset update, with the background b
 * read from device memory (float) and the subset's event range read from
 * the plan's device-side frame offsets when the kernels run.  A launch
 * sequence captured into a CUDA graph therefore stays valid after the plan
 * is rebound to another frame's events (up to its capacity) and b is
 * rewritten: one graph per plan serves every frame.
 */
int jp_osem_subset_tof_lm_dev(jp_plan p, int32_t f0, int32_t f1, float* x, const float* sens,
                              float sens_scale, const float* b_dev, const jp_tof* t, void* stream);

/*
 * Image-based resolution model H (paper Sec. 2.6: every listmode OSEM
 * reconstruction applies a shift-invariant isotropic 3D Gaussian of 4.5 mm
 * FWHM in image space; Sec. 4: two such convolutions per subset).  The
 * paper fixes no discretisation; this library uses: per axis a,
 * sigma_a = fwhm_mm[a] / sqrt(8 ln 2); taps = the Gaussian sampled at t*d_a
 * (d_a the voxel size) for |t| <= R_a = ceil(truncate * sigma_a / d_a),
 * normalised to sum 1 (fwhm 0: the single tap 1); the 3D kernel is the
 * product of the axis kernels; the image is zero outside its grid, so H is
 * symmetric (H^T = H).
 */
typedef struct jp_resolution {
  float fwhm_mm[3]; /* per-axis FWHM in mm, >= 0 (4.5 on every axis in the paper) */
  float truncate;   /* support half-width in sigmas, > 0 (4 is the usual value) */
} jp_resolution;

#define JP_MAX_RES_RADIUS 32 /* largest R_a in voxels */

/*
 * jp_gauss3d -- out = H img for n_images images of geometry g, each
 * nvox = n0*n1*n2 float32 (index (i0*n1 + i1)*n2 + i2), images back to back.
 *   work   device float32 scratch of n_images * nvox, caller-owned
 *   img, out and work are device pointers, 4-byte aligned and pairwise
 *   disjoint; n_images = 0 is a no-op.  Three separable passes (axis 2, 1,
 *   0), each one kernel, FP32 accumulation in ascending tap order.
 * Errors: JP_ERR_ARG (NULL or overlapping arrays, n_images < 0, fwhm < 0 or
 * not finite, truncate <= 0, a radius above JP_MAX_RES_RADIUS), JP_ERR_ALIGN,
 * JP_ERR_CUDA.
 */
int jp_gauss3d(const float* img, float* out, float* work, int32_t n_images, const jp_image_geom* g,
               const jp_resolution* r, void* stream);

/*
 * jp_osem_subset_tof_lm_ex -- listmode OSEM subset update, general form:
 *   x[j] <- sens[j] > 0 ? x[j] * (H^T A_S^T (1 / (A_S H x + b)))[j] / (sens[j] * sens_scale) : 0
 * with the resolution model H of r (paper Sec. 2.6), or H = identity when r
 * is NULL; sens is then the caller's H^T A^T 1.  Plan, frame range and TOF
 * rules as jp_osem_subset_tof_lm; b_dev non-NULL reads b from device memory
 * and the event range from the plan's device offsets (CUDA-graph
 * capturable, as jp_osem_subset_tof_lm_dev), otherwise the scalar b is used.
 *   path  JP_OSEM_PATH_QUADS: the projections go through the plan's
 *         zero-padded quad images (one 16-byte access per sample; an
 *         image-sized build, clear and fold per call);
 *         JP_OSEM_PATH_DIRECT: forward from the image, back projection by
 *         scalar atomics into an image (no quad traffic; cheaper for
 *         subsets of fewer than about nvox / 24 events, measured on GB300
 *         for 128x128x71 and 200x200x71 images);
 *         JP_OSEM_PATH_AUTO: DIRECT when b_dev is NULL and the subset holds
 *         fewer than nvox / JP_OSEM_DIRECT_VOXELS_PER_EVENT events, else
 *         QUADS.  All paths compute the same update.
 *   work  device float32 scratch of 2 * nvox, caller-owned, disjoint from x
 *         and sens; required when r is non-NULL, else unused (may be NULL).
 * Errors: those of jp_osem_subset_tof_lm and jp_gauss3d; JP_ERR_ARG for an
 * unknown path.
 */
#define JP_OSEM_PATH_AUTO 0
#define JP_OSEM_PATH_QUADS 1
#define JP_OSEM_PATH_DIRECT 2
#define JP_OSEM_DIRECT_VOXELS_PER_EVENT 24
int jp_osem_subset_tof_lm_ex(jp_plan p, int32_t f0, int32_t f1, float* x, const float* sens,
                             float sens_scale, float b, const float* b_dev, const jp_tof* t,
                             const jp_resolution* r, int32_t path, float* work, void* stream);

/*
 * Listmode Poisson log-likelihood of a forward projection p (the training
 * objective of unrolled reconstruction networks, paper Sec. 4):
 *   jp_poisson_loglik_value: *value (device float) = sum_e w_e log(p_e + b_f)
 *   jp_poisson_loglik_grad:  grad_e = scale * w_e / (p_e + b_f)
 * w may be NULL (all ones); b is device float [n_frames] with b_f the
 * background of event e's frame (frames from the plan's offsets in caller
 * order; plan NULL: one frame); scale is a device float or NULL (1).
 * The value is an FP32 compensated sum (error-free TwoSum steps, error of
 * order eps * sum_e |w_e log(p_e + b_f)| whatever n is) in two passes: block
 * partial sums go to work, device float[2 * JP_LOGLIK_BLOCKS] (8-byte
 * aligned, caller-owned scratch, contents undefined afterwards), and one
 * block adds them up.  Calls sharing a work buffer must not overlap.
 * Errors: JP_ERR_ARG, JP_ERR_ALIGN, JP_ERR_CUDA.
 */
#define JP_LOGLIK_BLOCKS 1024
int jp_poisson_loglik_value(jp_plan p, const float* proj, const float* w, const float* b, int64_t n,
                            float* value, float* work, void* stream);
int jp_poisson_loglik_grad(jp_plan p, const float* proj, const float* w, const float* b, const float* scale,
                           int64_t n, float* grad, void* stream);

/* listmode OSEM start image: x[j] = sens[j] > 0 ? 1 : 0 for nvox voxels */
int jp_osem_init(float* x, const float* sens, int64_t nvox, void* stream);

/* FP64 sum of a float32 device array into *out (device double).  Used only
 * for the sensitivity-normalisation check sum_j (A^T 1)_j = sum_i (A 1)_i. */
int jp_sum_f64(const float* x, int64_t n, double* out, void* stream);

/* Algorithmic work of the plan's LORs, summed into *out (device uint64,
 * overwritten): tof_mode 0 / 2, the plane samples the projector visits
 * (non-TOF / TOF listmode, whose samples are the planes of the TOF window);
 * tof_mode 1, the TOF bin evaluations of a TOF sinogram (over every plane
 * sample, the bins whose window holds it: the per-bin work of the sinogram
 * kernels).  Used to state the work of a launch (samples x bytes per sample,
 * bins x operations per bin). */
int jp_count_samples(jp_plan p, int32_t tof_mode, const jp_tof* t, uint64_t* out, void* stream);

/* Throughput ceiling of the TOF-sinogram kernels' per-bin work (measurement
 * helper): synthetic sample positions, each window's bins through the
 * bin-aligned shared-memory table of t (Gaussian kernels only) and
 * accumulated into per-thread shared-memory bins (direction 0, the
 * forward's operation) or dotted with per-thread shared-memory values
 * (direction 1, the back projection's), per_thread samples per thread on
 * every resident thread of the GPU, in CTAs of the projection's default
 * size (512 threads forward, 256 back).  *ms_out (host) is the time of one
 * timed launch after a warm-up one, *bins_out (device uint64) the bins it
 * evaluated.  Synchronises the stream.  Errors: JP_ERR_ARG, JP_ERR_ALIGN,
 * JP_ERR_CUDA. */
int jp_bench_tof_bins(const jp_tof* t, int32_t direction, int32_t per_thread, float* ms_out, uint64_t* bins_out,
                      void* stream);

/* Number of L2 reduction requests (32-byte sector operations) the plan's
 * quad-image back projection issues in the given mode (0 non-TOF, 2 TOF
 * listmode), counted on the device by replaying that kernel's schedule:
 * its warp chunks, its lane -> (LOR, plane) map and its quad entries, with
 * every LOR's input nonzero.  A warp instruction's 16-byte reductions
 * coalesce into one request per 32-byte sector and lane slot; a sector
 * holds two quad entries, so it costs the larger of their lane counts.
 * Frames are taken with their own image slots.  *out (device uint64) is
 * overwritten.  This is the work unit of the back projection's binding
 * roofline (the L2 reduction throughput).  Errors: JP_ERR_ARG, JP_ERR_ALIGN,
 * JP_ERR_STATE (tile, interleaved or one-LOR-per-thread plans), JP_ERR_CUDA. */
int jp_count_red_requests(jp_plan p, int32_t tof_mode, const jp_tof* t, uint64_t* out, void* stream);

/* total number of kernels this library has launched in the process */
uint64_t jp_launch_count(void);

/*
 * jp_back_tof_lm_noalloc -- TOF listmode back projection that allocates
 * nothing, for callers that cannot allocate device memory: engines whose
 * device memory is fully handed out by their own pool or a fixed real-time
 * budget, and callbacks or serving loops where a cudaMalloc (which may
 * synchronise the whole device) is not allowed to run.  The paper has no
 * counterpart; it is a service variant of jp_back_lors (tof_mode 2) with the
 * same arguments and result (img_accum += A^T proj, caller order, same
 * tolerance as the other back projections).
 * Its scratch is a workspace compiled into the library: 2^20 entries of 16
 * bytes (16 MiB), held by every GPU that loads the library until the process
 * exits.  The image must fit it: sum over a of n_a' (n_b + 2)(n_c + 2) <= 2^20
 * with n_a' = n_a rounded up to even (for instance 64 x 64 x 16, or about
 * 70^3), else JP_ERR_ARG.  The first call on a device looks the workspace
 * address up (cudaGetSymbolAddress, once per device), so make that first
 * call before any stream capture; the address is kept for the life of the
 * process, so a device reset (cudaDeviceReset) after that first call is not
 * supported.  Every call shares the one workspace (it is cleared at the
 * start of each call): calls that overlap on the GPU, on any stream, race
 * and give wrong results.
 * Errors: JP_ERR_ARG, JP_ERR_ALIGN, JP_ERR_CUDA.
 */
int jp_back_tof_lm_noalloc(const float* xstart, const float* xend, const int16_t* tof_bin,
                           const float* tof_center_offset, int64_t n_lor, const jp_image_geom* g,
                           const jp_tof* t, const float* proj, float* img_accum, void* stream);

/*
 * jp_bench_red -- measurement helper (not part of the projector): times
 * `iters` launches of a kernel in which every thread issues `per_thread`
 * 16-byte vector reductions (red.add of a float4) at pseudo-random 16-byte
 * aligned positions of the device buffer `buf` (n_entries float4, caller
 * allocated; its contents are changed).  *ms_out receives the mean time of
 * one launch; the rate is (blocks*threads*per_thread) / time.  It gives the
 * device's scattered-reduction ceiling that bounds the back projections.
 */
int jp_bench_red(float* buf, int64_t n_entries, int32_t per_thread, int32_t iters, float* ms_out,
                 void* stream);

/* Same, with an access pattern: 0 = every lane its own random 16-byte entry
 * (one 32-byte L2 sector per reduction), 1 = pairs of lanes on the two
 * halves of one random sector, 2 = a warp on 32 consecutive entries (512
 * contiguous bytes), 3 / 4 = groups of 4 / 8 lanes on the first 4 / 8
 * entries of one random 128-byte line (how much sharing lines, not only
 * sectors, saves).  Pattern 0 is jp_bench_red. */
int jp_bench_red_pattern(float* buf, int64_t n_entries, int32_t per_thread, int32_t iters, int32_t pattern,
                         float* ms_out, void* stream);

/* thread-local message of the last failing call ("" if none) */
const char* jp_last_error(void);

/* library version string */
const char* jp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* JOSEPH_H */
