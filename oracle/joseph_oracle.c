/*
 * FP64 reference Joseph projector.  TEST INFRASTRUCTURE ONLY: tests/,
 * the smoke check and the benchmark's CPU-baseline leg use it; the product
 * path never does.  It shares no code with the CUDA library.
 *
 * What it computes (paper Sec. 2.1 and Fig. 1, Joseph 1982):
 *   for a line of response (LOR) from xs to xe, d = xe - xs, L = |d|:
 *   1. principal axis a = argmax_i |d_i| (lowest index on exact ties), the
 *      other two axes b < c;
 *   2. every image plane k (coordinate X_k = o_a + k v_a) whose centre lies in
 *      the closed segment [min(xs_a,xe_a), max(xs_a,xe_a)] is visited;
 *   3. at the intersection P_k = xs + lambda_k d, lambda_k = (X_k - xs_a)/d_a,
 *      the continuous indices u = (P_b - o_b)/v_b, w = (P_c - o_c)/v_c give a
 *      bilinear interpolation of the 4 nearest voxels (zero outside the grid);
 *   4. the plane values are summed and multiplied by v_a / cos_a,
 *      cos_a = |d_a| / L  (the incidence-angle correction);
 *   5. TOF (Sec. 2.1, 2.2, 2.6): tau_k = (lambda_k - 1/2) L is the signed
 *      distance of the sample from the LOR midpoint along xs->xe.  A TOF bin
 *      with centre c has weight
 *        g = 1/2 [erf((tau-c+D/2)/(sqrt2 s)) - erf((tau-c-D/2)/(sqrt2 s))]
 *      when |tau - c| <= n_sigmas s + D/2, else 0 (Gaussian of width s
 *      convolved with a bin of width D, truncated).  Sinogram bin t of N has
 *      c_t = (t - (N-1)/2) D + delta; a listmode event with signed bin t_s has
 *      c = t_s D + delta (delta: optional per-LOR TOF centre offset).  An
 *      optional per-LOR sigma replaces s for that LOR (per-event TOF
 *      resolution);
 *   5b. tabulated kernel (Sec. 4: a 1D lookup table permits non-Gaussian
 *      TOF kernels): with a table of n values at d_e = -h + e 2h/(n-1), the
 *      weight at d = tau - c is the linear interpolation of the table, and 0
 *      when |d| > h (replacing the Gaussian and its truncation);
 *   6. back projection is the exact transpose (Sec. 2.2, matched pair).
 *
 * All arithmetic is double.  Outputs are double.  The single-thread mode is
 * deterministic; the threaded mode partitions LORs (forward) or uses private
 * per-thread images summed at the end (back).
 *
 * TOF truncation is a floating-point decision: a sample within `amb_eps` mm
 * of the truncation edge is "ambiguous" (FP32 and FP64 may decide it
 * differently).  The forward functions optionally report, per output, the
 * summed magnitude of such samples' contributions so that a comparison can
 * allow for either decision.
 *
 * Planted-mistake builds (-DOR_MUTANT=k) exist only so the pin tests can show
 * that each pin catches a plausible error; the default build has none.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef OR_MUTANT
#define OR_MUTANT 0
#endif

typedef struct {
  int64_t n[3];
  double o[3];
  double v[3];
} geom_t;

typedef struct {
  int mode;           /* 0 non-TOF, 1 TOF sinogram, 2 TOF listmode */
  double bin_width;   /* D */
  double sigma;       /* s */
  double n_sigmas;
  int64_t n_bins;     /* N (sinogram) */
  double amb_eps;     /* ambiguity band half-width (mm) */
  const double* table;  /* tabulated kernel or NULL (Gaussian) */
  int64_t table_nodes;
  double table_hw;      /* h */
} tof_t;

/* ---------------------------------------------------------------------- */
/* exact comparison |xe_i - xs_i| vs |xe_j - xs_j| (two-sum error terms)   */
/* ---------------------------------------------------------------------- */
static void two_diff(double a, double b, double* hi, double* lo) {
  double s = a - b;
  double bv = s - a;
  double av = s - bv;
  *hi = s;
  *lo = (a - av) + (-b - bv);
}

/* 1 if |d_i| > |d_j| exactly, else 0 */
static int abs_greater(double hi_i, double lo_i, double hi_j, double lo_j) {
  double ai = fabs(hi_i), aj = fabs(hi_j);
  if (ai != aj) return ai > aj;
  double ri = (hi_i > 0) ? lo_i : -lo_i;
  double rj = (hi_j > 0) ? lo_j : -lo_j;
  if (hi_i == 0) ri = 0;
  if (hi_j == 0) rj = 0;
  return ri > rj;
}

static int principal_axis(const double* xs, const double* xe) {
  double hi[3], lo[3];
  for (int i = 0; i < 3; ++i) two_diff(xe[i], xs[i], &hi[i], &lo[i]);
  int a = 0;
  for (int i = 1; i < 3; ++i)
    if (abs_greater(hi[i], lo[i], hi[a], lo[a])) a = i;
#if OR_MUTANT == 5
  /* planted: last axis wins ties */
  for (int i = 0; i < 3; ++i)
    if (!abs_greater(hi[a], lo[a], hi[i], lo[i]) && i > a) a = i;
#endif
  return a;
}

/* ---------------------------------------------------------------------- */
/* TOF weight of one bin (paper Sec. 2.1: Gaussian (x) rect -> erf diff)    */
/* ---------------------------------------------------------------------- */
double or_tof_weight(double tau, double centre, double bin_width, double sigma,
                     double n_sigmas) {
  double dist = tau - centre;
  double r = n_sigmas * sigma + 0.5 * bin_width;
  if (fabs(dist) > r) return 0.0;
  double k = 1.0 / (sqrt(2.0) * sigma);
#if OR_MUTANT == 3
  /* planted: dropped factor 1/2 */
  return (erf((dist + 0.5 * bin_width) * k) - erf((dist - 0.5 * bin_width) * k));
#else
  return 0.5 * (erf((dist + 0.5 * bin_width) * k) - erf((dist - 0.5 * bin_width) * k));
#endif
}

/* tabulated kernel: linear interpolation of the nodes, clamped to the table
 * (callers apply the support rule |dist| <= h) */
static double table_value(const tof_t* t, double dist) {
#if OR_MUTANT == 8
  /* planted: node spacing 2h / n instead of 2h / (n - 1) */
  double x = (dist + t->table_hw) * (double)(t->table_nodes) / (2.0 * t->table_hw);
#else
  double x = (dist + t->table_hw) * (double)(t->table_nodes - 1) / (2.0 * t->table_hw);
#endif
  double fl = floor(x);
  int64_t i = (int64_t)fl;
  if (i < 0) i = 0;
  if (i > t->table_nodes - 2) i = t->table_nodes - 2;
  double fr = x - (double)i;
  return t->table[i] + fr * (t->table[i + 1] - t->table[i]);
}

/* TOF weight of a bin with centre `centre` for a sample at tau, with the LOR's
 * sigma (Gaussian) or the table */
static double tof_w(const tof_t* t, double tau, double centre, double sigma) {
  if (t->table) {
    double dist = tau - centre;
    return fabs(dist) > t->table_hw ? 0.0 : table_value(t, dist);
  }
  return or_tof_weight(tau, centre, t->bin_width, sigma, t->n_sigmas);
}

/* untruncated value and ambiguity flag */
static double tof_weight_amb(double tau, double centre, const tof_t* t, double sigma, int* amb) {
  double dist = tau - centre;
  double r = t->table ? t->table_hw : t->n_sigmas * sigma + 0.5 * t->bin_width;
#if OR_MUTANT == 10
  /* planted: every sample inside the window flagged, not only the edge band */
  *amb = fabs(dist) <= r + t->amb_eps;
#else
  *amb = fabs(fabs(dist) - r) <= t->amb_eps;
#endif
  if (fabs(dist) > r && !*amb) return 0.0;
#if OR_MUTANT == 12
  /* planted: the truncated weight (0 just outside the edge) instead of the
   * untruncated one */
  if (fabs(dist) > r) return 0.0;
#endif
  if (t->table) return table_value(t, dist);
  double k = 1.0 / (sqrt(2.0) * sigma);
  double g = 0.5 * (erf((dist + 0.5 * t->bin_width) * k) - erf((dist - 0.5 * t->bin_width) * k));
  return g; /* caller applies the truncation rule itself for the main value */
}

static double bin_centre_sino(int64_t t, const tof_t* tp, double delta) {
#if OR_MUTANT == 4
  /* planted: bins counted from the xe end */
  return -((double)t - 0.5 * (double)(tp->n_bins - 1)) * tp->bin_width + delta;
#else
  return ((double)t - 0.5 * (double)(tp->n_bins - 1)) * tp->bin_width + delta;
#endif
}

/* ---------------------------------------------------------------------- */
/* one plane sample                                                        */
/* ---------------------------------------------------------------------- */
typedef struct {
  int64_t idx[4];  /* flat voxel indices, -1 when outside the grid */
  double wt[4];    /* bilinear weights */
  double tau;      /* along-LOR coordinate relative to the midpoint */
} sample_t;

typedef struct {
  int valid;   /* L > 0 */
  int a, b, c;
  double w0;   /* v_a / cos_a */
  double L;
} ray_t;

static ray_t ray_setup(const double* xs, const double* xe, const geom_t* g) {
  ray_t r;
  double d[3] = {xe[0] - xs[0], xe[1] - xs[1], xe[2] - xs[2]};
  r.L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  r.valid = r.L > 0;
  r.a = principal_axis(xs, xe);
  r.b = (r.a == 0) ? 1 : 0;
  r.c = (r.a == 2) ? 1 : 2;
  double cosa = r.valid ? fabs(d[r.a]) / r.L : 1.0;
#if OR_MUTANT == 2
  /* planted: angle correction dropped */
  r.w0 = g->v[r.a];
#else
  r.w0 = g->v[r.a] / cosa;
#endif
  return r;
}

static int64_t flat(const geom_t* g, const int64_t ijk[3]) {
  for (int i = 0; i < 3; ++i)
    if (ijk[i] < 0 || ijk[i] >= g->n[i]) return -1;
  return (ijk[0] * g->n[1] + ijk[1]) * g->n[2] + ijk[2];
}

/* returns 1 if plane k is visited and fills the sample */
static int plane_sample(const double* xs, const double* xe, const ray_t* r,
                        const geom_t* g, int64_t k, sample_t* s) {
  int a = r->a, b = r->b, c = r->c;
  double X = g->o[a] + (double)k * g->v[a];
  double lo = fmin(xs[a], xe[a]), hi = fmax(xs[a], xe[a]);
#if OR_MUTANT == 6
  /* planted: half-open plane range */
  if (X < lo || X >= hi) return 0;
#else
  if (X < lo || X > hi) return 0;
#endif
  double da = xe[a] - xs[a];
  double lam = (X - xs[a]) / da;
  double P[3];
  for (int i = 0; i < 3; ++i) P[i] = xs[i] + lam * (xe[i] - xs[i]);
  double u = (P[b] - g->o[b]) / g->v[b];
  double w = (P[c] - g->o[c]) / g->v[c];
  double fu = floor(u), fw = floor(w);
  double al = u - fu, be = w - fw;
#if OR_MUTANT == 1
  /* planted: fractions swapped between the two in-plane axes */
  { double tmp = al; al = be; be = tmp; }
#endif
  int64_t i = (int64_t)fu, j = (int64_t)fw;
  int64_t ijk[3];
  const int64_t di[4] = {0, 1, 0, 1};
  const int64_t dj[4] = {0, 0, 1, 1};
  for (int q = 0; q < 4; ++q) {
    ijk[a] = k;
    ijk[b] = i + di[q];
    ijk[c] = j + dj[q];
    s->idx[q] = flat(g, ijk);
    double wa = di[q] ? al : 1.0 - al;
    double wb = dj[q] ? be : 1.0 - be;
    s->wt[q] = wa * wb;
  }
#if OR_MUTANT == 7
  /* planted: TOF coordinate measured from xs instead of the midpoint */
  s->tau = lam * r->L;
#else
  s->tau = (lam - 0.5) * r->L;
#endif
  return 1;
}

static double interp(const sample_t* s, const double* img) {
  double acc = 0.0;
  for (int q = 0; q < 4; ++q)
    if (s->idx[q] >= 0) acc += s->wt[q] * img[s->idx[q]];
  return acc;
}

static void scatter(const sample_t* s, double val, double* img) {
  for (int q = 0; q < 4; ++q)
    if (s->idx[q] >= 0) img[s->idx[q]] += s->wt[q] * val;
}

/* ---------------------------------------------------------------------- */
/* per-LOR forward / back                                                   */
/* ---------------------------------------------------------------------- */
static void fwd_one(const double* xs, const double* xe, const geom_t* g, const tof_t* t,
                    int64_t tof_bin, double delta, double sigma, const double* img, double* out,
                    double* amb) {
  int nout = (t->mode == 1) ? (int)t->n_bins : 1;
  for (int q = 0; q < nout; ++q) {
    out[q] = 0.0;
    if (amb) amb[q] = 0.0;
  }
  ray_t r = ray_setup(xs, xe, g);
  if (!r.valid) return;
  sample_t s;
  for (int64_t k = 0; k < g->n[r.a]; ++k) {
    if (!plane_sample(xs, xe, &r, g, k, &s)) continue;
    double sk = interp(&s, img);
    if (t->mode == 0) {
      out[0] += sk;
    } else if (t->mode == 1) {
      for (int64_t b = 0; b < t->n_bins; ++b) {
        double cb = bin_centre_sino(b, t, delta);
        int ambf = 0;
        double graw = tof_weight_amb(s.tau, cb, t, sigma, &ambf);
        out[b] += tof_w(t, s.tau, cb, sigma) * sk;
        if (amb && ambf) amb[b] += fabs(graw * sk);
      }
    } else {
      double cb = (double)tof_bin * t->bin_width + delta;
      int ambf = 0;
      double graw = tof_weight_amb(s.tau, cb, t, sigma, &ambf);
      out[0] += tof_w(t, s.tau, cb, sigma) * sk;
      if (amb && ambf) amb[0] += fabs(graw * sk);
    }
  }
  for (int q = 0; q < nout; ++q) {
    out[q] *= r.w0;
#if OR_MUTANT != 11
    /* (planted mistake 11 leaves the ambiguity magnitude unscaled) */
    if (amb) amb[q] *= r.w0;
#endif
  }
}

static void back_one(const double* xs, const double* xe, const geom_t* g, const tof_t* t,
                     int64_t tof_bin, double delta, double sigma, const double* y, double* img) {
  ray_t r = ray_setup(xs, xe, g);
  if (!r.valid) return;
  sample_t s;
  for (int64_t k = 0; k < g->n[r.a]; ++k) {
    if (!plane_sample(xs, xe, &r, g, k, &s)) continue;
    double val;
    if (t->mode == 0) {
      val = y[0];
    } else if (t->mode == 1) {
      val = 0.0;
      for (int64_t b = 0; b < t->n_bins; ++b)
        val += tof_w(t, s.tau, bin_centre_sino(b, t, delta), sigma) * y[b];
    } else {
      val = tof_w(t, s.tau, (double)tof_bin * t->bin_width + delta, sigma) * y[0];
    }
    scatter(&s, r.w0 * val, img);
  }
}

/* ---------------------------------------------------------------------- */
/* threaded drivers                                                         */
/* ---------------------------------------------------------------------- */
typedef struct {
  const double *xs, *xe, *img, *y, *delta, *sigma;
  const int64_t* tof_bin;
  double *out, *amb, *img_out;
  const geom_t* g;
  const tof_t* t;
  int64_t lo, hi;
} job_t;

static void* fwd_job(void* p) {
  job_t* j = (job_t*)p;
  int nout = (j->t->mode == 1) ? (int)j->t->n_bins : 1;
  for (int64_t i = j->lo; i < j->hi; ++i)
#if OR_MUTANT == 9
    /* planted: the per-LOR sigma is ignored */
    fwd_one(j->xs + 3 * i, j->xe + 3 * i, j->g, j->t, j->tof_bin ? j->tof_bin[i] : 0,
            j->delta ? j->delta[i] : 0.0, j->t->sigma, j->img, j->out + nout * i,
            j->amb ? j->amb + nout * i : NULL);
#else
    fwd_one(j->xs + 3 * i, j->xe + 3 * i, j->g, j->t, j->tof_bin ? j->tof_bin[i] : 0,
            j->delta ? j->delta[i] : 0.0, j->sigma ? j->sigma[i] : j->t->sigma, j->img, j->out + nout * i,
            j->amb ? j->amb + nout * i : NULL);
#endif
  return NULL;
}

static void* back_job(void* p) {
  job_t* j = (job_t*)p;
  int nin = (j->t->mode == 1) ? (int)j->t->n_bins : 1;
  for (int64_t i = j->lo; i < j->hi; ++i)
    back_one(j->xs + 3 * i, j->xe + 3 * i, j->g, j->t, j->tof_bin ? j->tof_bin[i] : 0,
             j->delta ? j->delta[i] : 0.0, j->sigma ? j->sigma[i] : j->t->sigma, j->y + nin * i,
             j->img_out);
  return NULL;
}

static int fill(geom_t* g, tof_t* t, const int64_t* n, const double* o, const double* v,
                int mode, const double* tofp, int64_t n_bins, const double* table,
                int64_t table_nodes, double table_hw) {
  for (int i = 0; i < 3; ++i) {
    if (n[i] <= 0 || !(v[i] > 0)) return -1;
    g->n[i] = n[i];
    g->o[i] = o[i];
    g->v[i] = v[i];
  }
  t->mode = mode;
  t->bin_width = tofp ? tofp[0] : 1.0;
  t->sigma = tofp ? tofp[1] : 1.0;
  t->n_sigmas = tofp ? tofp[2] : 3.0;
  t->amb_eps = tofp ? tofp[3] : 0.0;
  t->n_bins = n_bins;
  t->table = table;
  t->table_nodes = table_nodes;
  t->table_hw = table_hw;
  if (mode < 0 || mode > 2) return -1;
  if (mode != 0 && !(t->bin_width > 0)) return -1;
  if (mode != 0 && table && (table_nodes < 2 || !(table_hw > 0))) return -1;
  if (mode != 0 && !table && (!(t->sigma > 0) || !(t->n_sigmas > 0))) return -1;
  if (mode == 1 && n_bins <= 0) return -1;
  return 0;
}

/*
 * or_fwd: forward projection of `nlor` LORs.
 *   xs, xe   [nlor*3] endpoints (mm)
 *   n, o, v  image shape, origin (centre of voxel 0), voxel size
 *   mode     0 non-TOF, 1 TOF sinogram, 2 TOF listmode
 *   tofp     [4] = bin width, sigma, n_sigmas, ambiguity band (mm); NULL for non-TOF
 *   n_bins   sinogram TOF bins (mode 1)
 *   tof_bin  [nlor] signed listmode bins (mode 2) or NULL
 *   delta    [nlor] TOF centre offsets or NULL (0)
 *   sigma    [nlor] per-LOR Gaussian sigma or NULL (tofp[1] for every LOR)
 *   table, table_nodes, table_hw   tabulated TOF kernel (5b) or NULL
 *   img      [n0*n1*n2] double image
 *   out      [nlor] or [nlor*n_bins] (TOF fastest)
 *   amb      same shape as out, or NULL
 */
int or_fwd_ex(const double* xs, const double* xe, int64_t nlor, const int64_t* n,
              const double* o, const double* v, int mode, const double* tofp, int64_t n_bins,
              const int64_t* tof_bin, const double* delta, const double* sigma,
              const double* table, int64_t table_nodes, double table_hw, const double* img,
              double* out, double* amb, int nthreads) {
  geom_t g;
  tof_t t;
  if (fill(&g, &t, n, o, v, mode, tofp, n_bins, table, table_nodes, table_hw)) return -1;
  if (mode == 2 && !tof_bin) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (nlor < nthreads * 64) nthreads = 1;
  job_t jobs[256];
  pthread_t th[256];
  for (int i = 0; i < nthreads; ++i) {
    job_t j = {xs, xe, img, NULL, delta, sigma, tof_bin, out, amb, NULL, &g, &t,
               nlor * i / nthreads, nlor * (i + 1) / nthreads};
    jobs[i] = j;
  }
  if (nthreads == 1) {
    fwd_job(&jobs[0]);
    return 0;
  }
  for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, fwd_job, &jobs[i]);
  for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
  return 0;
}

/*
 * or_back: img_out += A^T y  (accumulates; double image of n0*n1*n2).
 * y is [nlor] (modes 0, 2) or [nlor*n_bins] (mode 1).
 */
int or_back_ex(const double* xs, const double* xe, int64_t nlor, const int64_t* n,
               const double* o, const double* v, int mode, const double* tofp, int64_t n_bins,
               const int64_t* tof_bin, const double* delta, const double* sigma,
               const double* table, int64_t table_nodes, double table_hw, const double* y,
               double* img_out, int nthreads) {
  geom_t g;
  tof_t t;
  if (fill(&g, &t, n, o, v, mode, tofp, n_bins, table, table_nodes, table_hw)) return -1;
  if (mode == 2 && !tof_bin) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (nlor < nthreads * 64) nthreads = 1;
  int64_t nvox = n[0] * n[1] * n[2];
  job_t jobs[256];
  pthread_t th[256];
  double* priv = NULL;
  if (nthreads > 1) {
    priv = (double*)calloc((size_t)nvox * (size_t)nthreads, sizeof(double));
    if (!priv) return -2;
  }
  for (int i = 0; i < nthreads; ++i) {
    job_t j = {xs, xe, NULL, y, delta, sigma, tof_bin, NULL, NULL,
               nthreads > 1 ? priv + (size_t)nvox * i : img_out, &g, &t,
               nlor * i / nthreads, nlor * (i + 1) / nthreads};
    jobs[i] = j;
  }
  if (nthreads == 1) {
    back_job(&jobs[0]);
    return 0;
  }
  for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, back_job, &jobs[i]);
  for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
  for (int i = 0; i < nthreads; ++i) {
    const double* p = priv + (size_t)nvox * i;
    for (int64_t q = 0; q < nvox; ++q) img_out[q] += p[q];
  }
  free(priv);
  return 0;
}

/* principal axis as the oracle decides it (exported for tests) */
int or_principal_axis(const double* xs, const double* xe) { return principal_axis(xs, xe); }

int or_mutant(void) { return OR_MUTANT; }

/* the Gaussian-kernel forms with one sigma for every LOR */
int or_fwd(const double* xs, const double* xe, int64_t nlor, const int64_t* n,
           const double* o, const double* v, int mode, const double* tofp, int64_t n_bins,
           const int64_t* tof_bin, const double* delta, const double* img, double* out,
           double* amb, int nthreads) {
  return or_fwd_ex(xs, xe, nlor, n, o, v, mode, tofp, n_bins, tof_bin, delta, NULL, NULL, 0, 0.0,
                   img, out, amb, nthreads);
}

int or_back(const double* xs, const double* xe, int64_t nlor, const int64_t* n,
            const double* o, const double* v, int mode, const double* tofp, int64_t n_bins,
            const int64_t* tof_bin, const double* delta, const double* y, double* img_out,
            int nthreads) {
  return or_back_ex(xs, xe, nlor, n, o, v, mode, tofp, n_bins, tof_bin, delta, NULL, NULL, 0, 0.0,
                    y, img_out, nthreads);
}
