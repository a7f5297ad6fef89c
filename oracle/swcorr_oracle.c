/*
 * swcorr_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU implementation of the sliding-window
 * inter-channel Pearson correlation of Poyda & Zhizhin (arXiv:1807.06507).
 * Only the tests, the benchmark's CPU-baseline leg and the smoke check may
 * load this library; the product path (the CUDA library) never calls it and
 * shares no code, header or table with it.
 *
 * What it computes, per output window (Section "Introduction", Eq. 1, and
 * Section 3 for the centred output cell):
 *   - the window is the box of k_d cells per dimension centred on the output
 *     cell, clipped to the grid: [i - floor((k-1)/2), i + floor(k/2)] per
 *     dimension, intersected with [0, N-1].  n is the number of cells left.
 *   - if every x in the window is equal, or every y is equal, the variance is
 *     zero and the result is NaN.  This is the paper's exact-equality check
 *     for constant windows (Section 3, accuracy discussion).
 *   - otherwise the classical two-pass Pearson formula of Eq. 1 in double
 *     precision: means first, then the centred sums, then
 *     c = sxy / sqrt(sxx * syy), clamped to [-1, 1].
 *   - relvar_x = sxx / sum(x^2) (and likewise for y): the fraction of the
 *     second moment that is variance; it says how much cancellation a
 *     sums-form evaluation (Eq. 2) of that window suffers.
 * Border rule (border = 1, the paper's result convention, Section 3: the
 * paragraph on the result set): a window that reaches past an edge of the
 * grid in any dimension gives -2, and so does a window holding a missing
 * value (a value <= -999) in x or in y; the other windows follow the rules
 * above (they are never clipped).  border = 0 clips as above.
 * For uint16 data it also gives the five exact integer window sums
 * (sum x, sum y, sum x^2, sum y^2, sum xy) that the optimized algorithm's
 * steps 1-3 (Section 1) produce, by brute force over the window.
 *
 * Arrays are C-order: dimension 0 is the outermost, dimension ndim-1 the
 * contiguous one.  Output cell j has centre i_d = j_d * stride_d and the
 * output extent is ceil(N_d / stride_d) per dimension.
 *
 * Built with plain -O2 (no fast-math); one pthread per slice of outputs.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SWO_MAXDIM 8

enum { SWO_U16 = 1, SWO_F32 = 2 };

typedef struct {
  int ndim;
  int64_t shape[SWO_MAXDIM];
  int32_t k[SWO_MAXDIM];
  int32_t stride[SWO_MAXDIM];
  int64_t oshape[SWO_MAXDIM];
  int dtype;
  const void *x, *y;
  const int64_t *idx; /* flat output indices, or NULL for all outputs */
  int64_t n_out;
  double *c, *rvx, *rvy; /* each may be NULL */
  int64_t *sums;         /* n_out x 5, uint16 only; may be NULL */
  int border;            /* 0: clipped windows; 1: the paper's -2 convention */
  int64_t begin, end;
} swo_job;

static double value_at(int dtype, const void *p, int64_t off) {
  if (dtype == SWO_U16) return (double)((const uint16_t *)p)[off];
  return (double)((const float *)p)[off];
}

/* Window bounds [lo_d, hi_d] of output flat index o, clipped to the grid;
 * returns 1 if the unclipped window reaches past an edge in some dimension. */
static int window_of(const swo_job *J, int64_t o, int64_t *lo, int64_t *hi) {
  int64_t j[SWO_MAXDIM];
  for (int d = J->ndim - 1; d >= 0; d--) {
    j[d] = o % J->oshape[d];
    o /= J->oshape[d];
  }
  int outside = 0;
  for (int d = 0; d < J->ndim; d++) {
    int64_t centre = j[d] * (int64_t)J->stride[d];
    int64_t a = centre - (J->k[d] - 1) / 2;
    int64_t b = centre + J->k[d] / 2;
    if (a < 0 || b > J->shape[d] - 1) outside = 1;
    lo[d] = a < 0 ? 0 : a;
    hi[d] = b > J->shape[d] - 1 ? J->shape[d] - 1 : b;
  }
  return outside;
}

/* Visit every cell of the box [lo, hi] in C order; returns the flat input
 * offsets one at a time through *off.  state holds the current multi-index. */
typedef struct {
  int ndim;
  int64_t lo[SWO_MAXDIM], hi[SWO_MAXDIM], cur[SWO_MAXDIM];
  int64_t pitch[SWO_MAXDIM];
  int done;
} box_iter;

static void box_begin(box_iter *it, const swo_job *J, const int64_t *lo, const int64_t *hi) {
  it->ndim = J->ndim;
  int64_t p = 1;
  for (int d = J->ndim - 1; d >= 0; d--) {
    it->pitch[d] = p;
    p *= J->shape[d];
  }
  it->done = 0;
  for (int d = 0; d < J->ndim; d++) {
    it->lo[d] = lo[d];
    it->hi[d] = hi[d];
    it->cur[d] = lo[d];
    if (lo[d] > hi[d]) it->done = 1;
  }
}

static int box_next(box_iter *it, int64_t *off) {
  if (it->done) return 0;
  int64_t o = 0;
  for (int d = 0; d < it->ndim; d++) o += it->cur[d] * it->pitch[d];
  *off = o;
  for (int d = it->ndim - 1; d >= 0; d--) {
    if (it->cur[d] < it->hi[d]) {
      it->cur[d]++;
      return 1;
    }
    it->cur[d] = it->lo[d];
  }
  it->done = 1;
  return 1;
}

static void one_window(const swo_job *J, int64_t slot) {
  int64_t o = J->idx ? J->idx[slot] : slot;
  int64_t lo[SWO_MAXDIM], hi[SWO_MAXDIM], off;
  const int outside = window_of(J, o, lo, hi);
  box_iter it;

  /* The paper's convention: -2 for a window past an edge or holding a
   * missing value (<= -999) in either channel. */
  if (J->border == 1 && (J->c || J->rvx || J->rvy)) {
    int missing = outside;
    if (!missing) {
      box_begin(&it, J, lo, hi);
      while (box_next(&it, &off))
        if (value_at(J->dtype, J->x, off) <= -999.0 || value_at(J->dtype, J->y, off) <= -999.0) missing = 1;
    }
    if (missing) {
      if (J->c) J->c[slot] = -2.0;
      if (J->rvx) J->rvx[slot] = 0.0;
      if (J->rvy) J->rvy[slot] = 0.0;
      if (!J->sums) return;
    }
  }

  /* Exact integer sums (uint16 only): steps 1-3 of Section 1 by brute force. */
  if (J->sums) {
    int64_t sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
    const uint16_t *X = (const uint16_t *)J->x, *Y = (const uint16_t *)J->y;
    box_begin(&it, J, lo, hi);
    while (box_next(&it, &off)) {
      int64_t a = X[off], b = Y[off];
      sx += a;
      sy += b;
      sxx += a * a;
      syy += b * b;
      sxy += a * b;
    }
    int64_t *s = J->sums + 5 * slot;
    s[0] = sx;
    s[1] = sy;
    s[2] = sxx;
    s[3] = syy;
    s[4] = sxy;
  }
  if (!J->c && !J->rvx && !J->rvy) return;

  /* Pass 0: the equality check for constant windows, and n. */
  int64_t n = 0;
  double x0 = 0.0, y0 = 0.0;
  int x_const = 1, y_const = 1;
  box_begin(&it, J, lo, hi);
  while (box_next(&it, &off)) {
    double a = value_at(J->dtype, J->x, off), b = value_at(J->dtype, J->y, off);
    if (n == 0) {
      x0 = a;
      y0 = b;
    } else {
      if (a != x0) x_const = 0;
      if (b != y0) y_const = 0;
    }
    n++;
  }

  /* Pass 1: arithmetic means. */
  double sum_x = 0.0, sum_y = 0.0, sum_xx = 0.0, sum_yy = 0.0;
  box_begin(&it, J, lo, hi);
  while (box_next(&it, &off)) {
    double a = value_at(J->dtype, J->x, off), b = value_at(J->dtype, J->y, off);
    sum_x += a;
    sum_y += b;
    sum_xx += a * a;
    sum_yy += b * b;
  }
  double mx = sum_x / (double)n, my = sum_y / (double)n;

  /* Pass 2: centred sums of Eq. 1. */
  double sxy = 0.0, sxx = 0.0, syy = 0.0;
  box_begin(&it, J, lo, hi);
  while (box_next(&it, &off)) {
    double a = value_at(J->dtype, J->x, off) - mx;
    double b = value_at(J->dtype, J->y, off) - my;
    sxy += a * b;
    sxx += a * a;
    syy += b * b;
  }

  double c;
  if (x_const || y_const) {
    c = NAN;
  } else {
    c = sxy / sqrt(sxx * syy);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
  }
  if (J->c) J->c[slot] = c;
  if (J->rvx) J->rvx[slot] = (x_const || sum_xx == 0.0) ? 0.0 : sxx / sum_xx;
  if (J->rvy) J->rvy[slot] = (y_const || sum_yy == 0.0) ? 0.0 : syy / sum_yy;
}

static void *worker(void *arg) {
  swo_job *J = (swo_job *)arg;
  for (int64_t s = J->begin; s < J->end; s++) one_window(J, s);
  return NULL;
}

static int run_jobs(swo_job *proto, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (proto->n_out < nthreads) nthreads = proto->n_out > 0 ? (int)proto->n_out : 1;
  swo_job jobs[256];
  pthread_t th[256];
  int64_t per = (proto->n_out + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; t++) {
    jobs[t] = *proto;
    jobs[t].begin = per * t;
    jobs[t].end = per * (t + 1) > proto->n_out ? proto->n_out : per * (t + 1);
  }
  int started = 0;
  for (int t = 1; t < nthreads; t++) {
    if (pthread_create(&th[t], NULL, worker, &jobs[t]) != 0) break;
    started = t;
  }
  worker(&jobs[0]);
  for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
  /* Any slice whose thread could not start runs here. */
  for (int t = started + 1; t < nthreads; t++) worker(&jobs[t]);
  return 0;
}

static int setup(swo_job *J, int ndim, const int64_t *shape, const int32_t *k,
                 const int32_t *stride, int dtype, const void *x, const void *y,
                 const int64_t *idx, int64_t n_idx) {
  memset(J, 0, sizeof(*J));
  if (ndim < 1 || ndim > SWO_MAXDIM) return -1;
  if (dtype != SWO_U16 && dtype != SWO_F32) return -1;
  J->ndim = ndim;
  J->dtype = dtype;
  J->x = x;
  J->y = y;
  int64_t total = 1;
  for (int d = 0; d < ndim; d++) {
    if (shape[d] < 1 || k[d] < 1 || stride[d] < 1) return -1;
    J->shape[d] = shape[d];
    J->k[d] = k[d];
    J->stride[d] = stride[d];
    J->oshape[d] = (shape[d] + stride[d] - 1) / stride[d];
    total *= J->oshape[d];
  }
  J->idx = idx;
  J->n_out = idx ? n_idx : total;
  if (idx) {
    for (int64_t s = 0; s < n_idx; s++)
      if (idx[s] < 0 || idx[s] >= total) return -2;
  }
  return 0;
}

/* c, relvar_x and relvar_y (each optional) for the listed outputs, or for all
 * outputs in C order when idx is NULL.  Returns 0, or <0 on bad arguments. */
int swo_corr(int ndim, const int64_t *shape, const int32_t *k, const int32_t *stride,
             int dtype, const void *x, const void *y, const int64_t *idx, int64_t n_idx,
             double *c, double *relvar_x, double *relvar_y, int nthreads) {
  swo_job J;
  int rc = setup(&J, ndim, shape, k, stride, dtype, x, y, idx, n_idx);
  if (rc) return rc;
  J.c = c;
  J.rvx = relvar_x;
  J.rvy = relvar_y;
  return run_jobs(&J, nthreads);
}

/* swo_corr with a border rule: 0 clips the windows to the grid, 1 applies
 * the paper's -2 convention (see the file header). */
int swo_corr_border(int ndim, const int64_t *shape, const int32_t *k, const int32_t *stride,
                    int dtype, const void *x, const void *y, const int64_t *idx, int64_t n_idx,
                    double *c, double *relvar_x, double *relvar_y, int border, int nthreads) {
  swo_job J;
  int rc = setup(&J, ndim, shape, k, stride, dtype, x, y, idx, n_idx);
  if (rc) return rc;
  if (border != 0 && border != 1) return -1;
  J.c = c;
  J.rvx = relvar_x;
  J.rvy = relvar_y;
  J.border = border;
  return run_jobs(&J, nthreads);
}

/* Exact int64 window sums (uint16 inputs only): 5 per output, in the order
 * sum x, sum y, sum x^2, sum y^2, sum xy. */
int swo_sums_u16(int ndim, const int64_t *shape, const int32_t *k, const int32_t *stride,
                 const uint16_t *x, const uint16_t *y, const int64_t *idx, int64_t n_idx,
                 int64_t *sums, int nthreads) {
  swo_job J;
  int rc = setup(&J, ndim, shape, k, stride, SWO_U16, x, y, idx, n_idx);
  if (rc) return rc;
  J.sums = sums;
  return run_jobs(&J, nthreads);
}
