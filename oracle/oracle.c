/*
 * FP64 CPU oracle for wire-scan (differential-aperture) depth reconstruction.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg load it; the library in
 * paper_2201_13309_gb300/ never includes, links or calls it, and it shares
 * no code, header or constant with that library.
 *
 * What it computes (Sec. III-A and III-C of the paper: each pixel's
 * intensity differences between consecutive wire-step images are assigned
 * to depths and summed into a depth-resolved result; the geometry is the
 * differential-aperture method the paper cites, Larson et al. 2002):
 *
 *  1. Pixel centre Q(r,c) = det_origin + r*row_step + c*col_step.
 *  2. Everything is projected onto the plane perpendicular to the wire axis;
 *     a beam point at depth d (distance along the unit beam direction from
 *     beam_origin) projects to d*b', b' the projected unit beam direction.
 *  3. For wire step k the two lines through the projected pixel Q' that are
 *     tangent to the wire circle (centre C'_k, radius R) are built from the
 *     tangent-point construction (rotate the unit vector Q'->C'_k by
 *     +-asin(R/|C'_k-Q'|)) and intersected with the projected beam.  The two
 *     intersections bound the depths the wire hides from this pixel.  The
 *     leading edge is the end that moves in the wire's direction of travel
 *     (sign of (C'_{K-1}-C'_0).b'); the trailing edge is the other end.
 *  4. dI_k = I_k - I_{k+1} (int64) for the leading edge; the trailing edge
 *     sees the reverse change, I_{k+1} - I_k.
 *  5. dI_k is spread over [min(d_k,d_{k+1}), max(d_k,d_{k+1})) in proportion
 *     to the overlap with each bin [e_j, e_{j+1}); a zero-length interval
 *     puts all of dI_k in the bin holding it; mass outside [e_0, e_B] is
 *     dropped.
 *
 * Parity is pinned (tests/test_oracle_pins.py) against brute-force
 * ray-cylinder occlusion, the exact quadratic solution of the tangent
 * condition, the far-detector limit d = z + R, fine subdivision of the
 * intervals, conservation, invariance to the lengths of the direction
 * vectors and the sense of the wire axis, noise-free forward-model scans
 * (also for a path whose first step runs backwards and for rows asked for
 * by offset), and the refusal of geometries where the method has no answer.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_BAD_ARG = 1, OR_BAD_GEOMETRY = 2, OR_NO_MEMORY = 3 };
enum { OR_LEADING = 0, OR_TRAILING = 1 };

/* Flat geometry layout (19 doubles):
 *  [0..2] beam_origin  [3..5] beam_dir  [6..8] det_origin
 *  [9..11] row_step    [12..14] col_step [15..17] wire_axis  [18] radius */

static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
/* v minus its component along the unit vector a */
static void perp(const double *v, const double *a, double *o) {
  double s = dot3(v, a);
  o[0] = v[0] - s * a[0];
  o[1] = v[1] - s * a[1];
  o[2] = v[2] - s * a[2];
}

typedef struct {
  double axis[3];     /* unit wire axis */
  double bproj[3];    /* projected unit beam direction b' */
  double bb;          /* b'.b' */
  double origin[3];   /* beam origin */
  double radius;
  int travel;         /* +1: wire moves toward +depth, -1: toward -depth */
} or_frame;

static int make_frame(const double *g, const double *wires, int K,
                      or_frame *f) {
  double na = sqrt(dot3(g + 15, g + 15));
  double nb = sqrt(dot3(g + 3, g + 3));
  if (!(na > 0.0) || !(nb > 0.0) || !(g[18] > 0.0)) return OR_BAD_GEOMETRY;
  for (int i = 0; i < 3; ++i) f->axis[i] = g[15 + i] / na;
  double b[3] = {g[3] / nb, g[4] / nb, g[5] / nb};
  perp(b, f->axis, f->bproj);
  f->bb = dot3(f->bproj, f->bproj);
  if (!(f->bb > 1e-24)) return OR_BAD_GEOMETRY; /* beam along the wire */
  memcpy(f->origin, g, sizeof(double) * 3);
  f->radius = g[18];
  double move[3] = {wires[3 * (K - 1)] - wires[0], wires[3 * (K - 1) + 1] - wires[1],
                    wires[3 * (K - 1) + 2] - wires[2]};
  double m[3];
  perp(move, f->axis, m);
  double along = dot3(m, f->bproj);
  if (along == 0.0) return OR_BAD_GEOMETRY; /* no travel along the beam */
  f->travel = along > 0.0 ? 1 : -1;
  return OR_OK;
}

/* Depths of the two tangent lines from pixel q to the wire at centre c,
 * intersected with the beam.  Writes lo <= hi.  Tangent-point construction. */
static int tangent_depths(const or_frame *f, const double *q, const double *c,
                          double *lo, double *hi) {
  double qo[3] = {q[0] - f->origin[0], q[1] - f->origin[1], q[2] - f->origin[2]};
  double co[3] = {c[0] - f->origin[0], c[1] - f->origin[1], c[2] - f->origin[2]};
  double qp[3], cp[3];
  perp(qo, f->axis, qp);
  perp(co, f->axis, cp);
  double v[3] = {cp[0] - qp[0], cp[1] - qp[1], cp[2] - qp[2]};
  double D = sqrt(dot3(v, v));
  if (!(D > f->radius)) return OR_BAD_GEOMETRY; /* pixel inside the wire */
  double alpha = asin(f->radius / D);
  double w[3] = {v[0] / D, v[1] / D, v[2] / D};
  double aw[3];
  cross3(f->axis, w, aw); /* w turned by +90 degrees inside the plane */
  double qxb[3];
  cross3(qp, f->bproj, qxb);
  double d[2];
  for (int s = 0; s < 2; ++s) {
    double th = s == 0 ? alpha : -alpha;
    double u[3] = {w[0] * cos(th) + aw[0] * sin(th), w[1] * cos(th) + aw[1] * sin(th),
                   w[2] * cos(th) + aw[2] * sin(th)};
    /* qp + t*u = d*b'  ->  cross with b' and project on the axis */
    double uxb[3];
    cross3(u, f->bproj, uxb);
    double den = dot3(uxb, f->axis);
    if (den == 0.0) return OR_BAD_GEOMETRY; /* tangent parallel to beam */
    double t = -dot3(qxb, f->axis) / den;
    /* the beam must lie beyond the tangent point, seen from the pixel */
    if (!(t > sqrt(D * D - f->radius * f->radius))) return OR_BAD_GEOMETRY;
    double x[3] = {qp[0] + t * u[0], qp[1] + t * u[1], qp[2] + t * u[2]};
    d[s] = dot3(x, f->bproj) / f->bb;
  }
  *lo = d[0] < d[1] ? d[0] : d[1];
  *hi = d[0] < d[1] ? d[1] : d[0];
  return OR_OK;
}

static void pixel_centre(const double *g, int r, int c, double *q) {
  for (int i = 0; i < 3; ++i) q[i] = g[6 + i] + r * g[9 + i] + c * g[12 + i];
}

/* Depth sequence d_k (k = 0..K-1) of pixel (r, c) for the chosen edge. */
static int pixel_depths(const double *g, const or_frame *f, const double *wires,
                        int K, int edge, int r, int c, double *d) {
  double q[3];
  pixel_centre(g, r, c, q);
  for (int k = 0; k < K; ++k) {
    double lo, hi;
    int st = tangent_depths(f, q, wires + 3 * k, &lo, &hi);
    if (st) return st;
    int lead_is_hi = f->travel > 0;
    int want_hi = edge == OR_LEADING ? lead_is_hi : !lead_is_hi;
    d[k] = want_hi ? hi : lo;
  }
  return OR_OK;
}

/* Bin index j with e_j <= x < e_{j+1}, or -1 if x is outside [e_0, e_B). */
static int bin_of(const double *e, int B, double x) {
  if (!(x >= e[0]) || !(x < e[B])) return -1;
  int lo = 0, hi = B; /* e[lo] <= x < e[hi] */
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (e[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

/* Step 5 for one pixel: out[j * stride] += share of each difference. */
static void apportion_pixel(const double *d, const int64_t *dI, int K,
                            const double *e, int B, double *out,
                            size_t stride) {
  for (int k = 0; k + 1 < K; ++k) {
    if (dI[k] == 0) continue;
    double lo = d[k] < d[k + 1] ? d[k] : d[k + 1];
    double hi = d[k] < d[k + 1] ? d[k + 1] : d[k];
    if (hi > lo) {
      int j = bin_of(e, B, lo);
      if (j < 0) j = lo < e[0] ? 0 : B;
      for (; j < B && e[j] < hi; ++j) {
        double a = lo > e[j] ? lo : e[j];
        double b = hi < e[j + 1] ? hi : e[j + 1];
        if (b > a) out[(size_t)j * stride] += (double)dI[k] * (b - a) / (hi - lo);
      }
    } else {
      int j = bin_of(e, B, lo);
      if (j >= 0) out[(size_t)j * stride] += (double)dI[k];
    }
  }
}

/* ---- public entry points (called through ctypes from oracle.py) ---- */

/* Depths [nrows][cols][K] for rows r0 .. r0+nrows-1. */
int oracle_depths(const double *geom, int cols, const double *wires, int K,
                  int edge, int r0, int nrows, double *out) {
  if (K < 1 || cols < 0 || nrows < 0) return OR_BAD_ARG;
  or_frame f;
  int st = make_frame(geom, wires, K, &f);
  if (st) return st;
  for (int r = 0; r < nrows; ++r)
    for (int c = 0; c < cols; ++c) {
      st = pixel_depths(geom, &f, wires, K, edge, r0 + r, c,
                        out + ((size_t)r * cols + c) * K);
      if (st) return st;
    }
  return OR_OK;
}

/* Step 4: dI[k][p] = I[k][p] - I[k+1][p] for P pixels (int64, exact). */
void oracle_differences(const uint16_t *images, int K, long long P,
                        int64_t *out) {
  for (int k = 0; k + 1 < K; ++k)
    for (long long p = 0; p < P; ++p)
      out[(size_t)k * P + p] =
          (int64_t)images[(size_t)k * P + p] - (int64_t)images[(size_t)(k + 1) * P + p];
}

/* Step 5 alone, for given depths: depths [P][K], images [K][P] (uint16),
 * out [B][P] (overwritten).  edge selects the sign of the difference. */
int oracle_apportion(const double *depths, const uint16_t *images, int K,
                     long long P, int edge, const double *e, int B,
                     double *out) {
  if (K < 1 || B < 1 || P < 0) return OR_BAD_ARG;
  for (int j = 0; j + 1 <= B; ++j)
    if (!(e[j + 1] > e[j])) return OR_BAD_ARG;
  memset(out, 0, sizeof(double) * (size_t)B * (size_t)P);
  int64_t *dI = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K > 1 ? K : 1));
  if (!dI) return OR_NO_MEMORY;
  for (long long p = 0; p < P; ++p) {
    for (int k = 0; k + 1 < K; ++k) {
      int64_t a = images[(size_t)k * P + p], b = images[(size_t)(k + 1) * P + p];
      dI[k] = edge == OR_LEADING ? a - b : b - a;
    }
    apportion_pixel(depths + (size_t)p * K, dI, K, e, B, out + p, (size_t)P);
  }
  free(dI);
  return OR_OK;
}

typedef struct {
  const double *geom;
  const or_frame *f;
  const double *wires;
  int K, edge, cols, rows_total;
  const uint16_t *images; /* [K][rows_total][cols] */
  const double *e;
  int B;
  int r0, nrows;          /* output rows r0 .. r0+nrows-1 */
  double *out;            /* [B][nrows][cols] */
  int next_row;           /* shared work counter (guarded by mu) */
  pthread_mutex_t mu;
  int status;
} or_job;

static void *worker(void *arg) {
  or_job *J = (or_job *)arg;
  double *d = (double *)malloc(sizeof(double) * (size_t)J->K);
  int64_t *dI = (int64_t *)malloc(sizeof(int64_t) * (size_t)J->K);
  size_t plane = (size_t)J->rows_total * J->cols;
  size_t ostride = (size_t)J->nrows * J->cols;
  if (!d || !dI) {
    pthread_mutex_lock(&J->mu);
    J->status = OR_NO_MEMORY;
    pthread_mutex_unlock(&J->mu);
  }
  for (;;) {
    pthread_mutex_lock(&J->mu);
    int rr = J->status ? J->nrows : J->next_row++;
    pthread_mutex_unlock(&J->mu);
    if (rr >= J->nrows) break;
    int r = J->r0 + rr;
    for (int c = 0; c < J->cols; ++c) {
      int st = pixel_depths(J->geom, J->f, J->wires, J->K, J->edge, r, c, d);
      if (st) {
        pthread_mutex_lock(&J->mu);
        J->status = st;
        pthread_mutex_unlock(&J->mu);
        break;
      }
      size_t pix = (size_t)r * J->cols + c;
      for (int k = 0; k + 1 < J->K; ++k) {
        int64_t a = J->images[(size_t)k * plane + pix];
        int64_t b = J->images[(size_t)(k + 1) * plane + pix];
        dI[k] = J->edge == OR_LEADING ? a - b : b - a;
      }
      apportion_pixel(d, dI, J->K, J->e, J->B,
                      J->out + (size_t)rr * J->cols + c, ostride);
    }
  }
  free(d);
  free(dI);
  return NULL;
}

/* Full reconstruction of output rows r0 .. r0+nrows-1.
 * images: [K][rows][cols] uint16 (the whole ROI), out: [B][nrows][cols]
 * (overwritten), nthreads >= 1 worker threads over rows. */
int oracle_reconstruct(const double *geom, int rows, int cols,
                       const double *wires, int K, int edge,
                       const uint16_t *images, const double *e, int B, int r0,
                       int nrows, int nthreads, double *out) {
  if (K < 2 || B < 1 || rows < 0 || cols < 0 || r0 < 0 || nrows < 0 ||
      r0 + nrows > rows || nthreads < 1)
    return OR_BAD_ARG;
  for (int j = 0; j + 1 <= B; ++j)
    if (!(e[j + 1] > e[j])) return OR_BAD_ARG;
  or_frame f;
  int st = make_frame(geom, wires, K, &f);
  if (st) return st;
  memset(out, 0, sizeof(double) * (size_t)B * (size_t)nrows * (size_t)cols);
  or_job J = {geom, &f, wires, K, edge, cols, rows, images, e, B, r0, nrows,
              out, 0, PTHREAD_MUTEX_INITIALIZER, OR_OK};
  if (nthreads > nrows) nthreads = nrows > 0 ? nrows : 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  if (!th) return OR_NO_MEMORY;
  int started = 0;
  for (int i = 0; i < nthreads; ++i)
    if (pthread_create(&th[i], NULL, worker, &J) == 0) ++started;
  if (started == 0) worker(&J);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  free(th);
  return J.status;
}
