// Plan builder: FP64 per-pixel (or per-row) geometry constants, validation,
// device upload and launch-shape choice.  Host code.
//
// The depth model is the tangent condition described in dr_internal.h.  The
// plan computes, in FP64, the projected frame, the per-group constants
// (D, L0, Q0), the per-step constants (z_k, eta_k), every depth sequence
// needed for the monotonicity check, and the fixed-point scale that makes
// the kernels' position differences exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "dr_internal.h"

namespace dr {

static thread_local char g_msg[512];

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
}

dr_status cuda_fail(const char *what, int err) {
  set_error("%s: %s", what, cudaGetErrorString((cudaError_t)err));
  return DR_ERR_CUDA;
}

namespace {

struct V3 {
  double x, y, z;
};
V3 v3(const double *p) { return {p[0], p[1], p[2]}; }
V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
double norm(V3 a) { return std::sqrt(dot(a, a)); }
bool finite3(const double *p) {
  return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]);
}

// FP64 solution of the tangent condition for one (group, step): projected
// depth t.  Fixed point on the exact form t = z + Q0 + (a + sR dL(t))/(D-eta);
// the map contracts by ~R/D per pass, three passes reach rounding level.
double solve_t(double Y, double Z, double y0, double sR, double D, double L0,
               double Q0, double z, double eta) {
  double Dm = D - eta;
  double a = y0 * z + eta * (z - Z + Q0);
  double t = z + Q0 + a / Dm;
  for (int it = 0; it < 3; ++it) {
    double u = Z - t;
    double L = std::sqrt(Y * Y + u * u);
    double dL = t * (t - 2.0 * Z) / (L + L0);
    t = z + Q0 + (a + sR * dL) / Dm;
  }
  return t;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Device memory of plans: a stream-ordered pool per device (allocation and
// release on a library stream), so that building and destroying plans while
// other work runs neither waits for the device nor makes it wait, as
// cudaMalloc / cudaFree can.  The pool keeps up to 4 GiB of released blocks
// for later plans.
struct PlanMemory {
  cudaMemPool_t pool = nullptr;
  cudaStream_t stream = nullptr;
  bool ok = false;
};
std::mutex g_plan_mem_mu;
PlanMemory g_plan_mem[64];

dr_status plan_memory(int dev, PlanMemory **out) {
  if (dev < 0 || dev >= 64) {
    set_error("dr_plan: device %d out of range", dev);
    return DR_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_plan_mem_mu);
  PlanMemory &m = g_plan_mem[dev];
  if (!m.ok) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(&m.pool, &props);
    if (e == cudaSuccess) {
      uint64_t keep = uint64_t(4) << 30;
      e = cudaMemPoolSetAttribute(m.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail("dr_plan: memory pool", e);
    m.ok = true;
  }
  *out = &m;
  return DR_OK;
}

}  // namespace
}  // namespace dr

using namespace dr;

namespace {
struct Group64 {
  double Y, Z, D, L0, Q0;
};
}  // namespace

namespace dr {
// Launch shape: smem layout sizes for the two kernels (see dr_device.cuh).
int rows_smem_bytes(int K, int Kpad, int B, int tile_cols, bool f64) {
  size_t s = 128;                                          // mbarrier slot
  s += align_up((size_t)Kpad * tile_cols * 2, 16);         // image tile
  s += align_up((size_t)K * (f64 ? 8 : 4), 16);            // depth positions
  s += align_up((size_t)row_table_entries(B) * 8, 16);     // header + (k, f) table
  return (int)s;
}

int pixels_smem_bytes(int K, int Kpad, int B, int tile_cols, bool f64) {
  size_t s = 128;
  s += align_up((size_t)Kpad * tile_cols * 2, 16);                 // image tile
  s += align_up((size_t)K * tile_cols * (f64 ? 8 : 4), 16);        // depth positions
  s += align_up((size_t)(B + 1) * (f64 ? 8 : 4), 16);              // edges
  return (int)s;
}

int pixels_poly_smem_bytes(int K, int Kpad, int B, int tile_cols) {
  size_t s = 128;
  s += align_up((size_t)Kpad * tile_cols * 2, 16);                 // image tile
  s += align_up((size_t)K * 8, 16);                                // steps (dz, zfx)
  s += align_up((size_t)(B + 1) * 4, 16);                          // edges
  return (int)s;
}

// TMA chunks of kc steps: at most 256 steps per box, and every chunk's
// shared-memory destination (kc * tile_cols * 2 bytes apart) 128-byte aligned,
// as tensor copies require.  Picks the chunk count with the least padding.
void choose_chunks(int K, int tile_cols, int *kc, int *nchunks) {
  int g = 64, x = tile_cols;
  while (x % 2 == 0 && g > 1) {
    x /= 2;
    g /= 2;
  }
  const int m = g;  // kc must be a multiple of m = 64 / gcd(tile_cols, 64)
  int nmin = (K + 255) / 256;
  int best_n = nmin, best_c = 0, best_pad = 1 << 30;
  for (int n = nmin; n <= nmin + 4; ++n) {
    int c = (K + n - 1) / n;
    c = (c + m - 1) / m * m;
    if (c > 256) continue;
    int pad = n * c - K;
    if (pad < best_pad) {
      best_pad = pad;
      best_n = n;
      best_c = c;
    }
  }
  *nchunks = best_n;
  *kc = best_c;
}

}  // namespace dr

// One monotone plan.  side != 0 fixes the tangent side s (the wire edge
// chosen by the whole scan's travel), for the runs of a composite plan whose
// own travel may point the other way.
// shift_cap bounds the fixed-point scale (a retry after the check found a
// step too long for it or positions off the FP64 solution); max_mode bounds
// the form of the FP32 remainder (a retry after the check found a cheaper
// form not accurate enough).
static dr_status plan_one(bool intervals, const dr_geometry *g, const double *wires, int32_t K,
                          const double *edges, int32_t B, const dr_plan_options *opt_in,
                          int side, dr_plan_t **out, int shift_cap = 40,
                          int max_mode = kDepthPoly) {
  if (out) *out = nullptr;
  if (opt_in && opt_in->depth_form > 0) max_mode = std::min(max_mode, opt_in->depth_form - 1);
  if (!g || !wires || !edges || !out) {
    set_error("dr_plan: null argument");
    return DR_ERR_INVALID_ARG;
  }
  dr_plan_options opt;
  std::memset(&opt, 0, sizeof(opt));
  if (opt_in) opt = *opt_in;
  if (K < 2 || B < 1 || g->rows < 0 || g->cols < 0) {
    set_error("dr_plan: need K >= 2, B >= 1, rows, cols >= 0 (K=%d B=%d)", K, B);
    return DR_ERR_INVALID_ARG;
  }
  if (g->rows > 65535) {
    set_error("dr_plan: rows > 65535 not supported");
    return DR_ERR_UNSUPPORTED;
  }
  if (g->edge != DR_EDGE_LEADING && g->edge != DR_EDGE_TRAILING) {
    set_error("dr_plan: edge must be DR_EDGE_LEADING, DR_EDGE_TRAILING or DR_EDGE_BOTH");
    return DR_ERR_INVALID_ARG;
  }
  if ((opt.out_dtype != DR_OUT_F32 && opt.out_dtype != DR_OUT_BF16) ||
      (opt.geom_precision != DR_GEOM_FP32 && opt.geom_precision != DR_GEOM_FP64) ||
      opt.tile_cols < 0 || opt.bin_groups < 0 || opt.depth_form < 0 || opt.depth_form > 3) {
    set_error("dr_plan: bad options");
    return DR_ERR_INVALID_ARG;
  }
  for (int j = 0; j <= B; ++j) {
    if (!std::isfinite(edges[j]) || (j > 0 && !(edges[j] > edges[j - 1]))) {
      set_error("dr_plan: bin edges must be finite and strictly increasing (j=%d)", j);
      return DR_ERR_INVALID_ARG;
    }
  }
  for (int k = 0; k < K; ++k)
    if (!finite3(wires + 3 * k)) {
      set_error("dr_plan: wire centre %d not finite", k);
      return DR_ERR_INVALID_ARG;
    }
  if (!finite3(g->beam_origin) || !finite3(g->beam_dir) || !finite3(g->det_origin) ||
      !finite3(g->row_step) || !finite3(g->col_step) || !finite3(g->wire_axis) ||
      !std::isfinite(g->wire_radius) || !(g->wire_radius > 0.0)) {
    set_error("dr_plan: geometry not finite or radius <= 0");
    return DR_ERR_INVALID_ARG;
  }

  // ---- projected frame ----
  V3 ax = v3(g->wire_axis), bd = v3(g->beam_dir), O = v3(g->beam_origin);
  if (!(norm(ax) > 0) || !(norm(bd) > 0)) {
    set_error("dr_plan: zero wire axis or beam direction");
    return DR_ERR_GEOMETRY;
  }
  ax = (1.0 / norm(ax)) * ax;
  bd = (1.0 / norm(bd)) * bd;
  V3 bp = bd - dot(bd, ax) * ax;
  double nb = norm(bp);
  if (!(nb > 1e-9)) {
    set_error("dr_plan: beam runs along the wire axis");
    return DR_ERR_GEOMETRY;
  }
  V3 e2 = (1.0 / nb) * bp;
  V3 c0 = v3(wires) - O;
  V3 w = c0 - dot(c0, ax) * ax;
  w = w - dot(w, e2) * e2;
  if (!(norm(w) > 0)) {
    set_error("dr_plan: first wire centre lies on the beam");
    return DR_ERR_GEOMETRY;
  }
  V3 e1 = (1.0 / norm(w)) * w;
  const double R = g->wire_radius;

  std::vector<double> yk(K), zk(K);
  for (int k = 0; k < K; ++k) {
    V3 c = v3(wires + 3 * k) - O;
    yk[k] = dot(c, e1);
    zk[k] = dot(c, e2);
  }
  const double y0 = yk[0];
  const double travel = zk[K - 1] - zk[0];
  if (travel == 0.0) {
    set_error("dr_plan: wire does not travel along the projected beam");
    return DR_ERR_GEOMETRY;
  }
  const bool reverse = travel < 0.0;
  const double sgn = side != 0 ? (double)side
                               : (reverse ? -1.0 : 1.0) * (g->edge == DR_EDGE_LEADING ? 1.0 : -1.0);
  const double sR = sgn * R;
  bool has_eta = false;
  double ymin = yk[0], ymax = yk[0];
  for (int k = 0; k < K; ++k) {
    has_eta |= (yk[k] != y0);
    ymin = std::min(ymin, yk[k]);
    ymax = std::max(ymax, yk[k]);
  }
  if (!(ymin > R)) {
    set_error("dr_plan: wire overlaps the beam (distance %.6g <= radius)", ymin);
    return DR_ERR_GEOMETRY;
  }

  const int H = g->rows, W = g->cols;
  const long long P = (long long)H * W;
  V3 dorg = v3(g->det_origin) - O, rs = v3(g->row_step), cs = v3(g->col_step);
  // pixel coordinates are affine in (r, c): Y = Y00 + r*Yr + c*Yc
  double Y00 = dot(dorg, e1), Z00 = dot(dorg, e2);
  double Yr = dot(rs, e1), Zr = dot(rs, e2), Yc = dot(cs, e1), Zc = dot(cs, e2);
  if (P > 0) {
    double Ymin = 1e300;
    for (int cr = 0; cr < 4; ++cr) {
      double r = (cr & 1) ? H - 1 : 0, c = (cr & 2) ? W - 1 : 0;
      Ymin = std::min(Ymin, Y00 + r * Yr + c * Yc);
    }
    if (!(Ymin - ymax > R)) {
      set_error("dr_plan: wire not between beam and detector (min gap %.6g mm)",
                Ymin - ymax);
      return DR_ERR_GEOMETRY;
    }
  }
  double cs_n = norm(cs);
  bool rows_shared = std::fabs(Yc) + std::fabs(Zc) <= 1e-13 * std::max(cs_n, 1e-300);
  if (opt.force_pixels) rows_shared = false;
  if (W == 0 || H == 0) rows_shared = true;

  const long long G = rows_shared ? H : P;
  if (!rows_shared && P > (1LL << 31) / 2) {
    set_error("dr_plan: too many pixels for the per-pixel kernel");
    return DR_ERR_UNSUPPORTED;
  }
  auto group_at = [&](double r, double c) {
    Group64 q;
    q.Y = Y00 + r * Yr + c * Yc;
    q.Z = Z00 + r * Zr + c * Zc;
    q.D = q.Y - y0;
    q.L0 = std::sqrt(q.Y * q.Y + q.Z * q.Z);
    q.Q0 = (-y0 * q.Z + sR * q.L0) / q.D;
    return q;
  };

  // Steps in processing order (increasing depth).
  std::vector<double> zp(K), ep(K);
  double zlo = 1e300, zhi = -1e300;
  for (int k = 0; k < K; ++k) {
    int src = reverse ? K - 1 - k : k;
    zp[k] = zk[src];
    ep[k] = yk[src] - y0;
    zlo = std::min(zlo, zp[k]);
    zhi = std::max(zhi, zp[k]);
  }

  // ---- FP64 estimates on a sample of groups ----
  // The sample sets the fixed-point scale and the form of the remainder; the
  // device check after the upload computes every (group, step) as the
  // kernels will and decides whether the plan stands.  Rows: every 8th row
  // and the last; pixels: every 64th row and column and the last ones (all
  // four corners).  A sampled sequence that does not increase ends the plan
  // here.
  double tmin = 1e300, tmax = -1e300, minstep = 1e300, maxstep = 0.0, remmax = 0.0, qmax = 0.0;
  long long bad_r = -1, bad_c = -1;
  int bad_k = -1;
  auto sample = [&](double r, double c) {
    const Group64 q = group_at(r, c);
    qmax = std::max(qmax, std::fabs(q.Q0));
    double prev = 0;
    for (int k = 0; k < K; ++k) {
      const double t = solve_t(q.Y, q.Z, y0, sR, q.D, q.L0, q.Q0, zp[k], ep[k]);
      tmin = std::min(tmin, t);
      tmax = std::max(tmax, t);
      remmax = std::max(remmax, std::fabs(t - zp[k] - q.Q0));
      if (k > 0) {
        const double st = t - prev;
        if (intervals) {  // any order: only the smallest nonzero step is kept
          if (st != 0) minstep = std::min(minstep, std::fabs(st));
        } else if (!(st > 0)) {
          if (bad_k < 0) {
            bad_r = (long long)r;
            bad_c = (long long)c;
            bad_k = k;
          }
        } else {
          minstep = std::min(minstep, st);
          maxstep = std::max(maxstep, st);
        }
      }
      prev = t;
    }
  };
  if (P > 0) {
    auto picks = [](long long n, long long stride) {  // 0, stride, 2 stride, ..., n - 1
      std::vector<long long> v;
      for (long long i = 0; i < n; i += stride) v.push_back(i);
      if (v.back() != n - 1) v.push_back(n - 1);
      return v;
    };
    const std::vector<long long> prow = picks(H, rows_shared ? 8 : 64);
    const std::vector<long long> pcol = rows_shared ? std::vector<long long>{0} : picks(W, 64);
    for (long long r : prow)
      for (long long c : pcol) sample((double)r, (double)c);
    if (bad_k >= 0) {
      if (rows_shared)
        set_error("dr_plan: depth of row %lld not monotone at step %d", bad_r, bad_k);
      else
        set_error("dr_plan: depth of pixel (%lld,%lld) not monotone at step %d", bad_r, bad_c,
                  bad_k);
      return DR_ERR_NONMONOTONIC;
    }
  }
  if (P == 0) {
    tmin = edges[0] * nb;
    tmax = edges[B] * nb;
    minstep = 1.0;
  }

  // ---- fixed-point scale ----
  // positions (relative to the origin) get a budget of 2^29 grid units, four
  // times below the int32 limit, which covers any range the sample missed;
  // the device check measures the true range and the distance of every
  // position from FP64, and a plan whose positions went wrong is rebuilt on
  // a coarser grid
  double lo = std::min(tmin, edges[0] * nb), hi = std::max(tmax, edges[B] * nb);
  double origin = 0.5 * (lo + hi);
  double mag = 0.5 * (hi - lo) * 1.001 + 1e-9;
  for (int k = 0; k < K; ++k) mag = std::max(mag, std::fabs(zp[k] - origin));
  mag = std::max(mag, qmax * 1.05);
  mag = std::max(mag, remmax * 1.5);
  int shift = (int)std::floor(std::log2((double)(1 << 29) / mag));
  shift = std::min(shift, shift_cap);
  // FP32 geometry of the running-sum kernels: every step must stay below
  // 2^23 grid units (exact conversion of position differences); the check
  // below confirms it for every (group, step) and retries with a smaller
  // scale if a step the sample missed is longer
  const bool fx_walk = !intervals && opt.geom_precision == DR_GEOM_FP32;
  if (fx_walk && maxstep > 0.0)
    shift = std::min(shift, (int)std::floor(std::log2(0.9 * kMaxStepUnits / maxstep)));
  if (shift < 12) {
    set_error("dr_plan: depth range too large for 32-bit fixed point");
    return DR_ERR_UNSUPPORTED;
  }
  const double scale = std::ldexp(1.0, shift);
  if (minstep == 1e300) minstep = 0.0;  // interval kernel, no nonzero step seen
  // FP32 geometry positions carry a few grid units of error, so an interval
  // of the running-sum kernels must span many units; the interval kernel
  // apportions its shorter intervals with FP64 depths, and FP64 geometry
  // computes positions and fractions in FP64
  if (P > 0 && !intervals && opt.geom_precision == DR_GEOM_FP32 && minstep > 0.0 &&
      minstep * scale < kMinStepUnits) {
    set_error("dr_plan: depth steps (%.3g mm) too small for the fixed-point grid", minstep);
    return DR_ERR_UNSUPPORTED;
  }

  // ---- form of the FP32 remainder (dr_tables.h) ----
  // Polynomial: a wire at one distance from the beam (eta = 0) and a
  // remainder that rounds by the 1.5 * 2^23 construction.  Series: the
  // bound of its first dropped term, n / (2 L0) * 5/64 * x^3 / (1 - x), over
  // the ROI (|t| <= T, |Z| <= Zmax, L0 >= Y >= Ymin), carried into the
  // remainder (times R / D) in grid units, below 0.01.  Otherwise exact.
  // (the interval kernel evaluates the same FP32 positions, so its plans
  // take the same forms; the check below bounds their distance from FP64)
  int mode = kDepthExact;
  const bool fx_pos = opt.geom_precision == DR_GEOM_FP32;
  if (fx_pos && !has_eta && P > 0 && remmax * scale < (double)(1 << 20)) {
    double Zmax = 0.0, Ymin = 1e300;
    for (int cr = 0; cr < 4; ++cr) {
      const double r = (cr & 1) ? H - 1 : 0, cc = (cr & 2) ? W - 1 : 0;
      Zmax = std::max(Zmax, std::fabs(Z00 + r * Zr + cc * Zc));
      Ymin = std::min(Ymin, Y00 + r * Yr + cc * Yc);
    }
    const double T = std::max(std::fabs(tmin), std::fabs(tmax)) * 1.01 + 1e-6;
    const double n = T * (T + 2.0 * Zmax), x = n / (Ymin * Ymin);
    bool series_ok = false;
    if (Ymin > y0 && x < 0.5) {
      const double drop = n / (2.0 * Ymin) * (5.0 / 64.0) * x * x * x / (1.0 - x);
      series_ok = R / (Ymin - y0) * drop * scale < 0.01;
    }
    if (max_mode >= kDepthPoly)
      mode = kDepthPoly;
    else if (max_mode >= kDepthSeries && series_ok)
      mode = kDepthSeries;
  }
  const double zc = 0.5 * (zlo + zhi), zh = 0.5 * (zhi - zlo);

  // ---- host tables (steps, edges; the groups are computed on the device) ----
  std::vector<StepC> sc(K);
  std::vector<StepD> sd(K);
  for (int k = 0; k < K; ++k) {
    sc[k].zf = (float)zp[k];
    sc[k].eta = (float)ep[k];
    sc[k].zfx = (int32_t)std::llround((zp[k] - origin) * scale);
    sc[k].dz = (float)(zp[k] - zc);
    sd[k] = {zp[k], ep[k]};
  }
  std::vector<int32_t> efx(B + 1);
  std::vector<double> e64(B + 1);
  for (int j = 0; j <= B; ++j) {
    double t = edges[j] * nb - origin;
    e64[j] = t;
    double f = std::llround(t * scale);
    efx[j] = (int32_t)std::max(std::min(f, 2147483000.0), -2147483000.0);
  }

  // ---- launch shape ----
  dr_plan_t *p = new (std::nothrow) dr_plan_t();
  if (!p) {
    set_error("dr_plan: host allocation failed");
    return DR_ERR_OOM;
  }
  p->rows = H;
  p->cols = W;
  p->K = K;
  p->B = B;
  p->edge = g->edge;
  p->kernel = intervals ? DR_KERNEL_INTERVALS : rows_shared ? DR_KERNEL_ROWS : DR_KERNEL_PIXELS;
  p->pixel_groups = rows_shared ? 0 : 1;
  p->out_dtype = opt.out_dtype;
  p->geom_prec = opt.geom_precision;
  p->shift = shift;
  p->nb = nb;
  p->depth_min = tmin / nb;
  p->depth_max = tmax / nb;
  p->min_step = minstep / nb;
  const bool f64 = opt.geom_precision == DR_GEOM_FP64;
  Tuning t;
  auto smem_for = [&](int tc) {
    int kc, n;
    choose_chunks(K, tc, &kc, &n);
    if (rows_shared) return rows_smem_bytes(K, kc * n, B, tc, f64);
    return mode == kDepthPoly ? pixels_poly_smem_bytes(K, kc * n, B, tc)
                              : pixels_smem_bytes(K, kc * n, B, tc, f64);
  };
  if (intervals) {
    // 32 pixels x all steps per CTA; bins in windows of int32 accumulators
    // sized for three CTAs per SM (FP32 geometry), else two, else one: the
    // most CTAs whose windows still hold 256 bins (or all of them)
    t.ppt = 1;
    t.tile_cols = kIntervalTile;
    t.bin_groups = 1;
    p->threads = 512;  // lane = pixel, warp = a chunk of intervals
    if (K > 65535) {
      delete p;
      set_error("dr_plan: the interval kernel takes at most 65535 steps");
      return DR_ERR_UNSUPPORTED;
    }
  } else if (rows_shared) {
    t.ppt = (W % 4 == 0) ? 4 : 1;
    int tc = opt.tile_cols;
    if (tc == 0) {
      tc = 128;
      int wr = (W + 7) / 8 * 8;
      if (wr < tc) tc = std::max(wr, 8);
      // two CTAs per SM when the step count allows it
      while (tc > 32 && 2 * (smem_for(tc) + 1024) > kSmemPerSm) tc /= 2;
    }
    if (tc % 8 != 0 || tc > 256 || tc < 8 || tc % t.ppt != 0) {
      delete p;
      set_error("dr_plan: tile_cols must be a multiple of 8 in [8, 256]");
      return DR_ERR_INVALID_ARG;
    }
    t.tile_cols = tc;
    int lanes = tc / t.ppt;
    int bg = opt.bin_groups;
    if (bg == 0) {
      bg = std::max(1, 512 / lanes);
      while (bg > 1 && B / bg < 16) bg /= 2;
      while (lanes * bg > 512) bg /= 2;
    }
    if (bg < 1 || lanes * bg > 512) {
      delete p;
      set_error("dr_plan: bad bin_groups");
      return DR_ERR_INVALID_ARG;
    }
    t.bin_groups = bg;
    p->threads = lanes * bg;
  } else {
    // per-pixel kernel: tile_cols pixels (slabs of up to 32) x bin_groups shares
    t.ppt = 1;
    int tc = opt.tile_cols == 0 ? 32 : opt.tile_cols;
    if (!(tc == 8 || tc == 16 || (tc % 32 == 0 && tc <= 256))) {
      delete p;
      set_error("dr_plan: per-pixel tile_cols must be 8, 16 or a multiple of 32 up to 256");
      return DR_ERR_INVALID_ARG;
    }
    t.tile_cols = tc;
    int bg = opt.bin_groups;
    if (bg == 0) {
      bg = std::max(1, 512 / tc);
      while (bg > 1 && B / bg < 16) bg /= 2;
    }
    if (bg < 1 || tc * bg > 512) {
      delete p;
      set_error("dr_plan: per-pixel tile_cols x bin_groups must be at most 512");
      return DR_ERR_INVALID_ARG;
    }
    t.bin_groups = bg;
    p->threads = tc * bg;
  }
  choose_chunks(K, t.tile_cols, &t.kc, &t.nchunks);
  if (t.kc < 1 || t.kc > 256 || ((size_t)t.kc * t.tile_cols * 2) % 128 != 0) {
    delete p;
    set_error("dr_plan: no aligned TMA chunking for K=%d, tile_cols=%d", K, t.tile_cols);
    return DR_ERR_UNSUPPORTED;
  }
  if (intervals) {
    const bool per_pixel = !rows_shared;
    const size_t fixed = (size_t)intervals_smem(K, t.kc * t.nchunks, B, 0, f64, per_pixel);
    const size_t per_bin = (size_t)kIntervalTile * 4;
    const size_t want = fixed + per_bin * (size_t)std::min(B, 256);
    p->iv_ctas = (!f64 && want <= (size_t)(kSmemPerSm / 3 - 1024)) ? 3
                 : want <= (size_t)(kSmemPerSm / 2 - 1024)         ? 2
                                                                    : 1;
    const size_t budget = p->iv_ctas == 1 ? (size_t)kSmemPerCtaMax
                                          : (size_t)(kSmemPerSm / p->iv_ctas - 1024);
    const long long win = fixed < budget ? (long long)((budget - fixed) / per_bin) : 0;
    if (win < std::min(B, 32)) {
      delete p;
      set_error("dr_plan: %d steps x %d bins do not fit the interval kernel's shared memory", K,
                B);
      return DR_ERR_UNSUPPORTED;
    }
    p->window = (int)std::min<long long>(win, B);
    t.bin_groups = p->window;
    p->smem_bytes = intervals_smem(K, t.kc * t.nchunks, B, p->window, f64, per_pixel);
  } else {
    p->smem_bytes = smem_for(t.tile_cols);
  }
  if (p->smem_bytes > kSmemPerCtaMax) {
    delete p;
    set_error("dr_plan: %d steps x %d columns do not fit in shared memory", K, t.tile_cols);
    return DR_ERR_UNSUPPORTED;
  }
  p->tune = t;

  // ---- device upload (one allocation) ----
  // the small tables first (uploaded from the host), then the per-group
  // constants (computed on the device) and the row tables
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = align_up(off, 256);
    off = o + bytes;
    return o;
  };
  size_t o_sc = take(sizeof(StepC) * K), o_efx = take(sizeof(int32_t) * (B + 1));
  size_t o_sd = take(sizeof(StepD) * K), o_e64 = take(sizeof(double) * (B + 1));
  size_t o_err = take(sizeof(int32_t) * 4);
  size_t o_chk = take(sizeof(PlanCheck));
  const size_t host_bytes = align_up(off, 256);
  size_t o_gc = take(sizeof(GroupC) * (size_t)G), o_gd = take(sizeof(GroupD) * (size_t)G);
  // per-row (k, f) tables, built once on the device below (rows kernel only;
  // above 1 GiB the tiles build their own)
  const int tab_stride = row_table_entries(B);
  const size_t tab_bytes = (size_t)H * tab_stride * 8;
  const bool row_tables =
      p->kernel == DR_KERNEL_ROWS && H > 0 && W > 0 && tab_bytes <= (size_t(1) << 30);
  size_t o_tab = row_tables ? take(tab_bytes) : 0;
  size_t total = align_up(off, 256);
  void *blk = nullptr;
  PlanMemory *pm = nullptr;
  cudaError_t ce = cudaGetDevice(&p->device);
  if (ce != cudaSuccess) {
    delete p;
    return cuda_fail("dr_plan: cudaGetDevice", ce);
  }
  dr_status ms = plan_memory(p->device, &pm);
  if (ms != DR_OK) {
    delete p;
    return ms;
  }
  ce = cudaMallocFromPoolAsync(&blk, total, pm->pool, pm->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(pm->stream);
  if (ce != cudaSuccess) {
    delete p;
    if (ce == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      set_error("dr_plan: device allocation of %zu bytes failed", total);
      return DR_ERR_OOM;
    }
    return cuda_fail("dr_plan: device allocation", ce);
  }
  std::vector<char> host(host_bytes, 0);
  std::memcpy(host.data() + o_sc, sc.data(), sizeof(StepC) * K);
  std::memcpy(host.data() + o_efx, efx.data(), sizeof(int32_t) * (B + 1));
  std::memcpy(host.data() + o_sd, sd.data(), sizeof(StepD) * K);
  std::memcpy(host.data() + o_e64, e64.data(), sizeof(double) * (B + 1));
  ce = cudaMemcpy(blk, host.data(), host_bytes, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    cudaFreeAsync(blk, pm->stream);
    delete p;
    return cuda_fail("dr_plan: upload", ce);
  }
  char *b = (char *)blk;
  p->dev_block = blk;
  p->device_bytes = total;
  GroupsParams gq;
  std::memset(&gq, 0, sizeof(gq));
  gq.Y00 = Y00;
  gq.Yr = Yr;
  gq.Yc = Yc;
  gq.Z00 = Z00;
  gq.Zr = Zr;
  gq.Zc = Zc;
  gq.y0 = y0;
  gq.sR = sR;
  gq.scale = scale;
  gq.zc = zc;
  gq.zh = zh;
  gq.ngroups = G;
  gq.W = W;
  gq.rows_shared = rows_shared ? 1 : 0;
  gq.mode = mode;
  dr_status gs = run_groups(gq, reinterpret_cast<GroupC *>(b + o_gc),
                            reinterpret_cast<GroupD *>(b + o_gd));
  if (gs != DR_OK) {
    dr_plan_destroy(p);
    return gs;
  }
  Consts &c = p->c;
  c.grp = (const GroupC *)(b + o_gc);
  c.stp = (const StepC *)(b + o_sc);
  c.efx = (const int32_t *)(b + o_efx);
  c.grp64 = (const GroupD *)(b + o_gd);
  c.stp64 = (const StepD *)(b + o_sd);
  c.e64 = (const double *)(b + o_e64);
  c.err = (int32_t *)(b + o_err);
  c.K = K;
  c.H = H;
  c.W = W;
  c.B = B;
  c.has_eta = has_eta ? 1 : 0;
  c.reverse = reverse ? 1 : 0;
  c.y0 = (float)y0;
  c.sR = (float)sR;
  c.scale = (float)scale;
  c.y0d = y0;
  c.sRd = sR;
  c.origin = origin;
  c.nb = nb;
  // trailing edge: the reverse change; reversed step order: negated sweep
  c.out_sign = (float)((g->edge == DR_EDGE_LEADING ? 1.0 : -1.0) * (reverse ? -1.0 : 1.0));
  c.tab = nullptr;
  c.tab_stride = tab_stride;
  c.depth_mode = mode;
  p->checked_groups = 0;
  p->max_dev_units = -1;
  p->max_step_units = 0;
  p->one_adv = 0;
  if (P > 0) {
    // every (group, step) as the kernels compute it (and, for FP32
    // geometry, against FP64): order for the running-sum kernels, range and
    // accuracy for all
    PlanCheck res;
    dr_status st =
        run_plan_check(p, (int)G, !intervals, reinterpret_cast<PlanCheck *>(b + o_chk), &res);
    if (st != DR_OK) {
      dr_plan_destroy(p);
      return st;
    }
    if (res.bad != ~0ull) {
      const long long gi = (long long)(res.bad >> 32);
      const int k = (int)(res.bad & 0xffffffffu);
      dr_plan_destroy(p);
      if (fx_walk && res.max_step >= kMaxStepUnits && res.min_step >= kMinStepUnits &&
          shift > 12)
        return plan_one(intervals, g, wires, K, edges, B, opt_in, side, out, shift - 1,
                        max_mode);
      const long long r = rows_shared ? gi : gi / std::max(W, 1);
      const long long cc = rows_shared ? 0 : gi % std::max(W, 1);
      if (!fx_walk || res.min_step <= 0) {
        set_error("dr_plan: depth of %s (%lld,%lld) not increasing at step %d",
                  rows_shared ? "row" : "pixel", r, cc, k);
        return DR_ERR_NONMONOTONIC;
      }
      set_error("dr_plan: a depth step of %s (%lld,%lld) at step %d is outside the "
                "fixed-point grid's range", rows_shared ? "row" : "pixel", r, cc, k);
      return DR_ERR_UNSUPPORTED;
    }
    if (!f64) {
      if (mode != kDepthExact && res.max_dev > 4) {  // the cheaper form is not good enough
        dr_plan_destroy(p);
        return plan_one(intervals, g, wires, K, edges, B, opt_in, side, out, shift_cap,
                        mode - 1);
      }
      if (res.max_dev > 64) {  // positions off the FP64 solution: a coarser grid
        dr_plan_destroy(p);
        if (shift <= 12) {
          set_error("dr_plan: FP32 depth positions off the FP64 solution by %d grid units",
                    res.max_dev);
          return DR_ERR_UNSUPPORTED;
        }
        return plan_one(intervals, g, wires, K, edges, B, opt_in, side, out, shift - 1,
                        max_mode);
      }
      p->max_dev_units = res.max_dev;
    }
    p->checked_groups = G;
    p->depth_min = ((double)res.tmin / scale + origin) / nb;
    p->depth_max = ((double)res.tmax / scale + origin) / nb;
    if (!intervals) {
      p->max_step_units = res.max_step;
      p->min_step = (double)res.min_step / scale / nb;
    }
    if (fx_walk) {
      long long maxbin = 0;
      for (int j = 0; j < B; ++j) maxbin = std::max(maxbin, (long long)efx[j + 1] - efx[j]);
      p->one_adv = res.min_step >= maxbin ? 1 : 0;
    }
  }
  if (row_tables) {
    dr_status st = build_plan_tables(p, reinterpret_cast<int2 *>(b + o_tab));
    if (st != DR_OK) {
      dr_plan_destroy(p);
      return st;
    }
    c.tab = reinterpret_cast<const int2 *>(b + o_tab);
  }
  *out = p;
  return DR_OK;
}

// The public plan.  A wire path whose projected position along the beam
// changes direction (a back-and-forth scan) is split into monotone runs that
// share their turning steps; each run is a plan of its own that keeps the
// whole scan's wire edge, and the runs' outputs add up (the apportioning is a
// sum over intervals).  DR_EDGE_BOTH is the mean of the leading- and
// trailing-edge reconstructions.  Single-run, single-edge scans are one plan.
// Depth sequences that are not monotone within a run (a wire that also moves
// across the beam, two steps at the same position) take the interval kernel,
// which adds every interval by itself and accepts any order.
static dr_status plan_parts(bool intervals, const dr_geometry *g, const double *wires,
                            int32_t K, const double *edges, int32_t B,
                            const dr_plan_options *opt, const std::vector<int> &starts,
                            double travel, dr_plan_t **out) {
  const bool both = g->edge == DR_EDGE_BOTH;
  if (starts.size() == 1 && !both)
    return plan_one(intervals, g, wires, K, edges, B, opt, 0, out);
  dr_plan_t *top = new (std::nothrow) dr_plan_t();
  if (!top) {
    set_error("dr_plan: host allocation failed");
    return DR_ERR_OOM;
  }
  const int nedges = both ? 2 : 1;
  for (int ei = 0; ei < nedges; ++ei) {
    dr_geometry ge = *g;
    ge.edge = both ? (ei == 0 ? DR_EDGE_LEADING : DR_EDGE_TRAILING) : g->edge;
    const int side = (travel > 0 ? 1 : -1) * (ge.edge == DR_EDGE_LEADING ? 1 : -1);
    for (size_t r = 0; r < starts.size(); ++r) {
      const int k0 = starts[r];
      const int k1 = r + 1 < starts.size() ? starts[r + 1] : K - 1;  // inclusive
      dr_plan_t *part = nullptr;
      dr_status st =
          plan_one(intervals, &ge, wires + 3 * k0, k1 - k0 + 1, edges, B, opt, side, &part);
      if (st != DR_OK) {
        dr_plan_destroy(top);
        return st;
      }
      if (!top->parts.empty()) part->c.accumulate = 1;
      if (both) part->c.out_sign *= 0.5f;
      top->parts.push_back(part);
      top->part_k0.push_back(k0);
    }
  }
  const dr_plan_t *f = top->parts.front();
  top->rows = f->rows;
  top->cols = f->cols;
  top->K = K;
  top->B = B;
  top->edge = g->edge;
  top->kernel = f->kernel;
  top->pixel_groups = f->pixel_groups;
  top->window = f->window;
  top->iv_ctas = f->iv_ctas;
  top->out_dtype = f->out_dtype;
  top->geom_prec = f->geom_prec;
  top->shift = f->shift;
  top->nb = f->nb;
  top->depth_min = 1e300;
  top->depth_max = -1e300;
  top->min_step = 1e300;
  top->max_step_units = 0;
  top->max_dev_units = -1;
  top->one_adv = 1;
  top->checked_groups = 0;
  for (const dr_plan_t *q : top->parts) {
    top->depth_min = std::min(top->depth_min, q->depth_min);
    top->depth_max = std::max(top->depth_max, q->depth_max);
    top->min_step = std::min(top->min_step, q->min_step);
    top->device_bytes += q->device_bytes;
    top->max_step_units = std::max(top->max_step_units, q->max_step_units);
    top->max_dev_units = std::max(top->max_dev_units, q->max_dev_units);
    top->one_adv &= q->one_adv;
    top->checked_groups = std::max(top->checked_groups, q->checked_groups);
  }
  top->c = f->c;
  top->tune = f->tune;
  top->threads = f->threads;
  top->smem_bytes = f->smem_bytes;
  *out = top;
  return DR_OK;
}

extern "C" dr_status dr_plan(const dr_geometry *g, const double *wires, int32_t K,
                             const double *edges, int32_t B, const dr_plan_options *opt,
                             dr_plan_t **out) {
  TraceRange trace_("dr_plan");
  if (out) *out = nullptr;
  if (!g || !wires || !edges || !out) {
    set_error("dr_plan: null argument");
    return DR_ERR_INVALID_ARG;
  }
  if (K < 2 || B < 1) {
    set_error("dr_plan: need K >= 2, B >= 1 (K=%d B=%d)", K, B);
    return DR_ERR_INVALID_ARG;
  }
  const bool force_iv = opt && opt->force_intervals;
  // projected wire position along the beam (the plan's e2 coordinate):
  // monotone runs, or a repeated position (interval kernel)
  std::vector<int> starts{0};
  double travel = 0.0;
  bool repeated = false;
  {
    V3 ax = v3(g->wire_axis), bd = v3(g->beam_dir);
    if (norm(ax) > 0 && norm(bd) > 0 && finite3(wires) && finite3(wires + 3 * (K - 1))) {
      ax = (1.0 / norm(ax)) * ax;
      bd = (1.0 / norm(bd)) * bd;
      const V3 bp = bd - dot(bd, ax) * ax;
      if (norm(bp) > 1e-9) {
        const V3 e2 = (1.0 / norm(bp)) * bp;
        travel = dot(v3(wires + 3 * (K - 1)) - v3(wires), e2);
        int dir = 0;
        for (int k = 0; k + 1 < K && travel != 0.0; ++k) {
          if (!finite3(wires + 3 * k) || !finite3(wires + 3 * (k + 1))) break;
          const double dz = dot(v3(wires + 3 * (k + 1)) - v3(wires + 3 * k), e2);
          if (dz == 0.0) {
            repeated = true;
            break;
          }
          const int d = dz > 0 ? 1 : -1;
          if (dir != 0 && d != dir) starts.push_back(k);  // run turns at step k
          dir = d;
        }
      }
    }
  }
  if (travel == 0.0) {  // plan_one reports the geometry (or no travel)
    if (g->edge != DR_EDGE_BOTH) return plan_one(force_iv, g, wires, K, edges, B, opt, 0, out);
    set_error("dr_plan: the wire ends where it started along the beam (no travel)");
    return DR_ERR_GEOMETRY;
  }
  // Every kernel stages a tile's images for all the steps of a run in shared
  // memory; a run of more steps than kMaxRunSteps is cut into parts that
  // share their end steps (the apportioning is a sum over intervals, so the
  // parts add up to the whole; later parts add to the output).
  constexpr int kMaxRunSteps = 2048;
  auto cut_long = [&](const std::vector<int> &s) {
    std::vector<int> cut;
    for (size_t r = 0; r < s.size(); ++r) {
      const int k1 = r + 1 < s.size() ? s[r + 1] : K - 1;  // the run's last step
      for (int k = s[r]; k < k1; k += kMaxRunSteps - 1) cut.push_back(k);
    }
    return cut;
  };
  const std::vector<int> one = cut_long({0});
  starts = cut_long(starts);
  if (force_iv || repeated)
    return plan_parts(true, g, wires, K, edges, B, opt, one, travel, out);
  dr_status st = plan_parts(false, g, wires, K, edges, B, opt, starts, travel, out);
  if (st == DR_ERR_NONMONOTONIC)  // depth runs against its wire run somewhere
    return plan_parts(true, g, wires, K, edges, B, opt, one, travel, out);
  const bool shape_given = opt && (opt->tile_cols || opt->bin_groups);
  if (st == DR_ERR_UNSUPPORTED && !(opt && opt->force_pixels) && !shape_given) {
    // outside what the running-sum kernels take (depth steps too fine for
    // their fixed-point grid, tile memory): the interval kernel needs neither;
    // if it cannot take the scan either, the first reason is reported.  A
    // launch shape given by the caller is for the running-sum kernels, so a
    // shape that does not fit is reported rather than replaced by the
    // interval kernel.
    char first[sizeof(g_msg)];
    std::memcpy(first, g_msg, sizeof(g_msg));
    if (plan_parts(true, g, wires, K, edges, B, opt, one, travel, out) == DR_OK) return DR_OK;
    std::memcpy(g_msg, first, sizeof(g_msg));
  }
  return st;
}

extern "C" void dr_plan_destroy(dr_plan_t *p) {
  if (!p) return;
  for (dr_plan_t *q : p->parts) dr_plan_destroy(q);
  if (p->dev_block) {
    // stream-ordered release into the plan pool (no wait for the device)
    PlanMemory *pm = nullptr;
    if (plan_memory(p->device, &pm) == DR_OK) cudaFreeAsync(p->dev_block, pm->stream);
  }
  delete p;
}

extern "C" size_t dr_plan_device_bytes(const dr_plan_t *p) { return p ? p->device_bytes : 0; }

extern "C" dr_status dr_plan_get_info(const dr_plan_t *p, dr_plan_info *info) {
  if (!p || !info) {
    set_error("dr_plan_get_info: null argument");
    return DR_ERR_INVALID_ARG;
  }
  std::memset(info, 0, sizeof(*info));
  info->rows = p->rows;
  info->cols = p->cols;
  info->K = p->K;
  info->B = p->B;
  info->kernel = p->kernel;
  info->tile_cols = p->tune.tile_cols;
  info->pixels_per_thread = p->tune.ppt;
  info->bin_groups = p->tune.bin_groups;
  info->threads = p->threads;
  info->smem_bytes = p->smem_bytes;
  info->tma_chunk = p->tune.kc;
  info->tma_chunks = p->tune.nchunks;
  info->out_dtype = p->out_dtype;
  info->geom_precision = p->geom_prec;
  info->edge = p->edge;
  info->reversed = p->c.reverse;
  info->fixed_shift = p->shift;
  info->row_tables = p->c.tab != nullptr;
  info->parts = p->parts.empty() ? 1 : (int32_t)p->parts.size();
  info->depth_min = p->depth_min;
  info->depth_max = p->depth_max;
  info->min_step = p->min_step;
  const double unit = std::ldexp(1.0, -p->shift) / (p->nb > 0 ? p->nb : 1.0);
  info->max_step = p->max_step_units * unit;
  info->depth_err = p->max_dev_units >= 0 ? p->max_dev_units * unit : -1.0;
  info->depth_form = p->c.depth_mode;
  info->one_step_per_bin = p->one_adv;
  info->checked_groups = p->checked_groups;
  info->device_bytes = p->device_bytes;
  double P = (double)p->rows * p->cols;
  info->bytes_per_call = 2.0 * P * p->K + (p->out_dtype == DR_OUT_BF16 ? 2.0 : 4.0) * P * p->B;
  return DR_OK;
}

extern "C" const char *dr_status_string(dr_status s) {
  switch (s) {
    case DR_OK: return "ok";
    case DR_ERR_INVALID_ARG: return "invalid argument";
    case DR_ERR_GEOMETRY: return "invalid geometry";
    case DR_ERR_NONMONOTONIC: return "depth not monotone in the step index";
    case DR_ERR_OOM: return "out of memory";
    case DR_ERR_BUDGET: return "over the memory budget";
    case DR_ERR_CUDA: return "CUDA error";
    case DR_ERR_TIMEOUT: return "device wait timed out";
    case DR_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

extern "C" const char *dr_last_error(void) { return g_msg; }

extern "C" const char *dr_version(void) { return "1.0.0"; }

// ---------------------------------------------------------------------------
// Rows-kernel tables built into a fixed buffer (no allocation of any kind):
// the same FP64 frame, per-row constants, monotonicity check and fixed-point
// scale as dr_plan, restricted to detectors whose columns run along the wire
// axis and to FP32 geometry.
dr_status dr::build_rows_tables(const dr_geometry *g, const double *wires, int K,
                                const double *edges, int B, unsigned char *stage, size_t cap,
                                double *tmp, StaticTables *out) {
  if (!g || !wires || !edges || !stage || !tmp || !out) {
    set_error("null argument");
    return DR_ERR_INVALID_ARG;
  }
  if (K < 2 || B < 1 || g->rows < 0 || g->cols < 0 || g->rows > 65535 ||
      (g->edge != DR_EDGE_LEADING && g->edge != DR_EDGE_TRAILING)) {
    set_error("need K >= 2, B >= 1, 0 <= rows <= 65535, cols >= 0, a valid edge");
    return DR_ERR_INVALID_ARG;
  }
  for (int j = 0; j <= B; ++j)
    if (!std::isfinite(edges[j]) || (j > 0 && !(edges[j] > edges[j - 1]))) {
      set_error("bin edges must be finite and strictly increasing (j=%d)", j);
      return DR_ERR_INVALID_ARG;
    }
  for (int k = 0; k < K; ++k)
    if (!finite3(wires + 3 * k)) {
      set_error("wire centre %d not finite", k);
      return DR_ERR_INVALID_ARG;
    }
  if (!finite3(g->beam_origin) || !finite3(g->beam_dir) || !finite3(g->det_origin) ||
      !finite3(g->row_step) || !finite3(g->col_step) || !finite3(g->wire_axis) ||
      !std::isfinite(g->wire_radius) || !(g->wire_radius > 0.0)) {
    set_error("geometry not finite or radius <= 0");
    return DR_ERR_INVALID_ARG;
  }
  const int H = g->rows, W = g->cols;
  const size_t o_grp = 0;
  const size_t o_stp = align_up(o_grp + sizeof(GroupC) * (size_t)H, 256);
  const size_t o_efx = align_up(o_stp + sizeof(StepC) * (size_t)K, 256);
  const size_t o_err = align_up(o_efx + sizeof(int32_t) * (size_t)(B + 1), 256);
  const size_t bytes = o_err + 256;
  if (bytes > cap) {
    set_error("tables need %zu bytes of static scratch; the limit is %zu", bytes, cap);
    return DR_ERR_BUDGET;
  }
  V3 ax = v3(g->wire_axis), bd = v3(g->beam_dir), O = v3(g->beam_origin);
  if (!(norm(ax) > 0) || !(norm(bd) > 0)) {
    set_error("zero wire axis or beam direction");
    return DR_ERR_GEOMETRY;
  }
  ax = (1.0 / norm(ax)) * ax;
  bd = (1.0 / norm(bd)) * bd;
  const V3 bp = bd - dot(bd, ax) * ax;
  const double nb = norm(bp);
  if (!(nb > 1e-9)) {
    set_error("beam runs along the wire axis");
    return DR_ERR_GEOMETRY;
  }
  const V3 e2 = (1.0 / nb) * bp;
  V3 w = v3(wires) - O;
  w = w - dot(w, ax) * ax;
  w = w - dot(w, e2) * e2;
  if (!(norm(w) > 0)) {
    set_error("first wire centre lies on the beam");
    return DR_ERR_GEOMETRY;
  }
  const V3 e1 = (1.0 / norm(w)) * w;
  const double R = g->wire_radius;
  double *zp = tmp, *ep = tmp + K;
  const double z_first = dot(v3(wires) - O, e2);
  const double z_last = dot(v3(wires + 3 * (K - 1)) - O, e2);
  if (z_last == z_first) {
    set_error("wire does not travel along the projected beam");
    return DR_ERR_GEOMETRY;
  }
  const bool reverse = z_last < z_first;
  const double y_first = dot(v3(wires) - O, e1);
  double ymin = 1e300, ymax = -1e300;
  bool has_eta = false;
  for (int k = 0; k < K; ++k) {  // processing order: increasing depth
    const V3 c = v3(wires + 3 * (reverse ? K - 1 - k : k)) - O;
    zp[k] = dot(c, e2);
    const double yk = dot(c, e1);
    ep[k] = yk - y_first;
    has_eta |= (yk != y_first);
    ymin = std::min(ymin, yk);
    ymax = std::max(ymax, yk);
  }
  if (!(ymin > R)) {
    set_error("wire overlaps the beam");
    return DR_ERR_GEOMETRY;
  }
  const double sR = (reverse ? -1.0 : 1.0) * (g->edge == DR_EDGE_LEADING ? 1.0 : -1.0) * R;
  const V3 dorg = v3(g->det_origin) - O, rs = v3(g->row_step), cs = v3(g->col_step);
  const double Y00 = dot(dorg, e1), Z00 = dot(dorg, e2), Yr = dot(rs, e1), Zr = dot(rs, e2);
  if (std::fabs(dot(cs, e1)) + std::fabs(dot(cs, e2)) > 1e-13 * std::max(norm(cs), 1e-300)) {
    set_error("detector columns must run along the wire axis for this entry point");
    return DR_ERR_UNSUPPORTED;
  }
  if (H > 0 && W > 0 && !(std::min(Y00, Y00 + (H - 1) * Yr) - ymax > R)) {
    set_error("wire not between beam and detector");
    return DR_ERR_GEOMETRY;
  }
  // per-row constants (FP64), depth range and monotonicity
  double tmin = edges[0] * nb, tmax = edges[B] * nb, minstep = 1e300, maxstep = 0.0,
         remmax = 0.0, qmax = 0.0;
  for (int r = 0; r < H && W > 0; ++r) {
    const double Y = Y00 + r * Yr, Z = Z00 + r * Zr, D = Y - y_first;
    const double L0 = std::sqrt(Y * Y + Z * Z), Q0 = (-y_first * Z + sR * L0) / D;
    qmax = std::max(qmax, std::fabs(Q0));
    double prev = 0.0;
    for (int k = 0; k < K; ++k) {
      const double t = solve_t(Y, Z, y_first, sR, D, L0, Q0, zp[k], ep[k]);
      tmin = std::min(tmin, t);
      tmax = std::max(tmax, t);
      remmax = std::max(remmax, std::fabs(t - zp[k] - Q0));
      if (k > 0) {
        if (!(t - prev > 0)) {
          set_error("depth of row %d not monotone at step %d", r, k);
          return DR_ERR_NONMONOTONIC;
        }
        minstep = std::min(minstep, t - prev);
        maxstep = std::max(maxstep, t - prev);
      }
      prev = t;
    }
  }
  const double origin = 0.5 * (tmin + tmax);
  double mag = std::max(0.5 * (tmax - tmin) * 1.001 + 1e-9, std::max(qmax, remmax * 1.5));
  for (int k = 0; k < K; ++k) mag = std::max(mag, std::fabs(zp[k] - origin));
  int shift = std::min((int)std::floor(std::log2((double)(1 << 29) / mag)), 40);
  // every step below 2^23 grid units (exact conversion of position differences)
  if (maxstep > 0.0)
    shift = std::min(shift, (int)std::floor(std::log2(0.9 * kMaxStepUnits / maxstep)));
  if (shift < 12) {
    set_error("depth range too large for 32-bit fixed point");
    return DR_ERR_UNSUPPORTED;
  }
  const double scale = std::ldexp(1.0, shift);
  if (H > 0 && W > 0 && minstep * scale < kMinStepUnits) {
    set_error("depth steps too small for the fixed-point grid");
    return DR_ERR_UNSUPPORTED;
  }
  // launch shape: the dr_plan defaults
  Tuning t;
  t.ppt = (W % 4 == 0) ? 4 : 1;
  int tc = std::min(128, std::max((W + 7) / 8 * 8, 8));
  int kc, n;
  auto smem_for = [&](int c) {
    choose_chunks(K, c, &kc, &n);
    return rows_smem_bytes(K, kc * n, B, c, false);
  };
  while (tc > 32 && 2 * (smem_for(tc) + 1024) > kSmemPerSm) tc /= 2;
  const int smem = smem_for(tc);
  if (smem > kSmemPerCtaMax || kc < 1 || ((size_t)kc * tc * 2) % 128 != 0) {
    set_error("%d steps do not fit in shared memory", K);
    return DR_ERR_UNSUPPORTED;
  }
  t.tile_cols = tc;
  t.kc = kc;
  t.nchunks = n;
  const int lanes = tc / t.ppt;
  int bg = std::max(1, 512 / lanes);
  while (bg > 1 && B / bg < 16) bg /= 2;
  while (lanes * bg > 512) bg /= 2;
  t.bin_groups = bg;
  // tables
  std::memset(stage, 0, bytes);
  GroupC *gc = reinterpret_cast<GroupC *>(stage + o_grp);
  for (int r = 0; r < H; ++r) {
    const double Y = Y00 + r * Yr, Z = Z00 + r * Zr, D = Y - y_first;
    const double L0 = std::sqrt(Y * Y + Z * Z), Q0 = (-y_first * Z + sR * L0) / D;
    gc[r].Z = (float)Z;
    gc[r].Y2 = (float)(Y * Y);
    gc[r].L0 = (float)L0;
    gc[r].invD = (float)(1.0 / D);
    gc[r].D = (float)D;
    gc[r].Q0f = (float)Q0;
    gc[r].Q0fx = (int32_t)std::llround(Q0 * scale);
    gc[r].invL0 = (float)(1.0 / L0);
  }
  StepC *sc = reinterpret_cast<StepC *>(stage + o_stp);
  for (int k = 0; k < K; ++k) {
    sc[k].zf = (float)zp[k];
    sc[k].eta = (float)ep[k];
    sc[k].zfx = (int32_t)std::llround((zp[k] - origin) * scale);
  }
  int32_t *efx = reinterpret_cast<int32_t *>(stage + o_efx);
  for (int j = 0; j <= B; ++j) {
    const double f = (double)std::llround((edges[j] * nb - origin) * scale);
    efx[j] = (int32_t)std::max(std::min(f, 2147483000.0), -2147483000.0);
  }
  StaticTables &st = *out;
  std::memset(&st, 0, sizeof(st));
  st.off_grp = o_grp;
  st.off_stp = o_stp;
  st.off_efx = o_efx;
  st.off_err = o_err;
  st.bytes = bytes;
  st.tune = t;
  st.rows = H;
  st.cols = W;
  st.K = K;
  st.B = B;
  st.threads = lanes * bg;
  st.smem_bytes = smem;
  Consts &c = st.c;
  c.K = K;
  c.H = H;
  c.W = W;
  c.B = B;
  c.has_eta = has_eta ? 1 : 0;
  c.reverse = reverse ? 1 : 0;
  c.y0 = (float)y_first;
  c.sR = (float)sR;
  c.scale = (float)scale;
  c.y0d = y_first;
  c.sRd = sR;
  c.origin = origin;
  c.nb = nb;
  c.out_sign = (float)((g->edge == DR_EDGE_LEADING ? 1.0 : -1.0) * (reverse ? -1.0 : 1.0));
  return DR_OK;
}
