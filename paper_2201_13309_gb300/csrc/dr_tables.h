// Layouts of the tables the kernels read (shared by host and device code).
//
// Depth model (the tangent geometry of the differential-aperture method; in
// the paper's Sec. III-C the per-pixel routine assigns each difference to
// depth): everything is projected onto the plane perpendicular to the wire
// axis, with e2 along the projected beam and e1 toward the first wire centre.
// A beam point at projected depth t sits at (0, t); pixel p at (Y, Z); wire
// step k at (y_k, z_k), radius R.  The line from (0, t) to (Y, Z) touches the
// wire circle on the chosen edge (sign s = +-1) when
//
//     t (Y - y_k) = z_k Y - Z y_k + s R L(t),   L(t) = sqrt(Y^2 + (Z - t)^2).
//
// With y0 = y_0, eta_k = y_k - y0, D = Y - y0, L0 = sqrt(Y^2 + Z^2),
// dL(t) = L(t) - L0 = t (t - 2Z) / (L(t) + L0) and
// Q0 = (-y0 Z + s R L0) / D this is exactly
//
//     t_k = z_k + Q0 + (a_k + s R dL(t_k)) / (D - eta_k),
//     a_k = y0 z_k + eta_k (z_k - Z + Q0).
//
// z_k and Q0 are large (up to ~1 mm) and come from FP64; the remainder term
// is small (~5e-4 mm in the beamline set-up) and is all that FP32 computes
// per (pixel, step).  Positions are held as 32-bit fixed point in units of
// 2^-shift mm of projected depth relative to a plan origin, so differences of
// positions are exact.  dL enters scaled by R / D ~ 5e-5, so evaluating it
// at the estimate without the dL term leaves an error ~1e-10 mm.
//
// The remainder is computed in one of three forms (Consts::depth_mode):
//  * exact: dL = t (t - 2Z) / (L(t) + L0), a square root and a reciprocal;
//  * series: with n = t (t - 2Z) = L(t)^2 - L0^2 and x = n / L0^2,
//    dL = L0 (sqrt(1 + x) - 1) = n / (2 L0) (1 - x/4 + x^2/8 - 5x^3/64 + ...),
//    three terms (multiply-adds only);
//  * polynomial: when every wire centre has the same distance from the beam
//    (eta = 0) the remainder of a group is a smooth function of z_k alone;
//    the plan interpolates it in FP64 by a cubic in (z_k - z_c) through four
//    Chebyshev nodes of the path's z range, in grid units, so a position is
//    three multiply-adds and a rounding.
// A plan takes the cheapest form whose error it can bound far below one grid
// unit, and its check compares every depth the kernels compute with the FP64
// solution (falling back to the next form if the bound does not hold).
#pragma once

#include <cstddef>
#include <cstdint>

namespace dr {

// Per geometry group (a detector row when all pixels of a row share their
// projected position, else a single pixel).
struct GroupC {
  float Z, Y2, L0, invD;   // FP32 copies of FP64 values
  float D, Q0f;
  int32_t Q0fx;            // round(Q0 * 2^shift)
  float invL0;             // 1 / L0 (series form of dL)
};
static_assert(sizeof(GroupC) == 32, "GroupC layout");

// The same 32 bytes in the polynomial form: the remainder of the group in
// grid units is ((c3 d + c2) d + c1) d + c0 with d = z_k - z_c (StepC::dz),
// and q0fx = round(Q0 * 2^shift) - 0x4B400000 (the bias of the rounding by
// 1.5 * 2^23 folded in).
struct GroupPoly {
  float c0, c1, c2, c3;
  float unused0, unused1;
  int32_t q0fx;
  float unused2;
};
static_assert(sizeof(GroupPoly) == sizeof(GroupC), "GroupPoly layout");

struct StepC {
  float zf, eta;           // z_k, eta_k (FP32)
  int32_t zfx;             // round((z_k - origin) * 2^shift)
  float dz;                // z_k - z_c (polynomial form)
};
static_assert(sizeof(StepC) == 16, "StepC layout");

enum : int { kDepthExact = 0, kDepthSeries = 1, kDepthPoly = 2 };

// FP64 mirrors for the all-FP64 geometry variant.
struct GroupD {
  double Z, Y2, L0, D, Q0;
};
struct StepD {
  double z, eta;           // z_k - origin is formed on the fly
};

// Everything a reconstruction kernel needs besides the images/output.
struct Consts {
  const GroupC *grp;
  const StepC *stp;
  const int32_t *efx;      // [B+1] fixed-point edges (projected depth)
  const GroupD *grp64;
  const StepD *stp64;
  const double *e64;       // [B+1] edges relative to origin (projected depth)
  int K, H, W, B;
  int has_eta;             // wire centres do not all share y
  int reverse;             // plan's step order is the reverse of the images'
  float y0, sR, scale;     // y0, s*R, 2^shift
  double y0d, sRd, origin;  // origin of the fixed-point positions (mm)
  double nb;               // |projected unit beam direction|: d = t / nb
  float out_sign;          // +1 leading/forward; -1 trailing or reversed
  int32_t *err;            // device error word
  // Per-row tables built once by the plan (null: each tile builds its own):
  // row r holds tab_stride int2 entries at tab + r * tab_stride, [0] =
  // (first, end) of the bins that can hold data, [1 + j] = (k_j, f_j bits)
  // for edge j = 0..B.
  const int2 *tab;
  int tab_stride;
  // 1: add this plan's bins to the output instead of writing them (the later
  // parts of a composite plan: monotone runs, both wire edges)
  int accumulate;
  // form of the FP32 remainder (kDepthExact / kDepthSeries / kDepthPoly)
  int depth_mode;
};

// What the plan-time check of every (group, step) found (device, written by
// check_kernel): the first group whose FP32 depth positions are not strictly
// increasing with steps in [kMinStepUnits, kMaxStepUnits), the smallest and
// largest step, and the largest distance of an FP32 position from the FP64
// solution, all in grid units.
struct PlanCheck {
  unsigned long long bad;  // (group << 32) | step of the first failure; ~0 if none
  int32_t min_step, max_step;
  int32_t max_dev;         // max |t_fp32 - round(t_fp64 * 2^shift)|
  int32_t tmin, tmax;      // range of all positions
  int32_t pad;
};
// Steps of FP32 positions must span at least this many grid units (a few
// units of FP32 error then move a negligible part of an interval's
// difference across a bin edge) and fewer than 2^23 (so that a position
// difference converts to float exactly by the 2^23-bias construction).
constexpr int32_t kMinStepUnits = 64;
constexpr int32_t kMaxStepUnits = 1 << 23;

// Entries of one row table: a header, B + 1 edges, rounded up to an even
// count so that a row is a multiple of 16 bytes (bulk-copy granule).
__host__ __device__ inline int row_table_entries(int B) { return (B + 2 + 1) & ~1; }

// Error codes written to the device error word.
// The bounds-checked build (DR_CHECK_BOUNDS) writes kDevBounds | (line << 4),
// the device-source line of the first index found out of range.
enum : int32_t { kDevOk = 0, kDevTmaTimeout = 1, kDevBounds = 2 };

struct Tuning {
  int tile_cols;           // pixels per CTA along the row
  int ppt;                 // pixels per thread (1 or 4)
  int bin_groups;          // thread groups splitting the bins
  int kc, nchunks;         // TMA step chunk and chunk count
};

}  // namespace dr
