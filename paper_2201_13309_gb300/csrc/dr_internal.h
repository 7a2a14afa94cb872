// Internal definitions shared by the library's translation units.
//
// Depth model (the tangent geometry of the differential-aperture method; the
// paper's Sec. III-C "pixel reconstruction function" assigns each difference
// to depth): everything is projected onto the plane perpendicular to the wire
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
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/dr.h"

namespace dr {

// Per geometry group (a detector row when all pixels of a row share their
// projected position, else a single pixel).
struct GroupC {
  float Z, Y2, L0, invD;   // FP32 copies of FP64 values
  float D, Q0f;
  int32_t Q0fx;            // round(Q0 * 2^shift)
  float pad;
};
static_assert(sizeof(GroupC) == 32, "GroupC layout");

struct StepC {
  float zf, eta;           // z_k, eta_k (FP32)
  int32_t zfx;             // round((z_k - origin) * 2^shift)
  float pad;
};
static_assert(sizeof(StepC) == 16, "StepC layout");

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
};

// Error codes written to the device error word.
enum : int32_t { kDevOk = 0, kDevTmaTimeout = 1 };

struct Tuning {
  int tile_cols;           // pixels per CTA along the row
  int ppt;                 // pixels per thread (1 or 4)
  int bin_groups;          // thread groups splitting the bins
  int kc, nchunks;         // TMA step chunk and chunk count
};

}  // namespace dr

struct dr_plan {
  int rows, cols, K, B, edge;
  int kernel;              // DR_KERNEL_ROWS / DR_KERNEL_PIXELS
  int out_dtype, geom_prec;
  int shift;
  double nb;               // |projected beam direction|: depth = t / nb
  double depth_min, depth_max, min_step;
  dr::Consts c;            // device pointers + scalars
  dr::Tuning tune;         // for dr_reconstruct launches
  int threads, smem_bytes;
  size_t device_bytes;
  void *dev_block;         // single device allocation holding every table
};

namespace dr {

// Layout of the rows-kernel tables when they are built into a fixed buffer
// instead of a plan's own device allocation (offsets from the buffer start).
struct StaticTables {
  size_t off_grp, off_stp, off_efx, off_err, bytes;
  Consts c;                // pointers hold offsets until rebased
  Tuning tune;
  int rows, cols, K, B, threads, smem_bytes;
};

// Builds GroupC[rows] / StepC[K] / fixed-point edges / a zeroed error word
// into stage (cap bytes), using tmp (2*K doubles) as host scratch.  Only for
// detectors whose columns run along the wire axis (the rows kernel), FP32
// geometry; DR_ERR_BUDGET when the tables exceed cap.
dr_status build_rows_tables(const dr_geometry *g, const double *wires, int K,
                            const double *edges, int B, unsigned char *stage, size_t cap,
                            double *tmp, StaticTables *out);

void set_error(const char *fmt, ...);
dr_status cuda_fail(const char *what, int err);
}  // namespace dr
