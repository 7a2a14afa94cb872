// Host-side internals shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "../../include/dr.h"
#include "dr_tables.h"

struct dr_plan {
  int rows, cols, K, B, edge;
  int kernel;              // DR_KERNEL_ROWS / DR_KERNEL_PIXELS / DR_KERNEL_INTERVALS
  int pixel_groups;        // 1: geometry constants per pixel, 0: per row
  int window;              // interval kernel: bins per shared-memory window
  int iv_ctas = 2;         // interval kernel: CTAs per SM its tile is sized for
  int out_dtype, geom_prec;
  int shift;
  double nb;               // |projected beam direction|: depth = t / nb
  double depth_min, depth_max, min_step;
  dr::Consts c;            // device pointers + scalars
  dr::Tuning tune;         // for dr_reconstruct launches
  int threads, smem_bytes;
  size_t device_bytes;
  void *dev_block;         // single device allocation holding every table
  int device = 0;          // the device it lives on
  // what the plan-time check of every (group, step) found (FP32 geometry of
  // the running-sum kernels): groups checked, largest step and largest
  // distance from FP64 in grid units (-1: not checked), and whether every
  // step is at least as long as every bin (at most one step boundary per bin)
  long long checked_groups = 0;
  int max_step_units = 0, max_dev_units = -1, one_adv = 0;
  // composite plans (monotone runs of a back-and-forth scan, both wire
  // edges): the parts run in order on images + part_k0 planes, the first
  // writing the output and the others adding to it; empty for a plain plan
  std::vector<dr_plan *> parts;
  std::vector<int> part_k0;
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

constexpr int kSmemPerSm = 228 * 1024;       // shared memory per SM
constexpr int kSmemPerCtaMax = 227 * 1024;   // opt-in maximum per CTA

// Shared-memory bytes of one rows / pixels tile (layouts in dr_device.cuh).
int rows_smem_bytes(int K, int Kpad, int B, int tile_cols, bool f64);
int pixels_smem_bytes(int K, int Kpad, int B, int tile_cols, bool f64);
// The per-pixel kernel of the polynomial form (no depth table).
int pixels_poly_smem_bytes(int K, int Kpad, int B, int tile_cols);
// Interval kernel: pixels per CTA, and the shared-memory bytes of one tile:
// mbarrier, image tile [Kpad][32] uint16, depths [K][32] (per-pixel
// geometry) or [K] (shared along the row), edges [B + 1], the pixels' sums of
// |dI| (128 bytes), int32 accumulators [window][32] (dr_intervals.cuh).
constexpr int kIntervalTile = 32;
inline int intervals_smem(int K, int Kpad, int B, int window, bool f64, bool per_pixel) {
  const size_t ps = f64 ? 8 : 4, cols = per_pixel ? kIntervalTile : 1;
  auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  return (int)(128 + a16((size_t)Kpad * kIntervalTile * 2) + a16((size_t)K * cols * ps) +
               a16((size_t)(B + 1) * ps) + 4 * kIntervalTile +
               (size_t)window * kIntervalTile * 4);
}
// TMA chunking of K steps for a tile width (128-byte aligned destinations).
void choose_chunks(int K, int tile_cols, int *kc, int *nchunks);
// Raise a kernel's dynamic shared-memory limit (once per device).
dr_status allow_smem(const void *fn);
// [K][rows][cols] uint16 tensor map with a [kc][1][tile_cols] box (p->tune).
dr_status make_tensor_map(const dr_plan_t *p, const uint16_t *img, CUtensorMap *tm);
// Run check_kernel over the plan's ngroups groups into the device record
// d_res and copy the result to *h_res; synchronous.
dr_status run_plan_check(const dr_plan_t *p, int ngroups, bool monotone, PlanCheck *d_res,
                         PlanCheck *h_res);
// Inputs of the per-group constants (groups_kernel): affine pixel
// coordinates in the projected frame, the wire's y0 and signed radius, the
// grid scale, the z range of the path (centre, half width) and the form of
// the remainder.
struct GroupsParams {
  double Y00, Yr, Yc, Z00, Zr, Zc, y0, sR, scale, zc, zh;
  long long ngroups;
  int W, rows_shared, mode, pad;
};
// Compute every group's GroupC / GroupD on the device; synchronous.
dr_status run_groups(const GroupsParams &q, GroupC *gc, GroupD *gd);
// Build the plan's per-row (k, f) tables into tab (H rows of c.tab_stride
// entries) on the device; synchronous.
dr_status build_plan_tables(const dr_plan_t *p, int2 *tab);
// Load every reconstruction kernel on the current device (module loading is
// otherwise lazy, at the first launch).
dr_status preload_kernels();
// All launches of a plan (the parts of a composite plan in order).
dr_status launch_plan(const dr_plan_t *p, const uint16_t *img, void *out,
                      struct CUstream_st *st);
// Reconstruction launch of a plan (defined with the kernels).
dr_status launch_reconstruct(const dr_plan_t *p, const uint16_t *img, void *out,
                             struct CUstream_st *st);

// A named range for profilers' timelines (NVTX; nothing happens unless a
// tool is attached).
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

void set_error(const char *fmt, ...);
dr_status cuda_fail(const char *what, int err);
}  // namespace dr
