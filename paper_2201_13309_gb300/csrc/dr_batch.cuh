// The persistent batch kernel: many scans (each with its own plan tables,
// tensor map and tile shape) in one launch (dr_batch.cu).
#pragma once

#include "dr_device.cuh"
#include "dr_intervals.cuh"

namespace dr {

// Many scans (each with its own plan tables, tensor map and tile shape) in
// one launch: every CTA takes work items from a device counter until none
// are left.  An item is rows_per_item tiles of one scan at the same columns
// in consecutive rows, so the counter's round trip is paid once for them.
// Items are numbered scan by scan in the order of the descriptor array.

// Work-item kinds: a rows tile, a per-pixel tile (depth table or the
// polynomial form; with at most one step advance per bin, or the general
// walk), or an interval-kernel tile (depths in any order).
enum : int {
  kBatchRows = 0,
  kBatchPixelsOneAdv = 1,
  kBatchPixels = 2,
  kBatchPixelsPolyOneAdv = 3,
  kBatchPixelsPoly = 4,
  kBatchIntervals = 5
};

// Kernel instances by the kinds they hold: rows and per-pixel tiles; only
// per-pixel tiles of the polynomial form (three 512-thread CTAs per SM);
// rows, per-pixel and interval tiles (built only for a batch that has an
// interval plan, so the other instances keep their registers).
enum : int { kSetRunningSum = 0, kSetPolyOnly = 1, kSetAll = 2 };

struct BatchScan {
  CUtensorMap tmap;        // [K][rows][cols] images, box [kc][1][tile_cols]
  const uint16_t *img;
  void *out;
  Consts c;
  Tuning t;
  long long item_begin;    // first work item of this scan
  int tiles_per_row;
  int rows_per_item;       // an item is this many tiles down one column
  int kind;                // kBatchRows / ... / kBatchIntervals
  int pixel_groups;        // interval tiles: depths per pixel (1) or per row (0)
  int window;              // interval tiles: bins per shared-memory window
};

template <class OutT, int kSet>
__global__ void __launch_bounds__(512, kSet == kSetPolyOnly ? 3 : kSet == kSetAll ? 2 : 1)
    batch_kernel(const BatchScan *__restrict__ scans, int nscans, long long n_items,
                 unsigned long long *counter) {
  extern __shared__ __align__(128) unsigned char smem[];
  // the current tile, published by thread 0: scan (-1: no work left), row,
  // first column, and the end of the item's rows (bytes [0, 8) hold the
  // tiles' mbarrier, their data starts at 128)
  int *cur = reinterpret_cast<int *>(smem + 16);
  if (threadIdx.x == 0) {
    mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
    cur[1] = cur[3] = 0;  // no item yet: the first pass takes one
  }
  uint32_t parity = 0;
  for (;;) {
    __syncthreads();  // previous tile done with smem; barrier initialised
    if (threadIdx.x == 0) {
      if (++cur[1] >= cur[3]) {  // the item's rows are done: take the next item
        const long long item = (long long)atomicAdd(counter, 1ull);
        if (item >= n_items) {
          cur[0] = -1;
        } else {
          int lo = 0, hi = nscans - 1;  // last scan with item_begin <= item
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (scans[mid].item_begin <= item) lo = mid; else hi = mid - 1;
          }
          const BatchScan &S = scans[lo];
          const long long local = item - S.item_begin;
          cur[0] = lo;
          cur[1] = (int)(local / S.tiles_per_row) * S.rows_per_item;
          cur[2] = (int)(local % S.tiles_per_row) * S.t.tile_cols;
          cur[3] = min(cur[1] + S.rows_per_item, S.c.H);
        }
      }
    }
    __syncthreads();
    const int si = cur[0];
    if (si < 0) break;
    const BatchScan &S = scans[si];
    const int row = cur[1], c0 = cur[2];
    // the scan's constants as values of this thread, so that the tile's
    // stores to the output (global memory, like the descriptors) do not make
    // the compiler read them again
    const Consts c = S.c;
    const Tuning t = S.t;
    OutT *const o = reinterpret_cast<OutT *>(S.out);
    bool ok;
    if constexpr (kSet == kSetPolyOnly) {
      ok = S.kind == kBatchPixelsPolyOneAdv
               ? pixels_poly_tile<OutT, true, true>(&S.tmap, S.img, o, c, t, row, c0, smem,
                                                    parity)
               : pixels_poly_tile<OutT, true, false>(&S.tmap, S.img, o, c, t, row, c0,
                                                     smem, parity);
    } else if (kSet == kSetAll && S.kind == kBatchIntervals)
      ok = intervals_tile<GeoFx, OutT, true>(&S.tmap, S.img, o, c, t, S.pixel_groups, S.window,
                                             row, c0, smem, parity);
    else if (S.kind == kBatchRows)
      ok = rows_tile<GeoFx, OutT, true, 4>(&S.tmap, S.img, o, c, t, row, c0, smem, parity);
    else if (S.kind == kBatchPixelsPolyOneAdv)
      ok = pixels_poly_tile<OutT, true, true>(&S.tmap, S.img, o, c, t, row, c0, smem,
                                              parity);
    else if (S.kind == kBatchPixelsPoly)
      ok = pixels_poly_tile<OutT, true, false>(&S.tmap, S.img, o, c, t, row, c0, smem,
                                               parity);
    else if (S.kind == kBatchPixelsOneAdv)
      ok = pixels_tile<GeoFx, OutT, true, true>(&S.tmap, S.img, o, c, t, row, c0, smem,
                                                parity);
    else
      ok = pixels_tile<GeoFx, OutT, true, false>(&S.tmap, S.img, o, c, t, row, c0, smem,
                                                 parity);
    parity ^= 1u;
    if (!ok) break;
  }
}

}  // namespace dr
