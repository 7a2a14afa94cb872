// Interval kernel: apportioning for depth sequences in any order.
//
// The method spreads each image difference dI_k = I_k - I_{k+1} over the depth
// interval swept between steps k and k+1 in proportion to its overlap with
// each bin (Sec. III).  The rows and per-pixel kernels evaluate that sum as a
// running sum F, which needs the depths of a pixel to increase with k.  When
// they do not (a wire that also moves across the beam, repeated positions),
// the plan falls back to this kernel, which adds every interval by itself:
//
//   out_j = sum_k dI_k * (phi_k(e_{j+1}) - phi_k(e_j)),
//   phi_k(x) = clamp((x - lo_k) / (hi_k - lo_k), 0, 1),
//   lo_k = min(d_k, d_{k+1}), hi_k = max(d_k, d_{k+1}),
//
// and an interval of zero length puts its whole dI_k into the bin
// [e_j, e_{j+1}) that holds it.  Mass outside [e_0, e_B] is dropped.
//
// A CTA owns one row x 32 adjacent pixels x all K steps (image tile staged by
// TMA as in the other kernels; the depths in shared memory, per pixel, or
// once for the row when the geometry is shared along it).  Lane = pixel and
// warp = a chunk of consecutive intervals, so every shared-memory access of a
// warp touches 32 consecutive words, and one bin of the tile is a 128-byte
// line of its output plane.  The bins go through shared-memory windows of
// `window` int32 accumulators per pixel.
// Each thread splits its chunk into strictly monotone runs (and zero-length
// intervals) and walks each run once over the bins it spans; a chunk that
// its first pass finds to be a single run is walked without the split.  Over one run
// the sum of dI_k * phi_k at an edge e is s * G(e) with G(e) = V_0 - V(e):
// V interpolates the run's image values linearly in depth (clamped at both
// ends of the run), V_0 is the value at its shallowest point, and s = +1 when
// the depths rise with the step, -1 when they fall.  G is the per-pixel
// kernel's running sum F over that run, evaluated the same way in FP32; the
// bin gets s * (G(e_{j+1}) - G(e_j)), rounded onto the pixel's fixed-point
// grid and added with a shared-memory atomic.  The grid is 2^-q with q chosen
// from the pixel's M = sum_k |dI_k|, so that M 2^q < 2^29: every partial sum
// of a bin stays inside int32 (the parts added to all bins of a pixel come to
// M in absolute value, up to FP32 rounding), and a part is rounded by at most
// M 2^-30.  Integer sums do not depend on the order of the atomics, so the
// result is deterministic.
// FP32 positions carry a few units of their fixed-point grid.  An interval
// shorter than kMinStepUnits (a step next to a turning point of the depths,
// a repeated wire position) could then put its difference on the wrong side
// of a bin edge, so its two depths are computed again in FP64 from the plan's
// FP64 constants and it is apportioned against the FP64 edges by itself.
#pragma once

#include "dr_device.cuh"
#include "dr_internal.h"

namespace dr {

// 2^q as a float, -126 <= q <= 127
__device__ __forceinline__ float iv_pow2(int q) { return __int_as_float((127 + q) << 23); }
// the grid exponent q of a pixel whose sum of |dI| is M: M 2^q < 2^29
__device__ __forceinline__ int iv_grid(uint32_t M) { return 29 - (32 - __clz(M)); }
// 1 / (b - a) for a < b, and the position of e in [a, b] as a fraction (e
// clamped to the interval by the caller: a <= e <= b).  FP64 positions: the
// differences are taken in FP64 (exact where the positions are close) and
// the fraction in FP32, as for the fixed-point positions, so that the FP64
// pipe does two subtractions per step and bin, not a division.
__device__ __forceinline__ float iv_inv_len(int32_t lo, int32_t hi) {
  return rcp_approx(__uint2float_rn((uint32_t)hi - (uint32_t)lo));
}
__device__ __forceinline__ float iv_inv_len(double lo, double hi) {
  return rcp_approx(__double2float_rn(hi - lo));
}
__device__ __forceinline__ float iv_frac(int32_t e, int32_t lo, float inv) {
  return fminf(__fmul_rn(__uint2float_rn((uint32_t)e - (uint32_t)lo), inv), 1.f);
}
__device__ __forceinline__ float iv_frac(double e, double lo, float inv) {
  return fminf(__fmul_rn(__double2float_rn(e - lo), inv), 1.f);
}

// One tile: row `row`, columns c0 .. c0 + 31, all steps and bins.  The
// mbarrier at smem[0] must be initialised (by thread 0 before the call, or
// earlier with a barrier since); `parity` is its phase for this tile.
// Returns false (for every thread) if the bounded TMA wait ran out.
// Shared-memory layout (intervals_smem): [0, 128) mbarrier, the image tile
// [Kpad][32] uint16, the depths [K][32] (pixel_groups) or [K], the edges
// [B + 1], the pixels' sums of |dI| [32], the accumulators [window][32].
template <class Geo, class OutT, bool kTma>
__device__ __forceinline__ bool intervals_tile(const CUtensorMap *tmap, const uint16_t *img,
                                               OutT *out, const Consts &c, const Tuning &t,
                                               int pixel_groups, int window, int row, int c0,
                                               unsigned char *smem, uint32_t parity) {
  using pos_t = typename Geo::pos_t;
  constexpr int TC = kIntervalTile;
  const int K = c.K, B = c.B;
  const int Kpad = t.kc * t.nchunks;
  const int PS = pixel_groups ? TC : 1;  // depth columns
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  uint16_t *simg = reinterpret_cast<uint16_t *>(smem + 128);
  pos_t *spos = reinterpret_cast<pos_t *>(smem + 128 + align16((size_t)Kpad * TC * 2));
  pos_t *sedge = reinterpret_cast<pos_t *>(reinterpret_cast<unsigned char *>(spos) +
                                           align16((size_t)K * PS * sizeof(pos_t)));
  uint32_t *ssum = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(sedge) +
                                                align16((size_t)(B + 1) * sizeof(pos_t)));
  int32_t *acc = reinterpret_cast<int32_t *>(ssum + TC);
  const int tid = threadIdx.x, NT = blockDim.x;
  const int ncols = min(TC, c.W - c0);
  // thread = (pixel lc, chunk slot warp); with 32 pixels a slot is a warp
  const int lc = tid & (TC - 1), warp = tid / TC, nw = NT / TC;
  const int lcs = pixel_groups ? lc : 0;  // this pixel's depth column
  const bool valid = lc < ncols;

  stage_tile<kTma>(tmap, img, simg, bar, c, t, row, c0);
  {
    const auto *steps = Geo::steps(c);
    if (pixel_groups) {  // steps warp, warp + nw, ... of pixel lc, two at a time
      if (valid) {
        const auto g = Geo::group(c, row * c.W + c0 + lc);
        for (int k = warp; k < K; k += 2 * nw) {
          const int k2 = min(k + nw, K - 1);
          pos_t d0, d1;
          Geo::depth2(g, steps[k], steps[k2], c, d0, d1);
          spos[DR_IDX(k * TC + lc, K * PS, c.err)] = d0;
          if (k + nw < K) spos[DR_IDX((k + nw) * TC + lc, K * PS, c.err)] = d1;
        }
      }
    } else {  // the row's depths, one step per thread
      const auto g = Geo::group(c, row);
      for (int k = tid; k < K; k += NT)
        spos[DR_IDX(k, K * PS, c.err)] = Geo::depth(g, steps[k], c);
    }
  }
  for (int j = tid; j <= B; j += NT) sedge[DR_IDX(j, B + 1, c.err)] = Geo::edge(c, j);
  if (tid < TC) ssum[tid] = 0u;
  __syncthreads();  // also makes the mbarrier initialisation visible
  if constexpr (kTma) {
    const bool late = !mbar_wait_bounded(bar, parity, c.err);
    if (__syncthreads_or(late)) return false;
  }

  const bool rev = c.reverse != 0;
  const float sign = c.out_sign;
  const size_t plane = (size_t)c.H * c.W;
  const bool acc_out = c.accumulate != 0;
  // image value (biased float) of step m in the plan's travel order, and
  // dI of interval m (the step pair m, m + 1)
  auto step_V = [&](int m) {
    return biased(simg[DR_IDX((rev ? K - 1 - m : m) * TC + lc, Kpad * TC, c.err)]);
  };
  auto step_dI = [&](int m) { return (int)__fsub_rn(step_V(m), step_V(m + 1)); };
  constexpr bool kFx = std::is_same<Geo, GeoFx>::value;
  // intervals apportioned by themselves: zero length, and with FP32
  // positions anything shorter than kMinStepUnits
  auto is_short = [](pos_t a, pos_t b) {
    if constexpr (kFx) return (uint32_t)(a < b ? b - a : a - b) < (uint32_t)kMinStepUnits;
    return !(a < b) && !(b < a);
  };
  // b lies above a by an interval that is not short
  auto longer = [](pos_t a, pos_t b) {
    if constexpr (kFx) return b - a >= (pos_t)kMinStepUnits;
    return a < b;
  };
  // this thread's chunk of consecutive intervals m0 .. m1 - 1 of pixel lc
  // (one chunk per slot: C * nw >= K - 1), its range of depths, whether it
  // is a single run, and M = sum_k |dI_k| of each pixel (the chunks' sums,
  // one atomic per chunk)
  const int C = (K - 1 + nw - 1) / nw;
  const int m0 = warp * C, m1 = min(m0 + C, K - 1);
  const bool has_chunk = valid && m0 < m1;
  pos_t cmin = 0, cmax = 0;
  int one_run = 0;  // the chunk is one run with no short interval: 1 rising, 2 falling
  if (has_chunk) {
    uint32_t part = 0u;
    float Vp = step_V(m0);
    cmin = cmax = spos[DR_IDX(m0 * PS + lcs, K * PS, c.err)];
    pos_t dp = cmin;
    bool rise = true, fall = true;
    for (int m = m0; m < m1; ++m) {
      const float Vn = step_V(m + 1);
      part += (uint32_t)abs((int)__fsub_rn(Vp, Vn));
      Vp = Vn;
      const pos_t d = spos[DR_IDX((m + 1) * PS + lcs, K * PS, c.err)];
      cmin = d < cmin ? d : cmin;
      cmax = d > cmax ? d : cmax;
      rise = rise && longer(dp, d);
      fall = fall && longer(d, dp);
      dp = d;
    }
    one_run = rise ? 1 : fall ? 2 : 0;
    if (part) atomicAdd(&ssum[lc], part);
  }
  // number of edges e_i <= x (0..B+1): a guess from the mean bin width,
  // checked against its two neighbouring edges and moved by up to two edges;
  // a binary search when that does not settle it (uneven bins)
  const pos_t e0 = sedge[0];
  const float inv_w = (float)B / (float)(sedge[B] - e0);
  auto count_le = [&](pos_t x) {
    int g = (int)fminf(fmaxf((float)(x - e0) * inv_w + 1.f, 0.f), (float)(B + 1));
#pragma unroll
    for (int it = 0; it < 3; ++it) {
      const bool below_ok = g == 0 || sedge[DR_IDX(g - 1, B + 1, c.err)] <= x;  // e_{g-1} <= x
      const bool above_ok = g == B + 1 || sedge[DR_IDX(g, B + 1, c.err)] > x;   // e_g > x
      if (below_ok && above_ok) return g;
      g += below_ok ? 1 : -1;
    }
    int lo = 0, hi = B + 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sedge[DR_IDX(mid, B + 1, c.err)] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
  };

  float q_scale = 0.f;  // 2^q of pixel lc, read once the sums are complete
  // Interval m of pixel lc by itself, dI != 0, into the bins of the window
  // [wb0, wb1).  A zero-length interval puts dI into the bin [e_j, e_{j+1})
  // holding its depth; a longer one spreads it by overlap.  With FP32
  // positions the depths and edges are the FP64 ones (a binary search on the
  // FP64 edges); a0 is the interval's first position on the kernel's grid.
  auto short_interval = [&](int m, pos_t a0, int dI, int wb0, int wb1) {
    if constexpr (kFx) {
      const GroupD &gd = c.grp64[pixel_groups ? row * c.W + c0 + lc : row];
      const double d0 = depth_f64(gd, c.stp64[m], c), d1 = depth_f64(gd, c.stp64[m + 1], c);
      const double lo = fmin(d0, d1), hi = fmax(d0, d1);
      int j = 0, jh = B;  // first bin: the last edge <= lo, or 0
      if (!(c.e64[0] <= lo)) {
        j = -1;
      } else {
        while (j < jh) {
          const int mid = (j + jh + 1) >> 1;
          if (c.e64[mid] <= lo) j = mid; else jh = mid - 1;
        }
      }
      if (lo == hi) {
        if (j >= wb0 && j < wb1 && j < B)
          atomicAdd(&acc[DR_IDX((j - wb0) * TC + lc, window * TC, c.err)],
                    __float2int_rn(__fmul_rn((float)dI, q_scale)));
        return;
      }
      const double inv = 1.0 / (hi - lo);
      auto P = [&](double e) { return (double)dI * fmin(fmax((e - lo) * inv, 0.0), 1.0); };
      for (j = max(j, wb0); j < wb1 && c.e64[j] < hi; ++j) {
        const float v = (float)(P(c.e64[j + 1]) - P(c.e64[j]));
        if (v != 0.f)
          atomicAdd(&acc[DR_IDX((j - wb0) * TC + lc, window * TC, c.err)],
                    __float2int_rn(__fmul_rn(v, q_scale)));
      }
    } else {  // FP64 positions: only zero-length intervals come here
      const int j = count_le(a0) - 1;
      if (j >= wb0 && j < wb1)
        atomicAdd(&acc[DR_IDX((j - wb0) * TC + lc, window * TC, c.err)],
                  __float2int_rn(__fmul_rn((float)dI, q_scale)));
    }
  };
  for (int wb0 = 0; wb0 < B; wb0 += window) {
    const int wb1 = min(wb0 + window, B);
    const int nwin = (wb1 - wb0) * TC;  // 32 accumulators per bin
    for (int i = tid; i < nwin / 4; i += NT)
      reinterpret_cast<int4 *>(acc)[DR_IDX(i, window * TC / 4, c.err)] = make_int4(0, 0, 0, 0);
    __syncthreads();  // (first window: also the pixels' sums of |dI|)
    if (wb0 == 0) q_scale = iv_pow2(iv_grid(ssum[lc]));
    const pos_t ewlo = sedge[wb0], ewhi = sedge[wb1];
    // One strictly monotone run, intervals m .. n - 1, rising (up) or
    // falling.  Taken in increasing depth, its points are D(0) < ... <
    // D(len) (step m + i, or n - i when falling) with image values V(i);
    // G(e) = V(0) - V(e), V interpolated in depth and clamped to the run, is
    // formed as base + f * d with base = V(0) - V(i) and d = V(i) - V(i+1)
    // on the interval [D(i), D(i+1)] that holds e, as the per-pixel walk
    // forms its running sum.
    auto iv_run = [&](int m, int n, bool up) {
      // the run's points in increasing depth: positions at pd (stride ds)
      // and image values at pv (stride vs), starting at D(0)
      const int len = n - m, s0 = up ? m : n;
      const int ds = up ? PS : -PS, vs = (up != rev) ? TC : -TC;
      const pos_t *pd = spos + s0 * PS + lcs;
      const uint16_t *pv = simg + (rev ? K - 1 - s0 : s0) * TC + lc;
      const pos_t lo_run = *DR_PTR(pd, spos, K * PS, c.err);
      const pos_t hi_run = *DR_PTR(pd + len * ds, spos, K * PS, c.err);
      if (lo_run >= ewhi || hi_run < ewlo) return;  // nothing in this window
      pd += ds;
      pos_t t0 = lo_run, t1 = *DR_PTR(pd, spos, K * PS, c.err);
      const float V0 = biased(*DR_PTR(pv, simg, Kpad * TC, c.err));
      pv += vs;
      float V1 = biased(*DR_PTR(pv, simg, Kpad * TC, c.err));
      float base = 0.f, d = __fsub_rn(V0, V1);
      auto inv = iv_inv_len(t0, t1);
      auto G = [&](pos_t e) {
        const pos_t ec = e < hi_run ? e : hi_run;
        while (t1 < ec) {  // stops at the last point: t1 = D(len) >= ec
          t0 = t1;
          pd += ds;
          t1 = *DR_PTR(pd, spos, K * PS, c.err);
          pv += vs;
          const float Vn = biased(*DR_PTR(pv, simg, Kpad * TC, c.err));
          base = __fsub_rn(V0, V1);
          d = __fsub_rn(V1, Vn);
          V1 = Vn;
          inv = iv_inv_len(t0, t1);
        }
        return __fmaf_rn(iv_frac(ec > t0 ? ec : t0, t0, inv), d, base);
      };
      const float scale = up ? q_scale : -q_scale;  // the run's sign and the pixel's grid
      const int j0 = max(count_le(lo_run) - 1, wb0);
      if constexpr (kFx) {
        // bins j0 .. j1 - 1: those of the window whose lower edge lies below
        // the run's end.  Every upper edge e_{j+1} lies above the run's start
        // (e_{j0 + 1} > D(0), or e_{wb0} > D(0) when the run starts below
        // the window) and so above t0, and a bin's part is added whether or
        // not it is zero (one atomic, no branch)
        const int j1 = min(count_le(hi_run - 1), wb1);
        float g0 = G(sedge[DR_IDX(j0, B + 1, c.err)]);
        int32_t *pa = acc + (j0 - wb0) * TC + lc;
        for (int j = j0; j < j1; ++j, pa += TC) {
          const pos_t e = sedge[DR_IDX(j + 1, B + 1, c.err)];
          const pos_t ec = e < hi_run ? e : hi_run;
          while (t1 < ec) {  // stops at the last point: t1 = D(len) >= ec
            t0 = t1;
            pd += ds;
            t1 = *DR_PTR(pd, spos, K * PS, c.err);
            pv += vs;
            const float Vn = biased(*DR_PTR(pv, simg, Kpad * TC, c.err));
            base = __fsub_rn(V0, V1);
            d = __fsub_rn(V1, Vn);
            V1 = Vn;
            inv = iv_inv_len(t0, t1);
          }
          const float g1 = __fmaf_rn(iv_frac(ec, t0, inv), d, base);
          atomicAdd(DR_PTR(pa, acc, window * TC, c.err),
                    __float2int_rn(__fmul_rn(__fsub_rn(g1, g0), scale)));
          g0 = g1;
        }
        return;
      }
      const pos_t *pe = sedge + j0;
      int32_t *pa = acc + (j0 - wb0) * TC + lc;
      int32_t *const pa_end = acc + (wb1 - wb0) * TC;
      float g0 = G(*DR_PTR(pe, sedge, B + 1, c.err));
      for (; pa < pa_end && *DR_PTR(pe, sedge, B + 1, c.err) < hi_run; ++pe, pa += TC) {
        const float g1 = G(*DR_PTR(pe + 1, sedge, B + 1, c.err));
        const float v = __fsub_rn(g1, g0);
        if (v != 0.f)
          atomicAdd(DR_PTR(pa, acc, window * TC, c.err), __float2int_rn(__fmul_rn(v, scale)));
        g0 = g1;
      }
    };
    // the chunk splits into strictly monotone runs and zero-length
    // intervals, and each run is walked once over the bins it spans; a chunk
    // whose depths miss the window is skipped whole
    // (FP32 positions: a margin of kMinStepUnits for the short intervals'
    // FP64 depths)
    const pos_t margin = kFx ? (pos_t)kMinStepUnits : (pos_t)0;
    if (has_chunk && cmax + margin >= ewlo && cmin - margin < ewhi) {
      if (one_run) {  // the split below would find the one run
        iv_run(m0, m1, one_run == 1);
      } else {
        for (int m = m0; m < m1;) {
          const pos_t a = spos[DR_IDX(m * PS + lcs, K * PS, c.err)],
                      b = spos[DR_IDX((m + 1) * PS + lcs, K * PS, c.err)];
          if (is_short(a, b)) {
            const int dI = step_dI(m);
            if (dI != 0) short_interval(m, a, dI, wb0, wb1);
            ++m;
            continue;
          }
          const bool up = a < b;
          int n = m + 1;  // the run: intervals m .. n - 1
          for (pos_t prev = b; n < m1; ++n) {
            const pos_t nx = spos[DR_IDX((n + 1) * PS + lcs, K * PS, c.err)];
            if (!(up ? longer(prev, nx) : longer(nx, prev))) break;
            prev = nx;
          }
          iv_run(m, n, up);
          m = n;
        }
      }
    }
    __syncthreads();
    if (!acc_out && ncols == TC && c.W % 4 == 0 &&
        ((uintptr_t)out & (4 * sizeof(OutT) - 1)) == 0) {
      // 4 pixels per thread (the same 4 in every pass: NT is a multiple of
      // TC / 4), one 16-byte shared load and one vector store; TC / 4 threads
      // store a bin's line of 4 TC bytes
      const int p0 = (tid % (TC / 4)) * 4;
      float w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) w[u] = __fmul_rn(sign, iv_pow2(-iv_grid(ssum[p0 + u])));
      // thread tid stores bins wb0 + tid / (TC / 4) + i * NT / (TC / 4)
      const int4 *pq = reinterpret_cast<const int4 *>(acc) + tid;
      const int4 *const pq_end = reinterpret_cast<const int4 *>(acc) + nwin / 4;
      OutT *o = out + (size_t)(wb0 + tid / (TC / 4)) * plane + (size_t)row * c.W + c0 + p0;
      const size_t o_step = (size_t)(NT / (TC / 4)) * plane;
      for (; pq < pq_end; pq += NT, o += o_step) {
        const int4 a = *DR_PTR(pq, reinterpret_cast<const int4 *>(acc), window * TC / 4, c.err);
        st_cs4(DR_PTR(o, out, plane * B - 3, c.err), __fmul_rn(__int2float_rn(a.x), w[0]),
               __fmul_rn(__int2float_rn(a.y), w[1]), __fmul_rn(__int2float_rn(a.z), w[2]),
               __fmul_rn(__int2float_rn(a.w), w[3]));
      }
    } else {
      const float w = __fmul_rn(sign, iv_pow2(-iv_grid(ssum[lc])));
      for (int i = tid; i < nwin; i += NT) {  // i % TC = lc: NT is a multiple of TC
        if (!valid) continue;
        OutT *o = DR_PTR(out + (size_t)(wb0 + i / TC) * plane + (size_t)row * c.W + c0 + lc,
                         out, plane * B, c.err);
        const float v = __fmul_rn(__int2float_rn(acc[DR_IDX(i, window * TC, c.err)]), w);
        st_cs(o, acc_out ? __fadd_rn(out_load(o), v) : v);
      }
    }
    if (wb1 < B) __syncthreads();  // the window's accumulators are reused
  }
  return true;
}

// One CTA per tile (grid: tiles along the row x rows), kMinBlocks CTAs per
// SM: three (40 registers) when the plan's tile fits three times, else two
// with FP32 geometry (64 registers), one with FP64.
template <class Geo, class OutT, bool kTma, int kMinBlocks>
__global__ void __launch_bounds__(512, kMinBlocks)
    intervals_kernel(const __grid_constant__ CUtensorMap tmap, const uint16_t *__restrict__ img,
                     OutT *__restrict__ out, const Consts c, const Tuning t, int pixel_groups,
                     int window) {
  extern __shared__ __align__(128) unsigned char smem[];
  // thread 0 initialises the barrier and issues the copies; the others
  // first poll it after the tile's first __syncthreads
  if constexpr (kTma) {
    if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
  }
  intervals_tile<Geo, OutT, kTma>(&tmap, img, out, c, t, pixel_groups, window, blockIdx.y,
                                  blockIdx.x * kIntervalTile, smem, 0u);
}

}  // namespace dr
