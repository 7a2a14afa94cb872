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
// A CTA owns one row x 8 adjacent pixels x all K steps (image tile staged by
// TMA as in the other kernels, depths of the 8 pixels in shared memory); a
// warp covers 4 steps x the 8 pixels when it evaluates depths, and 4 chunks
// of consecutive intervals x the 8 pixels when it apportions.  The bins go
// through shared-memory windows of `window` int64 accumulators per pixel.
// Each thread splits its chunk into strictly monotone runs (and zero-length
// intervals) and walks each run once over the bins it spans, adding
// Phi(e_{j+1}) - Phi(e_j) summed over the run's intervals, Phi(e) =
// round(dI * phi(e) * 2^30) on the fixed-point grid 2^-30 (so the parts of
// one interval add up to dI exactly), with shared-memory atomics.  Integer
// sums do not depend on the order of the atomics, so the result is
// deterministic and does not depend on how the intervals are grouped.  The
// window is then written out, 8 pixels of one bin being one 32-byte sector.
#pragma once

#include "dr_device.cuh"
#include "dr_internal.h"

namespace dr {

constexpr float kIvScale = 1073741824.f;  // 2^30: fixed-point grid of the sums

// round(q * 2^30) for |q| < 2^31 without 64-bit conversions (those run on
// the FP64 pipe): q = i + r with i = trunc(q) and r = q - i exact, and
// r * 2^30 < 2^30 in magnitude
__device__ __forceinline__ long long iv_fix(float q) {
  const int i = __float2int_rz(q);
  const int r = __float2int_rn(__fmul_rn(__fsub_rn(q, (float)i), kIvScale));
  return (long long)i * (1ll << 30) + r;
}
// Phi(e) = round(dI * phi(e) * 2^30), phi(e) = clamp((e - lo) / (hi - lo), 0, 1);
// edges at or beyond an end give 0 or dI * 2^30 exactly
__device__ __forceinline__ long long iv_phi(int32_t e, int32_t lo, int32_t hi, float inv_len,
                                            int dI) {
  if (e <= lo) return 0;
  if (e >= hi) return (long long)dI * (1ll << 30);
  const float f = fminf(__fmul_rn(__uint2float_rn((uint32_t)e - (uint32_t)lo), inv_len), 1.f);
  return iv_fix(__fmul_rn((float)dI, f));
}
__device__ __forceinline__ long long iv_phi(double e, double lo, double hi, double inv_len,
                                            int dI) {
  if (e <= lo) return 0;
  if (e >= hi) return (long long)dI * (1ll << 30);
  const double f = fmin((e - lo) * inv_len, 1.0);
  return __double2ll_rn((double)dI * f * (double)kIvScale);
}
__device__ __forceinline__ float iv_inv_len(int32_t lo, int32_t hi) {
  return __frcp_rn(__uint2float_rn((uint32_t)hi - (uint32_t)lo));
}
__device__ __forceinline__ double iv_inv_len(double lo, double hi) { return 1.0 / (hi - lo); }
// accumulator (units of 2^-30) to FP32: hi * 4 + lo * 2^-30 with one
// rounding while |hi| < 2^24, i.e. for bin values below 2^26 counts (any
// real scan); larger values (extreme counts of thousands of steps piled into
// one bin) are within one ulp
__device__ __forceinline__ float iv_value(long long a) {
  const int hi = (int)(a >> 32);
  const uint32_t lo = (uint32_t)a;
  return __fmaf_rn(__uint2float_rn(lo), 1.f / kIvScale, __fmul_rn((float)hi, 4.f));
}

template <class Geo, class OutT, bool kTma>
__global__ void __launch_bounds__(512) intervals_kernel(const __grid_constant__ CUtensorMap tmap,
                                                        const uint16_t *__restrict__ img,
                                                        OutT *__restrict__ out, const Consts c,
                                                        const Tuning t, int pixel_groups,
                                                        int window) {
  using pos_t = typename Geo::pos_t;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  uint16_t *simg = reinterpret_cast<uint16_t *>(smem + 128);
  constexpr int TC = kIntervalTile;
  const int K = c.K, B = c.B;
  const int Kpad = t.kc * t.nchunks;
  pos_t *spos = reinterpret_cast<pos_t *>(smem + 128 + align16((size_t)Kpad * TC * 2));
  pos_t *sedge = reinterpret_cast<pos_t *>(reinterpret_cast<unsigned char *>(spos) +
                                           align16((size_t)K * TC * sizeof(pos_t)));
  unsigned long long *acc = reinterpret_cast<unsigned long long *>(
      reinterpret_cast<unsigned char *>(sedge) + align16((size_t)(B + 1) * sizeof(pos_t)));
  const int row = blockIdx.y, c0 = blockIdx.x * TC;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int ncols = min(TC, c.W - c0);

  if constexpr (kTma) {
    if (tid == 0) mbar_init(bar, 1);
  }
  stage_tile<kTma>(&tmap, img, simg, bar, c, t, row, c0);
  // a warp covers 4 steps x the 8 pixels (lane = 8 * step + pixel), so its
  // shared-memory accesses to the [step][pixel] arrays are contiguous
  const int warp = tid >> 5, lane = tid & 31, nwarps = NT >> 5;
  const int lc = lane & (TC - 1), s4 = warp * 4 + (lane >> 3), S = nwarps * 4;
  {  // depths of the tile: steps s4, s4 + S, ... of pixel lc, two at a time
    if (lc < ncols) {
      const auto g = Geo::group(c, pixel_groups ? row * c.W + c0 + lc : row);
      const auto *steps = Geo::steps(c);
      for (int k = s4; k < K; k += 2 * S) {
        const int k2 = min(k + S, K - 1);
        pos_t d0, d1;
        Geo::depth2(g, steps[k], steps[k2], c, d0, d1);
        spos[DR_IDX(k * TC + lc, K * TC, c.err)] = d0;
        if (k + S < K) spos[DR_IDX((k + S) * TC + lc, K * TC, c.err)] = d1;
      }
    }
  }
  for (int j = tid; j <= B; j += NT) sedge[DR_IDX(j, B + 1, c.err)] = Geo::edge(c, j);
  __syncthreads();  // also makes the mbarrier initialisation visible
  if constexpr (kTma) {
    const bool late = !mbar_wait_bounded(bar, 0, c.err);
    if (__syncthreads_or(late)) return;
  }

  const bool rev = c.reverse != 0;
  const float sign = c.out_sign;
  const size_t plane = (size_t)c.H * c.W;
  const bool acc_out = c.accumulate != 0;
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

  // dI of interval m (the step pair it joins, in the plan's travel order)
  auto step_dI = [&](int m) {
    const int ia = rev ? K - 1 - m : m, ib = rev ? K - 2 - m : m + 1;
    const int n_simg = Kpad * TC;
    return (int)simg[DR_IDX(ia * TC + lc, n_simg, c.err)] -
           (int)simg[DR_IDX(ib * TC + lc, n_simg, c.err)];
  };
  // intervals per chunk: one chunk per thread where K allows; odd, so that
  // the 4 chunks of a warp start in different banks
  const int C = ((K - 1 + S - 1) / S) | 1;

  for (int wb0 = 0; wb0 < B; wb0 += window) {
    const int wb1 = min(wb0 + window, B);
    const int nwin = (wb1 - wb0) * TC;  // even: 8 accumulators per bin
    for (int i = tid; i < nwin / 2; i += NT)
      reinterpret_cast<ulonglong2 *>(acc)[DR_IDX(i, window * TC / 2, c.err)] =
          make_ulonglong2(0ull, 0ull);
    __syncthreads();
    const pos_t ewlo = sedge[wb0], ewhi = sedge[wb1];
    // One strictly monotone run, intervals m .. n - 1, rising (up) or
    // falling.  Taken in increasing depth, its positions are D(0) < ... <
    // D(len) and interval i joins D(i) and D(i + 1).  At an edge e the sum
    // over the run's intervals of Phi_k(e) is P(e) = (sum of dI * 2^30 over
    // the intervals below e) + Phi of the interval holding e, so a bin gets
    // P(e_{j+1}) - P(e_j): the same integer as the sum of the intervals'
    // own differences, with one atomic per bin instead of one per interval.
    auto iv_run = [&](int m, int n, bool up) {
      const int len = n - m;
      auto D = [&](int i) { return spos[DR_IDX((up ? m + i : n - i) * TC + lc, K * TC, c.err)]; };
      const pos_t lo_run = D(0), hi_run = D(len);
      if (lo_run >= ewhi || hi_run < ewlo) return;  // nothing in this window
      int i = 0;
      pos_t lo_i = lo_run, hi_i = D(1);
      int dI = step_dI(up ? m : n - 1);
      auto inv = iv_inv_len(lo_i, hi_i);
      long long cum = 0;  // dI * 2^30 summed over the intervals below i
      auto P = [&](pos_t e) {
        while (i < len && !(e < hi_i)) {
          cum += (long long)dI * (1ll << 30);
          if (++i < len) {
            lo_i = hi_i;
            hi_i = D(i + 1);
            dI = step_dI(up ? m + i : n - 1 - i);
            inv = iv_inv_len(lo_i, hi_i);
          }
        }
        return i < len ? cum + iv_phi(e, lo_i, hi_i, inv, dI) : cum;
      };
      int j = max(count_le(lo_run) - 1, wb0);
      long long p0 = P(sedge[DR_IDX(j, B + 1, c.err)]);
      for (; j < wb1 && sedge[DR_IDX(j, B + 1, c.err)] < hi_run; ++j) {
        const long long p1 = P(sedge[DR_IDX(j + 1, B + 1, c.err)]);
        if (p1 != p0)
          atomicAdd(&acc[DR_IDX((j - wb0) * TC + lc, window * TC, c.err)],
                    (unsigned long long)(p1 - p0));
        p0 = p1;
      }
    };
    // chunks of C consecutive intervals of pixel lc, chunk q = s4, s4 + S,
    // ...; a chunk splits into strictly monotone runs and zero-length
    // intervals, and each run is walked once over the bins it spans
    for (int q = s4; q * C < K - 1 && lc < ncols; q += S) {
      const int m1 = min(q * C + C, K - 1);
      for (int m = q * C; m < m1;) {
        const pos_t a = spos[DR_IDX(m * TC + lc, K * TC, c.err)],
                    b = spos[DR_IDX((m + 1) * TC + lc, K * TC, c.err)];
        if (!(a < b) && !(b < a)) {  // zero length: the bin [e_j, e_{j+1}) holding a
          const int dI = step_dI(m);
          const int j = count_le(a) - 1;
          if (dI != 0 && j >= wb0 && j < wb1)
            atomicAdd(&acc[DR_IDX((j - wb0) * TC + lc, window * TC, c.err)],
                      (unsigned long long)((long long)dI * (1ll << 30)));
          ++m;
          continue;
        }
        const bool up = a < b;
        int n = m + 1;  // the run: intervals m .. n - 1
        for (pos_t prev = b; n < m1; ++n) {
          const pos_t nx = spos[DR_IDX((n + 1) * TC + lc, K * TC, c.err)];
          if (up ? !(prev < nx) : !(nx < prev)) break;
          prev = nx;
        }
        iv_run(m, n, up);
        m = n;
      }
    }
    __syncthreads();
    if (!acc_out && ncols == TC && c.W % 4 == 0 &&
        ((uintptr_t)out & (4 * sizeof(OutT) - 1)) == 0) {
      // 4 pixels per thread: two 16-byte shared loads, one vector store
      for (int q = tid; q < nwin / 4; q += NT) {
        const int jj = q >> 1, half = q & 1;
        const ulonglong2 a =
            reinterpret_cast<const ulonglong2 *>(acc)[DR_IDX(2 * q, window * TC / 2, c.err)];
        const ulonglong2 b =
            reinterpret_cast<const ulonglong2 *>(acc)[DR_IDX(2 * q + 1, window * TC / 2, c.err)];
        OutT *o = DR_PTR(out + (size_t)(wb0 + jj) * plane + (size_t)row * c.W + c0 + 4 * half,
                         out, plane * B - 3, c.err);
        st_cs4(o, __fmul_rn(sign, iv_value((long long)a.x)),
               __fmul_rn(sign, iv_value((long long)a.y)),
               __fmul_rn(sign, iv_value((long long)b.x)),
               __fmul_rn(sign, iv_value((long long)b.y)));
      }
    } else {
      for (int i = tid; i < nwin; i += NT) {
        const int jj = i / TC, px = i - jj * TC;
        if (px >= ncols) continue;
        OutT *o = DR_PTR(out + (size_t)(wb0 + jj) * plane + (size_t)row * c.W + c0 + px, out,
                         plane * B, c.err);
        const float v = __fmul_rn(sign, iv_value((long long)acc[DR_IDX(i, window * TC, c.err)]));
        st_cs(o, acc_out ? __fadd_rn(out_load(o), v) : v);
      }
    }
    __syncthreads();  // the window's accumulators are reused
  }
}

}  // namespace dr
