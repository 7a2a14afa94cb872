// Reconstruction kernels (sm_103a) and the launch side of the C ABI.
//
// Two kernels compute the same result:
//
//  rows_kernel    all pixels of a detector row share their projected
//                 position (columns run along the wire axis), so a CTA that
//                 owns a row segment computes the row's depth positions once,
//                 turns every bin edge e_j into a (step k_j, fraction f_j)
//                 pair, and then streams the bins: per pixel and edge
//                 F_j = S_k + f_j * dI_k with S_k = I_0 - I_k, dI_k = I_k -
//                 I_{k+1} (exact in FP32), out_j = F_{j+1} - F_j.
//  pixels_kernel  every pixel has its own depth sequence; each lane walks its
//                 steps and the bins in lockstep with the other lanes
//                 (merge-walk), evaluating depths as it goes.
//
// F is the running sum of the differences, linearly interpolated in depth
// between step depths, so F_{j+1} - F_j equals the sum over intervals of
// dI_k * |[d_k, d_{k+1}] intersect [e_j, e_{j+1})| / |d_{k+1} - d_k| (the
// paper's per-pixel accumulation of differences into depth, Sec. III-C),
// and each output element is written exactly once.  The image tile (a
// segment of one row x all steps) is staged into shared memory by TMA.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "dr_internal.h"

namespace dr {

// ------------------------------------------------------------------ PTX ---

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Wait for the TMA phase with a time limit.  On timeout the error word is
// set, the copies in flight get a second bounded wait to land, and the caller
// returns without touching the tile.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int32_t *err) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > kWaitLimitNs) {
      atomicExch(err, kDevTmaTimeout);
      uint64_t t1 = global_ns();
      while (!mbar_try_wait(bar, parity) && global_ns() - t1 < kWaitLimitNs) {
      }
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void st_cs(float *p, float v) {
  asm volatile("st.global.cs.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cs4(float *p, float a, float b, float c, float d) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}
__device__ __forceinline__ void st_cs(__nv_bfloat16 *p, float v) {
  __nv_bfloat16 h = __float2bfloat16_rn(v);
  unsigned short u = *reinterpret_cast<unsigned short *>(&h);
  asm volatile("st.global.cs.b16 [%0], %1;" ::"l"(p), "h"(u) : "memory");
}
__device__ __forceinline__ void st_cs4(__nv_bfloat16 *p, float a, float b, float c, float d) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  uint32_t ul = *reinterpret_cast<uint32_t *>(&lo), uh = *reinterpret_cast<uint32_t *>(&hi);
  asm volatile("st.global.cs.v2.b32 [%0], {%1, %2};" ::"l"(p), "r"(ul), "r"(uh) : "memory");
}

// --------------------------------------------------------- depth model ---

// FP32 depth position of (group, step) in fixed point (see dr_internal.h).
__device__ __forceinline__ int32_t depth_fx(const GroupC &g, const StepC &s, const Consts &c) {
  const float z = s.zf;
  float inv = g.invD;
  float a = __fmul_rn(c.y0, z);
  if (c.has_eta) {
    inv = rcp_approx(__fsub_rn(g.D, s.eta));
    a = __fmaf_rn(s.eta, __fadd_rn(__fsub_rn(z, g.Z), g.Q0f), a);
  }
  const float tap = __fmaf_rn(a, inv, __fadd_rn(z, g.Q0f));
  const float u = __fsub_rn(g.Z, tap);
  const float L = sqrt_approx(__fmaf_rn(u, u, g.Y2));
  const float num = __fmul_rn(tap, __fsub_rn(tap, __fadd_rn(g.Z, g.Z)));
  const float dL = __fmul_rn(num, rcp_approx(__fadd_rn(L, g.L0)));
  const float rem = __fmul_rn(__fmaf_rn(c.sR, dL, a), inv);
  const int32_t rfx = __float2int_rn(__fmul_rn(rem, c.scale));
  return (int32_t)((uint32_t)s.zfx + (uint32_t)g.Q0fx + (uint32_t)rfx);
}

// FP64 depth position of (group, step) relative to the plan origin.
__device__ __forceinline__ double depth_f64(const GroupD &g, const StepD &s, const Consts &c) {
  const double z = s.z, Dm = g.D - s.eta;
  const double a = c.y0d * z + s.eta * (z - g.Z + g.Q0);
  double rem = a / Dm;
  for (int it = 0; it < 2; ++it) {
    const double t = z + g.Q0 + rem;
    const double u = g.Z - t;
    const double L = sqrt(g.Y2 + u * u);
    const double dL = t * (t - 2.0 * g.Z) / (L + g.L0);
    rem = (a + c.sRd * dL) / Dm;
  }
  return ((z - c.origin) + g.Q0) + rem;
}

struct GeoFx {
  using pos_t = int32_t;
  using step_t = StepC;
  using group_t = GroupC;
  static __device__ __forceinline__ const StepC *steps(const Consts &c) { return c.stp; }
  static __device__ __forceinline__ const GroupC &group(const Consts &c, int i) {
    return c.grp[i];
  }
  static __device__ __forceinline__ pos_t depth(const GroupC &g, const StepC &s,
                                                const Consts &c) {
    return depth_fx(g, s, c);
  }
  static __device__ __forceinline__ pos_t edge(const Consts &c, int j) { return c.efx[j]; }
  // 1 / (b - a) for a < b (approximate reciprocal; same value in both kernels)
  static __device__ __forceinline__ float inv_len(pos_t a, pos_t b) {
    return rcp_approx(__int2float_rn(b - a));
  }
  static __device__ __forceinline__ float frac(pos_t e, pos_t a, float inv) {
    float f = __fmul_rn(__int2float_rn(e - a), inv);
    return fminf(fmaxf(f, 0.f), 1.f);
  }
  static __device__ __forceinline__ double to_mm(pos_t p, const Consts &c) {
    return ((double)p / (double)c.scale + c.origin) / c.nb;
  }
};

struct GeoF64 {
  using pos_t = double;
  using step_t = StepD;
  using group_t = GroupD;
  static __device__ __forceinline__ const StepD *steps(const Consts &c) { return c.stp64; }
  static __device__ __forceinline__ const GroupD &group(const Consts &c, int i) {
    return c.grp64[i];
  }
  static __device__ __forceinline__ pos_t depth(const GroupD &g, const StepD &s,
                                                const Consts &c) {
    return depth_f64(g, s, c);
  }
  static __device__ __forceinline__ pos_t edge(const Consts &c, int j) { return c.e64[j]; }
  static __device__ __forceinline__ double inv_len(pos_t a, pos_t b) { return 1.0 / (b - a); }
  static __device__ __forceinline__ float frac(pos_t e, pos_t a, double inv) {
    double f = (e - a) * inv;
    return (float)fmin(fmax(f, 0.0), 1.0);
  }
  static __device__ __forceinline__ double to_mm(pos_t p, const Consts &c) {
    return (p + c.origin) / c.nb;
  }
};

// ------------------------------------------------------ pixel values ---
// A uint16 count x is held as the float 2^23 + x (bit pattern 0x4B00_0000 | x):
// exact, and differences of two such values are the exact integer
// differences (|x - y| < 2^16 << 2^24).
__device__ __forceinline__ float biased_lo(uint32_t w) {
  return __uint_as_float(__byte_perm(w, 0x4B00u, 0x5410));
}
__device__ __forceinline__ float biased_hi(uint32_t w) {
  return __uint_as_float(__byte_perm(w, 0x4B00u, 0x5432));
}
__device__ __forceinline__ float biased(uint16_t x) {
  return __uint_as_float(0x4B000000u | (uint32_t)x);
}

// Exact difference I_k - I_{k+1} as the kernels form it.
__device__ __forceinline__ float step_delta(uint16_t a, uint16_t b) {
  return __fsub_rn(biased(a), biased(b));
}

template <int PPT>
__device__ __forceinline__ void load_px(const uint16_t *p, float (&v)[PPT]) {
  if constexpr (PPT == 4) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    v[0] = biased_lo(u.x);
    v[1] = biased_hi(u.x);
    v[2] = biased_lo(u.y);
    v[3] = biased_hi(u.y);
  } else {
#pragma unroll
    for (int i = 0; i < PPT; ++i) v[i] = biased(p[i]);
  }
}

template <class OutT, int PPT>
__device__ __forceinline__ void store_px(OutT *p, const float (&v)[PPT]) {
  if constexpr (PPT == 4) {
    st_cs4(p, v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int i = 0; i < PPT; ++i) st_cs(p + i, v[i]);
  }
}

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Stage rows r of the image tile [K][1][tile_cols] (columns c0..) into smem:
// by TMA when a tensor map is given, else with plain loads (zero-filled tail).
template <bool kTma>
__device__ __forceinline__ void stage_tile(const CUtensorMap *tmap, const uint16_t *img,
                                           uint16_t *simg, uint64_t *bar, const Consts &c,
                                           const Tuning &t, int row, int c0) {
  const int TC = t.tile_cols;
  if constexpr (kTma) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      mbar_expect_tx(bar, (uint32_t)(t.kc * t.nchunks * TC * 2));
      for (int ch = 0; ch < t.nchunks; ++ch)
        tma_load_3d(simg + (size_t)ch * t.kc * TC, tmap, bar, c0, row, ch * t.kc);
    }
  } else {
    const int n = c.K * TC;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int k = i / TC, cc = i - k * TC, col = c0 + cc;
      simg[i] = col < c.W ? img[((size_t)k * c.H + row) * c.W + col] : (uint16_t)0;
    }
  }
}

// --------------------------------------------------------- rows kernel ---

template <class Geo, class OutT, bool kTma, int PPT>
__global__ void __launch_bounds__(512) rows_kernel(const __grid_constant__ CUtensorMap tmap,
                                                   const uint16_t *__restrict__ img,
                                                   OutT *__restrict__ out, const Consts c,
                                                   const Tuning t) {
  using pos_t = typename Geo::pos_t;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  uint16_t *simg = reinterpret_cast<uint16_t *>(smem + 128);
  const int TC = t.tile_cols, K = c.K, B = c.B;
  const int Kpad = t.kc * t.nchunks;
  pos_t *spos = reinterpret_cast<pos_t *>(smem + 128 + align16((size_t)Kpad * TC * 2));
  int2 *stab = reinterpret_cast<int2 *>(reinterpret_cast<unsigned char *>(spos) +
                                        align16((size_t)K * sizeof(pos_t)));
  const int row = blockIdx.y, c0 = blockIdx.x * TC;
  const int tid = threadIdx.x, NT = blockDim.x;

  stage_tile<kTma>(&tmap, img, simg, bar, c, t, row, c0);

  int *zcount = reinterpret_cast<int *>(bar + 1);
  if (tid == 0) zcount[0] = zcount[1] = 0;
  // depth positions of this row (processing order: increasing depth)
  const auto &g = Geo::group(c, row);
  const auto *steps = Geo::steps(c);
  for (int k = tid; k < K; k += NT) spos[k] = Geo::depth(g, steps[k], c);
  __syncthreads();
  // each bin edge -> (k, f): k = last step below the edge (clamped to an
  // interval), f = position of the edge inside [d_k, d_{k+1}], clamped.
  // Edges at or below d_0 give F = 0 and edges at or above d_{K-1} give
  // F = S_{K-1}, so only bins [nz_lo, nz_hi) can hold data.
  int below = 0, above = 0;
  const pos_t tfirst = spos[0], tlast = spos[K - 1];
  for (int j = tid; j <= B; j += NT) {
    const pos_t e = Geo::edge(c, j);
    int lo = 0, hi = K;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (spos[mid] < e) lo = mid + 1; else hi = mid;
    }
    const int k = min(max(lo - 1, 0), K - 2);
    const float f = Geo::frac(e, spos[k], Geo::inv_len(spos[k], spos[k + 1]));
    stab[j] = make_int2(k, __float_as_int(f));
    below += !(e > tfirst);
    above += !(e < tlast);
  }
  if (below) atomicAdd(&zcount[0], below);
  if (above) atomicAdd(&zcount[1], above);
  __syncthreads();
  const int nz_hi = min(B + 1 - zcount[1], B);
  const int nz_lo = min(max(zcount[0] - 1, 0), nz_hi);
  if constexpr (kTma) {
    if (!mbar_wait_bounded(bar, 0, c.err)) return;
  }

  // stream the bins; thread = PPT adjacent pixels; the zero ranges and the
  // data range are each split evenly over the bin groups
  const int lanes = TC / PPT;
  const int lane = tid % lanes, grp = tid / lanes;
  const int lc = lane * PPT, col = c0 + lc;
  if (col >= c.W) return;
  const int G = t.bin_groups;
  auto slice_lo = [&](int lo, int hi) { return lo + (int)((long long)(hi - lo) * grp / G); };
  auto slice_hi = [&](int lo, int hi) { return lo + (int)((long long)(hi - lo) * (grp + 1) / G); };
  const float sign = c.out_sign;
  const size_t plane = (size_t)c.H * c.W;
  OutT *const o0 = out + (size_t)row * c.W + col;
  float zero[PPT];
#pragma unroll
  for (int i = 0; i < PPT; ++i) zero[i] = __fmul_rn(sign, 0.f);
  auto zero_fill = [&](int a, int b) {
    OutT *o = o0 + (size_t)a * plane;
#pragma unroll 4
    for (int j = a; j < b; ++j, o += plane) store_px<OutT, PPT>(o, zero);
  };
  zero_fill(slice_lo(0, nz_lo), slice_hi(0, nz_lo));
  zero_fill(slice_lo(nz_hi, B), slice_hi(nz_hi, B));

  const int a = slice_lo(nz_lo, nz_hi), b = slice_hi(nz_lo, nz_hi);
  if (a >= b) return;
  const bool rev = c.reverse != 0;
  auto srow = [&](int k) { return simg + (size_t)(rev ? K - 1 - k : k) * TC + lc; };
  float I0[PPT];
  load_px<PPT>(srow(0), I0);
  auto evalF = [&](int2 kf, float (&F)[PPT]) {
    float x[PPT], y[PPT];
    load_px<PPT>(srow(kf.x), x);
    load_px<PPT>(srow(kf.x + 1), y);
    const float f = __int_as_float(kf.y);
#pragma unroll
    for (int i = 0; i < PPT; ++i)
      F[i] = __fmaf_rn(f, __fsub_rn(x[i], y[i]), __fsub_rn(I0[i], x[i]));
  };
  float Fp[PPT];
  evalF(stab[a], Fp);
  OutT *o = o0 + (size_t)a * plane;
#pragma unroll 4
  for (int j = a; j < b; ++j, o += plane) {
    float Fn[PPT], v[PPT];
    evalF(stab[j + 1], Fn);
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      v[i] = __fmul_rn(sign, __fsub_rn(Fn[i], Fp[i]));
      Fp[i] = Fn[i];
    }
    store_px<OutT, PPT>(o, v);
  }
}

// ------------------------------------------------------- pixels kernel ---

template <class Geo, class OutT, bool kTma>
__global__ void __launch_bounds__(256) pixels_kernel(const __grid_constant__ CUtensorMap tmap,
                                                     const uint16_t *__restrict__ img,
                                                     OutT *__restrict__ out, const Consts c,
                                                     const Tuning t) {
  using pos_t = typename Geo::pos_t;
  using step_t = typename Geo::step_t;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  uint16_t *simg = reinterpret_cast<uint16_t *>(smem + 128);
  const int TC = t.tile_cols, K = c.K, B = c.B;
  const int Kpad = t.kc * t.nchunks;
  step_t *sstep = reinterpret_cast<step_t *>(smem + 128 + align16((size_t)Kpad * TC * 2));
  pos_t *sedge = reinterpret_cast<pos_t *>(reinterpret_cast<unsigned char *>(sstep) +
                                           align16((size_t)K * sizeof(step_t)));
  const int row = blockIdx.y, c0 = blockIdx.x * TC;
  const int tid = threadIdx.x, NT = blockDim.x;

  stage_tile<kTma>(&tmap, img, simg, bar, c, t, row, c0);
  const step_t *gsteps = Geo::steps(c);
  for (int k = tid; k < K; k += NT) sstep[k] = gsteps[k];
  for (int j = tid; j <= B; j += NT) sedge[j] = Geo::edge(c, j);
  __syncthreads();
  if constexpr (kTma) {
    if (!mbar_wait_bounded(bar, 0, c.err)) return;
  }
  const int col = c0 + tid;
  if (col >= c.W) return;
  const auto g = Geo::group(c, row * c.W + col);
  const bool rev = c.reverse != 0;
  auto spx = [&](int k) { return biased(simg[(size_t)(rev ? K - 1 - k : k) * TC + tid]); };

  // lockstep merge-walk: every lane handles bin edge j together, each with
  // its own step pointer k (t0 = d_k, t1 = d_{k+1})
  int k = 0;
  pos_t t0 = Geo::depth(g, sstep[0], c), t1 = Geo::depth(g, sstep[1], c);
  auto inv = Geo::inv_len(t0, t1);
  const float I0 = spx(0);
  float Ik = I0, Ik1 = spx(1);
  const float sign = c.out_sign;
  const size_t plane = (size_t)c.H * c.W;
  OutT *o = out + (size_t)row * c.W + col;
  float Fp = 0.f;
  for (int j = 0; j <= B; ++j) {
    const pos_t e = sedge[j];
    while (k < K - 2 && t1 < e) {
      ++k;
      t0 = t1;
      t1 = Geo::depth(g, sstep[k + 1], c);
      inv = Geo::inv_len(t0, t1);
      Ik = Ik1;
      Ik1 = spx(k + 1);
    }
    const float f = Geo::frac(e, t0, inv);
    const float F = __fmaf_rn(f, __fsub_rn(Ik, Ik1), __fsub_rn(I0, Ik));
    if (j > 0) {
      st_cs(o, __fmul_rn(sign, __fsub_rn(F, Fp)));
      o += plane;
    }
    Fp = F;
  }
}

// ------------------------------------------------ small helper kernels ---

__global__ void differences_kernel(const uint16_t *__restrict__ img, long long n_out,
                                   long long plane, int32_t *__restrict__ d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_out;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = __float2int_rn(step_delta(img[i], img[i + plane]));
}

template <class Geo>
__global__ void depths_kernel(const Consts c, int kernel, int r0, int nrows, double *out) {
  const long long n = (long long)nrows * c.W * c.K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i % c.K);
    const long long pc = i / c.K;
    const int col = (int)(pc % c.W), r = r0 + (int)(pc / c.W);
    const int gi = kernel == DR_KERNEL_ROWS ? r : r * c.W + col;
    const int kp = c.reverse ? c.K - 1 - k : k;
    out[i] = Geo::to_mm(Geo::depth(Geo::group(c, gi), Geo::steps(c)[kp], c), c);
  }
}

// ------------------------------------------------------------- launch ---

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                         cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }();
  return fn;
}

// Raise the dynamic shared-memory limit of a kernel once per device.
dr_status allow_smem(const void *fn) {
  static std::mutex mu;
  static const void *done[256][8];
  static int ndone[8];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
  int slot = dev & 7;
  std::lock_guard<std::mutex> lk(mu);
  for (int i = 0; i < ndone[slot]; ++i)
    if (done[i][slot] == fn) return DR_OK;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return cuda_fail("cudaFuncSetAttribute", e);
  if (ndone[slot] < 256) done[ndone[slot]++][slot] = fn;
  return DR_OK;
}

template <class Geo, class OutT, bool kTma, int PPT>
dr_status launch_rows(const dr_plan_t *p, const CUtensorMap &tm, const uint16_t *img, void *out,
                      cudaStream_t st) {
  auto fn = rows_kernel<Geo, OutT, kTma, PPT>;
  dr_status s = allow_smem((const void *)fn);
  if (s != DR_OK) return s;
  dim3 grid((p->cols + p->tune.tile_cols - 1) / p->tune.tile_cols, p->rows);
  fn<<<grid, p->threads, p->smem_bytes, st>>>(tm, img, (OutT *)out, p->c, p->tune);
  return DR_OK;
}

template <class Geo, class OutT, bool kTma>
dr_status launch_pixels(const dr_plan_t *p, const CUtensorMap &tm, const uint16_t *img,
                        void *out, cudaStream_t st) {
  auto fn = pixels_kernel<Geo, OutT, kTma>;
  dr_status s = allow_smem((const void *)fn);
  if (s != DR_OK) return s;
  dim3 grid((p->cols + p->tune.tile_cols - 1) / p->tune.tile_cols, p->rows);
  fn<<<grid, p->threads, p->smem_bytes, st>>>(tm, img, (OutT *)out, p->c, p->tune);
  return DR_OK;
}

template <class Geo, class OutT>
dr_status dispatch_out(const dr_plan_t *p, bool tma, const CUtensorMap &tm, const uint16_t *img,
                       void *out, cudaStream_t st) {
  if (p->kernel == DR_KERNEL_ROWS) {
    if (p->tune.ppt == 4)
      return tma ? launch_rows<Geo, OutT, true, 4>(p, tm, img, out, st)
                 : launch_rows<Geo, OutT, false, 4>(p, tm, img, out, st);
    return tma ? launch_rows<Geo, OutT, true, 1>(p, tm, img, out, st)
               : launch_rows<Geo, OutT, false, 1>(p, tm, img, out, st);
  }
  return tma ? launch_pixels<Geo, OutT, true>(p, tm, img, out, st)
             : launch_pixels<Geo, OutT, false>(p, tm, img, out, st);
}

}  // namespace

// Build the [K][rows][cols] uint16 tensor map with a [kc][1][tile_cols] box.
dr_status make_tensor_map(const dr_plan_t *p, const uint16_t *img, CUtensorMap *tm) {
  auto enc = encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return DR_ERR_CUDA;
  }
  cuuint64_t dims[3] = {(cuuint64_t)p->cols, (cuuint64_t)p->rows, (cuuint64_t)p->K};
  cuuint64_t strides[2] = {(cuuint64_t)p->cols * 2, (cuuint64_t)p->cols * p->rows * 2};
  cuuint32_t box[3] = {(cuuint32_t)p->tune.tile_cols, 1u, (cuuint32_t)p->tune.kc};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, (void *)img, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return DR_ERR_CUDA;
  }
  return DR_OK;
}

bool tma_usable(const dr_plan_t *p, const uint16_t *img) {
  return p->cols % 8 == 0 && ((uintptr_t)img & 15) == 0 && p->tune.tile_cols % 8 == 0 &&
         p->tune.kc <= 256 && p->tune.tile_cols <= 256;
}

dr_status launch_reconstruct(const dr_plan_t *p, const uint16_t *img, void *out,
                             cudaStream_t st) {
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  const bool tma = tma_usable(p, img);
  if (tma) {
    dr_status s = make_tensor_map(p, img, &tm);
    if (s != DR_OK) return s;
  }
  const bool bf16 = p->out_dtype == DR_OUT_BF16;
  if (p->geom_prec == DR_GEOM_FP64)
    return bf16 ? dispatch_out<GeoF64, __nv_bfloat16>(p, tma, tm, img, out, st)
                : dispatch_out<GeoF64, float>(p, tma, tm, img, out, st);
  return bf16 ? dispatch_out<GeoFx, __nv_bfloat16>(p, tma, tm, img, out, st)
              : dispatch_out<GeoFx, float>(p, tma, tm, img, out, st);
}

}  // namespace dr

using namespace dr;

extern "C" dr_status dr_reconstruct(const dr_plan_t *p, const uint16_t *img, void *out,
                                    dr_stream_t stream) {
  if (!p) {
    set_error("dr_reconstruct: null plan");
    return DR_ERR_INVALID_ARG;
  }
  if ((size_t)p->rows * p->cols == 0) return DR_OK;
  if (!img || !out) {
    set_error("dr_reconstruct: null buffer");
    return DR_ERR_INVALID_ARG;
  }
  const size_t align = p->out_dtype == DR_OUT_BF16 ? 2 : 4;
  if (((uintptr_t)out & (p->tune.ppt == 4 ? 4 * align - 1 : align - 1)) != 0 ||
      ((uintptr_t)img & 1) != 0 || (p->tune.ppt == 4 && ((uintptr_t)img & 7) != 0)) {
    set_error("dr_reconstruct: misaligned buffer");
    return DR_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  dr_status s = launch_reconstruct(p, img, out, st);
  if (s != DR_OK) return s;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct: launch", e);
  return DR_OK;
}

extern "C" dr_status dr_reconstruct_host(const dr_plan_t *p, const uint16_t *h_img, void *h_out,
                                         uint16_t *d_img, void *d_out, dr_stream_t stream) {
  if (!p || !h_img || !h_out || !d_img || !d_out) {
    if (p && (size_t)p->rows * p->cols == 0) return DR_OK;
    set_error("dr_reconstruct_host: null argument");
    return DR_ERR_INVALID_ARG;
  }
  const size_t P = (size_t)p->rows * p->cols;
  if (P == 0) return DR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t in_bytes = P * p->K * 2;
  const size_t out_bytes = P * p->B * (p->out_dtype == DR_OUT_BF16 ? 2 : 4);
  cudaError_t e = cudaMemcpyAsync(d_img, h_img, in_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct_host: upload", e);
  dr_status s = dr_reconstruct(p, d_img, d_out, stream);
  if (s != DR_OK) return s;
  e = cudaMemcpyAsync(h_out, d_out, out_bytes, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct_host: download", e);
  return DR_OK;
}

extern "C" dr_status dr_image_differences(const uint16_t *img, int32_t K, int32_t rows,
                                          int32_t cols, int32_t *d, dr_stream_t stream) {
  if (K < 1 || rows < 0 || cols < 0) {
    set_error("dr_image_differences: bad sizes");
    return DR_ERR_INVALID_ARG;
  }
  const long long plane = (long long)rows * cols, n = plane * (K - 1);
  if (n == 0) return DR_OK;
  if (!img || !d) {
    set_error("dr_image_differences: null buffer");
    return DR_ERR_INVALID_ARG;
  }
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  differences_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(img, n, plane, d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("dr_image_differences", e);
  return DR_OK;
}

extern "C" dr_status dr_plan_depths(const dr_plan_t *p, int32_t r0, int32_t nrows, double *d,
                                    dr_stream_t stream) {
  if (!p || r0 < 0 || nrows < 0 || r0 + nrows > p->rows) {
    set_error("dr_plan_depths: bad arguments");
    return DR_ERR_INVALID_ARG;
  }
  const long long n = (long long)nrows * p->cols * p->K;
  if (n == 0) return DR_OK;
  if (!d) {
    set_error("dr_plan_depths: null buffer");
    return DR_ERR_INVALID_ARG;
  }
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (p->geom_prec == DR_GEOM_FP64)
    depths_kernel<GeoF64><<<blocks, 256, 0, (cudaStream_t)stream>>>(p->c, p->kernel, r0, nrows, d);
  else
    depths_kernel<GeoFx><<<blocks, 256, 0, (cudaStream_t)stream>>>(p->c, p->kernel, r0, nrows, d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("dr_plan_depths", e);
  return DR_OK;
}

extern "C" dr_status dr_plan_check(const dr_plan_t *p) {
  if (!p) {
    set_error("dr_plan_check: null plan");
    return DR_ERR_INVALID_ARG;
  }
  int32_t v = 0, zero = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail("dr_plan_check: synchronize", e);
  e = cudaMemcpy(&v, p->c.err, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail("dr_plan_check: read", e);
  if (v != kDevOk) {
    e = cudaMemcpy(p->c.err, &zero, sizeof(zero), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail("dr_plan_check: clear", e);
    set_error("a kernel's bounded wait for its TMA tile ran out (code %d)", v);
    return DR_ERR_TIMEOUT;
  }
  return DR_OK;
}

// ------------------------------------------- no-allocation entry point ---
// The rows kernel with its geometry tables in a file-scope device array
// instead of a plan's cudaMalloc'd block, for callers that may not allocate
// device memory.  The array's host-side name is only a stand-in: the device
// address comes from cudaGetSymbolAddress, once per device, on the first
// call made with that device current.

namespace dr {
constexpr size_t kStaticScratchBytes = size_t(2) << 20;  // 2 MiB per device
constexpr int kStaticMaxK = 16384;
}  // namespace dr

static __device__ __align__(256) unsigned char g_dr_static_scratch[dr::kStaticScratchBytes];

namespace {
std::mutex g_static_mu;                                    // guards the three below
unsigned char g_static_stage[dr::kStaticScratchBytes];     // host staging (static)
double g_static_tmp[2 * dr::kStaticMaxK];                  // host FP64 temporaries
void *g_static_dev[64];                                    // device address per device
}  // namespace

extern "C" dr_status dr_reconstruct_rows_static(const dr_geometry *g, const double *wires,
                                               int32_t K, const double *edges, int32_t B,
                                               const uint16_t *d_images, float *d_out,
                                               int32_t *d_status, dr_stream_t stream) {
  if (K > kStaticMaxK) {
    set_error("dr_reconstruct_rows_static: K = %d exceeds %d steps", K, kStaticMaxK);
    return DR_ERR_BUDGET;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct_rows_static: cudaGetDevice", e);
  if (dev < 0 || dev >= 64) {
    set_error("dr_reconstruct_rows_static: device %d out of range", dev);
    return DR_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_dev[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_dr_static_scratch);
    if (e != cudaSuccess || !ptr)
      return cuda_fail("dr_reconstruct_rows_static: cudaGetSymbolAddress", e);
    g_static_dev[dev] = ptr;
  }
  StaticTables st;
  dr_status s = build_rows_tables(g, wires, K, edges, B, g_static_stage, kStaticScratchBytes,
                                  g_static_tmp, &st);
  if (s != DR_OK) return s;
  if ((size_t)st.rows * st.cols == 0) return DR_OK;
  if (!d_images || !d_out) {
    set_error("dr_reconstruct_rows_static: null buffer");
    return DR_ERR_INVALID_ARG;
  }
  if (((uintptr_t)d_out & (st.tune.ppt == 4 ? 15 : 3)) != 0 || ((uintptr_t)d_images & 1) != 0 ||
      (st.tune.ppt == 4 && ((uintptr_t)d_images & 7) != 0)) {
    set_error("dr_reconstruct_rows_static: misaligned buffer");
    return DR_ERR_INVALID_ARG;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  unsigned char *base = static_cast<unsigned char *>(g_static_dev[dev]);
  // the staged tables include a zeroed error word; pageable source: the call
  // returns once the bytes are staged, so the host buffer may be reused
  e = cudaMemcpyAsync(base, g_static_stage, st.bytes, cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct_rows_static: table upload", e);
  if (d_status) {
    e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), cs);
    if (e != cudaSuccess) return cuda_fail("dr_reconstruct_rows_static: status clear", e);
  }
  dr_plan_t p{};
  p.rows = st.rows;
  p.cols = st.cols;
  p.K = st.K;
  p.B = st.B;
  p.kernel = DR_KERNEL_ROWS;
  p.out_dtype = DR_OUT_F32;
  p.geom_prec = DR_GEOM_FP32;
  p.c = st.c;
  p.c.grp = reinterpret_cast<const GroupC *>(base + st.off_grp);
  p.c.stp = reinterpret_cast<const StepC *>(base + st.off_stp);
  p.c.efx = reinterpret_cast<const int32_t *>(base + st.off_efx);
  p.c.err = d_status ? d_status : reinterpret_cast<int32_t *>(base + st.off_err);
  p.tune = st.tune;
  p.threads = st.threads;
  p.smem_bytes = st.smem_bytes;
  s = launch_reconstruct(&p, d_images, d_out, cs);
  if (s != DR_OK) return s;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct_rows_static: launch", e);
  return DR_OK;
}
