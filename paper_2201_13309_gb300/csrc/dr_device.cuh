// Device code of the reconstruction: PTX helpers, the depth model, the two
// reconstruction kernels and two small helper kernels (sm_103a).
#pragma once

#include <cuda.h>
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dr_tables.h"
#include "../../include/dr.h"

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

// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load_1d(void *dst, const void *src, uint32_t bytes,
                                             uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Wait for the TMA phase with a time limit.  On timeout the error word is
// set, the copies in flight get a second bounded wait to land, and the caller
// returns without touching the tile.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ inline bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int32_t *err) {
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

// ------------------------------------------------------- checked build ---
// Built with -DDR_CHECK_BOUNDS (off by default: the normal build compiles
// every index unchanged), each shared-memory and global index of the
// reconstruction kernels goes through DR_IDX: an index outside [0, n)
// records kDevBounds with the source line in the error word (the first one
// found stays) and is replaced by 0, so the access stays inside its array and
// nothing traps.  DR_PTR does the same for a pointer walking an array.
#ifdef DR_CHECK_BOUNDS
#define DR_IDX(i, n, err) ::dr::checked_index((long long)(i), (long long)(n), (err), __LINE__)
#define DR_PTR(p, base, n, err) ((base) + DR_IDX((p) - (base), (n), (err)))
__device__ __forceinline__ long long checked_index(long long i, long long n, int32_t *err,
                                                   int line) {
  if (i >= 0 && i < n) return i;
  atomicCAS(err, 0, kDevBounds | (line << 4));
  return 0;
}
#else
#define DR_IDX(i, n, err) (i)
#define DR_PTR(p, base, n, err) (p)
#endif

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

__device__ __forceinline__ void st_cs_u4(void *p, uint4 v) {
  asm volatile("st.global.cs.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}
// 16 bytes of the output type's encoding of v (v is +0 or -0 here)
template <class OutT>
__device__ __forceinline__ uint4 zero_bits(float v);
template <>
__device__ __forceinline__ uint4 zero_bits<float>(float v) {
  const uint32_t b = __float_as_uint(v);
  return make_uint4(b, b, b, b);
}
template <>
__device__ __forceinline__ uint4 zero_bits<__nv_bfloat16>(float v) {
  __nv_bfloat16 h = __float2bfloat16_rn(v);
  const uint32_t u = *reinterpret_cast<unsigned short *>(&h);
  const uint32_t b = u | (u << 16);
  return make_uint4(b, b, b, b);
}

// --------------------------------------------------------- depth model ---

// float(x) for an integer 0 <= x < 2^23, exactly, on the FP32 pipe: the bit
// pattern 0x4B000000 | x is the float 2^23 + x.
__device__ __forceinline__ float cvt23(int32_t x) {
  return __fsub_rn(__int_as_float(0x4B000000 | x), 8388608.0f);
}

// Round v to the nearest integer (ties to even) for |v| < 2^22: adding
// 1.5 * 2^23 leaves the integer in the low mantissa bits.  rnd_bits returns
// the float whose bits are 0x4B400000 + round(v) (fused with the product).
constexpr float kRoundMagic = 12582912.0f;  // 1.5 * 2^23, bits 0x4B400000
constexpr int32_t kRoundMagicBits = 0x4B400000;

// FP32 depth position of (group, step) in fixed point (see dr_tables.h),
// series form of dL (no square root or reciprocal).
__device__ __forceinline__ int32_t depth_fx_series(const GroupC &g, const StepC &s,
                                                   const Consts &c) {
  const float z = s.zf;
  const float a = __fmul_rn(c.y0, z);
  const float tap = __fmaf_rn(a, g.invD, __fadd_rn(z, g.Q0f));
  const float n = __fmul_rn(tap, __fsub_rn(tap, __fadd_rn(g.Z, g.Z)));
  const float il = g.invL0;
  const float x = __fmul_rn(n, __fmul_rn(il, il));
  const float p = __fmaf_rn(x, __fmaf_rn(x, 0.0625f * il, -0.125f * il), 0.5f * il);
  const float dL = __fmul_rn(n, p);
  const float rem = __fmaf_rn(c.sR, dL, a);
  const float r = __fmaf_rn(rem, __fmul_rn(g.invD, c.scale), kRoundMagic);
  return (int32_t)((uint32_t)s.zfx + (uint32_t)g.Q0fx +
                   (uint32_t)(__float_as_int(r) - kRoundMagicBits));
}

// FP32 depth position of (group, step) in fixed point, exact form of dL.
__device__ __forceinline__ int32_t depth_fx_exact(const GroupC &g, const StepC &s,
                                                  const Consts &c) {
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

// The polynomial form (dr_tables.h): the group's 32 bytes read as GroupPoly.
__device__ __forceinline__ GroupPoly as_poly(const GroupC &g) {
  GroupPoly p;
  memcpy(&p, &g, sizeof(p));
  return p;
}

__device__ __forceinline__ int32_t depth_fx_poly(const GroupC &g, const StepC &s) {
  const GroupPoly p = as_poly(g);
  const float d = s.dz;
  const float r = __fmaf_rn(__fmaf_rn(__fmaf_rn(p.c3, d, p.c2), d, p.c1), d, p.c0);
  return (int32_t)((uint32_t)s.zfx + (uint32_t)p.q0fx +
                   (uint32_t)__float_as_int(__fadd_rn(r, kRoundMagic)));
}

__device__ __forceinline__ int32_t depth_fx(const GroupC &g, const StepC &s, const Consts &c) {
  if (c.depth_mode == kDepthPoly) return depth_fx_poly(g, s);
  return c.depth_mode == kDepthSeries ? depth_fx_series(g, s, c) : depth_fx_exact(g, s, c);
}

// Two steps of one group at once with Blackwell's packed FP32 ops (each
// half is an IEEE round-to-nearest operation, so both results are bitwise
// those of depth_fx); the approximate reciprocals and square roots and the
// conversions stay scalar.
struct f2 {
  unsigned long long v;
};
__device__ __forceinline__ f2 f2_pack(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2 x, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ f2 f2_rcp(f2 x) {
  float a, b;
  f2_unpack(x, a, b);
  return f2_pack(rcp_approx(a), rcp_approx(b));
}
__device__ __forceinline__ f2 f2_sqrt(f2 x) {
  float a, b;
  f2_unpack(x, a, b);
  return f2_pack(sqrt_approx(a), sqrt_approx(b));
}
__device__ __forceinline__ f2 f2_splat(float a) { return f2_pack(a, a); }

// depth_fx_series of steps s0 and s1 of group g, operation for operation
__device__ __forceinline__ void depth_fx2_series(const GroupC &g, const StepC &s0,
                                                 const StepC &s1, const Consts &c, int32_t &d0,
                                                 int32_t &d1) {
  const f2 z = f2_pack(s0.zf, s1.zf);
  const f2 a = f2_mul(f2_splat(c.y0), z);
  const f2 tap = f2_fma(a, f2_splat(g.invD), f2_add(z, f2_splat(g.Q0f)));
  const f2 n = f2_mul(tap, f2_sub(tap, f2_splat(__fadd_rn(g.Z, g.Z))));
  const float il = g.invL0;
  const f2 x = f2_mul(n, f2_splat(__fmul_rn(il, il)));
  const f2 p = f2_fma(x, f2_fma(x, f2_splat(0.0625f * il), f2_splat(-0.125f * il)),
                      f2_splat(0.5f * il));
  const f2 dL = f2_mul(n, p);
  const f2 rem = f2_fma(f2_splat(c.sR), dL, a);
  const f2 r = f2_fma(rem, f2_splat(__fmul_rn(g.invD, c.scale)), f2_splat(kRoundMagic));
  float r0, r1;
  f2_unpack(r, r0, r1);
  d0 = (int32_t)((uint32_t)s0.zfx + (uint32_t)g.Q0fx +
                 (uint32_t)(__float_as_int(r0) - kRoundMagicBits));
  d1 = (int32_t)((uint32_t)s1.zfx + (uint32_t)g.Q0fx +
                 (uint32_t)(__float_as_int(r1) - kRoundMagicBits));
}

// depth_fx_exact of steps s0 and s1 of group g, step for step the same operations
__device__ __forceinline__ void depth_fx2_exact(const GroupC &g, const StepC &s0,
                                                const StepC &s1, const Consts &c, int32_t &d0,
                                                int32_t &d1) {
  const f2 z = f2_pack(s0.zf, s1.zf);
  f2 inv = f2_splat(g.invD);
  f2 a = f2_mul(f2_splat(c.y0), z);
  if (c.has_eta) {
    const f2 eta = f2_pack(s0.eta, s1.eta);
    inv = f2_rcp(f2_sub(f2_splat(g.D), eta));
    a = f2_fma(eta, f2_add(f2_sub(z, f2_splat(g.Z)), f2_splat(g.Q0f)), a);
  }
  const f2 tap = f2_fma(a, inv, f2_add(z, f2_splat(g.Q0f)));
  const f2 u = f2_sub(f2_splat(g.Z), tap);
  const f2 L = f2_sqrt(f2_fma(u, u, f2_splat(g.Y2)));
  const f2 num = f2_mul(tap, f2_sub(tap, f2_splat(__fadd_rn(g.Z, g.Z))));
  const f2 dL = f2_mul(num, f2_rcp(f2_add(L, f2_splat(g.L0))));
  const f2 rem = f2_mul(f2_fma(f2_splat(c.sR), dL, a), inv);
  const f2 rs = f2_mul(rem, f2_splat(c.scale));
  float r0, r1;
  f2_unpack(rs, r0, r1);
  d0 = (int32_t)((uint32_t)s0.zfx + (uint32_t)g.Q0fx + (uint32_t)__float2int_rn(r0));
  d1 = (int32_t)((uint32_t)s1.zfx + (uint32_t)g.Q0fx + (uint32_t)__float2int_rn(r1));
}

// depth_fx_poly of steps s0 and s1 of one group, operation for operation
// (the coefficient pairs are formed by the caller once per group)
struct Poly2 {
  f2 c0, c1, c2, c3, magic;
  int32_t q0fx;
};
__device__ __forceinline__ Poly2 poly2_of(const GroupC &g) {
  const GroupPoly p = as_poly(g);
  return {f2_splat(p.c0), f2_splat(p.c1), f2_splat(p.c2), f2_splat(p.c3), f2_splat(kRoundMagic),
          p.q0fx};
}
__device__ __forceinline__ void depth_fx2_poly(const Poly2 &q, const StepC &s0, const StepC &s1,
                                               int32_t &d0, int32_t &d1) {
  const f2 d = f2_pack(s0.dz, s1.dz);
  const f2 r = f2_add(f2_fma(f2_fma(f2_fma(q.c3, d, q.c2), d, q.c1), d, q.c0), q.magic);
  float r0, r1;
  f2_unpack(r, r0, r1);
  d0 = (int32_t)((uint32_t)s0.zfx + (uint32_t)q.q0fx + (uint32_t)__float_as_int(r0));
  d1 = (int32_t)((uint32_t)s1.zfx + (uint32_t)q.q0fx + (uint32_t)__float_as_int(r1));
}

__device__ __forceinline__ void depth_fx2(const GroupC &g, const StepC &s0, const StepC &s1,
                                          const Consts &c, int32_t &d0, int32_t &d1) {
  if (c.depth_mode == kDepthPoly)
    depth_fx2_poly(poly2_of(g), s0, s1, d0, d1);
  else if (c.depth_mode == kDepthSeries)
    depth_fx2_series(g, s0, s1, c, d0, d1);
  else
    depth_fx2_exact(g, s0, s1, c, d0, d1);
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
  static constexpr int kPixelsMinBlocks = 3;  // three 512-thread CTAs per SM
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
  static __device__ __forceinline__ void depth2(const GroupC &g, const StepC &s0,
                                                const StepC &s1, const Consts &c, pos_t &d0,
                                                pos_t &d1) {
    depth_fx2(g, s0, s1, c, d0, d1);
  }
  static __device__ __forceinline__ pos_t edge(const Consts &c, int j) { return c.efx[j]; }
  // 1 / (b - a) for a < b, b - a < 2^23 (the plan checks every step):
  // approximate reciprocal of the exactly converted length; the same value
  // in every kernel
  static __device__ __forceinline__ float inv_len(pos_t a, pos_t b) {
    return rcp_approx(cvt23(b - a));
  }
  // Position of edge e in the interval [a, b] as a fraction: the edge is
  // clamped to the interval first, so the difference converts exactly
  static __device__ __forceinline__ float frac(pos_t e, pos_t a, pos_t b, float inv) {
    return __fmul_rn(cvt23(max(min(e, b), a) - a), inv);
  }
  static __device__ __forceinline__ double to_mm(pos_t p, const Consts &c) {
    return ((double)p / (double)c.scale + c.origin) / c.nb;
  }
};

struct GeoF64 {
  using pos_t = double;
  static constexpr int kPixelsMinBlocks = 1;  // the FP64 walk state needs more registers
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
  static __device__ __forceinline__ void depth2(const GroupD &g, const StepD &s0,
                                                const StepD &s1, const Consts &c, pos_t &d0,
                                                pos_t &d1) {
    d0 = depth_f64(g, s0, c);
    d1 = depth_f64(g, s1, c);
  }
  static __device__ __forceinline__ pos_t edge(const Consts &c, int j) { return c.e64[j]; }
  static __device__ __forceinline__ double inv_len(pos_t a, pos_t b) { return 1.0 / (b - a); }
  static __device__ __forceinline__ float frac(pos_t e, pos_t a, pos_t /*b*/, double inv) {
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

__device__ __forceinline__ float out_load(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float out_load(const __nv_bfloat16 *p) {
  return __bfloat162float(*p);
}

template <class OutT, int PPT>
__device__ __forceinline__ void load_out_px(const OutT *p, float (&v)[PPT]) {
  if constexpr (PPT == 4 && sizeof(OutT) == 4) {
    const float4 u = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = u.x;
    v[1] = u.y;
    v[2] = u.z;
    v[3] = u.w;
  } else {
#pragma unroll
    for (int i = 0; i < PPT; ++i) v[i] = out_load(p + i);
  }
}

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Stage the image tile [K][1][tile_cols] (row `row`, columns c0..) into
// smem: by TMA (thread 0 arms the already initialised mbarrier `bar` and
// issues the chunk copies) or with plain loads (zero-filled tail).
template <bool kTma>
__device__ __forceinline__ void stage_tile(const CUtensorMap *tmap, const uint16_t *img,
                                           uint16_t *simg, uint64_t *bar, const Consts &c,
                                           const Tuning &t, int row, int c0) {
  const int TC = t.tile_cols;
  if constexpr (kTma) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(bar, (uint32_t)(t.kc * t.nchunks * TC * 2));
      for (int ch = 0; ch < t.nchunks; ++ch)
        tma_load_3d(simg + (size_t)ch * t.kc * TC, tmap, bar, c0, row, ch * t.kc);
    }
  } else {
    const int n = c.K * TC;
    const size_t n_img = (size_t)c.K * c.H * c.W;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int k = i / TC, cc = i - k * TC, col = c0 + cc;
      simg[DR_IDX(i, (size_t)t.kc * t.nchunks * TC, c.err)] =
          col < c.W ? img[DR_IDX(((size_t)k * c.H + row) * c.W + col, n_img, c.err)]
                    : (uint16_t)0;
    }
  }
}

// --------------------------------------------------------- rows kernel ---
// Shared-memory layout of one rows tile: [0, 128) mbarrier, two counters and
// the persistent kernel's work slot; then the image tile [Kpad][tile_cols]
// uint16, the row's depth positions [K], and the (k, f) table [B + 1].

// The row's (k_j, f_j) table: depth positions of the row into spos (smem,
// K entries), then for every bin edge j: k = last step below the edge
// (clamped to an interval), f = position of the edge inside [d_k, d_{k+1}]
// (clamped), written to out1[j].  Edges at or below d_0 give F = 0 and edges
// at or above d_{K-1} give F = S_{K-1}, so only bins [nz_lo, nz_hi) can hold
// data.  zcount (2 ints, smem) must be zero before the first barrier here.
// Contains two __syncthreads; every thread of the CTA must call it.
template <class Geo>
__device__ __forceinline__ int2 build_row_table(const Consts &c, int row,
                                                typename Geo::pos_t *spos, int2 *out1,
                                                int *zcount) {
  using pos_t = typename Geo::pos_t;
  const int K = c.K, B = c.B, tid = threadIdx.x, NT = blockDim.x;
  const auto &g = Geo::group(c, row);
  const auto *steps = Geo::steps(c);
  for (int k = tid; k < K; k += NT) spos[DR_IDX(k, K, c.err)] = Geo::depth(g, steps[k], c);
  __syncthreads();
  int below = 0, above = 0;
  const pos_t tfirst = spos[0], tlast = spos[K - 1];
  for (int j = tid; j <= B; j += NT) {
    const pos_t e = Geo::edge(c, j);
    int lo = 0, hi = K;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (spos[DR_IDX(mid, K, c.err)] < e) lo = mid + 1; else hi = mid;
    }
    const int k = min(max(lo - 1, 0), K - 2);
    const pos_t a = spos[DR_IDX(k, K, c.err)], b = spos[DR_IDX(k + 1, K, c.err)];
    const float f = Geo::frac(e, a, b, Geo::inv_len(a, b));
    out1[DR_IDX(j, B + 1, c.err)] = make_int2(k, __float_as_int(f));
    below += !(e > tfirst);
    above += !(e < tlast);
  }
  if (below) atomicAdd(&zcount[0], below);
  if (above) atomicAdd(&zcount[1], above);
  __syncthreads();
  const int nz_hi = min(B + 1 - zcount[1], B);
  const int nz_lo = min(max(zcount[0] - 1, 0), nz_hi);
  return make_int2(nz_lo, nz_hi);
}

// Plan-time tables: one CTA per row writes its header and edge entries.
template <class Geo>
__global__ void __launch_bounds__(256) tables_kernel(const Consts c, int2 *tab) {
  extern __shared__ __align__(16) unsigned char tsmem[];
  int *zcount = reinterpret_cast<int *>(tsmem);
  auto *spos = reinterpret_cast<typename Geo::pos_t *>(tsmem + 16);
  const int row = blockIdx.x;
  if (threadIdx.x == 0) zcount[0] = zcount[1] = 0;
  int2 *trow = tab + (size_t)row * c.tab_stride;
  const int2 nz = build_row_table<Geo>(c, row, spos, trow + 1, zcount);
  if (threadIdx.x == 0) trow[0] = nz;
  for (int i = c.B + 2 + threadIdx.x; i < c.tab_stride; i += blockDim.x) trow[i] = make_int2(0, 0);
}

// One tile: row `row`, columns c0 .. c0 + tile_cols - 1, all steps and bins.
// The mbarrier at smem[0] must be initialised; `parity` is its phase for this
// tile.  Returns false (for every thread of the CTA) if the bounded TMA wait
// ran out; the tile is then left unwritten and the error word is set.
template <class Geo, class OutT, bool kTma, int PPT>
__device__ __forceinline__ bool rows_tile(const CUtensorMap *tmap, const uint16_t *img,
                                          OutT *out, const Consts &c, const Tuning &t,
                                          int row, int c0, unsigned char *smem,
                                          uint32_t parity) {
  using pos_t = typename Geo::pos_t;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  int *zcount = reinterpret_cast<int *>(smem + 8);
  uint16_t *simg = reinterpret_cast<uint16_t *>(smem + 128);
  const int TC = t.tile_cols, K = c.K, B = c.B;
  const int Kpad = t.kc * t.nchunks;
  pos_t *spos = reinterpret_cast<pos_t *>(smem + 128 + align16((size_t)Kpad * TC * 2));
  int2 *stab0 = reinterpret_cast<int2 *>(reinterpret_cast<unsigned char *>(spos) +
                                         align16((size_t)K * sizeof(pos_t)));
  int2 *stab = stab0 + 1;  // stab[j], j = 0..B
  const int tid = threadIdx.x, NT = blockDim.x;
  const bool pre = c.tab != nullptr;
  const int2 *grow = pre ? c.tab + (size_t)row * c.tab_stride : nullptr;

  // images (and the plan's row table) into shared memory
  if constexpr (kTma) {
    if (tid == 0) {
      const uint32_t tab_bytes = pre ? (uint32_t)c.tab_stride * 8u : 0u;
      mbar_expect_tx(bar, (uint32_t)(t.kc * t.nchunks * TC * 2) + tab_bytes);
      for (int ch = 0; ch < t.nchunks; ++ch)
        tma_load_3d(simg + (size_t)ch * t.kc * TC, tmap, bar, c0, row, ch * t.kc);
      if (pre) bulk_load_1d(stab0, grow, tab_bytes, bar);
    }
  } else {
    stage_tile<false>(tmap, img, simg, bar, c, t, row, c0);
    if (pre)
      for (int i = tid; i < c.tab_stride; i += NT) stab0[i] = grow[i];
  }
  int2 nz;
  if (!pre) {
    if (tid == 0) zcount[0] = zcount[1] = 0;
    nz = build_row_table<Geo>(c, row, spos, stab, zcount);
  }
  if constexpr (kTma) {
    const bool late = !mbar_wait_bounded(bar, parity, c.err);
    if (__syncthreads_or(late)) return false;
  } else {
    if (pre) __syncthreads();
  }
  if (pre) nz = stab0[0];
  const int nz_lo = nz.x, nz_hi = nz.y;

  // stream the bins; thread = PPT adjacent pixels; the zero ranges and the
  // data range are each split evenly over the bin groups
  const int lanes = TC / PPT;
  const int lane = tid % lanes, grp = tid / lanes;
  const int lc = lane * PPT, col = c0 + lc;
  if (col >= c.W || grp >= t.bin_groups) return true;
  const int G = t.bin_groups;
  auto slice_lo = [&](int lo, int hi) { return lo + (int)((long long)(hi - lo) * grp / G); };
  auto slice_hi = [&](int lo, int hi) { return lo + (int)((long long)(hi - lo) * (grp + 1) / G); };
  const float sign = c.out_sign;
  const size_t plane = (size_t)c.H * c.W;
  OutT *const o0 = out + (size_t)row * c.W + col;
  const bool acc = c.accumulate != 0;
  const size_t n_out = plane * B - (PPT - 1);  // first elements of in-range stores
  float zero[PPT];
#pragma unroll
  for (int i = 0; i < PPT; ++i) zero[i] = __fmul_rn(sign, 0.f);
  auto zero_fill = [&](int a, int b) {
    OutT *o = o0 + (size_t)a * plane;
#pragma unroll 4
    for (int j = a; j < b; ++j, o += plane)
      store_px<OutT, PPT>(DR_PTR(o, out, n_out, c.err), zero);
  };
  if (!acc) {  // bins without data: written as zero (nothing to add when accumulating)
    zero_fill(slice_lo(0, nz_lo), slice_hi(0, nz_lo));
    zero_fill(slice_lo(nz_hi, B), slice_hi(nz_hi, B));
  }

  const int a = slice_lo(nz_lo, nz_hi), b = slice_hi(nz_lo, nz_hi);
  if (a >= b) return true;
  const bool rev = c.reverse != 0;
  const size_t n_simg = (size_t)Kpad * TC - (PPT - 1);
  auto srow = [&](int k) {
    return simg + DR_IDX((size_t)(rev ? K - 1 - k : k) * TC + lc, n_simg, c.err);
  };
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
  // the data range; the accumulating form adds to what is there
  auto stream = [&](auto add) {
    constexpr bool kAdd = decltype(add)::value;
    float Fp[PPT];
    evalF(stab[DR_IDX(a, B + 1, c.err)], Fp);
    OutT *o = o0 + (size_t)a * plane;
#pragma unroll 4
    for (int j = a; j < b; ++j, o += plane) {
      float Fn[PPT], v[PPT];
      evalF(stab[DR_IDX(j + 1, B + 1, c.err)], Fn);
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        v[i] = __fmul_rn(sign, __fsub_rn(Fn[i], Fp[i]));
        Fp[i] = Fn[i];
      }
      if constexpr (kAdd) {
        float old[PPT];
        load_out_px<OutT, PPT>(DR_PTR(o, out, n_out, c.err), old);
#pragma unroll
        for (int i = 0; i < PPT; ++i) v[i] = __fadd_rn(old[i], v[i]);
      }
      store_px<OutT, PPT>(DR_PTR(o, out, n_out, c.err), v);
    }
  };
  if (acc)
    stream(std::true_type{});
  else
    stream(std::false_type{});
  return true;
}

// One CTA per tile (grid: tiles along the row x rows).
template <class Geo, class OutT, bool kTma, int PPT>
__global__ void __launch_bounds__(512) rows_kernel(const __grid_constant__ CUtensorMap tmap,
                                                   const uint16_t *__restrict__ img,
                                                   OutT *__restrict__ out, const Consts c,
                                                   const Tuning t) {
  extern __shared__ __align__(128) unsigned char smem[];
  if constexpr (kTma) {
    // every thread waits on this barrier: make its initialisation visible
    // to the CTA before any thread can poll it
    if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
    __syncthreads();
  }
  rows_tile<Geo, OutT, kTma, PPT>(&tmap, img, out, c, t, blockIdx.y, blockIdx.x * t.tile_cols,
                                  smem, 0u);
}

// ------------------------------------------------------- pixels kernel ---
// General geometry: every pixel has its own depth sequence.  A CTA owns one
// row x tile_cols pixels x all steps; its threads are (pixel, slab, share):
// a slab is 32 adjacent pixels (16 or 8 for narrower tiles), one per lane,
// and the bin_groups shares of a slab split its bins.
//  1. All threads evaluate the tile's K x tile_cols depth positions into
//     shared memory (thread (pixel, share) takes steps share, share + G, ...)
//     while the TMA copies the image tile.
//  2. Every warp finds the data span [jlo, jhi) of its slab (each warp holds
//     whole slabs): bin j can hold data for some pixel only if
//     e_{j+1} > min d_0 and e_j < max d_{K-1}.
//  3. Every share gets an equal part of the span, which it walks (search of
//     its first step, then bins and steps together), and an equal part of
//     the bins outside it, which are zero.  The bin loop is uniform over the
//     warp, so the 32 lanes store bin j as one coalesced line.  The searches
//     start from a linear guess and are exact (binary search as fallback).
// FP32 geometry (GeoFx): per bin a lane clamps the edge to its last depth,
// advances its step at most once (more often only when the plan found a step
// shorter than a bin), and evaluates F with integer clamps and exact 2^23-bias
// conversions, so the bin loop keeps the conversion pipe free; F is constant
// (and exactly zero below d_0) outside [d_0, d_{K-1}], so those bins come out
// as exact zeros with no test.  FP64 geometry keeps the general walk with the
// zero rule: a bin is zero for a pixel when e_{j+1} <= d_0 or e_j >= d_{K-1}.
// Both give the rows kernel's values bitwise on row-shared geometry: (k, f)
// come from the same device functions (GeoFx::frac / inv_len).
// Shared-memory layout: [0, 128) mbarrier, then the image tile
// [Kpad][tile_cols] uint16, the depth positions [K][tile_cols], the bin edges
// [B + 1].

// minimum / maximum over aligned groups of `width` lanes (a power of two
// <= 32); every lane of the warp takes part
template <class T>
__device__ __forceinline__ T group_min(T v, int width) {
  for (int m = width >> 1; m > 0; m >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}
template <class T>
__device__ __forceinline__ T group_max(T v, int width) {
  for (int m = width >> 1; m > 0; m >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}

// The bins of a slab outside its data span [sp.x, sp.y) are zero for all
// its pixels.  A full slab whose rows start on 16 bytes stores them with
// 16-byte stores: each of the slab's G * SW threads owns one 16-byte part of
// a bin row and walks the bins with a fixed stride; otherwise every valid
// lane stores its own pixel's zeros.
template <class OutT>
__device__ __forceinline__ void zero_outside_span(OutT *out, const Consts &c, int row, int c0,
                                                  int slab, int SW, int share, int sl, int G,
                                                  int2 sp, int ncols, bool valid, float zero,
                                                  size_t plane) {
  constexpr int kPer = 16 / sizeof(OutT);
  const int B = c.B;
  OutT *const os = out + (size_t)row * c.W + c0 + slab * SW;
  if (slab * SW + SW <= ncols && c.W % kPer == 0 && ((uintptr_t)out & 15) == 0) {
    const uint4 zv = zero_bits<OutT>(zero);
    const int kVec = SW / kPer, kvl = __ffs(kVec) - 1;  // 16-byte stores per bin row
    const int q = share * SW + sl;                      // 0 .. G * SW - 1
    const int part = q & (kVec - 1), first = q >> kvl, stride = (G * SW) >> kvl;
    const size_t step = (size_t)stride * plane;
    auto range = [&](int a, int b) {
      OutT *p = os + (size_t)(a + first) * plane + part * kPer;
      for (int j = a + first; j < b; j += stride, p += step)
        st_cs_u4(DR_PTR(p, out, plane * B - (kPer - 1), c.err), zv);
    };
    range(0, sp.x);
    range(sp.y, B);
  } else if (valid) {
    auto range = [&](int a, int b) {
      OutT *p = os + (size_t)(a + share) * plane + sl;
      for (int j = a + share; j < b; j += G, p += (size_t)G * plane)
        st_cs(DR_PTR(p, out, plane * B, c.err), zero);
    };
    range(0, sp.x);
    range(sp.y, B);
  }
}

// One tile: row `row`, columns c0 .. c0 + tile_cols - 1, all steps and bins.
// The mbarrier at smem[0] must be initialised (by thread 0 before the call,
// or earlier with a barrier since); `parity` is its phase for this tile.
// Returns false (for every thread) if the bounded TMA wait ran out.
template <class Geo, class OutT, bool kTma, bool kOneAdv>
__device__ __forceinline__ bool pixels_tile(const CUtensorMap *tmap, const uint16_t *img,
                                            OutT *out, const Consts &c, const Tuning &t,
                                            int row, int c0, unsigned char *smem,
                                            uint32_t parity) {
  using pos_t = typename Geo::pos_t;
  constexpr bool kFx = std::is_same<Geo, GeoFx>::value;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  uint16_t *simg = reinterpret_cast<uint16_t *>(smem + 128);
  const int TC = t.tile_cols, K = c.K, B = c.B, G = t.bin_groups;
  const int Kpad = t.kc * t.nchunks;
  pos_t *spos = reinterpret_cast<pos_t *>(smem + 128 + align16((size_t)Kpad * TC * 2));
  pos_t *sedge = reinterpret_cast<pos_t *>(reinterpret_cast<unsigned char *>(spos) +
                                           align16((size_t)K * TC * sizeof(pos_t)));
  const int tid = threadIdx.x, NT = blockDim.x;
  // slabs of SW adjacent pixels (32, or the whole tile when it is narrower);
  // thread = (pixel of its slab, slab, share)
  const int SW = min(TC, 32), nslab = TC / SW, swl = __ffs(SW) - 1;  // SW: 8, 16 or 32
  const int sl = tid & (SW - 1), grp = tid >> swl;
  const int slab = grp % nslab, share = grp / nslab;
  const int lc = slab * SW + sl;
  const int ncols = min(TC, c.W - c0);
  const bool valid = lc < ncols;

  stage_tile<kTma>(tmap, img, simg, bar, c, t, row, c0);
  if (valid) {
    const auto g = Geo::group(c, row * c.W + c0 + lc);
    const auto *gsteps = Geo::steps(c);
    auto fill = [&](auto depth2) {
      for (int k = share; k < K; k += 2 * G) {  // steps k and k + G together
        const int k2 = min(k + G, K - 1);
        pos_t d0, d1;
        depth2(g, gsteps[k], gsteps[k2], c, d0, d1);
        spos[DR_IDX(k * TC + lc, K * TC, c.err)] = d0;
        if (k + G < K) spos[DR_IDX((k + G) * TC + lc, K * TC, c.err)] = d1;
      }
    };
    if constexpr (kFx) {
      if (c.depth_mode == kDepthPoly) {
        const Poly2 q = poly2_of(g);  // coefficient pairs formed once per pixel
        fill([&q](const GroupC &, const StepC &s0, const StepC &s1, const Consts &, int32_t &d0,
                  int32_t &d1) { depth_fx2_poly(q, s0, s1, d0, d1); });
      } else if (c.depth_mode == kDepthSeries) {
        fill([](const GroupC &g, const StepC &s0, const StepC &s1, const Consts &c,
                int32_t &d0, int32_t &d1) { depth_fx2_series(g, s0, s1, c, d0, d1); });
      } else {
        fill([](const GroupC &g, const StepC &s0, const StepC &s1, const Consts &c,
                int32_t &d0, int32_t &d1) { depth_fx2_exact(g, s0, s1, c, d0, d1); });
      }
    } else {
      fill([](const auto &g, const auto &s0, const auto &s1, const Consts &c, pos_t &d0,
              pos_t &d1) { Geo::depth2(g, s0, s1, c, d0, d1); });
    }
  }
  for (int j = tid; j <= B; j += NT) sedge[DR_IDX(j, B + 1, c.err)] = Geo::edge(c, j);
  __syncthreads();  // also makes the mbarrier initialisation visible
  auto pos = [&](int k) { return spos[DR_IDX(k * TC + lc, K * TC, c.err)]; };
  // Counts on the sorted edges and depths, guessed by linear interpolation
  // (uniform bins, near-uniform depth steps), checked against the two
  // neighbours and moved by up to two places; a binary search otherwise.
  // below(i) must hold for a prefix of [0, n) and fail after it.
  auto count_prefix = [](float guess, int n, auto below) {
    int g = (int)fminf(fmaxf(guess, 0.f), (float)n);
#pragma unroll
    for (int it = 0; it < 3; ++it) {
      const bool lo_ok = g == 0 || below(g - 1);
      const bool hi_ok = g == n || !below(g);
      if (lo_ok && hi_ok) return g;
      g += lo_ok ? 1 : -1;
    }
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (below(mid)) lo = mid + 1; else hi = mid;
    }
    return lo;
  };
  const pos_t e0 = sedge[0];
  const float bins_per_pos = (float)B / ((float)sedge[B] - (float)e0);
  // the slab's data span [jlo, jhi): bin j can hold data for some pixel of
  // the slab only if e_{j+1} > min d_0 and e_j < max d_{K-1}; every warp
  // holds whole slabs, so each finds its own
  const pos_t lo_d = group_min(valid ? pos(0) : sedge[B], SW);
  const pos_t hi_d = group_max(valid ? pos(K - 1) : sedge[0], SW);
  const int n_le = count_prefix(((float)lo_d - (float)e0) * bins_per_pos + 1.f, B + 1,
                                [&](int i) { return !(sedge[DR_IDX(i, B + 1, c.err)] > lo_d); });
  const int n_lt = count_prefix(((float)hi_d - (float)e0) * bins_per_pos + 1.f, B + 1,
                                [&](int i) { return sedge[DR_IDX(i, B + 1, c.err)] < hi_d; });
  const int jlo = min(max(n_le - 1, 0), B);
  const int2 sp = make_int2(jlo, max(min(n_lt, B), jlo));
  if constexpr (kTma) {
    const bool late = !mbar_wait_bounded(bar, parity, c.err);
    if (__syncthreads_or(late)) return false;
  }
  const float sign = c.out_sign, zero = __fmul_rn(sign, 0.f);
  const size_t plane = (size_t)c.H * c.W;
  const bool acc = c.accumulate != 0;
  if (!acc)
    zero_outside_span(out, c, row, c0, slab, SW, share, sl, G, sp, ncols, valid, zero, plane);
  if (!valid) return true;
  OutT *const o0 = out + (size_t)row * c.W + c0 + lc;
  // this share's part of the span
  const int nd = sp.y - sp.x;
  const int jb = sp.x + (int)((long long)nd * share / G);
  const int je = sp.x + (int)((long long)nd * (share + 1) / G);
  if (jb >= je) return true;
  const pos_t tfirst = pos(0), tlast = pos(K - 1);
  // image of step k at ip[k * istep] (steps stored in reverse for a reversed plan)
  const bool rev = c.reverse != 0;
  const uint16_t *ip = simg + (rev ? (K - 1) * TC : 0) + lc;
  const int istep = rev ? -TC : TC;
  // k = last step below e_jb, clamped to an interval
  pos_t eb = sedge[DR_IDX(jb, B + 1, c.err)];
  const int n_below = count_prefix(
      ((float)eb - (float)tfirst) * ((float)(K - 1) / ((float)tlast - (float)tfirst)) + 1.f, K,
      [&](int i) { return pos(i) < eb; });
  int k = min(max(n_below - 1, 0), K - 2);
  const float I0 = biased(*DR_PTR(ip, simg, Kpad * TC, c.err));
  OutT *o = o0 + (size_t)jb * plane;
  if constexpr (kFx) {
    // Walk state: t0 = t_k, t1 = t_{k+1} (pp points at t1), the image of
    // step k + 1 (at ipn), base = I_0 - I_k, dI = I_k - I_{k+1}.  An edge
    // is first clamped to the last depth, so the walk never passes the last
    // interval; the clamped edge then lies in [t0, t1] (or below t0 on the
    // first interval), and F at an edge at or above t_{K-1} is the same
    // value for every such edge, as F below t_0 is exactly zero: the bins
    // outside [d_0, d_{K-1}] come out as exact zeros without a test.  Each
    // bin advances at most once when the plan found every step at least as
    // long as every bin (kOneAdv), else as often as needed.
    const int32_t *pp = spos + (k + 1) * TC + lc;
    int32_t t0 = *DR_PTR(pp - TC, spos, K * TC, c.err), t1 = *DR_PTR(pp, spos, K * TC, c.err);
    const uint16_t *ipn = ip + (k + 1) * istep;
    const int n_simg = Kpad * TC;
    float Ik1 = biased(*DR_PTR(ipn, simg, n_simg, c.err));
    const float Ik = biased(*DR_PTR(ipn - istep, simg, n_simg, c.err));
    float base = __fsub_rn(I0, Ik), dI = __fsub_rn(Ik, Ik1);
    float inv = GeoFx::inv_len(t0, t1);
    auto advance = [&]() {
      t0 = t1;
      pp += TC;
      t1 = *DR_PTR(pp, spos, K * TC, c.err);
      ipn += istep;
      const float In = biased(*DR_PTR(ipn, simg, n_simg, c.err));
      base = __fsub_rn(I0, Ik1);
      dI = __fsub_rn(Ik1, In);
      Ik1 = In;
      inv = GeoFx::inv_len(t0, t1);
    };
    // F at edge e: the same value as GeoFx::frac over the rows table
    auto F_at = [&](int32_t e) {
      const int32_t ec = min(e, tlast);
      if (t1 < ec) advance();
      if constexpr (!kOneAdv) {
        while (t1 < ec) advance();
      }
      return __fmaf_rn(__fmul_rn(cvt23(max(ec, t0) - t0), inv), dI, base);
    };
    float Fp = F_at(eb);
    const size_t n_out = plane * B;
    if (acc) {
      for (int j = jb; j < je; ++j, o += plane) {
        const int32_t e1 = sedge[DR_IDX(j + 1, B + 1, c.err)];
        const float F = F_at(e1);
        const float v = __fmul_rn(sign, __fsub_rn(F, Fp));
        OutT *oc = DR_PTR(o, out, n_out, c.err);
        if (e1 > tfirst && eb < tlast) st_cs(oc, __fadd_rn(out_load(oc), v));
        Fp = F;
        eb = e1;
      }
    } else {
#pragma unroll 4
      for (int j = jb; j < je; ++j, o += plane) {
        const float F = F_at(sedge[DR_IDX(j + 1, B + 1, c.err)]);
        st_cs(DR_PTR(o, out, n_out, c.err), __fmul_rn(sign, __fsub_rn(F, Fp)));
        Fp = F;
      }
    }
  } else {
    pos_t t0 = pos(k), t1 = pos(k + 1);
    auto inv = Geo::inv_len(t0, t1);
    const int n_simg = Kpad * TC;
    float Ik1 = biased(*DR_PTR(ip + (k + 1) * istep, simg, n_simg, c.err));
    const float Ik = biased(*DR_PTR(ip + k * istep, simg, n_simg, c.err));
    float base = __fsub_rn(I0, Ik), dI = __fsub_rn(Ik, Ik1);
    // F at edge e (k moves forward only): F = f (I_k - I_{k+1}) + (I_0 - I_k)
    auto F_at = [&](pos_t e) {
      while (k < K - 2 && t1 < e) {
        ++k;
        t0 = t1;
        t1 = pos(k + 1);
        inv = Geo::inv_len(t0, t1);
        const float Ikk = Ik1;
        Ik1 = biased(*DR_PTR(ip + (k + 1) * istep, simg, n_simg, c.err));
        base = __fsub_rn(I0, Ikk);
        dI = __fsub_rn(Ikk, Ik1);
      }
      return __fmaf_rn(Geo::frac(e, t0, t1, inv), dI, base);
    };
    float Fp = F_at(eb);
    const size_t n_out = plane * B;
    if (acc) {
      for (int j = jb; j < je; ++j, o += plane) {
        const pos_t e1 = sedge[DR_IDX(j + 1, B + 1, c.err)];
        const float F = F_at(e1);
        const float v = __fmul_rn(sign, __fsub_rn(F, Fp));
        OutT *oc = DR_PTR(o, out, n_out, c.err);
        if (e1 > tfirst && eb < tlast) st_cs(oc, __fadd_rn(out_load(oc), v));
        Fp = F;
        eb = e1;
      }
    } else {
      // below d_0 both edges give F = 0 exactly, so only the upper test is
      // needed for the zero rule
#pragma unroll 2
      for (int j = jb; j < je; ++j, o += plane) {
        const pos_t e1 = sedge[DR_IDX(j + 1, B + 1, c.err)];
        const float F = F_at(e1);
        const float v = __fmul_rn(sign, __fsub_rn(F, Fp));
        st_cs(DR_PTR(o, out, n_out, c.err), eb < tlast ? v : zero);
        Fp = F;
        eb = e1;
      }
    }
  }
  return true;
}

// One CTA per tile (grid: tiles along the row x rows).
template <class Geo, class OutT, bool kTma, bool kOneAdv>
__global__ void __launch_bounds__(512, Geo::kPixelsMinBlocks)
    pixels_kernel(const __grid_constant__ CUtensorMap tmap, const uint16_t *__restrict__ img,
                  OutT *__restrict__ out, const Consts c, const Tuning t) {
  extern __shared__ __align__(128) unsigned char smem[];
  // thread 0 initialises the barrier and issues the copies; the others
  // first poll it after the tile's first __syncthreads
  if constexpr (kTma) {
    if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
  }
  pixels_tile<Geo, OutT, kTma, kOneAdv>(&tmap, img, out, c, t, blockIdx.y,
                                        blockIdx.x * t.tile_cols, smem, 0u);
}

// ------------------------------------------ per-pixel kernel, cubic form ---
// The per-pixel kernel for plans whose remainder takes the polynomial form
// (dr_tables.h): a position is three multiply-adds and a rounding, so each
// lane computes its pixel's positions in the walk, as it reaches them,
// instead of a phase that fills a [K][tile_cols] table first.  Shared memory
// holds only the image tile, the step table (z_k - z_c, fixed-point z_k) and
// the edges, so several CTAs share an SM.  Thread mapping, data span, zero
// stores, the split of the span over the shares and the walk are those of
// pixels_tile with FP32 geometry, and the positions are those of
// depth_fx_poly, so the bins are bitwise the same.
// Shared-memory layout: [0, 128) mbarrier, the image tile [Kpad][tile_cols]
// uint16, the steps [K] of (dz bits, zfx), the bin edges [B + 1].
template <class OutT, bool kTma, bool kOneAdv>
__device__ __forceinline__ bool pixels_poly_tile(const CUtensorMap *tmap, const uint16_t *img,
                                                 OutT *out, const Consts &c, const Tuning &t,
                                                 int row, int c0, unsigned char *smem,
                                                 uint32_t parity) {
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  uint16_t *simg = reinterpret_cast<uint16_t *>(smem + 128);
  const int TC = t.tile_cols, K = c.K, B = c.B, G = t.bin_groups;
  const int Kpad = t.kc * t.nchunks;
  int2 *sstep = reinterpret_cast<int2 *>(smem + 128 + align16((size_t)Kpad * TC * 2));
  int32_t *sedge = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(sstep) +
                                               align16((size_t)K * sizeof(int2)));
  const int tid = threadIdx.x, NT = blockDim.x;
  const int SW = min(TC, 32), nslab = TC / SW, swl = __ffs(SW) - 1;  // SW: 8, 16 or 32
  const int sl = tid & (SW - 1), grp = tid >> swl;
  const int slab = grp % nslab, share = grp / nslab;
  const int lc = slab * SW + sl;
  const int ncols = min(TC, c.W - c0);
  const bool valid = lc < ncols;

  stage_tile<kTma>(tmap, img, simg, bar, c, t, row, c0);
  for (int k = tid; k < K; k += NT) {
    const StepC s = c.stp[k];
    sstep[DR_IDX(k, K, c.err)] = make_int2(__float_as_int(s.dz), s.zfx);
  }
  for (int j = tid; j <= B; j += NT) sedge[DR_IDX(j, B + 1, c.err)] = c.efx[j];
  const GroupPoly gp = as_poly(c.grp[valid ? row * c.W + c0 + lc : row * c.W + c0]);
  __syncthreads();  // also makes the mbarrier initialisation visible
  // position of step k: depth_fx_poly, operation for operation
  auto pos = [&](int k) {
    const int2 st = sstep[DR_IDX(k, K, c.err)];
    const float d = __int_as_float(st.x);
    const float r = __fmaf_rn(__fmaf_rn(__fmaf_rn(gp.c3, d, gp.c2), d, gp.c1), d, gp.c0);
    return (int32_t)((uint32_t)st.y + (uint32_t)gp.q0fx +
                     (uint32_t)__float_as_int(__fadd_rn(r, kRoundMagic)));
  };
  auto count_prefix = [](float guess, int n, auto below) {
    int g = (int)fminf(fmaxf(guess, 0.f), (float)n);
#pragma unroll
    for (int it = 0; it < 3; ++it) {
      const bool lo_ok = g == 0 || below(g - 1);
      const bool hi_ok = g == n || !below(g);
      if (lo_ok && hi_ok) return g;
      g += lo_ok ? 1 : -1;
    }
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (below(mid)) lo = mid + 1; else hi = mid;
    }
    return lo;
  };
  const int32_t tfirst = pos(0), tlast = pos(K - 1);
  const int32_t e0 = sedge[0];
  const float bins_per_pos = (float)B / ((float)sedge[B] - (float)e0);
  const int32_t lo_d = group_min(valid ? tfirst : sedge[B], SW);
  const int32_t hi_d = group_max(valid ? tlast : e0, SW);
  const int n_le = count_prefix(((float)lo_d - (float)e0) * bins_per_pos + 1.f, B + 1,
                                [&](int i) { return !(sedge[DR_IDX(i, B + 1, c.err)] > lo_d); });
  const int n_lt = count_prefix(((float)hi_d - (float)e0) * bins_per_pos + 1.f, B + 1,
                                [&](int i) { return sedge[DR_IDX(i, B + 1, c.err)] < hi_d; });
  const int jlo = min(max(n_le - 1, 0), B);
  const int2 sp = make_int2(jlo, max(min(n_lt, B), jlo));
  if constexpr (kTma) {
    const bool late = !mbar_wait_bounded(bar, parity, c.err);
    if (__syncthreads_or(late)) return false;
  }
  const float sign = c.out_sign, zero = __fmul_rn(sign, 0.f);
  const size_t plane = (size_t)c.H * c.W;
  const bool acc = c.accumulate != 0;
  if (!acc)
    zero_outside_span(out, c, row, c0, slab, SW, share, sl, G, sp, ncols, valid, zero, plane);
  if (!valid) return true;
  const int nd = sp.y - sp.x;
  const int jb = sp.x + (int)((long long)nd * share / G);
  const int je = sp.x + (int)((long long)nd * (share + 1) / G);
  if (jb >= je) return true;
  const bool rev = c.reverse != 0;
  const uint16_t *ip = simg + (rev ? (K - 1) * TC : 0) + lc;
  const int istep = rev ? -TC : TC;
  int32_t eb = sedge[DR_IDX(jb, B + 1, c.err)];
  const int n_below = count_prefix(
      ((float)eb - (float)tfirst) * ((float)(K - 1) / ((float)tlast - (float)tfirst)) + 1.f, K,
      [&](int i) { return pos(i) < eb; });
  const int k = min(max(n_below - 1, 0), K - 2);
  // walk state: t0 = t_k, t1 = t_{k+1} (step k1 = k + 1), the image of step
  // k + 1 at ipn, base = I_0 - I_k, dI = I_k - I_{k+1}
  int k1 = k + 1;
  int32_t t0 = pos(k), t1 = pos(k1);
  const int n_simg = Kpad * TC;
  const float I0 = biased(*DR_PTR(ip, simg, n_simg, c.err));
  const uint16_t *ipn = ip + k1 * istep;
  float Ik1 = biased(*DR_PTR(ipn, simg, n_simg, c.err));
  const float Ik = biased(*DR_PTR(ipn - istep, simg, n_simg, c.err));
  float base = __fsub_rn(I0, Ik), dI = __fsub_rn(Ik, Ik1);
  float inv = GeoFx::inv_len(t0, t1);
  auto advance = [&]() {
    t0 = t1;
    t1 = pos(++k1);
    ipn += istep;
    const float In = biased(*DR_PTR(ipn, simg, n_simg, c.err));
    base = __fsub_rn(I0, Ik1);
    dI = __fsub_rn(Ik1, In);
    Ik1 = In;
    inv = GeoFx::inv_len(t0, t1);
  };
  auto F_at = [&](int32_t e) {
    const int32_t ec = min(e, tlast);
    if (t1 < ec) advance();
    if constexpr (!kOneAdv) {
      while (t1 < ec) advance();
    }
    return __fmaf_rn(__fmul_rn(cvt23(max(ec, t0) - t0), inv), dI, base);
  };
  OutT *o = out + (size_t)row * c.W + c0 + lc + (size_t)jb * plane;
  float Fp = F_at(eb);
  const size_t n_out = plane * B;
  if (acc) {
    for (int j = jb; j < je; ++j, o += plane) {
      const int32_t e1 = sedge[DR_IDX(j + 1, B + 1, c.err)];
      const float F = F_at(e1);
      const float v = __fmul_rn(sign, __fsub_rn(F, Fp));
      OutT *oc = DR_PTR(o, out, n_out, c.err);
      if (e1 > tfirst && eb < tlast) st_cs(oc, __fadd_rn(out_load(oc), v));
      Fp = F;
      eb = e1;
    }
  } else {
#pragma unroll 4
    for (int j = jb; j < je; ++j, o += plane) {
      const float F = F_at(sedge[DR_IDX(j + 1, B + 1, c.err)]);
      st_cs(DR_PTR(o, out, n_out, c.err), __fmul_rn(sign, __fsub_rn(F, Fp)));
      Fp = F;
    }
  }
  return true;
}

template <class OutT, bool kTma, bool kOneAdv>
__global__ void __launch_bounds__(512, 3)
    pixels_poly_kernel(const __grid_constant__ CUtensorMap tmap, const uint16_t *__restrict__ img,
                       OutT *__restrict__ out, const Consts c, const Tuning t) {
  extern __shared__ __align__(128) unsigned char smem[];
  if constexpr (kTma) {
    if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t *>(smem), 1);
  }
  pixels_poly_tile<OutT, kTma, kOneAdv>(&tmap, img, out, c, t, blockIdx.y,
                                        blockIdx.x * t.tile_cols, smem, 0u);
}

// ------------------------------------------------- persistent batch kernel ---
// (in dr_batch.cuh, after the interval kernel it can also run)

// ------------------------------------------------ small helper kernels ---


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

}  // namespace dr

namespace dr {

// ---------------------------------------------------- pixel selection ---
// The paper's second experiment varies the percentage of pixels processed
// (Sec. IV-A).  Here a pixel's activity is its total intensity change
// sum_k |I_k - I_{k+1}| (exact); pixels at or above a threshold are
// compacted, in order, into an index list, and only those are reconstructed
// into a compacted [B][n] output.

constexpr int kSelChunk = 4096;  // pixels per block in the compaction kernels

// Reconstruction of listed pixels (compacted output out[j * n + i]).  With
// the plan's per-row tables (row-shared geometry) each lane reads its row's
// (k, f) entries and only the bins in the row's data range touch the images;
// otherwise it runs the per-pixel merge-walk of pixels_kernel on images read
// from global memory.  Both give the full reconstruction's values bitwise.
// A lane's image values come from global memory kSelBuf steps at a time
// into its own column of a shared-memory buffer, so that many loads are in
// flight (one at a time as the walk reached each step left the kernel
// waiting on memory latency).
constexpr int kSelBuf = 16;
constexpr int kSelThreads = 256;

template <class Geo, class OutT>
__global__ void __launch_bounds__(kSelThreads) selected_kernel(const Consts c, int kernel,
                                                       const uint16_t *__restrict__ img,
                                                       const int32_t *__restrict__ idx, int n,
                                                       OutT *__restrict__ out) {
  using pos_t = typename Geo::pos_t;
  __shared__ float sbuf[kSelBuf][kSelThreads];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = idx[i], K = c.K, B = c.B;
  if ((unsigned)p >= (unsigned)(c.H * c.W)) {  // not a pixel of the ROI: reported, not read
    atomicCAS(c.err, 0, kDevBounds | (__LINE__ << 4));
    return;
  }
  const size_t plane = (size_t)c.H * c.W;
  const int row = p / c.W;
  const bool rev = c.reverse != 0;
  auto px = [&](int k) { return biased(__ldg(img + (size_t)(rev ? K - 1 - k : k) * plane + p)); };
  float *const mybuf = &sbuf[0][threadIdx.x];
  int kb = 0, kend = 0;  // steps [kb, kend) are in this lane's buffer
  // image value of step k (k, k + 1 < K); refills the buffer from step k
  auto val = [&](int k) {
    if (k < kb || k >= kend) {
      float v[kSelBuf];
#pragma unroll
      for (int s = 0; s < kSelBuf; ++s) v[s] = k + s < K ? px(k + s) : 0.f;
#pragma unroll
      for (int s = 0; s < kSelBuf; ++s) mybuf[s * kSelThreads] = v[s];
      kb = k;
      kend = min(k + kSelBuf, K);
    }
    return mybuf[(k - kb) * kSelThreads];
  };
  const float sign = c.out_sign;
  const float I0 = px(0);
  OutT *o = out + i;
  if (kernel == DR_KERNEL_ROWS && c.tab != nullptr) {
    const int2 *trow = c.tab + (size_t)row * c.tab_stride;
    const int2 nz = __ldg(trow);
    const int2 *tab = trow + 1;
    const float zero = __fmul_rn(sign, 0.f);
    for (int j = 0; j < nz.x; ++j, o += n) st_cs(o, zero);
    int kcur = -2;  // nothing loaded yet: the first entry always loads both
    float Ik = 0.f, Ik1 = 0.f;
    auto evalF = [&](int2 kf) {
      if (kf.x != kcur) {
        if (kcur >= 0 && kf.x == kcur + 1) {
          Ik = Ik1;
        } else {
          Ik = val(kf.x);
        }
        Ik1 = val(kf.x + 1);
        kcur = kf.x;
      }
      return __fmaf_rn(__int_as_float(kf.y), __fsub_rn(Ik, Ik1), __fsub_rn(I0, Ik));
    };
    if (nz.x < nz.y) {
      float Fp = evalF(__ldg(tab + nz.x));
      for (int j = nz.x; j < nz.y; ++j, o += n) {
        const float F = evalF(__ldg(tab + j + 1));
        st_cs(o, __fmul_rn(sign, __fsub_rn(F, Fp)));
        Fp = F;
      }
    }
    for (int j = max(nz.y, nz.x); j < B; ++j, o += n) st_cs(o, zero);
    return;
  }
  const auto g = Geo::group(c, kernel == DR_KERNEL_ROWS ? row : p);
  const auto *steps = Geo::steps(c);
  int k = 0;
  pos_t t0 = Geo::depth(g, steps[0], c), t1 = Geo::depth(g, steps[1], c);
  // bins at or above the last depth are zero, as in pixels_kernel
  const pos_t tlast = Geo::depth(g, steps[K - 1], c);
  const float zero = __fmul_rn(sign, 0.f);
  auto inv = Geo::inv_len(t0, t1);
  float Ik = I0, Ik1 = val(1), Fp = 0.f;
  pos_t ep = 0;
  for (int j = 0; j <= B; ++j) {
    const pos_t e = Geo::edge(c, j);
    while (k < K - 2 && t1 < e) {
      ++k;
      t0 = t1;
      t1 = Geo::depth(g, steps[k + 1], c);
      inv = Geo::inv_len(t0, t1);
      Ik = Ik1;
      Ik1 = val(k + 1);
    }
    const float f = Geo::frac(e, t0, t1, inv);
    const float F = __fmaf_rn(f, __fsub_rn(Ik, Ik1), __fsub_rn(I0, Ik));
    if (j > 0) {
      st_cs(o, ep < tlast ? __fmul_rn(sign, __fsub_rn(F, Fp)) : zero);
      o += n;
    }
    Fp = F;
    ep = e;
  }
}


// First position i in the sorted list idx[0..n) with idx[i] >= target, found
// by one warp (32 probes per round); every lane returns it.
__device__ __forceinline__ int warp_lower_bound(const int32_t *idx, int n, int target) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = n;  // answer in [lo, hi]
  while (hi - lo > 31) {  // the final round covers hi - lo + 1 <= 32 positions
    const int m = hi - lo;
    const int pos = lo + (int)(((long long)m * lane) / 32);
    const bool ge = __ldg(idx + pos) >= target;
    const unsigned b = __ballot_sync(0xffffffffu, ge);
    if (b == 0) {
      lo = lo + (int)(((long long)m * 31) / 32) + 1;
    } else {
      const int f = __ffs(b) - 1;  // first probe >= target
      const int nhi = lo + (int)(((long long)m * f) / 32);
      const int nlo = f == 0 ? lo : lo + (int)(((long long)m * (f - 1)) / 32) + 1;
      lo = nlo;
      hi = nhi;
    }
  }
  const int pos = lo + lane;
  const bool ge = pos >= hi || __ldg(idx + pos) >= target;
  const unsigned b = __ballot_sync(0xffffffffu, ge);
  return lo + __ffs(b) - 1;
}

// Listed pixels of row-shared geometry, staged like rows_tile: one CTA per
// (row, column tile), the tile copied while its index range is searched; the
// listed pixels' bins are split over the threads, which stream them from
// shared memory into the compacted output out[j * n + i].  Needs the plan's
// row tables; TMA only.
template <class OutT>
__global__ void __launch_bounds__(512) selected_rows_kernel(const __grid_constant__ CUtensorMap tmap,
                                                            const Consts c, const Tuning t,
                                                            const int32_t *__restrict__ idx, int n,
                                                            OutT *__restrict__ out) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  int *range = reinterpret_cast<int *>(smem + 16);
  uint16_t *simg = reinterpret_cast<uint16_t *>(smem + 128);
  const int TC = t.tile_cols, K = c.K, B = c.B;
  const int Kpad = t.kc * t.nchunks;
  int2 *stab0 = reinterpret_cast<int2 *>(smem + 128 + align16((size_t)Kpad * TC * 2) +
                                         align16((size_t)K * sizeof(int32_t)));
  const int row = blockIdx.y, c0 = blockIdx.x * TC;
  const int tid = threadIdx.x, warp = tid >> 5;
  // the tile and the row table are requested first; meanwhile warps 0 and 1
  // find the tile's first and end positions in the index list
  if (tid == 0) {
    mbar_init(bar, 1);
    const uint32_t tab_bytes = (uint32_t)c.tab_stride * 8u;
    mbar_expect_tx(bar, (uint32_t)(Kpad * TC * 2) + tab_bytes);
    for (int ch = 0; ch < t.nchunks; ++ch)
      tma_load_3d(simg + (size_t)ch * t.kc * TC, &tmap, bar, c0, row, ch * t.kc);
    bulk_load_1d(stab0, c.tab + (size_t)row * c.tab_stride, tab_bytes, bar);
  }
  if (warp < 2) {
    const int first = row * c.W + c0;
    const int r = warp_lower_bound(idx, n, warp == 0 ? first : first + min(TC, c.W - c0));
    if ((tid & 31) == 0) range[warp] = r;
  }
  __syncthreads();
  const bool late = !mbar_wait_bounded(bar, 0, c.err);
  if (__syncthreads_or(late)) return;
  const int lo = range[0], hi = range[1];
  if (lo >= hi) return;  // nothing listed in this tile (its copies are complete)
  const int2 nz = stab0[0];
  const int2 *stab = stab0 + 1;
  const float sign = c.out_sign, zero = __fmul_rn(sign, 0.f);
  const bool rev = c.reverse != 0;
  // the m listed pixels x G bin groups (G the largest power of two with
  // m * G <= threads); consecutive threads take consecutive listed pixels,
  // so the stores of one bin are contiguous
  const int m = hi - lo, NT = blockDim.x;
  int G = 1;
  while (G < 32 && m * G * 2 <= NT) G *= 2;
  for (int sidx = tid; sidx < m * G; sidx += NT) {
    const int il = sidx % m, g = sidx / m, i = lo + il;
    const int jb = (int)((long long)B * g / G), je = (int)((long long)B * (g + 1) / G);
    const int lc = idx[i] - row * c.W - c0;
    if ((unsigned)lc >= (unsigned)min(TC, c.W - c0)) {  // a list not in increasing order
      atomicCAS(c.err, 0, kDevBounds | (__LINE__ << 4));
      continue;
    }
    auto pxs = [&](int k) { return biased(simg[(size_t)(rev ? K - 1 - k : k) * TC + lc]); };
    const float I0 = pxs(0);
    OutT *o = out + (size_t)jb * n + i;
    int j = jb;
    for (; j < min(je, nz.x); ++j, o += n) st_cs(o, zero);
    const int a = max(jb, nz.x), b = min(je, nz.y);
    if (a < b) {
      auto evalF = [&](int2 kf) {
        const float x = pxs(kf.x), y = pxs(kf.x + 1);
        return __fmaf_rn(__int_as_float(kf.y), __fsub_rn(x, y), __fsub_rn(I0, x));
      };
      float Fp = evalF(stab[a]);
#pragma unroll 4
      for (j = a; j < b; ++j, o += n) {
        const float F = evalF(stab[j + 1]);
        st_cs(o, __fmul_rn(sign, __fsub_rn(F, Fp)));
        Fp = F;
      }
    }
    for (j = max(j, max(jb, nz.y)); j < je; ++j, o += n) st_cs(o, zero);
  }
}
}  // namespace dr
