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
//  pixels_kernel  every pixel has its own depth sequence: the tile's depth
//                 positions go to shared memory once, then the warps split
//                 the bins evenly and each lane walks its pixel's steps and
//                 bins together (merge-walk), one step advance per bin when
//                 the plan found every step at least as long as every bin.
//  intervals_kernel  depths in any order (dr_intervals.cuh): every interval
//                 is added by itself into shared-memory accumulators.
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

#include <algorithm>
#include <cstring>
#include <mutex>

#include "dr_device.cuh"
#include "dr_internal.h"
#include "dr_intervals.cuh"

namespace dr {

// Plan-time check of every (group, step): one thread per group computes
// the K depth positions exactly as the kernels do (FP32 geometry: the
// plan's form of the remainder on its fixed-point grid; FP64 geometry: the
// FP64 depths) and records (PlanCheck) the first group whose positions are
// not strictly increasing with steps in [kMinStepUnits, kMaxStepUnits)
// (FP64: not increasing), the smallest and largest step, the range of the
// positions and, for FP32 geometry, the largest distance from the FP64
// solution, all in grid units.  monotone = 0 records the range and the
// distance only (the interval kernel takes any order).  res must hold
// bad = ~0, min_step = tmin = INT32_MAX, max_step = tmax = INT32_MIN and
// max_dev = 0 before the launch.
// The FP64 position of (group, step), as depth_f64 solves it, reached by one
// fixed-point pass from the FP32 position t (grid units).  The pass maps t
// to z + Q0 + (a + sR dL(t)) / (D - eta); dL has slope below 1 in t and sR
// is the wire radius, far below D - eta, so the pass shrinks any error in t
// by that ratio: from a start within a few grid units it lands within a
// small fraction of a unit of the solution, as depth_f64's passes from its
// own start do, with two of their five FP64 divisions and one of their two
// square roots.  inv_scale = 2^-shift.
__device__ __forceinline__ double depth_f64_from(const GroupD &g, const StepD &s,
                                                 const Consts &c, double t_units,
                                                 double inv_scale) {
  const double z = s.z, Dm = g.D - s.eta;
  const double a = c.y0d * z + s.eta * (z - g.Z + g.Q0);
  const double t = t_units * inv_scale + c.origin;
  const double u = g.Z - t;
  const double L = sqrt(g.Y2 + u * u);
  const double dL = t * (t - 2.0 * g.Z) / (L + g.L0);
  return ((z - c.origin) + g.Q0) + (a + c.sRd * dL) / Dm;
}

template <bool kF64>
__global__ void __launch_bounds__(256) check_kernel(const Consts c, int ngroups, int monotone,
                                                   PlanCheck *res) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t lmin = 0x7fffffff, lmax = (int32_t)0x80000000, ldev = 0;
  int32_t tlo = 0x7fffffff, thi = (int32_t)0x80000000;
  unsigned long long bad = ~0ull;
  if (i < ngroups) {
    const GroupD gd = c.grp64[i];
    const double scale = (double)c.scale;
    auto clamp32 = [](double v) {
      return (int32_t)fmin(fmax(rint(v), -2147483648.0), 2147483647.0);
    };
    double prev64 = 0.0;
    long long prev = 0;
    for (int k = 0; k < c.K; ++k) {
      double t64;  // grid units
      long long t;
      if constexpr (kF64) {
        t64 = depth_f64(gd, c.stp64[k], c) * scale;
        t = clamp32(t64);
        if (k > 0 && !(t64 > prev64) && bad == ~0ull && monotone)
          bad = ((unsigned long long)i << 32) | (unsigned)k;
      } else {
        t = depth_fx(c.grp[i], c.stp[k], c);
        t64 = depth_f64_from(gd, c.stp64[k], c, (double)(int32_t)t, 1.0 / scale) * scale;
        ldev = max(ldev, clamp32(fabs((double)t - rint(t64))));
      }
      tlo = min(tlo, (int32_t)t);
      thi = max(thi, (int32_t)t);
      if (k > 0) {
        const long long st = kF64 ? (long long)clamp32(t64 - prev64) : t - prev;
        lmin = (int32_t)min((long long)lmin, max(st, -2000000000ll));
        lmax = (int32_t)max((long long)lmax, min(st, 2000000000ll));
        if (!kF64 && monotone && (st < kMinStepUnits || st >= kMaxStepUnits) && bad == ~0ull)
          bad = ((unsigned long long)i << 32) | (unsigned)k;
      }
      prev = t;
      prev64 = t64;
    }
  }
  for (int m = 16; m > 0; m >>= 1) {
    lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, m));
    lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, m));
    ldev = max(ldev, __shfl_xor_sync(0xffffffffu, ldev, m));
    tlo = min(tlo, __shfl_xor_sync(0xffffffffu, tlo, m));
    thi = max(thi, __shfl_xor_sync(0xffffffffu, thi, m));
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, bad, m);
    bad = o < bad ? o : bad;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&res->min_step, lmin);
    atomicMax(&res->max_step, lmax);
    atomicMax(&res->max_dev, ldev);
    atomicMin(&res->tmin, tlo);
    atomicMax(&res->tmax, thi);
    if (bad != ~0ull) atomicMin(&res->bad, bad);
  }
}

// FP64 solution of the tangent condition (the plan's host solve_t, on the
// device): t = z + Q0 + (a + sR dL(t)) / (D - eta), three fixed-point passes.
__device__ double solve_t_dev(double Y, double Z, double y0, double sR, double D, double L0,
                              double Q0, double z, double eta) {
  const double Dm = D - eta;
  const double a = y0 * z + eta * (z - Z + Q0);
  double t = z + Q0 + a / Dm;
  for (int it = 0; it < 3; ++it) {
    const double u = Z - t;
    const double L = sqrt(Y * Y + u * u);
    const double dL = t * (t - 2.0 * Z) / (L + L0);
    t = z + Q0 + (a + sR * dL) / Dm;
  }
  return t;
}

// Per-group constants of a plan, in FP64, from the affine pixel coordinates
// Y = Y00 + r Yr + c Yc, Z = Z00 + r Zr + c Zc (group i is row i, or pixel
// (i / W, i % W)): the FP64 mirror (GroupD) and the FP32 constants of the
// plan's form of the remainder (GroupC; GroupPoly for the polynomial form:
// the cubic through the remainder at four Chebyshev nodes of [zc - zh,
// zc + zh], in grid units).
__global__ void __launch_bounds__(256) groups_kernel(const GroupsParams q, GroupC *gc,
                                                    GroupD *gd) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= q.ngroups) return;
  const double r = q.rows_shared ? (double)i : (double)(i / q.W);
  const double cc = q.rows_shared ? 0.0 : (double)(i % q.W);
  const double Y = q.Y00 + r * q.Yr + cc * q.Yc, Z = q.Z00 + r * q.Zr + cc * q.Zc;
  const double D = Y - q.y0, L0 = sqrt(Y * Y + Z * Z), Q0 = (-q.y0 * Z + q.sR * L0) / D;
  gd[i] = GroupD{Z, Y * Y, L0, D, Q0};
  const long long q0 = __double2ll_rn(Q0 * q.scale);
  GroupC g;
  if (q.mode == kDepthPoly) {
    const double node[4] = {0.92387953251128674, 0.38268343236508978, -0.38268343236508978,
                            -0.92387953251128674};
    double x[4], v[4];
    for (int n = 0; n < 4; ++n) {
      x[n] = q.zh * node[n];
      const double z = q.zc + x[n];
      v[n] = (solve_t_dev(Y, Z, q.y0, q.sR, D, L0, Q0, z, 0.0) - z - Q0) * q.scale;
    }
    // Newton divided differences, then the monomial coefficients in d = z - zc
    const double a0 = v[0];
    const double d01 = (v[1] - v[0]) / (x[1] - x[0]), d12 = (v[2] - v[1]) / (x[2] - x[1]),
                 d23 = (v[3] - v[2]) / (x[3] - x[2]);
    const double d012 = (d12 - d01) / (x[2] - x[0]), d123 = (d23 - d12) / (x[3] - x[1]);
    const double a1 = d01, a2 = d012, a3 = (d123 - d012) / (x[3] - x[0]);
    GroupPoly p;
    p.c3 = (float)a3;
    p.c2 = (float)(a2 - a3 * (x[0] + x[1] + x[2]));
    p.c1 = (float)(a1 - a2 * (x[0] + x[1]) + a3 * (x[0] * x[1] + x[0] * x[2] + x[1] * x[2]));
    p.c0 = (float)(a0 - a1 * x[0] + a2 * x[0] * x[1] - a3 * x[0] * x[1] * x[2]);
    p.unused0 = p.unused1 = p.unused2 = 0.f;
    p.q0fx = (int32_t)(q0 - kRoundMagicBits);
    memcpy(&g, &p, sizeof(g));
  } else {
    g.Z = (float)Z;
    g.Y2 = (float)(Y * Y);
    g.L0 = (float)L0;
    g.invD = (float)(1.0 / D);
    g.D = (float)D;
    g.Q0f = (float)Q0;
    g.Q0fx = (int32_t)q0;
    g.invL0 = (float)(1.0 / L0);
  }
  gc[i] = g;
}

dr_status run_groups(const GroupsParams &q, GroupC *gc, GroupD *gd) {
  if (q.ngroups <= 0) return DR_OK;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail("plan groups: stream", e);
  groups_kernel<<<(unsigned)((q.ngroups + 255) / 256), 256, 0, st>>>(q, gc, gd);
  e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail("plan groups", e);
  return DR_OK;
}

// Exact differences I_k - I_{k+1} as the kernels form them (int32 out).
__global__ void differences_kernel(const uint16_t *__restrict__ img, long long n_out,
                                   long long plane, int32_t *__restrict__ d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_out;
       i += (long long)gridDim.x * blockDim.x)
    d[i] = __float2int_rn(step_delta(img[i], img[i + plane]));
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

}  // namespace

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

namespace {

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
  // FP32 geometry: the walk takes at most one step per bin when the plan's
  // check found every step at least as long as every bin; the polynomial
  // form computes positions in the walk (pixels_poly_kernel)
  auto fn = pixels_kernel<Geo, OutT, kTma, false>;
  if constexpr (std::is_same<Geo, GeoFx>::value) {
    if (p->c.depth_mode == kDepthPoly)
      fn = p->one_adv ? pixels_poly_kernel<OutT, kTma, true> : pixels_poly_kernel<OutT, kTma, false>;
    else if (p->one_adv)
      fn = pixels_kernel<Geo, OutT, kTma, true>;
  }
  dr_status s = allow_smem((const void *)fn);
  if (s != DR_OK) return s;
  dim3 grid((p->cols + p->tune.tile_cols - 1) / p->tune.tile_cols, p->rows);
  fn<<<grid, p->threads, p->smem_bytes, st>>>(tm, img, (OutT *)out, p->c, p->tune);
  return DR_OK;
}

template <class Geo, class OutT, bool kTma>
dr_status launch_intervals(const dr_plan_t *p, const CUtensorMap &tm, const uint16_t *img,
                           void *out, cudaStream_t st) {
  constexpr bool kFx = std::is_same<Geo, GeoFx>::value;
  auto fn = p->iv_ctas == 3 ? intervals_kernel<Geo, OutT, kTma, kFx ? 3 : 1>
                            : intervals_kernel<Geo, OutT, kTma, kFx ? 2 : 1>;
  dr_status s = allow_smem((const void *)fn);
  if (s != DR_OK) return s;
  dim3 grid((p->cols + kIntervalTile - 1) / kIntervalTile, p->rows);
  fn<<<grid, p->threads, p->smem_bytes, st>>>(tm, img, (OutT *)out, p->c, p->tune,
                                              p->pixel_groups, p->window);
  return DR_OK;
}

template <class Geo, class OutT>
dr_status dispatch_out(const dr_plan_t *p, bool tma, const CUtensorMap &tm, const uint16_t *img,
                       void *out, cudaStream_t st) {
  if (p->kernel == DR_KERNEL_INTERVALS)
    return tma ? launch_intervals<Geo, OutT, true>(p, tm, img, out, st)
               : launch_intervals<Geo, OutT, false>(p, tm, img, out, st);
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

dr_status run_plan_check(const dr_plan_t *p, int ngroups, bool monotone, PlanCheck *d_res,
                         PlanCheck *h_res) {
  PlanCheck init;
  std::memset(&init, 0, sizeof(init));
  init.bad = ~0ull;
  init.min_step = init.tmin = 0x7fffffff;
  init.max_step = init.tmax = (int32_t)0x80000000;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail("plan check: stream", e);
  e = cudaMemcpyAsync(d_res, &init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && ngroups > 0) {
    if (p->geom_prec == DR_GEOM_FP64)
      check_kernel<true><<<(ngroups + 255) / 256, 256, 0, st>>>(p->c, ngroups, monotone, d_res);
    else
      check_kernel<false><<<(ngroups + 255) / 256, 256, 0, st>>>(p->c, ngroups, monotone, d_res);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_res, d_res, sizeof(*h_res), cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail("plan check", e);
  return DR_OK;
}

dr_status build_plan_tables(const dr_plan_t *p, int2 *tab) {
  const bool f64 = p->geom_prec == DR_GEOM_FP64;
  const size_t smem = 16 + (size_t)p->K * (f64 ? 8 : 4);
  const void *fn = f64 ? (const void *)tables_kernel<GeoF64> : (const void *)tables_kernel<GeoFx>;
  dr_status s = allow_smem(fn);
  if (s != DR_OK) return s;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail("plan tables: stream", e);
  if (f64)
    tables_kernel<GeoF64><<<p->rows, 256, smem, st>>>(p->c, tab);
  else
    tables_kernel<GeoFx><<<p->rows, 256, smem, st>>>(p->c, tab);
  e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail("plan tables", e);
  return DR_OK;
}

dr_status preload_kernels() {
  const void *fns[] = {
      (const void *)rows_kernel<GeoFx, float, true, 4>,
      (const void *)rows_kernel<GeoFx, float, false, 4>,
      (const void *)rows_kernel<GeoFx, float, true, 1>,
      (const void *)rows_kernel<GeoFx, float, false, 1>,
      (const void *)rows_kernel<GeoFx, __nv_bfloat16, true, 4>,
      (const void *)rows_kernel<GeoFx, __nv_bfloat16, false, 4>,
      (const void *)rows_kernel<GeoFx, __nv_bfloat16, true, 1>,
      (const void *)rows_kernel<GeoFx, __nv_bfloat16, false, 1>,
      (const void *)pixels_kernel<GeoFx, float, true, true>,
      (const void *)pixels_kernel<GeoFx, float, false, true>,
      (const void *)pixels_kernel<GeoFx, __nv_bfloat16, true, true>,
      (const void *)pixels_kernel<GeoFx, __nv_bfloat16, false, true>,
      (const void *)pixels_kernel<GeoFx, float, true, false>,
      (const void *)pixels_kernel<GeoFx, float, false, false>,
      (const void *)pixels_kernel<GeoFx, __nv_bfloat16, true, false>,
      (const void *)pixels_kernel<GeoFx, __nv_bfloat16, false, false>,
      (const void *)pixels_poly_kernel<float, true, true>,
      (const void *)pixels_poly_kernel<float, false, true>,
      (const void *)pixels_poly_kernel<__nv_bfloat16, true, true>,
      (const void *)pixels_poly_kernel<__nv_bfloat16, false, true>,
      (const void *)pixels_poly_kernel<float, true, false>,
      (const void *)pixels_poly_kernel<float, false, false>,
      (const void *)pixels_poly_kernel<__nv_bfloat16, true, false>,
      (const void *)pixels_poly_kernel<__nv_bfloat16, false, false>,
      (const void *)check_kernel<false>,
      (const void *)check_kernel<true>,
      (const void *)groups_kernel,
      (const void *)intervals_kernel<GeoFx, float, true, 2>,
      (const void *)intervals_kernel<GeoFx, float, false, 2>,
      (const void *)intervals_kernel<GeoFx, __nv_bfloat16, true, 2>,
      (const void *)intervals_kernel<GeoFx, __nv_bfloat16, false, 2>,
      (const void *)intervals_kernel<GeoFx, float, true, 3>,
      (const void *)intervals_kernel<GeoFx, float, false, 3>,
      (const void *)intervals_kernel<GeoFx, __nv_bfloat16, true, 3>,
      (const void *)intervals_kernel<GeoFx, __nv_bfloat16, false, 3>,
  };
  for (const void *f : fns) {
    dr_status s = allow_smem(f);
    if (s != DR_OK) return s;
  }
  return DR_OK;
}

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

// A plan's launches: one, or each part of a composite plan on its run's image
// planes (part 0 writes the output, later parts add to it).
dr_status launch_plan(const dr_plan_t *p, const uint16_t *img, void *out, cudaStream_t st) {
  if (p->parts.empty()) return launch_reconstruct(p, img, out, st);
  const size_t plane = (size_t)p->rows * p->cols;
  for (size_t i = 0; i < p->parts.size(); ++i) {
    dr_status s = launch_reconstruct(p->parts[i], img + (size_t)p->part_k0[i] * plane, out, st);
    if (s != DR_OK) return s;
  }
  return DR_OK;
}

}  // namespace dr

using namespace dr;

extern "C" dr_status dr_reconstruct(const dr_plan_t *p, const uint16_t *img, void *out,
                                    dr_stream_t stream) {
  TraceRange trace_("dr_reconstruct");
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
  dr_status s = launch_plan(p, img, out, st);
  if (s != DR_OK) return s;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct: launch", e);
  return DR_OK;
}

extern "C" dr_status dr_reconstruct_host(const dr_plan_t *p, const uint16_t *h_img, void *h_out,
                                         uint16_t *d_img, void *d_out, dr_stream_t stream) {
  TraceRange trace_("dr_reconstruct_host");
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
  TraceRange trace_("dr_image_differences");
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
  TraceRange trace_("dr_plan_depths");
  if (!p || r0 < 0 || nrows < 0 || r0 + nrows > p->rows) {
    set_error("dr_plan_depths: bad arguments");
    return DR_ERR_INVALID_ARG;
  }
  if (!p->parts.empty()) {
    set_error("dr_plan_depths: not available for plans of several runs or both edges");
    return DR_ERR_UNSUPPORTED;
  }
  const long long n = (long long)nrows * p->cols * p->K;
  if (n == 0) return DR_OK;
  if (!d) {
    set_error("dr_plan_depths: null buffer");
    return DR_ERR_INVALID_ARG;
  }
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  // the depth kernel picks the group layout from a kernel kind
  const int layout = p->pixel_groups ? DR_KERNEL_PIXELS : DR_KERNEL_ROWS;
  if (p->geom_prec == DR_GEOM_FP64)
    depths_kernel<GeoF64><<<blocks, 256, 0, (cudaStream_t)stream>>>(p->c, layout, r0, nrows, d);
  else
    depths_kernel<GeoFx><<<blocks, 256, 0, (cudaStream_t)stream>>>(p->c, layout, r0, nrows, d);
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
    if ((v & 15) == kDevBounds) {  // the bounds-checked build, or a bad pixel list
      set_error("a kernel index was out of range (device source line %d)", v >> 4);
      return DR_ERR_CUDA;
    }
    set_error("a kernel's bounded wait for its TMA tile ran out (code %d)", v);
    return DR_ERR_TIMEOUT;
  }
  return DR_OK;
}

// ------------------------------------------------ failure-path diagnostic ---
namespace dr {
// One CTA whose barrier nothing arrives at: the bounded wait runs out after
// limit_ns, the timeout code goes to *err, and every thread returns.
__global__ void wait_probe_kernel(int32_t *err, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(&bar, 0)) {
    if (global_ns() - t0 > limit_ns) {
      if (threadIdx.x == 0) atomicExch(err, kDevTmaTimeout);
      return;
    }
  }
}
}  // namespace dr

extern "C" dr_status dr_selftest_wait_timeout(int32_t *d_status, double wait_ms,
                                              dr_stream_t stream) {
  if (!d_status || !(wait_ms > 0.0) || wait_ms > 2000.0) {
    set_error("dr_selftest_wait_timeout: need a status word and 0 < wait_ms <= 2000");
    return DR_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_fail("dr_selftest_wait_timeout: clear", e);
  wait_probe_kernel<<<1, 32, 0, st>>>(d_status, (unsigned long long)(wait_ms * 1e6));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("dr_selftest_wait_timeout: launch", e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("dr_selftest_wait_timeout: synchronize", e);
  int32_t v = 0;
  e = cudaMemcpy(&v, d_status, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail("dr_selftest_wait_timeout: read", e);
  if (v == kDevTmaTimeout) {
    set_error("bounded wait ran out after %.1f ms (code %d)", wait_ms, v);
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
  // a captured copy would keep reading the library's host buffer, which
  // every later call overwrites: refuse to be captured
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct_rows_static: cudaStreamIsCapturing", e);
  if (cap != cudaStreamCaptureStatusNone) {
    set_error("dr_reconstruct_rows_static: cannot be captured into a CUDA graph");
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

// ------------------------------------------- streamed (out-of-core) form ---
// Row slabs of the scan flow through a small device workspace: host->device
// copy of a slab of every image (one 2-D copy: K planes, each slab_rows x cols
// uint16 at a pitch of rows x cols), the kernel on that slab, and a 2-D copy
// of the slab's bins back to the host.  Three streams overlap the two copy
// directions with the kernels; nbuf slab buffers rotate.  Used when the scan
// does not fit in device memory, and for the end-to-end form.

namespace {

struct StreamSet {
  cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
  cudaEvent_t start = nullptr, up_done[3] = {}, comp_done[3] = {}, down_done[3] = {};
  bool ok = false;
};
std::mutex g_streamset_mu;
StreamSet g_streamsets[64];

dr_status stream_set(StreamSet **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
  if (dev < 0 || dev >= 64) {
    set_error("device %d out of range", dev);
    return DR_ERR_UNSUPPORTED;
  }
  StreamSet &s = g_streamsets[dev];
  if (!s.ok) {
    const unsigned ev = cudaEventDisableTiming;
    e = cudaStreamCreateWithFlags(&s.up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.down, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.start, ev);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
      e = cudaEventCreateWithFlags(&s.up_done[i], ev);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.comp_done[i], ev);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.down_done[i], ev);
    }
    if (e != cudaSuccess) return cuda_fail("stream set", e);
    s.ok = true;
  }
  *out = &s;
  return DR_OK;
}

}  // namespace

extern "C" dr_status dr_reconstruct_streamed(const dr_plan_t *p, const uint16_t *h_img,
                                             void *h_out, void *d_ws, size_t ws_bytes,
                                             int32_t slab_rows, dr_stream_t stream) {
  TraceRange trace_("dr_reconstruct_streamed");
  if (!p) {
    set_error("dr_reconstruct_streamed: null plan");
    return DR_ERR_INVALID_ARG;
  }
  const int H = p->rows, W = p->cols, K = p->K, B = p->B;
  if ((size_t)H * W == 0) return DR_OK;
  if (!h_img || !h_out || !d_ws) {
    set_error("dr_reconstruct_streamed: null buffer");
    return DR_ERR_INVALID_ARG;
  }
  const size_t osz = p->out_dtype == DR_OUT_BF16 ? 2 : 4;
  auto slab_bytes = [&](int n) {
    return ((size_t)n * W * K * 2 + 255) / 256 * 256 + ((size_t)n * W * B * osz + 255) / 256 * 256;
  };
  const int nbuf = 3;
  if (slab_rows <= 0) {  // largest slab with three buffers in the workspace
    slab_rows = (int)std::min<size_t>(H, ws_bytes / nbuf / std::max<size_t>(slab_bytes(1), 1));
    if (slab_rows > 64) slab_rows = slab_rows / 8 * 8;
  }
  slab_rows = std::min(slab_rows, H);
  if (slab_rows < 1 || slab_bytes(slab_rows) * nbuf > ws_bytes || ((uintptr_t)d_ws & 255)) {
    set_error("dr_reconstruct_streamed: workspace of %zu bytes holds no three slabs of %d rows "
              "(%zu bytes each, 256-byte aligned)", ws_bytes, slab_rows, slab_bytes(std::max(slab_rows, 1)));
    return DR_ERR_BUDGET;
  }
  StreamSet *ss = nullptr;
  std::lock_guard<std::mutex> lk(g_streamset_mu);
  dr_status s = stream_set(&ss);
  if (s != DR_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaEventRecord(ss->start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ss->up, ss->start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ss->comp, ss->start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ss->down, ss->start, 0);
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct_streamed: fork", e);
  const int groups_per_row = p->pixel_groups ? W : 1;
  const int nslab = (H + slab_rows - 1) / slab_rows;
  // When h_out is pinned (mapped into the device's address space) and the
  // slabs are staged by TMA, the kernels store each slab's bins straight into
  // h_out over the host link: the output crosses the link once with no
  // download stage (full-detector scan: 86.7 ms for the kernel writing to
  // the host against 94 ms for one device->host copy of the same bytes).  The
  // kernels then take the whole scan's rows as their output plane.  Plans of
  // several parts (which add to their output) keep the download.
  unsigned char *h_out_dev = nullptr;
  if (p->parts.empty() && tma_usable(p, static_cast<const uint16_t *>(d_ws))) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, h_out) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer)
      h_out_dev = static_cast<unsigned char *>(at.devicePointer);
    else
      cudaGetLastError();  // an unregistered buffer: the download path
  }
  for (int i = 0; i < nslab; ++i) {
    const int b = i % nbuf, r0 = i * slab_rows, n = std::min(slab_rows, H - r0);
    unsigned char *buf = static_cast<unsigned char *>(d_ws) + slab_bytes(slab_rows) * b;
    uint16_t *dimg = reinterpret_cast<uint16_t *>(buf);
    void *dout = buf + ((size_t)slab_rows * W * K * 2 + 255) / 256 * 256;
    // upload: wait until the kernel that last read this buffer is done
    if (i >= nbuf) e = cudaStreamWaitEvent(ss->up, ss->comp_done[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(dimg, (size_t)n * W * 2, h_img + (size_t)r0 * W, (size_t)H * W * 2,
                            (size_t)n * W * 2, K, cudaMemcpyHostToDevice, ss->up);
    if (e == cudaSuccess) e = cudaEventRecord(ss->up_done[b], ss->up);
    // kernel: after the upload, and after the previous download of this buffer
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss->comp, ss->up_done[b], 0);
    if (e == cudaSuccess && i >= nbuf && !h_out_dev)
      e = cudaStreamWaitEvent(ss->comp, ss->down_done[b], 0);
    if (e != cudaSuccess) return cuda_fail("dr_reconstruct_streamed: upload", e);
    const size_t nparts = p->parts.empty() ? 1 : p->parts.size();
    for (size_t q = 0; q < nparts; ++q) {
      const dr_plan_t *part = p->parts.empty() ? p : p->parts[q];
      const int k0 = p->parts.empty() ? 0 : p->part_k0[q];
      dr_plan_t slab = *part;
      slab.parts.clear();
      slab.rows = n;
      slab.c.H = h_out_dev ? H : n;  // rows of the output plane
      slab.c.grp = part->c.grp + (size_t)r0 * groups_per_row;
      slab.c.grp64 = part->c.grp64 + (size_t)r0 * groups_per_row;
      if (part->c.tab) slab.c.tab = part->c.tab + (size_t)r0 * part->c.tab_stride;
      void *o = h_out_dev ? (void *)(h_out_dev + (size_t)r0 * W * osz) : dout;
      s = launch_reconstruct(&slab, dimg + (size_t)k0 * n * W, o, ss->comp);
      if (s != DR_OK) return s;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ss->comp_done[b], ss->comp);
    if (e != cudaSuccess) return cuda_fail("dr_reconstruct_streamed: kernel", e);
    if (h_out_dev) continue;  // the kernel wrote the slab's bins to the host
    // download the slab's bins into rows r0.. of every output plane
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss->down, ss->comp_done[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(static_cast<unsigned char *>(h_out) + (size_t)r0 * W * osz,
                            (size_t)H * W * osz, dout, (size_t)n * W * osz, (size_t)n * W * osz, B,
                            cudaMemcpyDeviceToHost, ss->down);
    if (e == cudaSuccess) e = cudaEventRecord(ss->down_done[b], ss->down);
    if (e != cudaSuccess) return cuda_fail("dr_reconstruct_streamed: download", e);
  }
  // join: the caller's stream continues after the last download (or the
  // last kernel when the kernels wrote to the host)
  cudaStream_t last = h_out_dev ? ss->comp : ss->down;
  e = cudaEventRecord(ss->down_done[0], last);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ss->down_done[0], 0);
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct_streamed: join", e);
  return DR_OK;
}

// ------------------------------------------------------ pixel selection ---

namespace dr {
// Two adjacent pixels per thread (one 32-bit load per step when P is even),
// steps unrolled so that several loads are in flight per thread.
__global__ void activity_kernel(const uint16_t *__restrict__ img, int K, long long P,
                                float *__restrict__ act) {
  const long long pairs = (P + 1) / 2;
  const bool even = (P % 2) == 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < pairs;
       q += (long long)gridDim.x * blockDim.x) {
    const long long p = 2 * q;
    const bool two = p + 1 < P;
    auto ld = [&](int k, int &a, int &b) {
      const size_t o = (size_t)k * P + p;
      if (even) {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(img + o));
        a = (int)(w & 0xFFFFu);
        b = (int)(w >> 16);
      } else {
        a = __ldg(img + o);
        b = two ? __ldg(img + o + 1) : 0;
      }
    };
    int pa, pb, sa = 0, sb = 0;
    ld(0, pa, pb);
    int k = 1;
    for (; k + 3 < K; k += 4) {
      int a0, b0, a1, b1, a2, b2, a3, b3;
      ld(k, a0, b0);
      ld(k + 1, a1, b1);
      ld(k + 2, a2, b2);
      ld(k + 3, a3, b3);
      sa += abs(pa - a0) + abs(a0 - a1) + abs(a1 - a2) + abs(a2 - a3);
      sb += abs(pb - b0) + abs(b0 - b1) + abs(b1 - b2) + abs(b2 - b3);
      pa = a3;
      pb = b3;
    }
    for (; k < K; ++k) {
      int a, b;
      ld(k, a, b);
      sa += abs(pa - a);
      sb += abs(pb - b);
      pa = a;
      pb = b;
    }
    act[p] = (float)sa;
    if (two) act[p + 1] = (float)sb;
  }
}

// Eight adjacent pixels per thread with one 16-byte load per step (P a
// multiple of 8, images 16-byte aligned): 64 bytes in flight per thread with
// the steps unrolled by 4, enough to cover the memory latency.
__global__ void activity8_kernel(const uint16_t *__restrict__ img, int K, long long P,
                                 float *__restrict__ act) {
  const long long oct = P / 8;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < oct;
       q += (long long)gridDim.x * blockDim.x) {
    const uint4 *src = reinterpret_cast<const uint4 *>(img) + q;
    const long long stride = P / 8;  // one step, in 16-byte units
    uint32_t prev[8], sum[8];
    auto unpack = [](const uint4 &w, uint32_t *v) {
      v[0] = w.x & 0xFFFFu; v[1] = w.x >> 16; v[2] = w.y & 0xFFFFu; v[3] = w.y >> 16;
      v[4] = w.z & 0xFFFFu; v[5] = w.z >> 16; v[6] = w.w & 0xFFFFu; v[7] = w.w >> 16;
    };
    unpack(__ldg(src), prev);
#pragma unroll
    for (int i = 0; i < 8; ++i) sum[i] = 0;
    auto add = [&](const uint4 &w) {
      uint32_t v[8];
      unpack(w, v);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        sum[i] = __sad((int)v[i], (int)prev[i], sum[i]);
        prev[i] = v[i];
      }
    };
    int k = 1;
    for (; k + 3 < K; k += 4) {
      const uint4 w0 = __ldg(src + (size_t)k * stride), w1 = __ldg(src + (size_t)(k + 1) * stride);
      const uint4 w2 = __ldg(src + (size_t)(k + 2) * stride), w3 = __ldg(src + (size_t)(k + 3) * stride);
      add(w0);
      add(w1);
      add(w2);
      add(w3);
    }
    for (; k < K; ++k) add(__ldg(src + (size_t)k * stride));
    float4 *dst = reinterpret_cast<float4 *>(act + 8 * q);
    dst[0] = make_float4((float)sum[0], (float)sum[1], (float)sum[2], (float)sum[3]);
    dst[1] = make_float4((float)sum[4], (float)sum[5], (float)sum[6], (float)sum[7]);
  }
}

// pass 1: selected pixels per chunk
__global__ void select_count_kernel(const float *__restrict__ act, long long n, float thr,
                                    int *__restrict__ counts) {
  __shared__ int total;
  if (threadIdx.x == 0) total = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSelChunk;
  int mine = 0;
  for (int i = threadIdx.x; i < kSelChunk; i += blockDim.x) {
    const long long p = base + i;
    mine += (p < n && act[p] >= thr);
  }
  atomicAdd(&total, mine);
  __syncthreads();
  if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// pass 2 (one block): exclusive scan of the chunk counts, total to *count
__global__ void select_scan_kernel(int *__restrict__ counts, int nchunks, int *__restrict__ count) {
  __shared__ int carry;
  __shared__ int warp_sums[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nchunks; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < nchunks ? counts[i] : 0;
    int x = v;  // inclusive warp scan
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
      int ws = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sums[lane] = ws;  // inclusive over warps
    }
    __syncthreads();
    const int before = carry + (w > 0 ? warp_sums[w - 1] : 0) + x - v;
    if (i < nchunks) counts[i] = before;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = carry;
}

// pass 3: each chunk writes its selected indices, in order, at its offset
__global__ void select_write_kernel(const float *__restrict__ act, long long n, float thr,
                                    const int *__restrict__ offsets, int32_t *__restrict__ idx) {
  __shared__ int warp_base[32];
  __shared__ int running;
  if (threadIdx.x == 0) running = offsets[blockIdx.x];
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSelChunk;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = 0; i0 < kSelChunk; i0 += blockDim.x) {
    const long long p = base + i0 + threadIdx.x;
    const bool sel = p < n && act[p] >= thr;
    const unsigned m = __ballot_sync(0xffffffffu, sel);
    if (lane == 0) warp_base[w] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {  // warp offsets in order
      int acc = running;
      for (int q = 0; q < nw; ++q) {
        const int c = warp_base[q];
        warp_base[q] = acc;
        acc += c;
      }
      running = acc;
    }
    __syncthreads();
    if (sel) idx[warp_base[w] + __popc(m & ((1u << lane) - 1u))] = (int32_t)p;
    __syncthreads();
  }
}

}  // namespace dr

extern "C" dr_status dr_pixel_activity(const uint16_t *img, int32_t K, int32_t rows, int32_t cols,
                                       float *act, dr_stream_t stream) {
  TraceRange trace_("dr_pixel_activity");
  const long long P = (long long)rows * cols;
  if (K < 1 || rows < 0 || cols < 0) {
    set_error("dr_pixel_activity: bad sizes");
    return DR_ERR_INVALID_ARG;
  }
  if (P == 0) return DR_OK;
  if (!img || !act) {
    set_error("dr_pixel_activity: null buffer");
    return DR_ERR_INVALID_ARG;
  }
  if ((long long)K * 65535 > 2147483647LL) {
    set_error("dr_pixel_activity: K too large for an exact int32 sum");
    return DR_ERR_UNSUPPORTED;
  }
  if (P % 2 == 0 && ((uintptr_t)img & 3) != 0) {
    set_error("dr_pixel_activity: images not 4-byte aligned");
    return DR_ERR_INVALID_ARG;
  }
  if (P % 8 == 0 && ((uintptr_t)img & 15) == 0 && ((uintptr_t)act & 15) == 0) {
    const int blocks = (int)std::min<long long>((P / 8 + 255) / 256, 152 * 64);
    activity8_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(img, K, P, act);
  } else {
    const int blocks = (int)std::min<long long>(((P + 1) / 2 + 255) / 256, 152 * 16);
    activity_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(img, K, P, act);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("dr_pixel_activity", e);
  return DR_OK;
}

extern "C" size_t dr_select_scratch_bytes(int64_t n) {
  const long long chunks = (n + kSelChunk - 1) / kSelChunk;
  return (size_t)std::max<long long>(chunks, 1) * sizeof(int);
}

extern "C" dr_status dr_select_pixels(const float *act, int64_t n, float threshold,
                                      int32_t *idx, int32_t *count, void *scratch,
                                      size_t scratch_bytes, dr_stream_t stream) {
  TraceRange trace_("dr_select_pixels");
  if (n < 0 || n > 2147483647LL || !act || !idx || !count || !scratch) {
    set_error("dr_select_pixels: bad arguments");
    return DR_ERR_INVALID_ARG;
  }
  if (scratch_bytes < dr_select_scratch_bytes(n)) {
    set_error("dr_select_pixels: scratch of %zu bytes, need %zu", scratch_bytes,
              dr_select_scratch_bytes(n));
    return DR_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int chunks = (int)((n + kSelChunk - 1) / kSelChunk);
  int *counts = static_cast<int *>(scratch);
  if (chunks == 0) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail("dr_select_pixels", e);
    return DR_OK;
  }
  select_count_kernel<<<chunks, 256, 0, st>>>(act, n, threshold, counts);
  select_scan_kernel<<<1, 1024, 0, st>>>(counts, chunks, count);
  select_write_kernel<<<chunks, 256, 0, st>>>(act, n, threshold, counts, idx);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("dr_select_pixels", e);
  return DR_OK;
}

extern "C" dr_status dr_reconstruct_selected(const dr_plan_t *p, const uint16_t *img,
                                             const int32_t *idx, int32_t n, void *out,
                                             dr_stream_t stream) {
  TraceRange trace_("dr_reconstruct_selected");
  if (!p || n < 0) {
    set_error("dr_reconstruct_selected: bad arguments");
    return DR_ERR_INVALID_ARG;
  }
  if (!p->parts.empty() || p->kernel == DR_KERNEL_INTERVALS) {
    set_error("dr_reconstruct_selected: not available for plans of several runs or both edges"
              " or for the interval kernel");
    return DR_ERR_UNSUPPORTED;
  }
  if (n == 0 || (size_t)p->rows * p->cols == 0) return DR_OK;
  if (!img || !idx || !out) {
    set_error("dr_reconstruct_selected: null buffer");
    return DR_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool bf16 = p->out_dtype == DR_OUT_BF16;
  // Staged tiles load every image row segment that holds a listed pixel and
  // split the listed pixels' bins over the CTA's threads; they pay off when
  // nearly all pixels are listed (measured on the full-detector scan: the
  // per-lane walk, images read from global memory in runs of steps, is
  // faster up to at least three quarters of the pixels, where the staged
  // tiles' short compacted output runs per tile leave partial 32-byte
  // sectors; the staged tiles win at all pixels).
  const bool dense = (double)n >= 0.9 * (double)p->rows * p->cols;
  if (dense && p->kernel == DR_KERNEL_ROWS && p->c.tab && tma_usable(p, img)) {
    // staged: one CTA per (row, tile of at most 128 columns, two CTAs per
    // SM), 512 threads (listed pixels x bin groups)
    dr_plan_t q;
    q.rows = p->rows;
    q.cols = p->cols;
    q.K = p->K;
    q.tune = p->tune;
    q.tune.tile_cols = std::min(p->tune.tile_cols, 128);
    choose_chunks(p->K, q.tune.tile_cols, &q.tune.kc, &q.tune.nchunks);
    const int smem = rows_smem_bytes(p->K, q.tune.kc * q.tune.nchunks, p->B, q.tune.tile_cols,
                                     false);
    CUtensorMap tm;
    dr_status s = make_tensor_map(&q, img, &tm);
    if (s != DR_OK) return s;
    const void *fn = bf16 ? (const void *)selected_rows_kernel<__nv_bfloat16>
                          : (const void *)selected_rows_kernel<float>;
    s = allow_smem(fn);
    if (s != DR_OK) return s;
    dim3 grid((p->cols + q.tune.tile_cols - 1) / q.tune.tile_cols, p->rows);
    if (bf16)
      selected_rows_kernel<__nv_bfloat16><<<grid, 512, smem, st>>>(tm, p->c, q.tune, idx, n,
                                                                    (__nv_bfloat16 *)out);
    else
      selected_rows_kernel<float><<<grid, 512, smem, st>>>(tm, p->c, q.tune, idx, n,
                                                            (float *)out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail("dr_reconstruct_selected", e);
    return DR_OK;
  }
  const int blocks = (n + kSelThreads - 1) / kSelThreads;
  if (p->geom_prec == DR_GEOM_FP64) {
    if (bf16)
      selected_kernel<GeoF64, __nv_bfloat16><<<blocks, kSelThreads, 0, st>>>(
          p->c, p->kernel, img, idx, n, (__nv_bfloat16 *)out);
    else
      selected_kernel<GeoF64, float><<<blocks, kSelThreads, 0, st>>>(p->c, p->kernel, img, idx,
                                                                     n, (float *)out);
  } else {
    if (bf16)
      selected_kernel<GeoFx, __nv_bfloat16><<<blocks, kSelThreads, 0, st>>>(
          p->c, p->kernel, img, idx, n, (__nv_bfloat16 *)out);
    else
      selected_kernel<GeoFx, float><<<blocks, kSelThreads, 0, st>>>(p->c, p->kernel, img, idx,
                                                                    n, (float *)out);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("dr_reconstruct_selected", e);
  return DR_OK;
}
