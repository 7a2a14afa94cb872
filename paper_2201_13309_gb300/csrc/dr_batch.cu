// Many scans in one persistent launch, replayed from a captured CUDA graph.
//
// A batch is built once from (plan, images, output) jobs: every job gets a
// descriptor (its plan's tables, a TMA tensor map of its images and a tile
// shape for 512-thread CTAs), the (scan, row, tile) work items of all jobs
// are numbered with the most expensive items first, and a device counter
// hands them out to a grid of one CTA per SM slot.  The counter reset and
// the launch are captured once into a CUDA graph; dr_batch_launch replays it.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "dr_batch.cuh"
#include "dr_internal.h"

struct dr_batch {
  int n = 0, out_dtype = 0;
  long long n_items = 0;
  int grid = 0, threads = 512, smem = 0;
  size_t device_bytes = 0;
  void *dev = nullptr;
  dr::BatchScan *d_scans = nullptr;
  unsigned long long *d_counter = nullptr;
  int32_t *d_err = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

using namespace dr;

namespace {

constexpr int kBatchThreads = 512;
// tiles per work item (consecutive rows, same columns): the work counter's
// round trip and the scan lookup are paid once per item
constexpr int kRowsPerItem = 4;

void destroy(dr_batch_t *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->dev) cudaFree(b->dev);
  delete b;
}

template <class OutT>
const void *batch_fn(int set) {
  return set == kSetPolyOnly ? (const void *)batch_kernel<OutT, kSetPolyOnly>
         : set == kSetAll    ? (const void *)batch_kernel<OutT, kSetAll>
                             : (const void *)batch_kernel<OutT, kSetRunningSum>;
}

}  // namespace

extern "C" dr_status dr_batch_create(const dr_job *jobs, int32_t n,
                                     const dr_batch_options *opt_in, dr_batch_t **out) {
  TraceRange trace_("dr_batch_create");
  if (out) *out = nullptr;
  if (!jobs || n < 1 || !out) {
    set_error("dr_batch_create: need at least one job");
    return DR_ERR_INVALID_ARG;
  }
  dr_batch_options opt;
  std::memset(&opt, 0, sizeof(opt));
  if (opt_in) opt = *opt_in;
  if (opt.ctas_per_sm < 0 || opt.ctas_per_sm > 3 || opt.max_tile_cols < 0 ||
      (opt.threads != 0 && opt.threads != 256 && opt.threads != 512)) {
    set_error("dr_batch_create: ctas_per_sm must be 0..3 and threads 0, 256 or 512");
    return DR_ERR_INVALID_ARG;
  }
  const int nthreads = opt.threads ? opt.threads : kBatchThreads;
  // shared memory each CTA may use so that ctas_per_sm CTAs share an SM
  const int want_per_sm = opt.ctas_per_sm == 0 ? 1 : opt.ctas_per_sm;
  const int smem_budget = std::min(kSmemPerCtaMax, kSmemPerSm / want_per_sm - 1024);
  std::vector<BatchScan> desc(n);
  std::vector<double> cost(n);
  int smem_max = 0, out_dtype = -1;
  bool poly_only = true, any_intervals = false;
  for (int i = 0; i < n; ++i) {
    const dr_plan_t *p = jobs[i].plan;
    if (!p) {
      set_error("dr_batch_create: job %d has no plan", i);
      return DR_ERR_INVALID_ARG;
    }
    const bool rows = p->kernel == DR_KERNEL_ROWS, iv = p->kernel == DR_KERNEL_INTERVALS;
    const char *why = !p->parts.empty() ? "a composite plan (monotone runs or both edges)"
                      : p->geom_prec != DR_GEOM_FP32  ? "FP64 geometry"
                      : p->cols % 8 != 0              ? "a width not a multiple of 8"
                      : (rows && p->tune.ppt != 4)    ? "one pixel per thread"
                                                      : nullptr;
    if (why) {
      set_error("dr_batch_create: job %d is %s; the batch runs single-run, single-edge plans "
                "with FP32 geometry on widths that are multiples of 8",
                i, why);
      return DR_ERR_UNSUPPORTED;
    }
    if (out_dtype >= 0 && p->out_dtype != out_dtype) {
      set_error("dr_batch_create: all jobs must share the output type");
      return DR_ERR_UNSUPPORTED;
    }
    out_dtype = p->out_dtype;
    const size_t P = (size_t)p->rows * p->cols;
    if (P > 0 && (!jobs[i].d_images || !jobs[i].d_out || ((uintptr_t)jobs[i].d_images & 15) ||
                  ((uintptr_t)jobs[i].d_out & 15))) {
      set_error("dr_batch_create: job %d: null or misaligned buffer", i);
      return DR_ERR_INVALID_ARG;
    }
    // tile shape for the batch's CTAs.  Rows tiles: the plan's width (capped
    // by the options), narrowed until the tile fits the per-CTA budget, four
    // pixels per thread.  Per-pixel tiles: one pixel per lane, the bins
    // shared among nthreads / tile_cols threads per pixel.
    Tuning t = p->tune;
    int smem = 0, lanes = 0, window = 0;
    if (iv) {
      // interval tiles keep the plan's 32 columns and step chunks; the bin
      // window shrinks to the per-CTA budget if it must
      lanes = kIntervalTile;
      const int fixed = intervals_smem(p->K, t.kc * t.nchunks, p->B, 0, false, p->pixel_groups);
      const int per_bin = kIntervalTile * 4;
      window = std::min(p->window, std::max(0, (smem_budget - fixed) / per_bin));
      if (window < std::min(p->B, 32)) window = p->window;  // reported below as not fitting
      smem = intervals_smem(p->K, t.kc * t.nchunks, p->B, window, false, p->pixel_groups);
    } else if (rows) {
      if (opt.max_tile_cols >= 32 && t.tile_cols > opt.max_tile_cols)
        t.tile_cols = opt.max_tile_cols / 32 * 32;
      for (;;) {
        choose_chunks(p->K, t.tile_cols, &t.kc, &t.nchunks);
        smem = rows_smem_bytes(p->K, t.kc * t.nchunks, p->B, t.tile_cols, false);
        if (smem <= smem_budget || t.tile_cols <= 32) break;
        t.tile_cols /= 2;
      }
      lanes = t.tile_cols / 4;
    } else {
      // the polynomial form's tile holds no depth table: 128 columns (4
      // threads per pixel at 512 threads, the standalone kernel's fastest
      // shape on the full detector) when they fit the budget and the cap,
      // else narrower
      const bool poly = p->c.depth_mode == kDepthPoly;
      t.tile_cols = poly ? (nthreads >= 512 ? 128 : 64) : 32;
      while (opt.max_tile_cols >= 8 && t.tile_cols > opt.max_tile_cols && t.tile_cols > 8)
        t.tile_cols /= 2;  // a power of two: whole 8-, 16- or 32-pixel slabs
      for (;;) {
        choose_chunks(p->K, t.tile_cols, &t.kc, &t.nchunks);
        smem = poly ? pixels_poly_smem_bytes(p->K, t.kc * t.nchunks, p->B, t.tile_cols)
                    : pixels_smem_bytes(p->K, t.kc * t.nchunks, p->B, t.tile_cols, false);
        if (smem <= smem_budget || t.tile_cols <= 8) break;
        t.tile_cols /= 2;
      }
      lanes = t.tile_cols;
    }
    if (smem > smem_budget || lanes > nthreads || t.kc < 1 ||
        ((size_t)t.kc * t.tile_cols * 2) % 128 != 0) {
      set_error("dr_batch_create: job %d (%d steps) does not fit in shared memory", i, p->K);
      return DR_ERR_UNSUPPORTED;
    }
    t.bin_groups = iv ? window : nthreads / lanes;
    smem_max = std::max(smem_max, smem);
    BatchScan &d = desc[i];
    std::memset(&d, 0, sizeof(d));
    d.img = jobs[i].d_images;
    d.out = jobs[i].d_out;
    d.c = p->c;
    d.t = t;
    d.tiles_per_row = (p->cols + t.tile_cols - 1) / t.tile_cols;
    d.rows_per_item = kRowsPerItem;
    d.pixel_groups = p->pixel_groups;
    d.window = window;
    if (iv)
      d.kind = kBatchIntervals;
    else if (rows)
      d.kind = kBatchRows;
    else if (p->c.depth_mode == kDepthPoly)
      d.kind = p->one_adv ? kBatchPixelsPolyOneAdv : kBatchPixelsPoly;
    else
      d.kind = p->one_adv ? kBatchPixelsOneAdv : kBatchPixels;
    poly_only &= d.kind == kBatchPixelsPolyOneAdv || d.kind == kBatchPixelsPoly;
    any_intervals |= iv;
    if (P > 0) {
      dr_plan_t tmp = *p;
      tmp.tune = t;
      dr_status s = make_tensor_map(&tmp, jobs[i].d_images, &d.tmap);
      if (s != DR_OK) return s;
    }
    // per-pixel tiles cost about twice a rows tile of the same size, interval
    // tiles about three times
    cost[i] = (double)t.tile_cols * p->B * (rows ? 1.0 : iv ? 3.0 : 2.0);
  }
  // most expensive items first (the counter hands items out in order)
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<BatchScan> sorted;
  long long items = 0;
  for (int i : order) {
    BatchScan d = desc[i];
    d.item_begin = items;
    items += (long long)((jobs[i].plan->rows + d.rows_per_item - 1) / d.rows_per_item) *
             d.tiles_per_row;
    if (d.c.H * (long long)d.c.W == 0) continue;  // empty ROI: no items
    sorted.push_back(d);
  }
  dr_batch_t *b = new (std::nothrow) dr_batch_t();
  if (!b) {
    set_error("dr_batch_create: host allocation failed");
    return DR_ERR_OOM;
  }
  b->n = n;
  b->threads = nthreads;
  b->n_items = items;
  b->out_dtype = out_dtype;
  b->smem = smem_max;
  const int set = any_intervals ? kSetAll : poly_only ? kSetPolyOnly : kSetRunningSum;
  const void *fn = out_dtype == DR_OUT_BF16 ? batch_fn<__nv_bfloat16>(set)
                                            : batch_fn<float>(set);
  dr_status s = allow_smem(fn);
  if (s != DR_OK) {
    destroy(b);
    return s;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nthreads, smem_max);
  if (e != cudaSuccess) {
    destroy(b);
    return cuda_fail("dr_batch_create: occupancy", e);
  }
  b->grid = std::max(1, sms * std::max(per_sm, 1));
  if ((long long)b->grid > items) b->grid = (int)std::max(items, 1LL);
  // device block: descriptors, work counter, error word
  const size_t o_desc = 0, n_desc = std::max<size_t>(sorted.size(), 1);
  const size_t o_cnt = (sizeof(BatchScan) * n_desc + 255) / 256 * 256;
  const size_t total = o_cnt + 256;
  e = cudaMalloc(&b->dev, total);
  if (e != cudaSuccess) {
    b->dev = nullptr;
    destroy(b);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      set_error("dr_batch_create: cudaMalloc failed");
      return DR_ERR_OOM;
    }
    return cuda_fail("dr_batch_create: cudaMalloc", e);
  }
  b->device_bytes = total;
  b->d_scans = reinterpret_cast<BatchScan *>((char *)b->dev + o_desc);
  b->d_counter = reinterpret_cast<unsigned long long *>((char *)b->dev + o_cnt);
  b->d_err = reinterpret_cast<int32_t *>((char *)b->dev + o_cnt + 64);
  for (auto &d : sorted) d.c.err = b->d_err;
  e = cudaMemset(b->dev, 0, total);
  if (e == cudaSuccess && !sorted.empty())
    e = cudaMemcpy(b->d_scans, sorted.data(), sizeof(BatchScan) * sorted.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    destroy(b);
    return cuda_fail("dr_batch_create: upload", e);
  }
  // capture: counter reset + persistent launch
  e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), b->cap);
    if (items > 0) {
      const int ns = (int)sorted.size();
      void *args[] = {&b->d_scans, const_cast<int *>(&ns), &items, &b->d_counter};
      e = cudaLaunchKernel(fn, dim3(b->grid), dim3(nthreads), args, smem_max, b->cap);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &b->graph);
    e = e2 != cudaSuccess ? e2 : cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    destroy(b);
    return cuda_fail("dr_batch_create: graph capture", e);
  }
  *out = b;
  return DR_OK;
}

extern "C" dr_status dr_batch_launch(dr_batch_t *b, dr_stream_t stream) {
  TraceRange trace_("dr_batch_launch");
  if (!b) {
    set_error("dr_batch_launch: null batch");
    return DR_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail("dr_batch_launch", e);
  return DR_OK;
}

extern "C" dr_status dr_batch_check(dr_batch_t *b) {
  if (!b) {
    set_error("dr_batch_check: null batch");
    return DR_ERR_INVALID_ARG;
  }
  int32_t v = 0, zero = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, b->d_err, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail("dr_batch_check", e);
  if (v != kDevOk) {
    cudaMemcpy(b->d_err, &zero, sizeof(zero), cudaMemcpyHostToDevice);
    set_error("a batch tile's bounded wait for its TMA tile ran out (code %d)", v);
    return DR_ERR_TIMEOUT;
  }
  return DR_OK;
}

extern "C" dr_status dr_batch_get_info(const dr_batch_t *b, dr_batch_info *info) {
  if (!b || !info) {
    set_error("dr_batch_get_info: null argument");
    return DR_ERR_INVALID_ARG;
  }
  std::memset(info, 0, sizeof(*info));
  info->scans = b->n;
  info->items = b->n_items;
  info->grid = b->grid;
  info->threads = b->threads;
  info->smem_bytes = b->smem;
  info->device_bytes = b->device_bytes;
  return DR_OK;
}

extern "C" void dr_batch_destroy(dr_batch_t *b) { destroy(b); }

extern "C" dr_status dr_batch_reconstruct(const dr_job *jobs, int32_t n,
                                          const dr_batch_options *options, dr_stream_t stream) {
  TraceRange trace_("dr_batch_reconstruct");
  dr_batch_t *b = nullptr;
  dr_status st = dr_batch_create(jobs, n, options, &b);
  if (st != DR_OK) return st;
  st = dr_batch_launch(b, stream);
  if (st == DR_OK) {
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    st = e == cudaSuccess ? dr_batch_check(b) : cuda_fail("dr_batch_reconstruct", e);
  }
  destroy(b);
  return st;
}
