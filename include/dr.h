/*
 * dr.h -- C ABI of the GB300 wire-scan depth reconstruction library (libdr).
 *
 * Method: differential-aperture depth reconstruction (the paper's Sec. III:
 * per pixel, the intensity difference between consecutive wire-step images is
 * assigned to depth and summed into a depth-resolved result; Sec. III-C
 * describes the per-pixel routine).  For every detector pixel and wire step k
 * the library computes the beam depth d_k at which the ray from that pixel
 * grazes the chosen wire edge (tangent to the wire circle in the plane
 * perpendicular to the wire axis, intersected with the incident beam), takes
 * the exact integer difference dI_k = I_k - I_{k+1}, and spreads dI_k over
 * the output depth bins in proportion to the overlap of [d_k, d_{k+1}] with
 * each bin.  Mass outside [e_0, e_B] is dropped.
 *
 * Units: lengths in millimetres, lab frame.  Depth is the signed distance
 * along beam_dir (normalised internally) from beam_origin.
 *
 * Layouts (row-major, no padding):
 *   images  [K][rows][cols]  uint16   (Sec. III-B: p images of m rows x n cols,
 *                                      stored as one flat array)
 *   output  [B][rows][cols]  float32 or bfloat16 (plan option)
 *
 * Ownership: a plan owns its device constants; the caller owns every image and
 * output buffer.  Device pointers must come from cudaMalloc (or torch) on the
 * current device.  No call throws; every call returns a dr_status, and
 * dr_last_error() gives a one-line explanation of the last failure on the
 * calling thread.  Kernels are launched asynchronously on the caller's stream.
 */
#ifndef DR_H_
#define DR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st *dr_stream_t;

typedef enum {
  DR_OK = 0,
  DR_ERR_INVALID_ARG = 1,   /* null pointer, bad size, unsorted bin edges */
  DR_ERR_GEOMETRY = 2,      /* beam along the wire, pixel inside the wire, wire
                               not between beam and detector, no travel */
  DR_ERR_NONMONOTONIC = 3,  /* depth sequence not strictly monotone where an
                               entry point needs it (the no-allocation rows
                               entry); dr_plan itself takes any order */
  DR_ERR_OOM = 4,           /* device or host allocation failed */
  DR_ERR_BUDGET = 5,        /* request does not fit the memory budget */
  DR_ERR_CUDA = 6,          /* a CUDA runtime call failed */
  DR_ERR_TIMEOUT = 7,       /* a kernel gave up waiting (bounded wait) */
  DR_ERR_UNSUPPORTED = 8    /* valid request outside what this build handles */
} dr_status;

enum { DR_EDGE_LEADING = 0, DR_EDGE_TRAILING = 1, DR_EDGE_BOTH = 2 };
enum { DR_OUT_F32 = 0, DR_OUT_BF16 = 1 };
enum { DR_GEOM_FP32 = 0, DR_GEOM_FP64 = 1 };
enum { DR_KERNEL_ROWS = 0, DR_KERNEL_PIXELS = 1, DR_KERNEL_INTERVALS = 2 };

/* Scan geometry.  Pixel (r, c) has its centre at
 * det_origin + r*row_step + c*col_step.  The wire is an infinite cylinder of
 * radius wire_radius whose axis runs along wire_axis through each wire centre.
 * edge selects the wire edge whose passage is reconstructed: the leading edge
 * (the one moving in the direction of travel; a pixel's intensity drops as it
 * covers a scatterer), the trailing edge (intensity comes back), or
 * DR_EDGE_BOTH, the mean of the two reconstructions.  The direction of travel
 * is that of the whole scan (first to last wire centre); a path that turns
 * back along the beam is reconstructed run by run with that same edge. */
typedef struct {
  double beam_origin[3];
  double beam_dir[3];
  double det_origin[3];
  double row_step[3];
  double col_step[3];
  int32_t rows;
  int32_t cols;
  double wire_axis[3];
  double wire_radius;
  int32_t edge;
} dr_geometry;

/* Optional plan settings; a null pointer means all zero (defaults). */
typedef struct {
  int32_t out_dtype;        /* DR_OUT_F32 (default) or DR_OUT_BF16 */
  int32_t geom_precision;   /* DR_GEOM_FP32 (default): per-step depth in FP32
                               on FP64 per-pixel constants, positions on a
                               grid of 2^-fixed_shift mm (a few units of
                               error, so an interval of L units may move
                               about 8/L of its difference across a bin edge:
                               below the 1e-4 bar for steps above ~60 nm at
                               the beamline scale); DR_GEOM_FP64: the whole
                               depth computation in FP64 on the GPU */
  int32_t tile_cols;        /* pixels per CTA along a row; 0 = tuned */
  int32_t bin_groups;       /* warps-groups splitting the bins; 0 = tuned */
  int32_t force_pixels;     /* 1: use the per-pixel kernel even when all
                               pixels of a row share their depths */
  int32_t force_intervals;  /* 1: use the interval kernel (depths in any
                               order) even when every sequence is monotone */
  int32_t depth_form;       /* FP32 geometry: 0 = the plan's choice; else the
                               cheapest form the plan may use for the depth
                               remainder, plus one: 1 exact, 2 up to the
                               series of dL, 3 up to the per-pixel cubic */
  int32_t reserved;
} dr_plan_options;

typedef struct dr_plan dr_plan_t;

/* What a plan decided (for reports and tests). */
typedef struct {
  int32_t rows, cols, K, B;
  int32_t kernel;           /* DR_KERNEL_ROWS, DR_KERNEL_PIXELS or
                               DR_KERNEL_INTERVALS */
  int32_t tile_cols, pixels_per_thread;
  int32_t bin_groups;       /* thread groups splitting the bins; for the
                               interval kernel, bins per shared-memory window */
  int32_t threads;
  int32_t smem_bytes, tma_chunk, tma_chunks;
  int32_t out_dtype, geom_precision, edge, reversed;
  int32_t fixed_shift;      /* depth positions in units of 2^-fixed_shift mm
                               of projected depth (FP32 geometry) */
  int32_t row_tables;       /* 1: the per-row (k, f) tables were built once at
                               plan time; 0: each tile builds its own */
  int32_t parts;            /* launches per reconstruction: monotone runs of
                               the wire path (each cut into runs of at most
                               2048 steps) x wire edges (1 for most scans) */
  double depth_min, depth_max;   /* range of all d_k (mm) */
  double min_step;               /* smallest |d_{k+1} - d_k| (mm) */
  size_t device_bytes;           /* device memory held by the plan */
  double bytes_per_call;         /* algorithmic HBM bytes of one
                                    dr_reconstruct: 2*P*K + out*P*B */
  /* FP32 geometry of the rows and per-pixel kernels: the plan computes every
   * (row or pixel, step) depth exactly as the kernels will, checks that each
   * sequence increases by steps the fixed-point grid takes, and compares
   * each depth with the FP64 solution of the same geometry. */
  double max_step;               /* largest |d_{k+1} - d_k| (mm) */
  double depth_err;              /* largest distance of a kernel depth from
                                    the FP64 solution (mm); -1: not checked */
  int32_t depth_form;            /* form of the FP32 remainder: 0 exact (a
                                    square root and a reciprocal), 1 series
                                    of dL, 2 per-pixel cubic in the wire
                                    position (multiply-adds only) */
  int32_t one_step_per_bin;      /* 1: every step at least as long as every
                                    bin, so a bin holds at most one step */
  int64_t checked_groups;        /* rows or pixels checked at every step */
} dr_plan_info;

/* Build a plan: validate the geometry, compute the per-pixel (or per-row,
 * when all pixels of a row share their depths) constants in FP64, upload them
 * and pick the kernel and tile shape.  The apportioning of Sec. III spreads
 * each difference over the interval between two consecutive depths.  When
 * every depth sequence is strictly monotone within each run of the wire path
 * (the path may turn back along the beam) the plan uses the running-sum
 * kernels (rows or per-pixel); otherwise (a wire that also moves across the
 * beam, two centres at the same position along the beam) it uses the
 * interval kernel, which adds each interval by itself in any order; a
 * zero-length interval puts its difference in the bin that holds it.  The
 * interval kernel also takes scans that the running-sum kernels cannot
 * (depth steps too fine for their fixed-point grid, tiles too large for
 * shared memory), unless options give tile_cols or bin_groups: a launch
 * shape that does not fit is then reported (DR_ERR_UNSUPPORTED).  With FP32
 * geometry the interval kernel apportions each interval shorter than its
 * positions' grid resolves (next to a turning point of the depths, a
 * repeated wire position) with that interval's depths in FP64.  The wire
 * must travel along the beam between its first and last centre
 * (DR_ERR_GEOMETRY otherwise).
 *   wire_centres  host [K][3] FP64, K >= 2
 *   bin_edges     host [B+1] FP64 strictly increasing (depth, mm), B >= 1
 * rows or cols may be 0 (an empty ROI: dr_reconstruct then does nothing).
 * Allocates device memory on the current device; *out is null on failure. */
dr_status dr_plan(const dr_geometry *geometry, const double *wire_centres,
                  int32_t K, const double *bin_edges, int32_t B,
                  const dr_plan_options *options, dr_plan_t **out);

/* Free a plan (null is ignored).  The caller must make sure no kernel that
 * uses the plan is still running. */
void dr_plan_destroy(dr_plan_t *plan);

dr_status dr_plan_get_info(const dr_plan_t *plan, dr_plan_info *info);
size_t dr_plan_device_bytes(const dr_plan_t *plan);

/* Reconstruct one scan (the per-pixel routine of Sec. III-C, for every pixel
 * of the ROI: exact differences between consecutive wire-step images, each
 * spread over the depth bins its wire-edge interval overlaps, Sec. III-A):
 * d_images [K][rows][cols] uint16 in device memory,
 * d_out [B][rows][cols] (float or bf16 per the plan) in device memory.  Every
 * output element is written exactly once (no prior clearing needed).  Allocates
 * nothing; asynchronous on stream.  A plan may be used from several streams at
 * once.  Input rows whose byte pitch is a multiple of 16 and a 16-byte aligned
 * d_images are staged by TMA; other inputs take a plain-load path. */
dr_status dr_reconstruct(const dr_plan_t *plan, const uint16_t *d_images,
                         void *d_out, dr_stream_t stream);

/* End-to-end form with host buffers: copies h_images (pinned host memory for
 * full speed) into the caller's device buffer d_images_ws, reconstructs into
 * d_out_ws, and copies the result into h_out, all in order on stream.  The
 * call returns once everything is queued; synchronize the stream before
 * reading h_out.  Sizes are those of dr_reconstruct. */
dr_status dr_reconstruct_host(const dr_plan_t *plan, const uint16_t *h_images,
                              void *h_out, uint16_t *d_images_ws,
                              void *d_out_ws, dr_stream_t stream);

/* Streamed (out-of-core) form, the row-slab chunking of the paper's Sec. III-B
 * with the transfer overlap its Sec. II motivates: the scan moves through a
 * device workspace of ws_bytes (256-byte aligned) in slabs of slab_rows rows
 * (0 = as large as three slab buffers allow).  For each slab: one 2-D
 * host->device copy of its rows of every image, the reconstruction kernel,
 * and one 2-D device->host copy of its rows of every bin; three internal
 * streams overlap uploads, kernels and downloads across slabs.  When h_out is
 * pinned (page-locked and mapped) and the images are staged by TMA, the
 * kernels store the bins straight into h_out instead (no download stage;
 * plans of several runs or both edges keep the download).  h_images
 * [K][rows][cols] and h_out [B][rows][cols] are host memory (pinned for full
 * speed).  Ordered after prior work on stream; later work on stream waits
 * for the last download.  Calls are serialised by the library (one internal
 * stream set per device).  DR_ERR_BUDGET if three slabs do not fit. */
dr_status dr_reconstruct_streamed(const dr_plan_t *plan, const uint16_t *h_images,
                                  void *h_out, void *d_workspace, size_t workspace_bytes,
                                  int32_t slab_rows, dr_stream_t stream);

/* ---- Pixel selection (the paper's pixel-percentage experiment, Sec. IV-A) --
 * Only some pixels carry signal (diffraction spots); these calls reconstruct
 * only the selected ones into a compacted output.
 * dr_pixel_activity: d_activity[p] = sum_k |I_k(p) - I_{k+1}(p)| for the
 *   [K][rows][cols] stack, p row-major; summed exactly in 32-bit integers
 *   (K <= 32768) and stored as float, i.e. exact up to 2^24 and rounded to
 *   nearest above (possible only for K > 257).
 * dr_select_pixels: the indices p (0..n-1) with d_activity[p] >= threshold,
 *   in increasing order, into d_index (room for n entries); the number of them
 *   into the device int32 *d_count.  Needs dr_select_scratch_bytes(n) bytes of
 *   device scratch (caller-owned).
 * dr_reconstruct_selected: bins of the listed pixels only, compacted:
 *   d_out[j * n + i] is bin j of pixel d_index[i] (FP32 or BF16 per the plan),
 *   bitwise equal to dr_reconstruct's value for that pixel.  n is the host
 *   count of listed pixels; d_index holds n row-major pixel numbers in
 *   increasing order, each in [0, rows * cols) (as dr_select_pixels writes
 *   them).  A list with numbers outside the ROI or out of order makes the
 *   kernels read nothing outside the images, but the output columns of
 *   those numbers are undefined; where such a number reaches a kernel's
 *   walk, the plan's error word records it (dr_plan_check: DR_ERR_CUDA). */
dr_status dr_pixel_activity(const uint16_t *d_images, int32_t K, int32_t rows, int32_t cols,
                            float *d_activity, dr_stream_t stream);
size_t dr_select_scratch_bytes(int64_t n);
dr_status dr_select_pixels(const float *d_activity, int64_t n, float threshold,
                           int32_t *d_index, int32_t *d_count, void *d_scratch,
                           size_t scratch_bytes, dr_stream_t stream);
dr_status dr_reconstruct_selected(const dr_plan_t *plan, const uint16_t *d_images,
                                  const int32_t *d_index, int32_t n, void *d_out,
                                  dr_stream_t stream);

/* The exact integer differences the kernels use (Sec. III-C: each pixel's
 * change of intensity between steps): d_diff[k][p] = images[k][p] - images[k+1][p] as
 * int32, k = 0..K-2, for a [K][rows][cols] uint16 device stack. */
dr_status dr_image_differences(const uint16_t *d_images, int32_t K,
                               int32_t rows, int32_t cols, int32_t *d_diff,
                               dr_stream_t stream);

/* The depths d_k (mm) the plan's kernels use, for rows r0 .. r0+nrows-1:
 * d_depths [nrows][cols][K] FP64 in device memory.  Computed on the GPU by the
 * same device code as dr_reconstruct (for checks against the oracle). */
dr_status dr_plan_depths(const dr_plan_t *plan, int32_t r0, int32_t nrows,
                         double *d_depths, dr_stream_t stream);

/* Read and clear the plan's device error word (set by a kernel whose bounded
 * wait ran out).  Synchronizes the device.  DR_OK or DR_ERR_TIMEOUT; in the
 * bounds-checked test build of the library (compiled with DR_CHECK_BOUNDS)
 * also DR_ERR_CUDA when a kernel index was out of range (dr_last_error names
 * the device-source line). */
dr_status dr_plan_check(const dr_plan_t *plan);

/* Failure-path diagnostic (no counterpart in the paper): launches one CTA on
 * stream whose barrier is never completed, so its bounded wait (the form the
 * reconstruction kernels use for their tile copies) runs out after wait_ms
 * milliseconds (0 < wait_ms <= 2000); it records the timeout code in the
 * caller's device word *d_status and returns, leaving the device usable.
 * Synchronizes the stream; returns DR_ERR_TIMEOUT when the timeout was
 * recorded (the expected outcome), DR_OK if the wait completed. */
dr_status dr_selftest_wait_timeout(int32_t *d_status, double wait_ms, dr_stream_t stream);

/* ---- Many scans in one persistent launch ---------------------------------
 * A batch reconstructs several scans (each with its own plan, image stack and
 * output; different ROI sizes, step and bin counts) in ONE launch of a
 * persistent kernel: every CTA takes work items (a tile column of four rows
 * of one scan) from a device counter until none are left, biggest items
 * first, so uneven scans do not leave the GPU idle between per-scan
 * launches.  The counter reset and the launch are captured into a CUDA graph
 * at creation; dr_batch_launch replays it.  Jobs must use single-run,
 * single-edge plans (rows, per-pixel or interval kernel) with FP32
 * geometry, widths that are multiples of 8, 16-byte aligned buffers and one
 * output type (DR_ERR_UNSUPPORTED, naming the job and the reason,
 * otherwise).  The buffers are bound at creation: a batch always
 * reads and writes the same device buffers (refill the image buffers between
 * launches).  The result of every scan is bitwise identical to
 * dr_reconstruct's. */
typedef struct {
  const dr_plan_t *plan;
  const uint16_t *d_images;   /* [K][rows][cols] of the plan, device */
  void *d_out;                /* [B][rows][cols] of the plan, device */
} dr_job;

typedef struct dr_batch dr_batch_t;

/* Optional batch settings; null means all zero (defaults). */
typedef struct {
  int32_t ctas_per_sm;        /* 1 (default, up to 227 KB of shared memory per
                                 CTA), 2 (up to 113 KB each: narrower tiles,
                                 two CTAs overlapping on each SM) or 3 (up to
                                 75 KB each; reached with 512-thread CTAs when
                                 every job is a per-pixel plan of the
                                 polynomial form) */
  int32_t max_tile_cols;      /* cap on each job's tile width (rows tiles:
                                 multiples of 32; per-pixel tiles: powers
                                 of two from 8); 0 = the default width */
  int32_t threads;            /* threads per CTA: 256 or 512 (0 = 512) */
  int32_t reserved;
} dr_batch_options;

typedef struct {
  int32_t scans;
  int64_t items;              /* (scan, row, tile) work items */
  int32_t grid, threads, smem_bytes;
  size_t device_bytes;
} dr_batch_info;

/* Build descriptors, upload them and capture the launch graph (allocates a
 * few KB of device memory; synchronous).  Each job keeps its plan's tile
 * width, narrowed until it fits the per-CTA shared-memory budget of
 * options->ctas_per_sm.  The plans must outlive the batch. */
dr_status dr_batch_create(const dr_job *jobs, int32_t n, const dr_batch_options *options,
                          dr_batch_t **out);
/* Replay the captured launch on stream (asynchronous). */
dr_status dr_batch_launch(dr_batch_t *batch, dr_stream_t stream);
/* Synchronize, read and clear the batch's device error word. */
dr_status dr_batch_check(dr_batch_t *batch);
dr_status dr_batch_get_info(const dr_batch_t *batch, dr_batch_info *info);
void dr_batch_destroy(dr_batch_t *batch);

/* One-shot form: dr_batch_create, dr_batch_launch on stream, wait for the
 * stream, dr_batch_check, dr_batch_destroy.  For a set of scans reconstructed
 * once; a set replayed many times should keep its batch (graph capture and
 * tables are built at creation).  Synchronizes the stream and the device. */
dr_status dr_batch_reconstruct(const dr_job *jobs, int32_t n, const dr_batch_options *options,
                               dr_stream_t stream);

/* ---- Serving: a stream of requests ----------------------------------------
 * A server takes reconstruction requests of any ROI, step and bin count as
 * they arrive and runs them concurrently on one GPU (the paper's Sec. II names
 * host<->device transfers as the cost to hide by overlapping them with
 * computation; here each request's pinned-host upload overlaps other
 * requests' kernels).  At creation the server reserves budget_bytes of device
 * memory (one cudaMalloc) and starts a scheduler thread and planner threads.
 * Plans are cached by geometry, wire path and bins; a submitted request whose
 * plan is not cached has it built by a planner thread while earlier requests
 * upload and run.  Requests are admitted in arrival order as soon as their
 * plan is ready, a slot (a stream) is free and their image and output blocks
 * fit in the reserved memory; a request larger than the whole budget fails
 * with DR_ERR_BUDGET.  A request's image block is returned when its kernel finishes;
 * its output stays on the device until dr_server_release.  Results are
 * bitwise identical to dr_reconstruct's, alone or in any mix. */
typedef struct dr_server dr_server_t;

typedef struct {
  size_t budget_bytes;        /* device memory for images + outputs */
  int32_t slots;              /* requests on the GPU at once (streams); 0 = 4 */
  int32_t plan_cache;         /* plans kept; 0 = 64 */
  int32_t reserved[2];
} dr_server_options;

enum { DR_REQ_QUEUED = 0, DR_REQ_UPLOADING = 1, DR_REQ_RUNNING = 2, DR_REQ_DONE = 3,
       DR_REQ_FAILED = 4 };

/* Seconds since the server was created (host steady clock): submitted,
 * planned (the request's plan was ready: found in the cache at submission,
 * or built by a planner thread while the request waited), admitted (plan
 * ready, slot and memory reserved), uploaded (the upload, which waits behind
 * earlier uploads, is done, as its host callback saw it), done (kernel done,
 * as its host callback saw it); issued (the upload was queued on the upload
 * stream) and copy (the device's duration of the upload copy itself, from
 * CUDA events; -1 if unknown). */
typedef struct {
  double submitted, admitted, planned, uploaded, done, issued, copy;
} dr_request_times;

typedef struct {
  int64_t queued, in_flight, admitted, completed, failed, plans_built, plans_cached;
  size_t arena_bytes, arena_used;
} dr_server_stats;

dr_status dr_server_create(const dr_server_options *options, dr_server_t **out);
/* Queue one scan.  h_images [K][rows][cols] uint16 host memory (pinned for
 * overlap) must stay valid and unchanged until the request is done.  The
 * geometry, wire path and bins are copied. */
dr_status dr_server_submit(dr_server_t *server, const dr_geometry *geometry,
                           const double *wire_centres, int32_t K, const double *bin_edges,
                           int32_t B, const uint16_t *h_images, uint64_t *id);
/* Current state (DR_REQ_*) of a request. */
dr_status dr_server_poll(dr_server_t *server, uint64_t id, int32_t *state);
/* Block until the request is done or failed (DR_ERR_TIMEOUT after timeout_s). */
dr_status dr_server_wait(dr_server_t *server, uint64_t id, double timeout_s);
/* The device address of a done request's [B][rows][cols] FP32 output (valid
 * until released) and its timestamps. */
dr_status dr_server_fetch(dr_server_t *server, uint64_t id, const void **d_out,
                          dr_request_times *times);
/* Copy a done request's output into dst (device or host memory) on stream. */
dr_status dr_server_fetch_into(dr_server_t *server, uint64_t id, void *dst,
                               size_t dst_bytes, dr_stream_t stream);
/* Give a done (or failed) request's output memory back and forget it. */
dr_status dr_server_release(dr_server_t *server, uint64_t id);
dr_status dr_server_get_stats(dr_server_t *server, dr_server_stats *stats);
/* Stop the scheduler, wait for work in flight and free everything. */
void dr_server_destroy(dr_server_t *server);

/* ---- Reconstruction that allocates nothing -------------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot call cudaMalloc themselves and so cannot build a plan (dr_plan keeps
 * its tables in device memory it allocates): for example a program whose
 * device memory is all handed out by another allocator (a framework's caching
 * pool that reserves the GPU), or an acquisition pipeline that forbids device
 * allocation once running because cudaMalloc/cudaFree may block or
 * synchronize the device.
 *
 * It runs the same rows kernel as dr_reconstruct for detectors whose columns
 * run along the wire axis, FP32 geometry and FP32 output.  Its geometry
 * tables (per-row constants, per-step constants, fixed-point bin edges and an
 * error word) live in one file-scope device array of 2 MiB
 * (DR_STATIC_SCRATCH_BYTES) inside the library; every GPU that loads the
 * library holds that array until the process exits.  The tables of a call
 * need 32*rows + 16*K + 4*(B+1) bytes plus alignment (at most 2 MiB, and
 * K <= 16384); larger requests return DR_ERR_BUDGET, detectors whose columns
 * do not run along the wire axis DR_ERR_UNSUPPORTED.  Arguments are those of
 * dr_plan + dr_reconstruct; d_status is an optional device int32 that is
 * cleared and then receives a device-side error code (nonzero: a bounded wait
 * ran out).  With d_status null no error is reported: the code goes to a
 * word in the library's array that nothing reads and the next call clears,
 * so pass a status word wherever a timeout must be seen.  The library cannot
 * see buffer sizes: d_images and d_out must hold the full [K][rows][cols] and
 * [B][rows][cols] arrays (the Python binding checks this).
 *
 * The call cannot be captured into a CUDA graph: while stream is capturing
 * it returns DR_ERR_UNSUPPORTED and queues nothing (a captured copy would
 * keep reading the host buffer below, which later calls overwrite).  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Each call writes its tables into a host
 * buffer inside the library and copies them into the array with an
 * asynchronous copy from that (pageable) buffer on stream: the copy first
 * waits for the work already queued on stream, and the call returns once
 * the bytes are staged, so the host buffer is reused by the next call.  A
 * lock serialises the calls' host side.  Every call shares the array and
 * leaves its own tables there: calls on one stream are ordered, but calls
 * whose work overlaps on the GPU (other streams, other threads) race on the
 * array and must not be issued. */
#define DR_STATIC_SCRATCH_BYTES (2u << 20)
dr_status dr_reconstruct_rows_static(const dr_geometry *geometry,
                                     const double *wire_centres, int32_t K,
                                     const double *bin_edges, int32_t B,
                                     const uint16_t *d_images, float *d_out,
                                     int32_t *d_status, dr_stream_t stream);

const char *dr_status_string(dr_status status);
/* One line describing the last failure on the calling thread ("" if none). */
const char *dr_last_error(void);
/* Library version, e.g. "1.0.0". */
const char *dr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DR_H_ */
