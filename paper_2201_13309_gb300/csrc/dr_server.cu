// Reconstruction server: continuous admission of scans of any ROI, step and
// bin count against an HBM budget, pinned host->device uploads overlapped with
// other requests' kernels on per-slot streams, results kept on the device
// until fetched.  (The paper's related work, Sec. II, names host-device
// transfers over PCI Express as the bottleneck to hide by overlapping them
// with computation; this runtime does that for a stream of requests.)
//
// Planner threads build the plans of submitted requests while earlier
// requests upload and run (plans are cached by their geometry, wire path and
// bins; a queued request holds its plan).  One scheduler thread owns
// admission: in arrival order, a request is admitted when its plan is ready,
// a slot is free and its image and output blocks fit in the arena (one
// cudaMalloc of the budget made at creation, sub-allocated first-fit).  Per
// request, on the slot's stream: upload, host callback (upload time),
// dr_reconstruct, host callback (done time).  The image block returns to the
// arena as soon as the kernel is done; the output block when the client
// releases the request.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dr_internal.h"

using namespace dr;

namespace {

constexpr int kPlanners = 3;  // planner threads per server

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit sub-allocator over [0, size) with coalescing free list.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
    used_ = 0;
  }
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        used_ += bytes;
        return off;
      }
    }
    return kNone;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    if (bytes == 0) bytes = 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }
  static constexpr size_t kNone = ~size_t(0);

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0;
};

enum { kPlanBuilding = 0, kPlanReady = 1, kPlanFailed = 2 };

struct PlanEntry {
  dr_plan_t *plan = nullptr;
  int refs = 0;                // requests holding it (queued to released)
  int state = kPlanBuilding;
  dr_status status = DR_OK;    // of a failed build
  double ready = 0;            // seconds since server creation
  bool in_lru = false;
  std::list<std::string>::iterator lru;
};

struct Request {
  uint64_t id = 0;
  int state = DR_REQ_QUEUED;
  dr_status status = DR_OK;
  dr_geometry g{};
  std::vector<double> wires, edges;
  int K = 0, B = 0;
  const uint16_t *h_images = nullptr;
  std::string key;
  PlanEntry *pe = nullptr;
  size_t img_off = Arena::kNone, out_off = Arena::kNone, img_bytes = 0, out_bytes = 0;
  int slot = -1;
  bool done_seen = false;      // completion handled by the scheduler
  dr_server_t *srv = nullptr;
  dr_request_times t{};
};

}  // namespace

struct dr_server {
  dr_server_options opt{};
  unsigned char *base = nullptr;
  Arena arena;
  std::vector<cudaStream_t> streams;   // one compute stream per slot
  std::vector<cudaEvent_t> up_start;   // per slot: before its request's upload (timing)
  std::vector<cudaEvent_t> up_done;    // per slot: its request's upload is done (timing)
  cudaStream_t up = nullptr;           // uploads, one at a time in admission order
  std::vector<int> slot_busy;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request *> queue;
  std::vector<Request *> finished;     // kernels done, blocks not yet returned
  std::unordered_map<uint64_t, Request *> reqs;
  std::unordered_map<std::string, PlanEntry> plans;
  std::list<std::string> lru;          // ready or failed plans, oldest use first
  std::deque<Request *> plan_jobs;     // first request of each plan to build
  std::condition_variable cv_plan;
  std::vector<std::thread> planners;
  std::thread sched;
  bool stop = false;
  uint64_t next_id = 1;
  int device = 0;
  uint64_t admitted = 0, completed = 0, rejected = 0, plan_builds = 0;
  double t0 = 0;
};

namespace {

std::string plan_key(const Request &r) {
  // field by field: the struct's padding bytes are not part of the key
  std::string k;
  auto put = [&](const void *p, size_t n) { k.append(reinterpret_cast<const char *>(p), n); };
  put(r.g.beam_origin, sizeof(r.g.beam_origin));
  put(r.g.beam_dir, sizeof(r.g.beam_dir));
  put(r.g.det_origin, sizeof(r.g.det_origin));
  put(r.g.row_step, sizeof(r.g.row_step));
  put(r.g.col_step, sizeof(r.g.col_step));
  put(&r.g.rows, sizeof(r.g.rows));
  put(&r.g.cols, sizeof(r.g.cols));
  put(r.g.wire_axis, sizeof(r.g.wire_axis));
  put(&r.g.wire_radius, sizeof(r.g.wire_radius));
  put(&r.g.edge, sizeof(r.g.edge));
  k.append(reinterpret_cast<const char *>(&r.K), sizeof(r.K));
  k.append(reinterpret_cast<const char *>(&r.B), sizeof(r.B));
  k.append(reinterpret_cast<const char *>(r.wires.data()), r.wires.size() * sizeof(double));
  k.append(reinterpret_cast<const char *>(r.edges.data()), r.edges.size() * sizeof(double));
  return k;
}

// Host callbacks (CUDA's callback thread: no CUDA calls in here).
// The upload's callback can run after the kernel's (both only note times):
// uploaded is then the done time.
void CUDART_CB on_uploaded(void *arg) {
  Request *r = static_cast<Request *>(arg);
  std::lock_guard<std::mutex> lk(r->srv->mu);
  if (r->state == DR_REQ_UPLOADING) {
    r->t.uploaded = now_s() - r->srv->t0;
    r->state = DR_REQ_RUNNING;
  }
}

void CUDART_CB on_done(void *arg) {
  Request *r = static_cast<Request *>(arg);
  dr_server_t *s = r->srv;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->t.done = now_s() - s->t0;
    if (r->state == DR_REQ_UPLOADING) r->t.uploaded = r->t.done;
    r->state = DR_REQ_DONE;
    s->finished.push_back(r);
    s->completed++;
  }
  s->cv_sched.notify_all();
  s->cv_done.notify_all();
}

// Plans that no request holds, beyond the cache size, least recently used
// first: taken out of the cache under the lock, destroyed by the caller after
// unlocking (no CUDA call under the lock).
void evict_plans(dr_server_t *s, std::vector<dr_plan_t *> *dead) {
  while ((int)s->plans.size() > std::max(1, s->opt.plan_cache)) {
    bool evicted = false;
    for (auto l = s->lru.begin(); l != s->lru.end(); ++l) {
      auto pe = s->plans.find(*l);
      if (pe != s->plans.end() && pe->second.refs == 0) {
        if (pe->second.plan) dead->push_back(pe->second.plan);
        s->plans.erase(pe);
        s->lru.erase(l);
        evicted = true;
        break;
      }
    }
    if (!evicted) break;
  }
}

// A planner thread: builds the plan of the first request of each new key
// (the request outlives the build: it cannot finish before its plan is
// ready), without the lock while dr_plan runs.
void planner(dr_server_t *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    while (!s->stop && s->plan_jobs.empty()) s->cv_plan.wait(lk);
    if (s->stop) return;
    Request *r = s->plan_jobs.front();
    s->plan_jobs.pop_front();
    PlanEntry *pe = r->pe;
    const dr_geometry g = r->g;
    const std::vector<double> wires = r->wires, edges = r->edges;
    const int K = r->K, B = r->B;
    const std::string key = r->key;
    lk.unlock();
    dr_plan_t *p = nullptr;
    dr_status st;
    {
      TraceRange trace_("server: plan of one request");
      st = dr_plan(&g, wires.data(), K, edges.data(), B, nullptr, &p);
    }
    lk.lock();
    pe->plan = p;
    pe->state = st == DR_OK ? kPlanReady : kPlanFailed;
    pe->status = st;
    pe->ready = now_s() - s->t0;
    if (st == DR_OK) s->plan_builds++;
    s->lru.push_back(key);
    pe->lru = std::prev(s->lru.end());
    pe->in_lru = true;
    s->cv_sched.notify_all();
  }
}

void fail(dr_server_t *s, Request *r, dr_status st) {
  r->status = st;
  r->state = DR_REQ_FAILED;
  r->t.done = now_s() - s->t0;
  s->rejected++;
  s->cv_done.notify_all();
}

// The scheduler never holds the mutex while it calls CUDA: the host
// callbacks of requests in flight take the same mutex, and several CUDA calls
// (allocation, synchronous copies, freeing) can wait for those callbacks.
void scheduler(dr_server_t *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    // kernels that finished: the device time of their uploads (the slot's
    // events, read without the lock), then their image blocks and slots go back
    if (!s->finished.empty()) {
      std::vector<Request *> fin;
      fin.swap(s->finished);
      lk.unlock();
      std::vector<float> copy_ms(fin.size(), -1.f);
      for (size_t i = 0; i < fin.size(); ++i)
        if (cudaEventElapsedTime(&copy_ms[i], s->up_start[fin[i]->slot],
                                 s->up_done[fin[i]->slot]) != cudaSuccess) {
          cudaGetLastError();
          copy_ms[i] = -1.f;
        }
      lk.lock();
      for (size_t i = 0; i < fin.size(); ++i) {
        Request *r = fin[i];
        r->t.copy = copy_ms[i] >= 0.f ? copy_ms[i] * 1e-3 : -1.0;
        s->arena.release(r->img_off, r->img_bytes);
        r->img_off = Arena::kNone;
        s->slot_busy[r->slot] = 0;
        r->done_seen = true;
      }
      progress = true;
    }
    if (progress) s->cv_done.notify_all();
    // choose admissions in arrival order while the head's plan is ready and
    // a slot and memory are free
    std::vector<Request *> admit;
    while (!s->queue.empty()) {
      Request *r = s->queue.front();
      if (r->pe->state == kPlanBuilding) break;
      if (r->pe->state == kPlanFailed) {
        s->queue.pop_front();
        const dr_status st = r->pe->status;
        r->pe->refs--;
        r->pe = nullptr;
        fail(s, r, st);
        progress = true;
        continue;
      }
      int slot = -1;
      for (int i = 0; i < (int)s->slot_busy.size(); ++i)
        if (!s->slot_busy[i]) {
          slot = i;
          break;
        }
      if (slot < 0) break;
      if (r->img_bytes + r->out_bytes + 512 > s->arena.size()) {
        s->queue.pop_front();
        fail(s, r, DR_ERR_BUDGET);
        progress = true;
        continue;
      }
      const size_t io = s->arena.alloc(r->img_bytes);
      if (io == Arena::kNone) break;
      const size_t oo = s->arena.alloc(r->out_bytes);
      if (oo == Arena::kNone) {
        s->arena.release(io, r->img_bytes);
        break;
      }
      s->queue.pop_front();
      r->img_off = io;
      r->out_off = oo;
      r->slot = slot;
      s->slot_busy[slot] = 1;
      r->state = DR_REQ_UPLOADING;
      r->t.admitted = now_s() - s->t0;
      r->t.planned = std::max(r->t.submitted, r->pe->ready);
      s->admitted++;
      if (r->pe->in_lru) s->lru.splice(s->lru.end(), s->lru, r->pe->lru);
      admit.push_back(r);
    }
    std::vector<dr_plan_t *> dead;
    evict_plans(s, &dead);
    if (admit.empty() && dead.empty()) {
      if (!progress) s->cv_sched.wait(lk);
      continue;
    }
    lk.unlock();  // ---- CUDA calls below, without the lock ----
    std::vector<std::pair<Request *, dr_status>> failed;
    for (Request *r : admit) {
      TraceRange trace_("server: upload and launch of one request");
      dr_status st = DR_OK;
      cudaStream_t cs = s->streams[r->slot];
      uint16_t *d_img = reinterpret_cast<uint16_t *>(s->base + r->img_off);
      void *d_out = s->base + r->out_off;
      if (st == DR_OK) {
        // uploads share the host link: one at a time, in admission order, so
        // each finishes as early as possible; the slot's kernel waits for the
        // copy itself (its event), not for the host callback that notes the
        // time, so a late callback does not hold the kernel back
        cudaError_t e = cudaEventRecord(s->up_start[r->slot], s->up);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(d_img, r->h_images, r->img_bytes, cudaMemcpyHostToDevice, s->up);
        if (e == cudaSuccess) {
          std::lock_guard<std::mutex> g(s->mu);
          r->t.issued = now_s() - s->t0;
        }
        if (e == cudaSuccess) e = cudaEventRecord(s->up_done[r->slot], s->up);
        if (e == cudaSuccess) e = cudaLaunchHostFunc(s->up, on_uploaded, r);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, s->up_done[r->slot], 0);
        st = e == cudaSuccess ? dr_reconstruct(r->pe->plan, d_img, d_out, (dr_stream_t)cs)
                              : cuda_fail("server upload", e);
        if (st == DR_OK) {
          e = cudaLaunchHostFunc(cs, on_done, r);
          if (e != cudaSuccess) st = cuda_fail("server completion callback", e);
        }
        if (st != DR_OK) {  // let the slot (and its upload) drain before reuse
          cudaStreamSynchronize(s->up);
          cudaStreamSynchronize(cs);
        }
      }
      if (st != DR_OK) failed.emplace_back(r, st);
    }
    for (dr_plan_t *p : dead) dr_plan_destroy(p);
    lk.lock();
    for (auto &f : failed) {
      Request *r = f.first;
      s->arena.release(r->img_off, r->img_bytes);
      s->arena.release(r->out_off, r->out_bytes);
      r->img_off = r->out_off = Arena::kNone;
      if (r->pe) r->pe->refs--;
      r->pe = nullptr;
      s->slot_busy[r->slot] = 0;
      fail(s, r, f.second);
    }
  }
}

Request *find(dr_server_t *s, uint64_t id) {
  auto it = s->reqs.find(id);
  return it == s->reqs.end() ? nullptr : it->second;
}

}  // namespace

extern "C" dr_status dr_server_create(const dr_server_options *o, dr_server_t **out) {
  TraceRange trace_("dr_server_create");
  if (out) *out = nullptr;
  if (!o || !out || o->budget_bytes < (size_t(1) << 20) || o->slots < 0 || o->slots > 64) {
    set_error("dr_server_create: need options with budget_bytes >= 1 MiB and 0..64 slots");
    return DR_ERR_INVALID_ARG;
  }
  dr_server_t *s = new (std::nothrow) dr_server_t();
  if (!s) {
    set_error("dr_server_create: host allocation failed");
    return DR_ERR_OOM;
  }
  s->opt = *o;
  if (s->opt.slots == 0) s->opt.slots = 4;
  if (s->opt.plan_cache <= 0) s->opt.plan_cache = 64;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&s->base), o->budget_bytes);
  if (e != cudaSuccess) {
    s->base = nullptr;
    delete s;
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      set_error("dr_server_create: cannot reserve %zu bytes of device memory", o->budget_bytes);
      return DR_ERR_OOM;
    }
    return cuda_fail("dr_server_create", e);
  }
  s->arena.reset(o->budget_bytes);
  s->streams.assign(s->opt.slots, nullptr);
  s->up_start.assign(s->opt.slots, nullptr);
  s->up_done.assign(s->opt.slots, nullptr);
  s->slot_busy.assign(s->opt.slots, 0);
  e = cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking);
  for (int i = 0; i < s->opt.slots && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s->up_start[i]);
    if (e == cudaSuccess) e = cudaEventCreate(&s->up_done[i]);
  }
  if (e != cudaSuccess) {
    dr_server_destroy(s);
    return cuda_fail("dr_server_create: streams", e);
  }
  // load the kernels now, while no stream has work: loading a module later
  // can synchronize the context
  dr_status ps = preload_kernels();
  if (ps != DR_OK) {
    dr_server_destroy(s);
    return ps;
  }
  s->t0 = now_s();
  s->sched = std::thread(scheduler, s);
  for (int i = 0; i < kPlanners; ++i) s->planners.emplace_back(planner, s);
  *out = s;
  return DR_OK;
}

extern "C" dr_status dr_server_submit(dr_server_t *s, const dr_geometry *g, const double *wires,
                                      int32_t K, const double *edges, int32_t B,
                                      const uint16_t *h_images, uint64_t *id) {
  TraceRange trace_("dr_server_submit");
  if (!s || !g || !wires || !edges || !id || K < 2 || B < 1 || g->rows < 0 || g->cols < 0) {
    set_error("dr_server_submit: bad arguments");
    return DR_ERR_INVALID_ARG;
  }
  const size_t P = (size_t)g->rows * g->cols;
  if (P > 0 && !h_images) {
    set_error("dr_server_submit: null images");
    return DR_ERR_INVALID_ARG;
  }
  Request *r = new (std::nothrow) Request();
  if (!r) {
    set_error("dr_server_submit: host allocation failed");
    return DR_ERR_OOM;
  }
  r->g = *g;
  r->wires.assign(wires, wires + 3 * (size_t)K);
  r->edges.assign(edges, edges + (size_t)B + 1);
  r->K = K;
  r->B = B;
  r->h_images = h_images;
  r->img_bytes = P * K * 2;
  r->out_bytes = P * B * 4;
  r->t.copy = -1.0;
  r->key = plan_key(*r);
  r->srv = s;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->t.submitted = now_s() - s->t0;
    s->reqs[r->id] = r;
    auto it = s->plans.find(r->key);
    if (it == s->plans.end()) {  // a new plan: to the planners
      it = s->plans.emplace(r->key, PlanEntry()).first;
      r->pe = &it->second;
      s->plan_jobs.push_back(r);
    }
    it->second.refs++;
    r->pe = &it->second;
    s->queue.push_back(r);
    *id = r->id;
  }
  s->cv_plan.notify_one();
  s->cv_sched.notify_all();
  return DR_OK;
}

extern "C" dr_status dr_server_poll(dr_server_t *s, uint64_t id, int32_t *state) {
  if (!s || !state) {
    set_error("dr_server_poll: null argument");
    return DR_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  Request *r = find(s, id);
  if (!r) {
    set_error("dr_server_poll: unknown request %llu", (unsigned long long)id);
    return DR_ERR_INVALID_ARG;
  }
  *state = r->state;
  return DR_OK;
}

extern "C" dr_status dr_server_wait(dr_server_t *s, uint64_t id, double timeout_s) {
  if (!s) {
    set_error("dr_server_wait: null server");
    return DR_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  Request *r = find(s, id);
  if (!r) {
    set_error("dr_server_wait: unknown request %llu", (unsigned long long)id);
    return DR_ERR_INVALID_ARG;
  }
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(timeout_s));
  while (r->state != DR_REQ_DONE && r->state != DR_REQ_FAILED) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
        r->state != DR_REQ_DONE && r->state != DR_REQ_FAILED) {
      set_error("dr_server_wait: request %llu not done after %.3f s",
                (unsigned long long)id, timeout_s);
      return DR_ERR_TIMEOUT;
    }
  }
  if (r->state == DR_REQ_FAILED) {
    set_error("request %llu failed: %s", (unsigned long long)id, dr_status_string(r->status));
    return r->status;
  }
  return DR_OK;
}

extern "C" dr_status dr_server_fetch(dr_server_t *s, uint64_t id, const void **d_out,
                                     dr_request_times *times) {
  if (!s) {
    set_error("dr_server_fetch: null server");
    return DR_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  Request *r = find(s, id);
  if (!r) {
    set_error("dr_server_fetch: unknown request %llu", (unsigned long long)id);
    return DR_ERR_INVALID_ARG;
  }
  // a done request's upload time is read by the scheduler right after
  while (r->state == DR_REQ_DONE && !r->done_seen)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(1));
  if (times) *times = r->t;
  if (r->state == DR_REQ_FAILED) {
    set_error("request %llu failed: %s", (unsigned long long)id, dr_status_string(r->status));
    return r->status;
  }
  if (r->state != DR_REQ_DONE) {
    set_error("dr_server_fetch: request %llu not done", (unsigned long long)id);
    return DR_ERR_INVALID_ARG;
  }
  if (d_out) *d_out = s->base + r->out_off;
  return DR_OK;
}

extern "C" dr_status dr_server_fetch_into(dr_server_t *s, uint64_t id, void *dst,
                                          size_t dst_bytes, dr_stream_t stream) {
  TraceRange trace_("dr_server_fetch_into");
  const void *src = nullptr;
  dr_status st = dr_server_fetch(s, id, &src, nullptr);
  if (st != DR_OK) return st;
  size_t bytes;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    bytes = find(s, id)->out_bytes;
  }
  if (!dst || dst_bytes < bytes) {
    set_error("dr_server_fetch_into: destination holds %zu of %zu bytes", dst_bytes, bytes);
    return DR_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail("dr_server_fetch_into", e);
  return DR_OK;
}

extern "C" dr_status dr_server_release(dr_server_t *s, uint64_t id) {
  if (!s) {
    set_error("dr_server_release: null server");
    return DR_ERR_INVALID_ARG;
  }
  {
    std::unique_lock<std::mutex> lk(s->mu);
    Request *r = find(s, id);
    if (!r) {
      set_error("dr_server_release: unknown request %llu", (unsigned long long)id);
      return DR_ERR_INVALID_ARG;
    }
    if (r->state != DR_REQ_DONE && r->state != DR_REQ_FAILED) {
      set_error("dr_server_release: request %llu still in flight", (unsigned long long)id);
      return DR_ERR_INVALID_ARG;
    }
    // the scheduler must have returned the image block first
    while (r->state == DR_REQ_DONE && !r->done_seen) s->cv_done.wait_for(lk, std::chrono::milliseconds(1));
    if (r->out_off != Arena::kNone) s->arena.release(r->out_off, r->out_bytes);
    if (r->pe) r->pe->refs--;
    s->reqs.erase(id);
    delete r;
  }
  s->cv_sched.notify_all();
  return DR_OK;
}

extern "C" dr_status dr_server_get_stats(dr_server_t *s, dr_server_stats *st) {
  if (!s || !st) {
    set_error("dr_server_get_stats: null argument");
    return DR_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->queued = (int64_t)s->queue.size();
  int inflight = 0;
  for (int b : s->slot_busy) inflight += b;
  st->in_flight = inflight;
  st->admitted = s->admitted;
  st->completed = s->completed;
  st->failed = s->rejected;
  st->plans_built = s->plan_builds;
  st->plans_cached = (int64_t)s->plans.size();
  st->arena_bytes = s->arena.size();
  st->arena_used = s->arena.used();
  return DR_OK;
}

extern "C" void dr_server_destroy(dr_server_t *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  s->cv_plan.notify_all();
  if (s->sched.joinable()) s->sched.join();
  for (auto &t : s->planners)
    if (t.joinable()) t.join();
  if (s->up) {
    cudaStreamSynchronize(s->up);
    cudaStreamDestroy(s->up);
  }
  for (auto st : s->streams)
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (auto ev : s->up_start)
    if (ev) cudaEventDestroy(ev);
  for (auto ev : s->up_done)
    if (ev) cudaEventDestroy(ev);
  for (auto &kv : s->reqs) delete kv.second;
  for (auto &kv : s->plans)
    if (kv.second.plan) dr_plan_destroy(kv.second.plan);
  if (s->base) cudaFree(s->base);
  delete s;
}
