// Request server with continuous batching.
//
// Callers submit correlation requests (host input, host taps, host output
// buffer) at any time.  A worker thread
//   1. admits queued requests in arrival order while the device-resident
//      pool (allocated once at creation) has room for their input and output
//      buffers -- admission by free device memory;
//   2. forms a batch from admitted requests as soon as a stream slot is free
//      and either the batch is full, the device is idle, or the oldest
//      admitted request has waited max_wait_s -- so requests that arrive
//      while others run join the next batch (continuous batching), and up to
//      n_streams batches are in flight at once, their copies and kernels
//      overlapping on the device;
//   3. per batch: copies the inputs in, runs the persistent batched kernel
//      over a table built for the batch (or, in plain mode, one plain
//      correlation launch per request), copies the outputs back and records
//      an event;
//   4. retires finished batches: frees their pool memory and records each
//      request's latency (submission to the worker seeing the batch done).
// Results are bitwise identical to a request served alone (every tile uses
// the plain kernel's tap order).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batched_internal.h"
#include "platform.h"
#include "runtime.h"

namespace convtune {
namespace {

constexpr size_t kAlign = 256;
constexpr int kTapFloats = kMaxK * ((kMaxK + 3) / 4 * 4);

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing.
class PoolAlloc {
 public:
  explicit PoolAlloc(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct Request {
  long long id = 0;
  const float* in_host = nullptr;
  long in_pitch = 0;
  float taps[kMaxK * kMaxK];
  int k = 0;
  float* out_host = nullptr;
  long out_pitch = 0;
  int out_h = 0, out_w = 0;
  double t_submit = 0, t_done = 0;
  size_t off = 0, bytes = 0, in_bytes = 0;
  bool done = false;
  int status = CT_OK;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  std::vector<Request*> reqs;
  ct_server_trace_entry trace;  // the batch in flight (timeline)
  cudaEvent_t tev[4] = {};       // timeline: start, copies in, kernels, copies out
  BatchImage* d_table = nullptr;
  float* d_taps = nullptr;
  unsigned* d_counter = nullptr;
  BatchImage* h_table = nullptr;  // pinned staging
  float* h_taps = nullptr;        // pinned staging
};

}  // namespace
}  // namespace convtune

using namespace convtune;

struct ct_server {
  ct_server_options opt;
  int device = 0;
  unsigned char* pool = nullptr;
  size_t pool_bytes = 0;
  unsigned char* slot_mem = nullptr;
  PoolAlloc* alloc = nullptr;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queued;    // submitted, not yet admitted
  std::deque<Request*> admitted;  // buffers reserved, not yet dispatched
  std::unordered_map<long long, Request*> all;
  long long next_id = 1;
  bool stop = false;
  int fatal = CT_OK;
  std::thread worker;
  // statistics since the last reset
  std::vector<double> lat;
  long long submitted = 0, completed = 0, rejected = 0, batches = 0, batched_reqs = 0;
  double flop = 0, t0 = 0, t_last = 0;
  unsigned long long e0 = 0;
  bool have_energy = false;
  ct_platform_ops ops;
  // timeline of completed batches (ring of trace_cap entries)
  std::vector<ct_server_trace_entry> trace;
  size_t trace_next = 0, trace_count = 0;

  void run();
  int dispatch(Slot& sl, std::vector<Request*>& batch);
  ~ct_server();
};

int ct_server::dispatch(Slot& sl, std::vector<Request*>& batch) {
  cudaError_t e;
  int rc = CT_OK;
  const bool timed = sl.tev[0] != nullptr;
  if (timed && (e = cudaEventRecord(sl.tev[0], sl.s)) != cudaSuccess) return cuda_status(e);
  // inputs in: whole pitched rows in one contiguous copy (the pool's copy of
  // the caller's padding columns is never read)
  for (Request* r : batch) {
    const size_t bytes = sizeof(float) * (size_t)r->in_pitch * (r->out_h + r->k - 1);
    e = cudaMemcpyAsync(pool + r->off, r->in_host, bytes, cudaMemcpyHostToDevice, sl.s);
    if (e != cudaSuccess) return cuda_status(e);
    sl.trace.bytes_in += (double)bytes;
  }
  if (timed && (e = cudaEventRecord(sl.tev[1], sl.s)) != cudaSuccess) return cuda_status(e);
  if (opt.plain) {
    for (Request* r : batch) {
      ct_problem p;
      p.in = reinterpret_cast<const float*>(pool + r->off);
      p.in_pitch = r->in_pitch;
      p.filt = r->taps;
      p.fh = p.fw = r->k;
      p.out = reinterpret_cast<float*>(pool + r->off + r->in_bytes);
      p.out_pitch = r->out_pitch;
      p.out_h = r->out_h;
      p.out_w = r->out_w;
      ct_batch_item it;
      it.in = p.in;
      it.in_pitch = p.in_pitch;
      it.filt = r->taps;
      it.k = r->k;
      it.out = p.out;
      it.out_pitch = p.out_pitch;
      it.out_h = p.out_h;
      it.out_w = p.out_w;
      BatchImage im;
      rc = batch_image_from_item(it, opt.use_tiles ? &opt.tiles : nullptr, &im);
      if (rc != CT_OK) return rc;
      ct_config c;
      c.block_x = im.bx;
      c.block_y = im.threads / im.bx;
      c.tile_x = kBatchTileX;
      c.tile_y = std::min(im.ty, 4);  // (the single-image kernel's tiles are at most 4 high)
      c.staging = CT_STAGE_SMEM;
      c.filter_mem = CT_FILTER_CONST;
      c.vec_width = im.vw;
      if ((rc = ct_conv2d_run(&p, &c, sl.s)) != CT_OK) return rc;
    }
  } else {
    // the table runs in filter-side order (so in class order too: one
    // persistent kernel per class, whose CTAs then take one side's items in
    // a row); the caller's order of `batch` does not matter beyond this
    std::stable_sort(batch.begin(), batch.end(),
                     [](const Request* x, const Request* y) { return x->k < y->k; });
    const double t_plan0 = now_s();
    long long first = 0;
    for (size_t q = 0; q < batch.size(); ++q) {
      Request* r = batch[q];
      ct_batch_item it;
      it.in = reinterpret_cast<const float*>(pool + r->off);
      it.in_pitch = r->in_pitch;
      it.filt = r->taps;
      it.k = r->k;
      it.out = reinterpret_cast<float*>(pool + r->off + r->in_bytes);
      it.out_pitch = r->out_pitch;
      it.out_h = r->out_h;
      it.out_w = r->out_w;
      BatchImage& im = sl.h_table[q];
      rc = batch_image_from_item(it, opt.use_tiles ? &opt.tiles : nullptr, &im);
      if (rc != CT_OK) return rc;
      const int kp = (r->k + 3) / 4 * 4;
      float* ht = sl.h_taps + q * kTapFloats;
      for (int j = 0; j < r->k; ++j)
        for (int i = 0; i < kp; ++i) ht[j * kp + i] = i < r->k ? r->taps[j * r->k + i] : 0.0f;
      im.filt = sl.d_taps + q * kTapFloats;
      im.first_item = first;
      first += (long long)im.tiles_x * im.tiles_y;
    }
    const size_t n = batch.size();
    // the plan places the 13..17 taps in parameter blocks and sets tap_off:
    // the table goes to the device after it
    std::vector<const float*> host_taps(n);
    for (size_t q = 0; q < n; ++q) host_taps[q] = batch[q]->taps;
    BatchPlan plan;
    if ((rc = plan_batch(sl.h_table, (int)n, host_taps.data(), &plan)) != CT_OK) return rc;
    sl.trace.plan_s = now_s() - t_plan0;
    if ((e = cudaMemcpyAsync(sl.d_taps, sl.h_taps, sizeof(float) * kTapFloats * n,
                             cudaMemcpyHostToDevice, sl.s)) != cudaSuccess)
      return cuda_status(e);
    if ((e = cudaMemcpyAsync(sl.d_table, sl.h_table, sizeof(BatchImage) * n,
                             cudaMemcpyHostToDevice, sl.s)) != cudaSuccess)
      return cuda_status(e);
    int err = CT_OK;
    unsigned* status = device_status_word(&err);
    if (!status) return err;
    if ((rc = enqueue_batch_plan(plan, sl.d_table, sl.d_counter, status, sl.s)) != CT_OK)
      return rc;
  }
  if (timed && (e = cudaEventRecord(sl.tev[2], sl.s)) != cudaSuccess) return cuda_status(e);
  // outputs back: only the out_w computed columns of each row (the caller's
  // padding columns are left untouched)
  for (Request* r : batch) {
    sl.trace.bytes_out += sizeof(float) * (double)r->out_w * r->out_h;
    const size_t pitch = sizeof(float) * (size_t)r->out_pitch;
    if (r->out_pitch == r->out_w)  // no padding columns: one contiguous copy
      e = cudaMemcpyAsync(r->out_host, pool + r->off + r->in_bytes, pitch * r->out_h,
                          cudaMemcpyDeviceToHost, sl.s);
    else
      e = cudaMemcpy2DAsync(r->out_host, pitch, pool + r->off + r->in_bytes, pitch,
                            sizeof(float) * (size_t)r->out_w, r->out_h, cudaMemcpyDeviceToHost,
                            sl.s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (timed && (e = cudaEventRecord(sl.tev[3], sl.s)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaEventRecord(sl.ev, sl.s)) != cudaSuccess) return cuda_status(e);
  sl.busy = true;
  sl.reqs = batch;
  return CT_OK;
}

void ct_server::run() {
  cudaSetDevice(device);
  double t_iter = now_s(), max_gap = 0;
  int n_queued = 0;
  for (;;) {
    {
      // pauses of this thread between iterations (timeline)
      const double t = now_s();
      max_gap = std::max(max_gap, t - t_iter);
      t_iter = t;
    }
    bool idle = true;
    std::vector<Request*> finished;
    // retire finished batches
    for (Slot& sl : slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      idle = false;
      const double t = now_s();
      std::lock_guard<std::mutex> lk(mu);
      for (Request* r : sl.reqs) {
        r->t_done = t;
        r->done = true;
        if (q != cudaSuccess) r->status = cuda_status(q);
        alloc->release(r->off, r->bytes);
        lat.push_back(t - r->t_submit);
        ++completed;
        flop += 2.0 * r->k * r->k * (double)r->out_h * r->out_w;
        t_last = t;
      }
      if (!trace.empty()) {
        sl.trace.t_done = t;
        if (sl.tev[0] && q == cudaSuccess) {
          float ms[3] = {0, 0, 0};
          for (int k = 0; k < 3; ++k)
            if (cudaEventElapsedTime(&ms[k], sl.tev[k], sl.tev[k + 1]) != cudaSuccess) {
              cudaGetLastError();
              ms[k] = NAN;
            }
          sl.trace.h2d_ms = ms[0];
          sl.trace.kernels_ms = ms[1];
          sl.trace.d2h_ms = ms[2];
        }
        trace[trace_next] = sl.trace;
        trace_next = (trace_next + 1) % trace.size();
        trace_count = std::min(trace_count + 1, trace.size());
      }
      sl.busy = false;
      sl.reqs.clear();
      cv.notify_all();
    }
    std::vector<Request*> batch;
    Slot* free_slot = nullptr;
    bool any_busy = false;
    for (Slot& sl : slots) {
      if (sl.busy) any_busy = true;
      else if (!free_slot) free_slot = &sl;
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      if (stop && queued.empty() && admitted.empty() && !any_busy) break;
      n_queued = (int)queued.size();
      // admission: arrival order, while the pool has room
      while (!queued.empty()) {
        Request* r = queued.front();
        if (!alloc->alloc(r->bytes, &r->off)) break;
        queued.pop_front();
        admitted.push_back(r);
        idle = false;
      }
      if (free_slot && !admitted.empty()) {
        const double wait = now_s() - admitted.front()->t_submit;
        if ((int)admitted.size() >= opt.max_batch || !any_busy || wait >= opt.max_wait_s) {
          while (!admitted.empty() && (int)batch.size() < opt.max_batch) {
            batch.push_back(admitted.front());
            admitted.pop_front();
          }
        }
      }
    }
    if (!batch.empty()) {
      idle = false;
      ct_server_trace_entry& te = free_slot->trace;
      memset(&te, 0, sizeof(te));
      te.t_dispatch = now_s();
      te.oldest_wait_s = te.t_dispatch - batch.front()->t_submit;
      te.loop_gap_s = max_gap;
      te.n_requests = (int)batch.size();
      te.slot = (int)(free_slot - slots.data());
      te.queued = n_queued;
      for (const Slot& o : slots) te.busy_slots += o.busy ? 1 : 0;
      max_gap = 0;
      const int rc = dispatch(*free_slot, batch);
      te.dispatch_s = now_s() - te.t_dispatch;
      std::lock_guard<std::mutex> lk(mu);
      ++batches;
      batched_reqs += (long long)batch.size();
      if (rc != CT_OK) {
        // fail the batch's requests; keep serving
        cudaStreamSynchronize(free_slot->s);
        const double t = now_s();
        for (Request* r : batch) {
          r->status = rc;
          r->done = true;
          r->t_done = t;
          alloc->release(r->off, r->bytes);
        }
        free_slot->busy = false;
        free_slot->reqs.clear();
        cv.notify_all();
      }
    }
    if (idle) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

ct_server::~ct_server() {
  for (Slot& sl : slots) {
    if (sl.s) {
      cudaStreamSynchronize(sl.s);
      cudaStreamDestroy(sl.s);
    }
    if (sl.ev) cudaEventDestroy(sl.ev);
    for (cudaEvent_t te : sl.tev)
      if (te) cudaEventDestroy(te);
    if (sl.h_table) cudaFreeHost(sl.h_table);
    if (sl.h_taps) cudaFreeHost(sl.h_taps);
  }
  if (pool) cudaFree(pool);
  if (slot_mem) cudaFree(slot_mem);
  delete alloc;
  for (auto& kv : all) delete kv.second;
}

extern "C" {

int ct_server_create(const ct_server_options* opt, ct_server** out) {
  if (!opt || !out) return CT_EINVAL;
  *out = nullptr;
  if (opt->n_streams < 1 || opt->n_streams > 64 || opt->max_batch < 1 ||
      opt->max_batch > 4096 || opt->pool_bytes <= 0 || !(opt->max_wait_s >= 0) ||
      opt->trace_cap < 0 || opt->trace_cap > (1 << 20))
    return CT_EINVAL;
  ct_server* sv = new (std::nothrow) ct_server();
  if (!sv) return CT_ENOMEM;
  sv->opt = *opt;
  cudaError_t e = cudaGetDevice(&sv->device);
  // the request pool never exceeds 90 % of the device memory free right now
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    delete sv;
    return cuda_status(e);
  }
  sv->pool_bytes = std::min<size_t>((size_t)opt->pool_bytes, free_b / 10 * 9);
  int err = CT_OK;
  if (!device_status_word(&err)) {
    delete sv;
    return err;
  }
  if ((e = cudaMalloc(&sv->pool, sv->pool_bytes)) != cudaSuccess) {
    delete sv;
    return cuda_status(e);
  }
  sv->alloc = new PoolAlloc(sv->pool_bytes);
  const size_t per_slot_table = sizeof(BatchImage) * opt->max_batch;
  const size_t per_slot_taps = sizeof(float) * kTapFloats * opt->max_batch;
  const size_t per_slot =
      (per_slot_table + per_slot_taps + kBatchCounterBytes + kAlign - 1) / kAlign * kAlign;
  if ((e = cudaMalloc(&sv->slot_mem, per_slot * opt->n_streams)) != cudaSuccess) {
    delete sv;
    return cuda_status(e);
  }
  sv->slots.resize(opt->n_streams);
  for (int i = 0; i < opt->n_streams; ++i) {
    Slot& sl = sv->slots[i];
    unsigned char* base = sv->slot_mem + per_slot * i;
    sl.d_counter = reinterpret_cast<unsigned*>(base);  // one work counter per launch
    sl.d_table = reinterpret_cast<BatchImage*>(base + kBatchCounterBytes);
    sl.d_taps = reinterpret_cast<float*>(base + kBatchCounterBytes + per_slot_table);
    if (opt->trace_cap > 0)
      for (cudaEvent_t& te : sl.tev)
        if ((e = cudaEventCreate(&te)) != cudaSuccess) {
          delete sv;
          return cuda_status(e);
        }
    if ((e = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMallocHost(&sl.h_table, per_slot_table)) != cudaSuccess ||
        (e = cudaMallocHost(&sl.h_taps, per_slot_taps)) != cudaSuccess) {
      delete sv;
      return cuda_status(e);
    }
  }
  // Load every kernel the worker can launch before the first request: code
  // is loaded on first use, and a first launch inside a busy worker held up
  // every request queued behind it (plain mode: one variant per bucket,
  // ~40 ms stalls measured at 5000 requests/s; batched: the class kernels).
  {
    BatchPlan warm;
    int rc = plan_batch(nullptr, 0, nullptr, &warm);
    for (int k = 1; rc == CT_OK && opt->plain && k <= kMaxK; k += 2)
      for (int cls = 0; rc == CT_OK && cls < 2; ++cls) {
        ct_batch_item it;
        memset(&it, 0, sizeof(it));
        it.k = k;
        it.out_h = it.out_w = cls ? 1024 : 256;  // a shape of the size class
        it.in_pitch = it.out_pitch = 1024 + k;
        it.in = it.out = reinterpret_cast<float*>(sv->pool);
        it.filt = reinterpret_cast<const float*>(sv->pool);
        BatchImage im;
        if ((rc = batch_image_from_item(it, opt->use_tiles ? &opt->tiles : nullptr, &im)) !=
            CT_OK)
          break;
        ct_config c;
        c.block_x = im.bx;
        c.block_y = im.threads / im.bx;
        c.tile_x = kBatchTileX;
        c.tile_y = std::min(im.ty, 4);
        c.staging = CT_STAGE_SMEM;
        c.filter_mem = CT_FILTER_CONST;
        c.vec_width = 4;
        rc = prime_conv_kernel(k, c);
      }
    if (rc != CT_OK) {
      delete sv;
      return rc;
    }
  }
  if (opt->trace_cap > 0) sv->trace.resize((size_t)opt->trace_cap);
  sv->ops = platform_ops();
  sv->t0 = now_s();
  sv->have_energy = sv->ops.energy_mj && sv->ops.energy_mj(sv->ops.ctx, &sv->e0) == CT_OK;
  sv->worker = std::thread([sv] { sv->run(); });
  *out = sv;
  return CT_OK;
}

int ct_server_submit(ct_server* sv, const float* in_host, long in_pitch, const float* filt, int k,
                     float* out_host, long out_pitch, int out_h, int out_w, long long* id) {
  if (!sv || !in_host || !filt || !out_host || !id) return CT_EINVAL;
  if (k < 1 || k > kMaxK || !(k & 1) || out_h <= 0 || out_w <= 0) return CT_EINVAL;
  if (in_pitch < (long)out_w + k - 1 || out_pitch < out_w) return CT_EINVAL;
  Request* r = new (std::nothrow) Request();
  if (!r) return CT_ENOMEM;
  r->in_host = in_host;
  r->in_pitch = in_pitch;
  memcpy(r->taps, filt, sizeof(float) * k * k);
  r->k = k;
  r->out_host = out_host;
  r->out_pitch = out_pitch;
  r->out_h = out_h;
  r->out_w = out_w;
  r->in_bytes = (sizeof(float) * (size_t)(out_h + k - 1) * in_pitch + kAlign - 1) / kAlign * kAlign;
  r->bytes = r->in_bytes + sizeof(float) * (size_t)out_h * out_pitch;
  r->t_submit = now_s();
  std::lock_guard<std::mutex> lk(sv->mu);
  if (r->bytes > sv->pool_bytes) {
    ++sv->rejected;
    delete r;
    return CT_ENOMEM;  // can never be admitted
  }
  if (sv->stop) {
    delete r;
    return CT_EINVAL;
  }
  r->id = sv->next_id++;
  sv->all[r->id] = r;
  sv->queued.push_back(r);
  ++sv->submitted;
  *id = r->id;
  return CT_OK;
}

int ct_server_wait(ct_server* sv, long long id, double timeout_s, double* latency_s) {
  if (!sv) return CT_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(id);
  if (it == sv->all.end()) return CT_EINVAL;
  Request* r = it->second;
  const bool ok = sv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                  [r] { return r->done; });
  if (!ok) return CT_ETIMEOUT;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  const int st = r->status;
  sv->all.erase(it);
  delete r;
  return st;
}

int ct_server_drain(ct_server* sv, double timeout_s) {
  if (!sv) return CT_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  const bool ok = sv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [sv] {
    for (auto& kv : sv->all)
      if (!kv.second->done) return false;
    return true;
  });
  if (!ok) return CT_ETIMEOUT;
  for (auto& kv : sv->all) delete kv.second;
  sv->all.clear();
  return CT_OK;
}

int ct_server_stats_get(ct_server* sv, int reset, ct_server_stats* out) {
  if (!sv || !out) return CT_EINVAL;
  memset(out, 0, sizeof(*out));
  std::lock_guard<std::mutex> lk(sv->mu);
  const double t = now_s();
  std::vector<double> v = sv->lat;
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) -> double {
    if (v.empty()) return (double)NAN;
    const size_t i = (size_t)std::min<double>(v.size() - 1, floor(q * (v.size() - 1) + 0.5));
    return v[i];
  };
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->rejected = sv->rejected;
  out->p50_s = pct(0.50);
  out->p99_s = pct(0.99);
  out->max_s = v.empty() ? NAN : v.back();
  double acc = 0;
  for (double x : v) acc += x;
  out->mean_s = v.empty() ? NAN : acc / v.size();
  out->wall_s = (sv->completed ? sv->t_last : t) - sv->t0;
  out->flop = sv->flop;
  out->batches = sv->batches;
  out->mean_batch = sv->batches ? (double)sv->batched_reqs / sv->batches : 0.0;
  out->pool_used_bytes = (long long)sv->alloc->used();
  out->energy_j = NAN;
  if (sv->have_energy) {
    unsigned long long e1 = 0;
    if (sv->ops.energy_mj(sv->ops.ctx, &e1) == CT_OK) out->energy_j = (e1 - sv->e0) / 1000.0;
    if (reset) sv->e0 = e1;
  }
  if (reset) {
    sv->lat.clear();
    sv->submitted = sv->completed = sv->rejected = sv->batches = sv->batched_reqs = 0;
    sv->flop = 0;
    sv->t0 = t;
    sv->t_last = t;
  }
  return CT_OK;
}

int ct_server_trace_get(ct_server* sv, ct_server_trace_entry* out, int cap, int* n) {
  if (!sv || !n || cap < 0) return CT_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->trace.empty()) return CT_ENOTSUP;
  *n = (int)sv->trace_count;
  if ((int)sv->trace_count > cap || (!out && sv->trace_count > 0)) return CT_ENOMEM;
  const size_t m = sv->trace.size();
  const size_t first = (sv->trace_next + m - sv->trace_count) % m;
  for (size_t i = 0; i < sv->trace_count; ++i) out[i] = sv->trace[(first + i) % m];
  return CT_OK;
}

int ct_server_destroy(ct_server* sv) {
  if (!sv) return CT_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  if (sv->worker.joinable()) sv->worker.join();
  delete sv;
  return CT_OK;
}

}  // extern "C"
