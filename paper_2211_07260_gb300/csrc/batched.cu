// Persistent, CUDA-graph-captured batched correlation (many images of
// uneven sizes and odd filter sides in one launch), its per-bucket tile
// tuning with the energy objective, and the plain one-launch-per-image
// comparison.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "batched.cuh"
#include "batched_internal.h"
#include "measure.h"
#include "platform.h"
#include "runtime.h"

namespace convtune {

template <int KK>
__device__ __forceinline__ void run_tile_k(const BatchArgs& a, const BatchImage& im, int t,
                                           const float* buf, const float* sfilt) {
  if (im.ty == 1) batch_tile<KK, 1>(a, im, t, buf, sfilt);
  else if (im.ty == 2) batch_tile<KK, 2>(a, im, t, buf, sfilt);
  else if constexpr (KK <= kBatchMaxK8) {
    if (im.ty == 8) batch_tile<KK, 8>(a, im, t, buf, sfilt);
    else batch_tile<KK, 4>(a, im, t, buf, sfilt);
  } else {
    batch_tile<KK, 4>(a, im, t, buf, sfilt);
  }
}

// One tile of a class-CLS image; a filter side outside the class (a table
// the host did not split correctly) only raises the status bit.
template <int CLS>
__device__ __forceinline__ void run_tile(const BatchArgs& a, const BatchImage& im, int t,
                                         const float* buf, const float* sfilt, unsigned* status) {
  switch (im.k) {
#define CT_BATCH_CASE(KK)                                                        \
  case KK:                                                                       \
    if constexpr (batch_class_of(KK) == CLS) {                                   \
      run_tile_k<KK>(a, im, t, buf, sfilt);                                      \
      return;                                                                    \
    }                                                                            \
    break;
    CT_BATCH_CASE(1)
    CT_BATCH_CASE(3)
    CT_BATCH_CASE(5)
    CT_BATCH_CASE(7)
    CT_BATCH_CASE(9)
    CT_BATCH_CASE(11)
    CT_BATCH_CASE(13)
    CT_BATCH_CASE(15)
    CT_BATCH_CASE(17)
#undef CT_BATCH_CASE
    default:
      break;
  }
  if (threadIdx.x == 0) atomicOr(status, kStatusBadItem);
}

// resident CTAs per SM each class kernel is compiled for (registers <= 80,
// 80, 128 per thread; sides 1-7 measured 164 -> 148 us with 80 registers
// and 3 CTAs instead of 64 and 4, whose spills cost more than the fourth CTA
// gave)
__host__ __device__ constexpr int batch_class_min_ctas(int cls) { return cls == 2 ? 2 : 3; }

// largest filter side of a class (its shared-memory tap area)
__host__ __device__ constexpr int batch_class_max_k(int cls) { return cls == 0 ? 7 : (cls == 1 ? 11 : 17); }

// Images whose first work items a CTA keeps in shared memory for the lookup
// (larger launches search the table in global memory).
constexpr int kBatchFirstCache = 512;

// Claim state, touched by lane 0 of warp 0 only.
struct BatchClaimState {
  unsigned cur, end;     // items [cur, end) of the current chunk
  long long first, last;  // table items [first, last) of image `img`
  int img;
};

// Lane 0 of warp 0: the launch item after the current one (taking the
// prefetched chunk, and prefetching the next, when the current chunk is
// used up), or n_items past the end.
__device__ __forceinline__ unsigned batch_next_item(const BatchArgs& a, BatchClaimState* c,
                                                    unsigned* next_chunk) {
  if (c->cur >= c->end) {
    const unsigned long long lo = (unsigned long long)*next_chunk * a.claim_items;
    if (lo >= (unsigned long long)a.n_items) return (unsigned)a.n_items;
    c->cur = (unsigned)lo;
    const unsigned long long hi = lo + a.claim_items;
    c->end = (unsigned)(hi < (unsigned long long)a.n_items ? hi : (unsigned long long)a.n_items);
    *next_chunk = atomicAdd(a.counter, 1u);
  }
  return c->cur++;
}

// Lane 0 of warp 0: the image and tile of launch item w, or -1 past the end
// of the launch's items and -2 for an item outside its image.  The range of
// the last image found is kept; otherwise a binary search over first_item
// (from shared memory when the launch has at most kBatchFirstCache images).
__device__ __forceinline__ int batch_resolve(const BatchArgs& a, unsigned w, BatchClaimState* c,
                                             const long long* s_first, long long* tile) {
  if ((long long)w >= a.n_items) return -1;
  const long long gw = a.item_base + (long long)w;
  if (gw < c->first || gw >= c->last) {
    const bool cached = a.n_images <= kBatchFirstCache;
    int lo = 0, hi = a.n_images - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if ((cached ? s_first[mid] : a.images[mid].first_item) <= gw) lo = mid;
      else hi = mid - 1;
    }
    const BatchImage& im = a.images[lo];
    c->img = lo;
    c->first = im.first_item;
    c->last = im.first_item + (long long)im.tiles_x * im.tiles_y;
    if (gw < c->first || gw >= c->last) return -2;
  }
  *tile = gw - c->first;
  return c->img;
}

// Warp 0: slot `dst` of the work-item ring describes item w (its image entry
// copied from the table, or from slot `prev` when the image is the same).
__device__ __forceinline__ void batch_fill_slot(const BatchArgs& a, unsigned w, int dst, int prev,
                                                BatchClaimState* c, const long long* s_first,
                                                BatchImage* s_desc, long long* s_tile,
                                                int* s_img) {
  const int lane = threadIdx.x & 31;
  int img = 0;
  if (lane == 0) {
    long long tl = 0;
    img = batch_resolve(a, w, c, s_first, &tl);
    s_img[dst] = img;
    s_tile[dst] = tl;
  }
  img = __shfl_sync(0xffffffffu, img, 0);
  if (img >= 0) {
    const uint2* src = prev >= 0 && s_img[prev] == img
                           ? reinterpret_cast<const uint2*>(&s_desc[prev])
                           : reinterpret_cast<const uint2*>(a.images + img);
    reinterpret_cast<uint2*>(&s_desc[dst])[lane] = src[lane];
  }
  __syncwarp();
}

template <int CLS>
__global__ void __launch_bounds__(kBatchThreads, batch_class_min_ctas(CLS))
    batched_conv_kernel(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int kFilt = batch_filt_floats(batch_class_max_k(CLS));
  float* const sfilt = reinterpret_cast<float*>(smem_raw);
  float* const bufs = sfilt + kFilt;  // nb staging buffers of a.buf_floats
  constexpr int nb = batch_class_stages(CLS);
  constexpr int nslot = nb + 1;
  __shared__ __align__(8) uint64_t mbar[kBatchMaxStages];
  // Work-item ring: item i's image entry (copied from the table), image index
  // and tile sit in slot i % (nb + 1).  At the start of item i lane 0 starts
  // the input copy of item i + nb - 1 into staging buffer (i + nb - 1) % nb
  // (the one item i - 1 used) and warp 0 describes item i + nb in the slot
  // item i - 1 held; the CTA then computes item i.  Claims run a chunk ahead.
  __shared__ __align__(128) BatchImage s_desc[kBatchMaxStages + 1];
  __shared__ long long s_tile[kBatchMaxStages + 1];
  __shared__ int s_img[kBatchMaxStages + 1];
  __shared__ long long s_first[kBatchFirstCache];
  __shared__ BatchClaimState s_claim;
  const int tid = threadIdx.x;
  const bool warp0 = tid < 32;
  unsigned next_chunk = 0;  // lane 0: the chunk claimed ahead
  if (a.n_images <= kBatchFirstCache)
    for (int q = tid; q < a.n_images; q += blockDim.x) s_first[q] = a.images[q].first_item;
  if (tid == 0) {
    for (int q = 0; q < nb; ++q) mbar_init(&mbar[q]);
    mbar_init_fence();
    s_claim.cur = s_claim.end = 0;
    s_claim.first = s_claim.last = -1;
    s_claim.img = 0;
    next_chunk = atomicAdd(a.counter, 1u);
  }
  __syncthreads();
  if (warp0) {
    // prologue: items 0 .. nb-1 described, the copies of items 0 .. nb-2
    // started
    for (int q = 0; q < nb; ++q) {
      unsigned w = (unsigned)a.n_items;
      if (tid == 0 && (q == 0 || s_img[q - 1] != -1)) w = batch_next_item(a, &s_claim, &next_chunk);
      batch_fill_slot(a, w, q, q - 1, &s_claim, s_first, s_desc, s_tile, s_img);
    }
    if (tid == 0)
      for (int q = 0; q + 1 < nb; ++q)
        if (s_img[q] >= 0 && s_desc[q].use_tma)
          batch_issue_tma(&s_desc[q], a.images + s_img[q], (int)s_tile[q], bufs + q * a.buf_floats,
                          &mbar[q]);
  }
  __syncthreads();
  unsigned phase = 0;  // bit b: parity of mbar[b]'s next phase
  for (int i = 0;; ++i) {
    const int cs = i % nslot;               // item i's slot
    const int ls = (i + nb - 1) % nslot;    // the last described item's slot
    const int fs = (i + nb) % nslot;        // the slot item i - 1 held
    const int b = i % nb;
    const int img = s_img[cs];
    if (img == -1) break;
    float* const buf = bufs + b * a.buf_floats;
    if (warp0) {
      const int lb = (i + nb - 1) % nb;
      if (tid == 0 && s_img[ls] >= 0 && s_desc[ls].use_tma)
        batch_issue_tma(&s_desc[ls], a.images + s_img[ls], (int)s_tile[ls],
                        bufs + lb * a.buf_floats, &mbar[lb]);
      unsigned w = (unsigned)a.n_items;
      if (tid == 0 && s_img[ls] != -1) w = batch_next_item(a, &s_claim, &next_chunk);
      batch_fill_slot(a, w, fs, ls, &s_claim, s_first, s_desc, s_tile, s_img);
    }
    bool ok = true;
    if (img >= 0) {
      const BatchImage& im = s_desc[cs];
      const int tl = (int)s_tile[cs];  // tiles of one image fit 32 bits
      const bool param_taps = im.tap_off >= 0;  // CTA-uniform, like use_tma
      if (!param_taps) {
        const int kp = (im.k + 3) / 4 * 4;
        for (int q = tid; q < im.k * kp; q += blockDim.x) sfilt[q] = im.filt[q];
      }
      if (im.use_tma) {
        ok = mbar_wait(&mbar[b], (phase >> b) & 1u);
        phase ^= 1u << b;
        if (!param_taps) __syncthreads();
      } else {
        batch_stage_cp_async(im, tl, buf);
        __syncthreads();
      }
      if (ok) run_tile<CLS>(a, im, tl, buf, sfilt, a.status);
    } else if (tid == 0) {
      atomicOr(a.status, kStatusBadItem);
    }
    // the buffers and the ring slots are rewritten only after this point
    if (__syncthreads_or(!ok)) {
      // a copy never completed: report it, give the copies still in flight
      // (this item's and those of the next nb - 1 items) a bounded wait to
      // land, and stop this CTA
      if (tid == 0) {
        atomicOr(a.status, kStatusTmaTimeout);
        mbar_wait(&mbar[b], ((phase >> b) & 1u) ^ 1u);
        for (int d = 1; d < nb; ++d) {
          const int sl = (i + d) % nslot, bb = (i + d) % nb;
          if (s_img[sl] >= 0 && s_desc[sl].use_tma) mbar_wait(&mbar[bb], (phase >> bb) & 1u);
        }
      }
      return;
    }
  }
}

const void* batched_kernel_fn(int cls) {
  switch (cls) {
    case 0: return (const void*)batched_conv_kernel<0>;
    case 1: return (const void*)batched_conv_kernel<1>;
    default: return (const void*)batched_conv_kernel<2>;
  }
}

namespace {

constexpr size_t kBatchBranches = 8;  // parallel branches of a captured batch graph
// Parallel branches of the launches graph (GB300, 256-image batch ordered
// by filter side: 8, 10 and 12 branches 856-857 us, 16 branches 878-885 us,
// 24 branches 890-893 us).
constexpr size_t kBatchLaunchBranches = 12;
// Launches-mode candidates of the per-bucket tuner: (block_x, block_y,
// tile_y), 128 or 256 threads and 4-wide tiles, as in the single-image
// kernel's fastest configurations (4096^2 / 17 x 17 and 1024^2 / 7 x 7).
constexpr int kLaunchCandidates = 9;
constexpr int kLaunchCand[kLaunchCandidates][3] = {
    {16, 8, 4}, {32, 4, 4}, {32, 2, 4}, {16, 4, 4}, {64, 2, 4},
    {32, 8, 2}, {32, 4, 2}, {64, 4, 2}, {128, 2, 2}};

inline int round_up(int x, int a) { return (x + a - 1) / a * a; }

// Dynamic shared memory of a class launch whose largest staging buffer is
// buf_floats: the class's shared-memory tap area and `stages` buffers.
size_t batch_launch_smem(int cls, int buf_floats, int stages) {
  return sizeof(float) *
         (size_t)(batch_filt_floats(batch_class_max_k(cls)) + stages * buf_floats);
}

bool valid_tile(int bx, int ty, int k, int threads) {
  return (bx == 16 || bx == 32 || bx == 64 || bx == 128) && bx <= threads &&
         (ty == 1 || ty == 2 || ty == 4 || (ty == 8 && k <= kBatchMaxK8));
}

// CTA size of filter side k's class launch.
int class_threads(const ct_batch_tiles* tiles, int k) {
  const int t = tiles ? tiles->class_threads[batch_class_of(k)] : 0;
  return batch_valid_threads(t) ? t : kBatchThreads;
}

// Work items per claim of filter side k's class launch.
int class_claim(const ct_batch_tiles* tiles, int k) {
  const int c = tiles ? tiles->claim_items[batch_class_of(k)] : 0;
  return c >= 1 && c <= 8 ? c : batch_default_claim(batch_class_of(k));
}

int size_class(int h, int w) { return (long long)h * w >= 512LL * 512LL ? 1 : 0; }

}  // namespace

int plan_batch(BatchImage* table, int n, const float* const* host_taps, BatchPlan* plan) {
  *plan = BatchPlan();
  int dev = 0, sms = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= 64) return CT_ENOTSUP;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
          cudaSuccess)
    return cuda_status(e);
  {
    // once per device: every class kernel may use the device's whole opt-in
    // shared memory (a per-plan value could undercut another live plan)
    static std::mutex mu;
    static bool raised[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (!raised[dev]) {
      for (int c = 0; c < kBatchClasses; ++c) {
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, batched_kernel_fn(c))) != cudaSuccess ||
            (e = cudaFuncSetAttribute(batched_kernel_fn(c),
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      optin - (int)fa.sharedSizeBytes)) != cudaSuccess)
          return cuda_status(e);
      }
      raised[dev] = true;
    }
  }
  for (int q = 1; q < n; ++q)
    if (batch_class_of(table[q].k) < batch_class_of(table[q - 1].k)) return CT_EINVAL;
  // Launches: one per class, cut into runs whose taps fit one parameter
  // block (the last launches fall back to taps in shared memory if the
  // counters would run out).
  auto finish = [&](BatchClassLaunch& L) -> int {
    L.n = L.hi - L.lo;
    if (L.n == 0) return CT_OK;
    int buf = 32;
    for (int q = L.lo; q < L.hi; ++q) {
      L.items += (long long)table[q].tiles_x * table[q].tiles_y;
      buf = std::max(buf, table[q].g.buf_floats);
    }
    L.item_base = table[L.lo].first_item;
    L.threads = table[L.lo].threads;
    L.claim = table[L.lo].claim;
    for (int q = L.lo; q < L.hi; ++q)  // one CTA size and claim size per launch
      if (table[q].threads != L.threads || table[q].claim != L.claim) return CT_EINVAL;
    L.buf_floats = buf;
    cudaFuncAttributes fa;
    cudaError_t e2 = cudaFuncGetAttributes(&fa, batched_kernel_fn(L.cls));
    if (e2 != cudaSuccess) return cuda_status(e2);
    L.stages = batch_class_stages(L.cls);
    L.smem = batch_launch_smem(L.cls, buf, L.stages);
    if (L.smem + fa.sharedSizeBytes > (size_t)optin) return CT_ECONFIG;
    int per_sm = 0;
    if ((e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel_fn(L.cls),
                                                            L.threads, L.smem)) != cudaSuccess)
      return cuda_status(e2);
    if (per_sm < 1) return CT_ECONFIG;
    L.grid = (int)std::max<long long>(1, std::min<long long>((long long)per_sm * sms, L.items));
    plan->total_grid += L.grid;
    plan->max_smem = std::max(plan->max_smem, L.smem);
    plan->launches.push_back(std::move(L));
    return CT_OK;
  };
  int q = 0;
  for (int c = 0; c < kBatchClasses; ++c) {
    BatchClassLaunch L;
    L.cls = c;
    L.lo = q;
    int used = 0;  // floats of the parameter block in use
    for (; q < n && batch_class_of(table[q].k) == c; ++q) {
      table[q].tap_off = -1;
      if (!host_taps) continue;
      const int k = table[q].k, kp = (k + 3) / 4 * 4;
      if (used + k * kp > kBatchParamTaps) {  // this run is full: start the next
        L.hi = q;
        int rc = finish(L);
        if (rc != CT_OK) return rc;
        L = BatchClassLaunch();
        L.cls = c;
        L.lo = q;
        used = 0;
      }
      if ((int)plan->launches.size() + 2 < kBatchMaxLaunches) {
        table[q].tap_off = used;
        L.taps.resize(used + k * kp, 0.0f);
        for (int j = 0; j < k; ++j)
          for (int i = 0; i < k; ++i) L.taps[used + j * kp + i] = host_taps[q][j * k + i];
        used += k * kp;
      }
    }
    L.hi = q;
    int rc = finish(L);
    if (rc != CT_OK) return rc;
  }
  if ((int)plan->launches.size() > kBatchMaxLaunches) return CT_ENOTSUP;
  return CT_OK;
}

int enqueue_batch_plan(const BatchPlan& plan, const BatchImage* d_table, unsigned* counters,
                       unsigned* status, cudaStream_t s, const cudaStream_t* branches,
                       const cudaEvent_t* events, int n_branches) {
  const int nl = (int)plan.launches.size();
  if (nl == 0) return CT_OK;
  cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(unsigned) * nl, s);
  if (e != cudaSuccess) return cuda_status(e);
  // launch l runs on branch l % n_branches (when given): s forks after the
  // counter reset and joins every branch at the end
  const int nb = (branches && events) ? std::min(n_branches, nl) : 0;
  if (nb > 0 && (e = cudaEventRecord(events[nb], s)) != cudaSuccess) return cuda_status(e);
  for (int b = 0; b < nb; ++b)
    if ((e = cudaStreamWaitEvent(branches[b], events[nb], 0)) != cudaSuccess)
      return cuda_status(e);
  // the parameter block is copied into the launch (and into a captured graph)
  static thread_local BatchArgs a;
  for (int l = 0; l < nl; ++l) {
    const BatchClassLaunch& L = plan.launches[l];
    const cudaStream_t ls = nb > 0 ? branches[l % nb] : s;
    a.images = d_table + L.lo;
    a.n_images = L.n;
    a.n_items = L.items;
    a.item_base = L.item_base;
    a.counter = counters + l;
    a.status = status;
    a.buf_floats = L.buf_floats;
    a.claim_items = (unsigned)L.claim;
    if (!L.taps.empty()) memcpy(a.w, L.taps.data(), sizeof(float) * L.taps.size());
    if (L.cls == 0) batched_conv_kernel<0><<<L.grid, L.threads, L.smem, ls>>>(a);
    else if (L.cls == 1) batched_conv_kernel<1><<<L.grid, L.threads, L.smem, ls>>>(a);
    else batched_conv_kernel<2><<<L.grid, L.threads, L.smem, ls>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
  }
  for (int b = 0; b < nb; ++b)
    if ((e = cudaEventRecord(events[b], branches[b])) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, events[b], 0)) != cudaSuccess)
      return cuda_status(e);
  return CT_OK;
}
}  // namespace convtune

using namespace convtune;

struct ct_batch {
  int device = 0;
  std::vector<BatchImage> host_images;   // sorted by (k, class)
  std::vector<int> order;                // host image index of each table entry
  std::vector<ct_batch_item> items;      // caller's items (input order)
  std::vector<std::vector<float>> taps;  // host taps, input order
  BatchImage* d_images = nullptr;
  float* d_filters = nullptr;
  unsigned* d_counter = nullptr;
  long long n_items = 0;
  BatchPlan plan;        // class ranges, shared memory and grids
  size_t smem = 0;       // largest class's dynamic shared memory
  int grid = 0;          // CTAs over all class launches
  double flop = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  // branches of the captured graph (launch l on branch l % kBatchBranches),
  // so that one launch's last tiles overlap the next launch's first ones
  std::vector<cudaStream_t> branches;
  std::vector<cudaEvent_t> events;  // one per branch + the fork
  // launches graph: one single-image kernel per image, by filter side, then area
  std::vector<ct_problem> lprob;
  std::vector<ct_config> lcfg;
  cudaGraphExec_t exec_launch = nullptr;
  std::vector<cudaStream_t> lbranches;
  std::vector<cudaEvent_t> levents;  // one per branch + the fork
  int mode = CT_BATCH_PERSISTENT;    // the graph ct_batch_run replays
  ~ct_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (exec_launch) cudaGraphExecDestroy(exec_launch);
    for (cudaStream_t bs : lbranches) cudaStreamDestroy(bs);
    for (cudaEvent_t ev : levents) cudaEventDestroy(ev);
    for (cudaStream_t bs : branches) cudaStreamDestroy(bs);
    for (cudaEvent_t ev : events) cudaEventDestroy(ev);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    if (d_images) cudaFree(d_images);
    if (d_filters) cudaFree(d_filters);
    if (d_counter) cudaFree(d_counter);
  }
};

namespace {

// Enqueue one batched run: counter reset + one persistent kernel per class.
int enqueue_batch(ct_batch* b, cudaStream_t s) {
  if (b->n_items == 0) return CT_OK;
  int err = CT_OK;
  unsigned* status = device_status_word(&err);
  if (!status) return err;
  return enqueue_batch_plan(b->plan, b->d_images, b->d_counter, status, s,
                            b->branches.empty() ? nullptr : b->branches.data(),
                            b->events.empty() ? nullptr : b->events.data(),
                            (int)b->branches.size());
}

// The plain comparison: one ct_conv2d_run per image, configuration from the
// image's bucket (taps from the parameter space).
int enqueue_plain(ct_batch* b, cudaStream_t s) {
  for (size_t i = 0; i < b->host_images.size(); ++i) {
    const BatchImage& im = b->host_images[i];
    const ct_batch_item& it = b->items[b->order[i]];
    ct_problem p;
    p.in = it.in;
    p.in_pitch = it.in_pitch;
    p.filt = b->taps[b->order[i]].data();
    p.fh = p.fw = it.k;
    p.out = it.out;
    p.out_pitch = it.out_pitch;
    p.out_h = it.out_h;
    p.out_w = it.out_w;
    ct_config c;
    c.block_x = im.bx;
    c.block_y = im.threads / im.bx;
    c.tile_x = kBatchTileX;
    c.tile_y = std::min(im.ty, 4);  // (the single-image kernel's tiles are at most 4 high)
    c.staging = CT_STAGE_SMEM;
    c.filter_mem = CT_FILTER_CONST;
    c.vec_width = im.vw;
    const int rc = ct_conv2d_run(&p, &c, s);
    if (rc != CT_OK) return rc;
  }
  return CT_OK;
}

// Launches mode, one image: the bucket's block and tile height (defaults
// 16 x 8 threads, tile_y 4: the single-image kernel's energy optimum at
// 4096^2 / 17 x 17), taps in the parameter block, TMA staging with 4-wide
// loads where the buffers allow it, else shared-memory staging with the
// widest loads they allow.
int launch_config(const ct_batch_item& it, const float* taps, const ct_batch_tiles* tiles,
                  ct_problem* p, ct_config* c) {
  p->in = it.in;
  p->in_pitch = it.in_pitch;
  p->filt = taps;
  p->fh = p->fw = it.k;
  p->out = it.out;
  p->out_pitch = it.out_pitch;
  p->out_h = it.out_h;
  p->out_w = it.out_w;
  int bx = 16, by = 8, ty = 4;
  if (tiles) {
    const int cls = size_class(it.out_h, it.out_w);
    const int tbx = tiles->launch_block_x[cls][it.k], tby = tiles->launch_block_y[cls][it.k];
    const int tty = tiles->launch_tile_y[cls][it.k];
    if ((tbx == 16 || tbx == 32 || tbx == 64 || tbx == 128) &&
        (tby == 1 || tby == 2 || tby == 4 || tby == 8) && (tty == 1 || tty == 2 || tty == 4)) {
      bx = tbx;
      by = tby;
      ty = tty;
    }
  }
  const int stage[5] = {CT_STAGE_TMA, CT_STAGE_SMEM, CT_STAGE_SMEM, CT_STAGE_SMEM,
                        CT_STAGE_DIRECT};
  const int vec[5] = {4, 4, 2, 1, 1};
  int rc = CT_ECONFIG;
  for (int q = 0; q < 5; ++q) {
    c->block_x = bx;
    c->block_y = by;
    c->tile_x = kBatchTileX;
    c->tile_y = ty;
    c->staging = stage[q];
    c->filter_mem = CT_FILTER_CONST;
    c->vec_width = vec[q];
    if ((rc = ct_conv2d_check(p, c, nullptr, 0)) == CT_OK) return CT_OK;
  }
  return rc;
}

// The launches graph's work: fork `s` to the branches, one single-image
// launch per image (in the order above) on branch n % branches, join.
int enqueue_launches(ct_batch* b, cudaStream_t s) {
  const int nb = (int)b->lbranches.size();
  if (nb == 0) return CT_ENOTSUP;
  cudaError_t e = cudaEventRecord(b->levents[nb], s);
  if (e != cudaSuccess) return cuda_status(e);
  for (int q = 0; q < nb; ++q)
    if ((e = cudaStreamWaitEvent(b->lbranches[q], b->levents[nb], 0)) != cudaSuccess)
      return cuda_status(e);
  for (size_t n = 0; n < b->lprob.size(); ++n) {
    const int rc = ct_conv2d_run(&b->lprob[n], &b->lcfg[n], b->lbranches[n % nb]);
    if (rc != CT_OK) return rc;
  }
  for (int q = 0; q < nb; ++q)
    if ((e = cudaEventRecord(b->levents[q], b->lbranches[q])) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, b->levents[q], 0)) != cudaSuccess)
      return cuda_status(e);
  return CT_OK;
}

int build_batch(const ct_batch_item* items, int n, const ct_batch_tiles* tiles, ct_batch* b) {
  b->items.assign(items, items + n);
  b->taps.resize(n);
  std::vector<BatchImage> imgs;
  std::vector<int> order;
  for (int i = 0; i < n; ++i) {
    const ct_batch_item& it = items[i];
    if (!it.filt || it.k < 1 || it.k > kMaxK || (it.k & 1) == 0) return CT_EINVAL;
    if (it.out_h < 0 || it.out_w < 0) return CT_EINVAL;
    b->taps[i].assign(it.filt, it.filt + it.k * it.k);
    if (it.out_h == 0 || it.out_w == 0) continue;
    BatchImage im;
    const int rc = batch_image_from_item(it, tiles, &im);
    if (rc != CT_OK) return rc;
    imgs.push_back(im);
    order.push_back(i);
    b->flop += 2.0 * it.k * it.k * (double)it.out_h * it.out_w;
  }
  // bucket order: filter side, then size class, then input order
  std::vector<int> idx(imgs.size());
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
    const int cx = size_class(imgs[x].out_h, imgs[x].out_w);
    const int cy = size_class(imgs[y].out_h, imgs[y].out_w);
    return std::make_pair(imgs[x].k, cx) < std::make_pair(imgs[y].k, cy);
  });
  long long first = 0;
  size_t filt_floats = 0;
  for (int j : idx) {
    BatchImage im = imgs[j];
    im.first_item = first;
    first += (long long)im.tiles_x * im.tiles_y;
    filt_floats += (size_t)im.k * round_up(im.k, 4);
    b->host_images.push_back(im);
    b->order.push_back(order[j]);
  }
  b->n_items = first;
  // device copies: padded taps, then the table pointing at them
  cudaError_t e;
  std::vector<float> padded(std::max<size_t>(filt_floats, 1), 0.0f);
  size_t off = 0;
  std::vector<size_t> offs;
  for (size_t q = 0; q < b->host_images.size(); ++q) {
    const int k = b->host_images[q].k, kp = round_up(k, 4);
    const std::vector<float>& t = b->taps[b->order[q]];
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) padded[off + j * kp + i] = t[j * k + i];
    offs.push_back(off);
    off += (size_t)k * kp;
  }
  if ((e = cudaMalloc(&b->d_filters, sizeof(float) * padded.size())) != cudaSuccess)
    return cuda_status(e);
  if ((e = cudaMemcpy(b->d_filters, padded.data(), sizeof(float) * padded.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_status(e);
  for (size_t q = 0; q < b->host_images.size(); ++q) b->host_images[q].filt = b->d_filters + offs[q];
  // persistent grids: resident CTAs per SM x SMs per launch, capped by the
  // work; the plan also places the 13..17 taps in parameter blocks (it sets
  // tap_off, so the table goes to the device after it)
  std::vector<const float*> host_taps(b->host_images.size());
  for (size_t q = 0; q < b->host_images.size(); ++q) host_taps[q] = b->taps[b->order[q]].data();
  const int rc = plan_batch(b->host_images.data(), (int)b->host_images.size(), host_taps.data(),
                            &b->plan);
  if (rc != CT_OK) return rc;
  b->grid = b->plan.total_grid;
  b->smem = std::max<size_t>(b->plan.max_smem, 16);
  const size_t tb = sizeof(BatchImage) * std::max<size_t>(b->host_images.size(), 1);
  if ((e = cudaMalloc(&b->d_images, tb)) != cudaSuccess) return cuda_status(e);
  if (!b->host_images.empty() &&
      (e = cudaMemcpy(b->d_images, b->host_images.data(),
                      sizeof(BatchImage) * b->host_images.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
    return cuda_status(e);
  if ((e = cudaMalloc(&b->d_counter, kBatchCounterBytes)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaMemset(b->d_counter, 0, kBatchCounterBytes)) != cudaSuccess) return cuda_status(e);
  // launches mode: every image's problem and configuration, by filter side
  // (largest first), then by output area (largest first; stable: ties keep
  // input order).  Round-robin over the branches, the kernels running side
  // by side then mostly share one filter side's code in the instruction
  // caches (GB300, 256-image batch: 877-883 us, against 977-984 us with the
  // images ordered by work alone, sides mixed).
  if (b->host_images.size() <= (size_t)CT_BATCH_LAUNCH_MAX_IMAGES) {
    std::vector<int> by_work(b->order);
    std::stable_sort(by_work.begin(), by_work.end(), [&](int x, int y) {
      if (items[x].k != items[y].k) return items[x].k > items[y].k;
      return (double)items[x].out_h * items[x].out_w > (double)items[y].out_h * items[y].out_w;
    });
    for (int i : by_work) {
      ct_problem p;
      ct_config c;
      const int rc2 = launch_config(items[i], b->taps[i].data(), tiles, &p, &c);
      if (rc2 != CT_OK) return rc2;
      b->lprob.push_back(p);
      b->lcfg.push_back(c);
    }
  }
  return CT_OK;
}

// Capture the launches graph (batches of at most CT_BATCH_LAUNCH_MAX_IMAGES
// images).
int capture_launches(ct_batch* b) {
  if (b->lprob.empty()) return CT_OK;
  cudaError_t e;
  const size_t nb = std::min<size_t>(b->lprob.size(), kBatchLaunchBranches);
  for (size_t q = 0; q < nb; ++q) {
    cudaStream_t bs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_status(e);
    b->lbranches.push_back(bs);
  }
  for (size_t q = 0; q <= nb; ++q) {
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_status(e);
    b->levents.push_back(ev);
  }
  // one uncaptured run first: first-use kernel attributes and module loads
  // happen outside the capture
  int rc = enqueue_launches(b, b->capture_stream);
  if (rc != CT_OK) return rc;
  if ((e = cudaStreamSynchronize(b->capture_stream)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return cuda_status(e);
  rc = enqueue_launches(b, b->capture_stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->capture_stream, &g);
  if (rc != CT_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaGraphInstantiate(&b->exec_launch, g, 0);
  cudaGraphDestroy(g);
  return cuda_status(e);
}

int capture_batch(ct_batch* b) {
  // allocations are not allowed while capturing: make the status word exist
  int err = CT_OK;
  if (!device_status_word(&err)) return err;
  cudaError_t e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_status(e);
  const size_t nl = std::min<size_t>(b->plan.launches.size(), kBatchBranches);
  for (size_t l = 0; l < nl; ++l) {
    cudaStream_t bs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_status(e);
    b->branches.push_back(bs);
  }
  for (size_t l = 0; l <= nl; ++l) {
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_status(e);
    b->events.push_back(ev);
  }
  if ((e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return cuda_status(e);
  int rc = enqueue_batch(b, b->capture_stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->capture_stream, &g);
  if (rc != CT_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  return cuda_status(e);
}

}  // namespace

extern "C" {

int ct_batch_create(const ct_batch_item* items, int n, const ct_batch_tiles* tiles,
                    ct_batch** out) {
  if (!out || n < 0 || (n > 0 && !items)) return CT_EINVAL;
  *out = nullptr;
  ct_batch* b = new (std::nothrow) ct_batch();
  if (!b) return CT_ENOMEM;
  cudaError_t e = cudaGetDevice(&b->device);
  int rc = e == cudaSuccess ? build_batch(items, n, tiles, b) : cuda_status(e);
  if (rc == CT_OK) rc = capture_batch(b);
  const int req = tiles ? tiles->mode : CT_BATCH_AUTO;
  if (rc == CT_OK && req != CT_BATCH_PERSISTENT) rc = capture_launches(b);
  if (rc == CT_OK) {
    double px = 0;
    for (const BatchImage& im : b->host_images) px += (double)im.out_h * im.out_w;
    const bool big = !b->host_images.empty() && px >= 65536.0 * b->host_images.size();
    if (req == CT_BATCH_LAUNCHES)
      rc = b->exec_launch || b->host_images.empty() ? CT_OK : CT_ENOTSUP;
    else if (req != CT_BATCH_AUTO && req != CT_BATCH_PERSISTENT)
      rc = CT_EINVAL;
    b->mode = (req == CT_BATCH_LAUNCHES || (req == CT_BATCH_AUTO && big)) && b->exec_launch
                  ? CT_BATCH_LAUNCHES
                  : CT_BATCH_PERSISTENT;
  }
  if (rc != CT_OK) {
    delete b;
    return rc;
  }
  *out = b;
  return CT_OK;
}

int ct_batch_run(ct_batch* b, void* stream) {
  if (!b) return CT_EINVAL;
  if (b->n_items == 0) return CT_OK;
  return cuda_status(cudaGraphLaunch(b->mode == CT_BATCH_LAUNCHES ? b->exec_launch : b->exec,
                                     (cudaStream_t)stream));
}

int ct_batch_run_mode(ct_batch* b, int which, void* stream) {
  if (!b) return CT_EINVAL;
  switch (which) {
    case CT_BATCH_RUN_DEFAULT:
      return ct_batch_run(b, stream);
    case CT_BATCH_RUN_PLAIN:
      return enqueue_plain(b, (cudaStream_t)stream);
    case CT_BATCH_RUN_PERSISTENT:
      if (b->n_items == 0) return CT_OK;
      return cuda_status(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    case CT_BATCH_RUN_LAUNCHES:
      if (b->n_items == 0) return CT_OK;
      if (!b->exec_launch) return CT_ENOTSUP;
      return cuda_status(cudaGraphLaunch(b->exec_launch, (cudaStream_t)stream));
    default:
      return CT_EINVAL;
  }
}

int ct_batch_run_plain(ct_batch* b, void* stream) {
  if (!b) return CT_EINVAL;
  return enqueue_plain(b, (cudaStream_t)stream);
}

int ct_batch_info(const ct_batch* b, ct_batch_stats* st) {
  if (!b || !st) return CT_EINVAL;
  memset(st, 0, sizeof(*st));
  st->n_images = (int)b->host_images.size();
  st->n_items = b->n_items;
  st->grid = b->grid;
  st->smem_bytes = (long)b->smem;
  st->flop = b->flop;
  st->launches = (int)b->plan.launches.size();
  st->mode = b->mode;
  st->has_launch_graph = b->exec_launch ? 1 : 0;
  for (const BatchImage& im : b->host_images)
    st->bytes += 4.0 * ((double)im.in_h * im.in_w + (double)im.out_h * im.out_w + im.k * im.k);
  return CT_OK;
}

int ct_batch_destroy(ct_batch* b) {
  if (!b) return CT_OK;
  cudaStreamSynchronize(b->capture_stream);
  delete b;
  return CT_OK;
}

int ct_measure_batch(ct_batch* b, int which, const ct_measure_options* opt, void* stream,
                     ct_record* out) {
  if (!b || !out) return CT_EINVAL;
  if (b->n_items == 0) return CT_EINVAL;
  if (which == CT_BATCH_RUN_DEFAULT)
    which = b->mode == CT_BATCH_LAUNCHES ? CT_BATCH_RUN_LAUNCHES : CT_BATCH_RUN_PERSISTENT;
  if (which == CT_BATCH_RUN_LAUNCHES && !b->exec_launch) return CT_ENOTSUP;
  if (which < CT_BATCH_RUN_PLAIN || which > CT_BATCH_RUN_LAUNCHES) return CT_EINVAL;
  MeasureUnit u;
  u.kind = CT_UNIT_CONV;
  u.work = b->flop;
  u.eager = which == CT_BATCH_RUN_PLAIN;
  if (which == CT_BATCH_RUN_PLAIN)
    u.launch = [b](cudaStream_t s) { return enqueue_plain(b, s); };
  else if (which == CT_BATCH_RUN_LAUNCHES)
    u.launch = [b](cudaStream_t s) { return enqueue_launches(b, s); };
  else
    u.launch = [b](cudaStream_t s) { return enqueue_batch(b, s); };
  return measure_unit(u, resolve_options(opt), platform_ops(), (cudaStream_t)stream, 0, out);
}

int ct_batch_tune(const ct_batch_item* items, int n, int objective,
                  const ct_measure_options* opt, void* stream, ct_batch_tiles* tiles,
                  ct_record* records, int cap, int* n_records) {
  if (!items || n <= 0 || !tiles || !n_records) return CT_EINVAL;
  if (objective < CT_OBJ_TIME || objective > CT_OBJ_GFLOPS_PER_W) return CT_EINVAL;
  // start from the caller's table: its class CTA sizes and claim sizes are
  // kept, its valid tiles are the starting point of the search
  ct_batch_tiles cur;
  memset(&cur, 0, sizeof(cur));
  // (the launches-mode fields and the mode pass through unchanged)
  memcpy(cur.launch_block_x, tiles->launch_block_x, sizeof(cur.launch_block_x));
  memcpy(cur.launch_block_y, tiles->launch_block_y, sizeof(cur.launch_block_y));
  memcpy(cur.launch_tile_y, tiles->launch_tile_y, sizeof(cur.launch_tile_y));
  cur.mode = tiles->mode;
  for (int c = 0; c < kBatchClasses; ++c) {
    cur.class_threads[c] = batch_valid_threads(tiles->class_threads[c]) ? tiles->class_threads[c] : 0;
    cur.claim_items[c] =
        tiles->claim_items[c] >= 1 && tiles->claim_items[c] <= 8 ? tiles->claim_items[c] : 0;
  }
  for (int sc = 0; sc < 2; ++sc)
    for (int k = 1; k <= kMaxK; k += 2)
      if (valid_tile(tiles->block_x[sc][k], tiles->tile_y[sc][k], k, class_threads(&cur, k))) {
        cur.block_x[sc][k] = tiles->block_x[sc][k];
        cur.tile_y[sc][k] = tiles->tile_y[sc][k];
      }
  const ct_measure_options mo = resolve_options(opt);
  const ct_platform_ops ops = platform_ops();
  std::vector<std::vector<int>> bucket(2 * (kMaxK + 1));
  std::vector<std::vector<int>> klass(kBatchClasses);
  for (int i = 0; i < n; ++i) {
    if (items[i].out_h <= 0 || items[i].out_w <= 0) continue;
    if (items[i].k < 1 || items[i].k > kMaxK || !(items[i].k & 1)) return CT_EINVAL;
    bucket[size_class(items[i].out_h, items[i].out_w) * (kMaxK + 1) + items[i].k].push_back(i);
    klass[batch_class_of(items[i].k)].push_back(i);
  }
  const int bxs[4] = {16, 32, 64, 128}, tys[4] = {1, 2, 4, 8};
  auto n_ty = [](int k) { return k <= kBatchMaxK8 ? 4 : 3; };
  int written = 0, needed = 0;
  for (size_t q = 0; q < bucket.size(); ++q)
    needed += bucket[q].empty() ? 0 : 4 * n_ty((int)(q % (kMaxK + 1)));
  *n_records = needed;
  if (records && cap < needed) return CT_ENOMEM;
  // One bucket (size class, filter side) at a time, each candidate tile
  // measured on the whole filter-side class the bucket belongs to, with the
  // class's other buckets at their current tiles: a class launch's staging
  // buffers and occupancy follow its largest tile, so a tile that is best
  // for its bucket alone can slow the rest of its class (measured on the
  // 256-image batch: tuning buckets alone gave a 9 % slower batch).
  for (int c = 0; c < kBatchClasses; ++c) {
    if (klass[c].empty()) continue;
    std::vector<ct_batch_item> sub;
    for (int i : klass[c]) sub.push_back(items[i]);
    for (int k = 1; k <= kMaxK; k += 2) {
      if (batch_class_of(k) != c) continue;
      for (int sc = 0; sc < 2; ++sc) {
        if (bucket[sc * (kMaxK + 1) + k].empty()) continue;
        std::vector<ct_record> recs;
        for (int bx : bxs)
          for (int qt = 0; qt < n_ty(k); ++qt) {
            const int ty = tys[qt];
            ct_batch_tiles t = cur;
            t.mode = CT_BATCH_PERSISTENT;  // (no launches graph to capture)
            if (bx > class_threads(&t, k)) continue;  // wider than the CTA
            t.block_x[sc][k] = bx;
            t.tile_y[sc][k] = ty;
            ct_batch* b = nullptr;
            int rc = ct_batch_create(sub.data(), (int)sub.size(), &t, &b);
            if (rc != CT_OK) return rc;
            MeasureUnit u;
            u.kind = CT_UNIT_CONV;
            u.work = b->flop;
            u.launch = [b](cudaStream_t s) { return enqueue_batch(b, s); };
            ct_record r;
            rc = measure_unit(u, mo, ops, (cudaStream_t)stream, 0, &r);
            ct_batch_destroy(b);
            if (rc != CT_OK) return rc;
            r.cfg.block_x = bx;
            r.cfg.block_y = class_threads(&t, k) / bx;
            r.cfg.tile_x = kBatchTileX;
            r.cfg.tile_y = ty;
            r.cfg.staging = CT_STAGE_TMA;
            r.cfg.filter_mem = CT_FILTER_SHARED;  // taps staged into shared memory
            r.cfg.vec_width = 4;
            recs.push_back(r);
            if (records) records[written] = r;
            ++written;
          }
        int best = 0;
        ct_select_best(recs.data(), (int)recs.size(), objective, nullptr, 0, &best);
        if (best < 0) best = 0;
        cur.block_x[sc][k] = recs[best].cfg.block_x;
        cur.tile_y[sc][k] = recs[best].cfg.tile_y;
      }
    }
  }
  *tiles = cur;
  *n_records = written;
  return CT_OK;
}

int ct_batch_tune_launches(const ct_batch_item* items, int n, int objective,
                           const ct_measure_options* opt, void* stream, ct_batch_tiles* tiles,
                           ct_record* records, int cap, int* n_records) {
  if (!items || n <= 0 || !tiles || !n_records) return CT_EINVAL;
  if (objective < CT_OBJ_TIME || objective > CT_OBJ_GFLOPS_PER_W) return CT_EINVAL;
  std::vector<std::vector<int>> bucket(2 * (kMaxK + 1));
  for (int i = 0; i < n; ++i) {
    if (items[i].out_h <= 0 || items[i].out_w <= 0) continue;
    if (items[i].k < 1 || items[i].k > kMaxK || !(items[i].k & 1)) return CT_EINVAL;
    bucket[size_class(items[i].out_h, items[i].out_w) * (kMaxK + 1) + items[i].k].push_back(i);
  }
  int needed = 0;
  for (const auto& v : bucket) needed += v.empty() ? 0 : kLaunchCandidates;
  *n_records = needed;
  if (records && cap < needed) return CT_ENOMEM;
  const ct_measure_options mo = resolve_options(opt);
  ct_batch_tiles cur = *tiles;
  int written = 0;
  for (int sc = 0; sc < 2; ++sc)
    for (int k = 1; k <= kMaxK; k += 2) {
      const std::vector<int>& v = bucket[sc * (kMaxK + 1) + k];
      if (v.empty()) continue;
      std::vector<ct_batch_item> sub;
      for (int i : v) sub.push_back(items[i]);
      std::vector<ct_record> recs;
      for (int q = 0; q < kLaunchCandidates; ++q) {
        ct_batch_tiles t = cur;
        t.mode = CT_BATCH_LAUNCHES;
        t.launch_block_x[sc][k] = kLaunchCand[q][0];
        t.launch_block_y[sc][k] = kLaunchCand[q][1];
        t.launch_tile_y[sc][k] = kLaunchCand[q][2];
        ct_batch* b = nullptr;
        int rc = ct_batch_create(sub.data(), (int)sub.size(), &t, &b);
        if (rc != CT_OK) return rc;
        ct_record r;
        rc = ct_measure_batch(b, CT_BATCH_RUN_LAUNCHES, &mo, stream, &r);
        // the configuration the bucket's first image ran with (its staging
        // may have fallen back from TMA)
        const ct_config c = b->lcfg.empty() ? ct_config{} : b->lcfg.front();
        ct_batch_destroy(b);
        if (rc != CT_OK) return rc;
        r.cfg = c;
        recs.push_back(r);
        if (records) records[written] = r;
        ++written;
      }
      int best = 0;
      ct_select_best(recs.data(), (int)recs.size(), objective, nullptr, 0, &best);
      if (best < 0) best = 0;
      cur.launch_block_x[sc][k] = kLaunchCand[best][0];
      cur.launch_block_y[sc][k] = kLaunchCand[best][1];
      cur.launch_tile_y[sc][k] = kLaunchCand[best][2];
    }
  *tiles = cur;
  *n_records = written;
  return CT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched correlation without any device allocation.
//
// Some callers cannot allocate device memory: code running where a framework
// or memory pool owns all of the GPU's memory, or under a policy that forbids
// cudaMalloc after start-up (allocation can synchronise the device and fail
// under memory pressure at the worst moment).  For them the batched kernel
// also runs out of a fixed scratch area compiled into the library: a
// file-scope device array that every GPU loading the library holds until the
// process exits.  The caller still owns and passes the inputs and outputs.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxImages = 256;
constexpr int kNoAllocTapFloats = kMaxK * ((kMaxK + 3) / 4 * 4);  // 17 rows of 20
constexpr size_t kNoAllocHeaderBytes = kBatchCounterBytes;  // work counters, status word
constexpr size_t kNoAllocTableBytes = sizeof(BatchImage) * kNoAllocMaxImages;
constexpr size_t kNoAllocTapBytes = sizeof(float) * (size_t)kNoAllocTapFloats * kNoAllocMaxImages;
constexpr size_t kNoAllocBytes = kNoAllocHeaderBytes + kNoAllocTableBytes + kNoAllocTapBytes;

struct NoAllocDevice {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of the scratch array
};

std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];
// host mirror of the scratch's table and tap regions, per thread: one copy
// sends the image table and the padded taps of a call
struct NoAllocHostBlock {
  BatchImage table[kNoAllocMaxImages];
  float taps[(size_t)kNoAllocTapFloats * kNoAllocMaxImages];
};
static_assert(sizeof(BatchImage) * kNoAllocMaxImages == kNoAllocTableBytes, "table region");
thread_local NoAllocHostBlock t_noalloc_host;

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

// Once per device, with that device current: resolve the array's device
// address.
int noalloc_device(NoAllocDevice* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= 64) return CT_ENOTSUP;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return cuda_status(e);
    d.base = static_cast<unsigned char*>(p);
    d.ready = true;
  }
  *out = d;
  return CT_OK;
}

// The status word sits in the last word of the counter header.
unsigned* noalloc_status_word(const NoAllocDevice& nd) {
  return reinterpret_cast<unsigned*>(nd.base) + kBatchMaxLaunches;
}

}  // namespace

extern "C" int ct_batch_run_noalloc(const ct_batch_item* items, int n,
                                    const ct_batch_tiles* tiles, void* stream) {
  if (n < 0 || (n > 0 && !items)) return CT_EINVAL;
  if (n > kNoAllocMaxImages) {
    set_last_error("ct_batch_run_noalloc: more images than the fixed scratch holds (limit 256)");
    return CT_EINVAL;
  }
  NoAllocDevice nd;
  int rc = noalloc_device(&nd);
  if (rc != CT_OK) return rc;

  // validate, and order the images by (filter side, size class)
  int idx[kNoAllocMaxImages];
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const ct_batch_item& it = items[i];
    if (!it.filt || it.k < 1 || it.k > kMaxK || (it.k & 1) == 0) return CT_EINVAL;
    if (it.out_h < 0 || it.out_w < 0) return CT_EINVAL;
    if (it.out_h == 0 || it.out_w == 0) continue;
    if (!it.in || !it.out) return CT_EINVAL;
    if (it.in_pitch < (long)it.out_w + it.k - 1 || it.out_pitch < it.out_w) return CT_EINVAL;
    if ((long long)it.out_w + it.k > (1LL << 30) || (long long)it.out_h + it.k > (1LL << 30))
      return CT_EINVAL;
    int q = m++;
    const int key = it.k * 2 + size_class(it.out_h, it.out_w);
    while (q > 0) {  // stable insertion by key
      const ct_batch_item& prev = items[idx[q - 1]];
      if (prev.k * 2 + size_class(prev.out_h, prev.out_w) <= key) break;
      idx[q] = idx[q - 1];
      --q;
    }
    idx[q] = i;
  }
  if (m == 0) return CT_OK;

  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  // header: one work counter per launch, the status word in its last word
  unsigned* counters = reinterpret_cast<unsigned*>(nd.base);
  unsigned* status = noalloc_status_word(nd);
  BatchImage* d_table = reinterpret_cast<BatchImage*>(nd.base + kNoAllocHeaderBytes);
  float* d_taps = reinterpret_cast<float*>(nd.base + kNoAllocHeaderBytes + kNoAllocTableBytes);
  NoAllocHostBlock& hb = t_noalloc_host;
  long long first = 0;
  for (int q = 0; q < m; ++q) {
    const ct_batch_item& it = items[idx[q]];
    BatchImage& im = hb.table[q];
    rc = batch_image_from_item(it, tiles, &im);
    if (rc != CT_OK) return rc;
    im.first_item = first;
    first += (long long)im.tiles_x * im.tiles_y;
    // taps: k rows padded to round_up(k, 4) floats (the padding is never used
    // as a tap) in this image's slot of the tap region
    const int kp = round_up(it.k, 4);
    float* slot = hb.taps + (size_t)q * kNoAllocTapFloats;
    for (int j = 0; j < it.k; ++j)
      for (int i = 0; i < kp; ++i) slot[j * kp + i] = i < it.k ? it.filt[j * it.k + i] : 0.0f;
    im.filt = d_taps + (size_t)q * kNoAllocTapFloats;
  }
  // the plan places taps in parameter blocks where they fit (it sets tap_off,
  // so the table goes to the device after it)
  const float* host_taps[kNoAllocMaxImages];
  for (int q = 0; q < m; ++q) host_taps[q] = items[idx[q]].filt;
  BatchPlan plan;
  rc = plan_batch(hb.table, m, host_taps, &plan);
  if (rc != CT_OK) return rc;
  // one copy: the whole table region, then the m tap slots right behind it
  // (the two regions are adjacent in the scratch and in the host mirror)
  static_assert(offsetof(NoAllocHostBlock, taps) == kNoAllocTableBytes, "host mirror layout");
  const size_t bytes = kNoAllocTableBytes + sizeof(float) * (size_t)kNoAllocTapFloats * m;
  if ((e = cudaMemcpyAsync(d_table, &hb, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_status(e);
  // the counters are zeroed with the launches; the status word (zero when
  // the library loads) keeps its bits until ct_batch_noalloc_status clears it
  return enqueue_batch_plan(plan, d_table, counters, status, s);
}

extern "C" int ct_batch_noalloc_status(unsigned* bits, int clear, void* stream) {
  if (!bits) return CT_EINVAL;
  NoAllocDevice nd;
  int rc = noalloc_device(&nd);
  if (rc != CT_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* status = noalloc_status_word(nd);
  cudaError_t e = cudaMemcpyAsync(bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && clear) e = cudaMemsetAsync(status, 0, sizeof(unsigned), s);
  return cuda_status(e);
}

// ---------------------------------------------------------------------------
// Helpers for other units of the library (the request server) that build
// batch tables in their own memory and launch the batched kernel.
// ---------------------------------------------------------------------------
namespace convtune {

int batch_image_from_item(const ct_batch_item& it, const ct_batch_tiles* tiles, BatchImage* im) {
  if (!it.filt || it.k < 1 || it.k > kMaxK || (it.k & 1) == 0) return CT_EINVAL;
  if (it.out_h <= 0 || it.out_w <= 0 || !it.in || !it.out) return CT_EINVAL;
  if (it.in_pitch < (long)it.out_w + it.k - 1 || it.out_pitch < it.out_w) return CT_EINVAL;
  if ((long long)it.out_w + it.k > (1LL << 30) || (long long)it.out_h + it.k > (1LL << 30))
    return CT_EINVAL;
  memset(im, 0, sizeof(*im));
  im->tap_off = -1;
  im->in = it.in;
  im->out = it.out;
  im->in_pitch = it.in_pitch;
  im->out_pitch = it.out_pitch;
  im->in_h = it.out_h + it.k - 1;
  im->in_w = it.out_w + it.k - 1;
  im->out_h = it.out_h;
  im->out_w = it.out_w;
  im->k = it.k;
  const int cls = size_class(it.out_h, it.out_w);
  const int threads = class_threads(tiles, it.k);
  int bx = 32, ty = 2;
  if (tiles && valid_tile(tiles->block_x[cls][it.k], tiles->tile_y[cls][it.k], it.k, threads)) {
    bx = tiles->block_x[cls][it.k];
    ty = tiles->tile_y[cls][it.k];
  }
  im->bx = bx;
  im->ty = ty;
  im->threads = threads;
  im->claim = class_claim(tiles, it.k);
  const bool aligned = (uintptr_t)it.in % 16 == 0 && it.in_pitch % 4 == 0 &&
                       (uintptr_t)it.out % 16 == 0 && it.out_pitch % 4 == 0;
  im->vw = aligned ? 4 : 1;
  im->tiles_x = (it.out_w + bx * kBatchTileX - 1) / (bx * kBatchTileX);
  const int rows = batch_item_rows(it.k, bx, ty, threads);
  im->tiles_y = (it.out_h + rows - 1) / rows;
  im->g = batch_stage_geom(it.k, bx, ty, threads);
  // TMA staging wants a 16-byte aligned input and row stride; the box
  // (<= 144 x 144 floats here) is within the 256-element limit
  const bool in_aligned = (uintptr_t)it.in % 16 == 0 && it.in_pitch % 4 == 0;
  auto enc = in_aligned ? tensor_map_encoder() : nullptr;
  if (enc) {
    const cuuint64_t dims[2] = {(cuuint64_t)im->in_w, (cuuint64_t)im->in_h};
    const cuuint64_t strides[1] = {(cuuint64_t)it.in_pitch * 4};
    const cuuint32_t box[2] = {(cuuint32_t)im->g.box_w, (cuuint32_t)im->g.tile_h};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&im->tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)it.in, dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    im->use_tma = r == CUDA_SUCCESS ? 1 : 0;
  }
  return CT_OK;
}

}  // namespace convtune
