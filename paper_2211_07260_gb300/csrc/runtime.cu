// libconvtune runtime: validation and launch of the tuned correlation, the
// device status word, the host-buffer entry point and device facts.
#include <cudaTypedefs.h>
#include <limits.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <set>
#include <vector>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "runtime.h"

namespace convtune {

namespace {

struct DeviceState {
  unsigned* status = nullptr;
  int smem_optin = 0;
  int sm_count = 0;
  std::set<const void*> smem_raised;  // kernels whose dynamic shared-memory cap is raised
  // buffers of the host-buffer entry point: two sets, used by alternate
  // calls, so that a call's copies in overlap the previous call's kernels
  // and copies out
  float* din[2] = {nullptr, nullptr};
  size_t din_bytes[2] = {0, 0};
  float* dout[2] = {nullptr, nullptr};
  size_t dout_bytes[2] = {0, 0};
  int host_slot = 0;  // the set the next call uses
  // streams and events of the pipelined host-buffer entry point
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  cudaEvent_t ev_slot_k[2] = {nullptr, nullptr};    // last kernel of the set's last call
  cudaEvent_t ev_slot_out[2] = {nullptr, nullptr};  // last copy out of the set's last call
  std::vector<cudaEvent_t> ev_in, ev_k;
};

constexpr int kHostMaxBands = 64;

std::mutex g_mu;        // guards g_dev
std::mutex g_host_mu;   // serialises the host-buffer entry point
std::map<int, DeviceState> g_dev;

DeviceState* current_state(int* dev_out, int* err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *err = cuda_status(e);
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceState& st = g_dev[dev];
  if (st.smem_optin == 0) {
    int v = 0;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) {
      *err = cuda_status(e);
      return nullptr;
    }
    st.smem_optin = v;
    e = cudaDeviceGetAttribute(&st.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      *err = cuda_status(e);
      return nullptr;
    }
  }
  if (dev_out) *dev_out = dev;
  *err = CT_OK;
  return &st;
}

const void* pick_specialised(int k, int tx, int ty, bool staged, bool fs, bool big) {
  switch (k) {
    case 1: return pick_k1(tx, ty, staged, fs, big);
    case 3: return pick_k3(tx, ty, staged, fs, big);
    case 5: return pick_k5(tx, ty, staged, fs, big);
    case 7: return pick_k7(tx, ty, staged, fs, big);
    case 9: return pick_k9(tx, ty, staged, fs, big);
    case 11: return pick_k11(tx, ty, staged, fs, big);
    case 13: return pick_k13(tx, ty, staged, fs, big);
    case 15: return pick_k15(tx, ty, staged, fs, big);
    case 17: return pick_k17(tx, ty, staged, fs, big);
    default: return nullptr;
  }
}

KernelLauncher launcher_for(int k) {
  switch (k) {
    case 1: return launch_k1;
    case 3: return launch_k3;
    case 5: return launch_k5;
    case 7: return launch_k7;
    case 9: return launch_k9;
    case 11: return launch_k11;
    case 13: return launch_k13;
    case 15: return launch_k15;
    case 17: return launch_k17;
    default: return nullptr;
  }
}

inline int round_up(int x, int a) { return (x + a - 1) / a * a; }
inline bool one_of_124(int v) { return v == 1 || v == 2 || v == 4; }

// Raise a kernel's dynamic shared-memory cap to the device's opt-in limit
// once (the attribute is per kernel: setting it per launch size would let a
// smaller later value break an earlier, larger plan).  Caller holds g_mu.
cudaError_t raise_smem_cap(DeviceState* st, const void* fn) {
  if (st->smem_raised.count(fn)) return cudaSuccess;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           st->smem_optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) st->smem_raised.insert(fn);
  return e;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

namespace {
thread_local char g_last_error[256] = "";
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return CT_OK;
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e),
           cudaGetErrorString(e));
  if (e == cudaErrorInvalidConfiguration || e == cudaErrorLaunchOutOfResources) {
    cudaGetLastError();
    return CT_ECONFIG;
  }
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return CT_ENOMEM;
  }
  cudaGetLastError();
  return CT_ECUDA;
}

unsigned* device_status_word(int* err) {
  DeviceState* st = current_state(nullptr, err);
  if (!st) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!st->status) {
    unsigned* p = nullptr;
    cudaError_t e = cudaMalloc(&p, 256);
    if (e == cudaSuccess) e = cudaMemset(p, 0, 256);
    if (e != cudaSuccess) {
      *err = cuda_status(e);
      return nullptr;
    }
    st->status = p;
  }
  return st->status;
}

double conv_flop(const ct_problem& p) {
  return 2.0 * p.fh * p.fw * (double)p.out_h * (double)p.out_w;
}

double conv_bytes(const ct_problem& p) {
  const double in_elems = (double)(p.out_h + p.fh - 1) * (double)(p.out_w + p.fw - 1);
  return 4.0 * (in_elems + (double)p.out_h * p.out_w + (double)p.fh * p.fw);
}

int plan_conv(const ct_problem& p, const ct_config& c, ConvPlan* plan, std::string* why,
              bool device_checks) {
  auto fail = [&](int code, const char* msg) {
    if (why) *why = msg;
    return code;
  };
  *plan = ConvPlan{};
  if (p.out_h < 0 || p.out_w < 0) return fail(CT_EINVAL, "negative output size");
  if (!p.filt) return fail(CT_EINVAL, "null filter");
  if (p.fh < 1 || p.fw < 1 || p.fh > 32 || p.fw > 32 || p.fh * p.fw > kGenericMaxTaps)
    return fail(CT_EINVAL, "filter sides must be 1..32 with fh*fw <= 1024");
  if (p.out_h == 0 || p.out_w == 0) {
    plan->empty = true;
    return CT_OK;
  }
  if (!p.in || !p.out) return fail(CT_EINVAL, "null input or output");
  const long long in_w = (long long)p.out_w + p.fw - 1;
  const long long in_h = (long long)p.out_h + p.fh - 1;
  if (in_w > (1LL << 30) || in_h > (1LL << 30)) return fail(CT_EINVAL, "problem too large");
  if (p.in_pitch < in_w) return fail(CT_EINVAL, "in_pitch < out_w + fw - 1");
  if (p.out_pitch < p.out_w) return fail(CT_EINVAL, "out_pitch < out_w");

  if (c.block_x < 16 || c.block_x > 1024 || (c.block_x != 16 && c.block_x % 32 != 0))
    return fail(CT_ECONFIG, "block_x must be 16 or a multiple of 32, <= 1024");
  if (c.block_y < 1 || c.block_x * c.block_y > 1024)
    return fail(CT_ECONFIG, "block_x * block_y must be 16..1024");
  if (!one_of_124(c.tile_x) || !one_of_124(c.tile_y)) return fail(CT_ECONFIG, "tile sides 1, 2, 4");
  if (c.staging < CT_STAGE_DIRECT || c.staging > CT_STAGE_TMA) return fail(CT_ECONFIG, "staging");
  if (c.filter_mem != CT_FILTER_SHARED && c.filter_mem != CT_FILTER_CONST)
    return fail(CT_ECONFIG, "filter_mem");
  if (!one_of_124(c.vec_width)) return fail(CT_ECONFIG, "vec_width 1, 2, 4");

  ConvLaunch& L = plan->L;
  L.in = p.in;
  L.out = p.out;
  L.in_pitch = p.in_pitch;
  L.out_pitch = p.out_pitch;
  L.in_h = (int)in_h;
  L.in_w = (int)in_w;
  L.out_h = p.out_h;
  L.out_w = p.out_w;
  L.fh = p.fh;
  L.fw = p.fw;
  L.taps = p.filt;
  L.bx = c.block_x;
  L.by = c.block_y;

  const bool specialised = p.fh == p.fw && (p.fh & 1) && p.fh <= kMaxK;
  plan->specialised = specialised;
  plan->block = dim3(c.block_x, c.block_y);
  if (!specialised) {
    L.tx = L.ty = 1;
    L.staging = kStageDirect;
    L.filt_smem = 1;
    L.vw = 1;
    L.smem_bytes = sizeof(float) * p.fh * p.fw;
    plan->fn = pick_generic();
    plan->grid = dim3((p.out_w + c.block_x - 1) / c.block_x, (p.out_h + c.block_y - 1) / c.block_y);
  } else {
    const int K = p.fh;
    L.tx = c.tile_x;
    L.ty = c.tile_y;
    L.staging = c.staging;
    L.filt_smem = c.filter_mem == CT_FILTER_SHARED;
    L.vw = c.vec_width;
    const bool staged = c.staging != CT_STAGE_DIRECT;
    plan->fn = pick_specialised(K, c.tile_x, c.tile_y, staged, L.filt_smem != 0,
                                c.block_x * c.block_y >= kRingRemFirstThreads);
    if (!plan->fn) return fail(CT_ECONFIG, "variant not compiled");
    plan->grid = dim3((p.out_w + c.block_x * c.tile_x - 1) / (c.block_x * c.tile_x),
                      (p.out_h + c.block_y * c.tile_y - 1) / (c.block_y * c.tile_y));
    const int lw = staged ? c.vec_width : (c.vec_width < c.tile_x ? c.vec_width : c.tile_x);
    const int sw = c.vec_width < c.tile_x ? c.vec_width : c.tile_x;
    if (lw > 1 && ((uintptr_t)p.in % (4 * lw) != 0 || p.in_pitch % lw != 0))
      return fail(CT_ECONFIG, "input pointer / pitch not aligned to the load width");
    if (sw > 1 && ((uintptr_t)p.out % (4 * sw) != 0 || p.out_pitch % sw != 0))
      return fail(CT_ECONFIG, "output pointer / pitch not aligned to the store width");
    size_t smem = L.filt_smem ? sizeof(float) * round_up(K * round_up(K, 4), 32) : 0;
    if (staged) {
      L.tile_w = round_up(c.block_x * c.tile_x + K - 1, 4);
      L.tile_h = c.block_y * c.tile_y + K - 1;
      L.group_x = c.block_x;
      L.group_stride = 0;
      L.groups = 1;
      if (c.staging == CT_STAGE_TMA) {
        if (L.tile_h > 256) return fail(CT_ECONFIG, "TMA box taller than 256 elements");
        if ((uintptr_t)p.in % 16 != 0 || (p.in_pitch * 4) % 16 != 0)
          return fail(CT_ECONFIG, "TMA needs a 16-byte aligned input and row stride");
        // a tile wider than one 256-float box: one box per group of
        // threads in x, each with its own halo (the widest power-of-two
        // group whose box fits)
        while (L.tile_w > 256 && L.group_x > 1) {
          L.group_x /= 2;
          L.tile_w = round_up(L.group_x * c.tile_x + K - 1, 4);
        }
        if (L.tile_w > 256) return fail(CT_ECONFIG, "TMA box wider than 256 elements");
        L.groups = c.block_x / L.group_x;
        L.smem_pitch = L.tile_w;
        L.group_stride = L.groups > 1 ? round_up(L.tile_w * L.tile_h, 32) : 0;
        smem += sizeof(float) * (size_t)(L.groups > 1 ? L.groups * L.group_stride
                                                       : L.tile_h * L.smem_pitch);
      } else {
        L.smem_pitch = L.tile_w;
        // half-warp rows of 16 lanes reading 4-byte words: put consecutive
        // tile rows 16 banks apart
        if (c.block_x == 16 && c.tile_x == 1)
          while (L.smem_pitch % 32 != 16) L.smem_pitch += 4;
        smem += sizeof(float) * (size_t)L.tile_h * L.smem_pitch;
      }
    }
    L.smem_bytes = smem;
  }
  if (plan->grid.y > 65535u) return fail(CT_ECONFIG, "grid y exceeds 65535");

  if (!device_checks) return CT_OK;
  // device-dependent checks
  int err = CT_OK;
  DeviceState* st = current_state(nullptr, &err);
  if (!st) return fail(err, "no CUDA device");
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, plan->fn);
  if (e != cudaSuccess) return fail(cuda_status(e), "cudaFuncGetAttributes failed");
  if (c.block_x * c.block_y > fa.maxThreadsPerBlock)
    return fail(CT_ECONFIG, "block larger than the kernel's register budget allows");
  if (L.smem_bytes + fa.sharedSizeBytes > (size_t)st->smem_optin)
    return fail(CT_ECONFIG, "shared memory exceeds the per-block limit");
  if (c.staging == CT_STAGE_TMA && specialised && !tensor_map_encoder())
    return fail(CT_ENOTSUP, "cuTensorMapEncodeTiled unavailable");
  return CT_OK;
}

int prime_conv_kernel(int k, const ct_config& c) {
  if (k < 1 || k > kMaxK || !(k & 1)) return CT_EINVAL;
  const void* fn = pick_specialised(k, c.tile_x, c.tile_y, c.staging != CT_STAGE_DIRECT,
                                    c.filter_mem == CT_FILTER_SHARED,
                                    c.block_x * c.block_y >= kRingRemFirstThreads);
  if (!fn) return CT_ECONFIG;
  int err = CT_OK;
  DeviceState* st = current_state(nullptr, &err);
  if (!st) return err;
  std::lock_guard<std::mutex> lk(g_mu);
  return cuda_status(raise_smem_cap(st, fn));  // queries (and so loads) the kernel
}

int launch_plan(ConvPlan& plan, cudaStream_t s) {
  if (plan.empty) return CT_OK;
  int err = CT_OK;
  DeviceState* st = current_state(nullptr, &err);
  if (!st) return err;
  unsigned* status = device_status_word(&err);
  if (!status) return err;
  ConvLaunch& L = plan.L;
  L.status = status;
  if (L.smem_bytes > 48 * 1024) {
    std::lock_guard<std::mutex> lk(g_mu);
    const cudaError_t e = raise_smem_cap(st, plan.fn);
    if (e != cudaSuccess) return cuda_status(e);
  }
  L.tmap = nullptr;
  if (plan.specialised && L.staging == kStageTma) {
    auto enc = tensor_map_encoder();
    if (!enc) return CT_ENOTSUP;
    const cuuint64_t dims[2] = {(cuuint64_t)L.in_w, (cuuint64_t)L.in_h};
    const cuuint64_t strides[1] = {(cuuint64_t)L.in_pitch * 4};
    const cuuint32_t box[2] = {(cuuint32_t)L.tile_w, (cuuint32_t)L.tile_h};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&plan.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)L.in, dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return CT_ECONFIG;
    L.tmap = &plan.tmap;
  }
  cudaError_t e;
  if (plan.specialised) {
    KernelLauncher fn = launcher_for(L.fh);
    if (!fn) return CT_ECONFIG;
    e = fn(L, s);
  } else {
    e = launch_generic(L, s);
  }
  return cuda_status(e);
}

}  // namespace convtune

using namespace convtune;

extern "C" {

const char* ct_strerror(int status) {
  switch (status) {
    case CT_OK: return "ok";
    case CT_EINVAL: return "invalid argument";
    case CT_ENOTSUP: return "not supported on this device or driver";
    case CT_EPERM: return "clock control not permitted";
    case CT_ECUDA: return "CUDA call failed";
    case CT_ENOMEM: return "capacity too small or allocation failed";
    case CT_ETIMEOUT: return "bounded device wait gave up";
    case CT_ECONFIG: return "configuration invalid for this problem or device";
    case CT_EIO: return "results cache I/O failed";
    default: return "unknown status";
  }
}

const char* ct_version(void) { return "convtune 0.1 sm_103a"; }

const char* ct_last_error(void) { return g_last_error; }

}  // extern "C"

namespace convtune {
void set_last_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
}  // namespace convtune

extern "C" {

int ct_conv2d_check(const ct_problem* p, const ct_config* c, char* why, int why_cap) {
  if (!p || !c) return CT_EINVAL;
  ConvPlan plan;
  std::string w;
  const int rc = plan_conv(*p, *c, &plan, &w);
  if (why && why_cap > 0) {
    snprintf(why, (size_t)why_cap, "%s", rc == CT_OK ? "" : w.c_str());
  }
  return rc;
}

int ct_conv2d_run(const ct_problem* p, const ct_config* c, void* stream) {
  if (!p || !c) return CT_EINVAL;
  ConvPlan plan;
  const int rc = plan_conv(*p, *c, &plan, nullptr);
  if (rc != CT_OK) return rc;
  return launch_plan(plan, (cudaStream_t)stream);
}

}  // extern "C"

namespace {

// Default row bands of the host-buffer entry point: an even split into
// n = max(min(out_h / 256, 8), ceil(out_h / 512)) bands (at least 1, at most
// kHostMaxBands).  Each band costs a few microseconds of copy and launch
// set-up, and the first input copy and the last output copy overlap nothing,
// so bands of a few hundred rows balance the two; on GB300, 4096 rows ran
// fastest as 8 bands (4, 16 and 32 bands, and bands ramping from 64 rows at
// both ends, were slower).
std::vector<int> default_host_bands(int out_h) {
  const long long h = out_h;
  long long n = std::max(std::min(h / 256, 8LL), (h + 511) / 512);
  n = std::max(1LL, std::min(n, (long long)kHostMaxBands));
  std::vector<int> rows;
  for (long long b = 0; b < n; ++b) rows.push_back((int)(h / n + (b < h % n ? 1 : 0)));
  return rows;
}

// One host-buffer call over the given row bands.  sync: start after the
// caller's earlier work on `stream`, make `stream` wait for the last copy
// out and return when the output is in out_host.  Otherwise: return once
// everything is enqueued, ordered only after the earlier host-buffer calls
// (ct_conv2d_host_wait waits for it).
int run_host_bands(const float* in_host, long in_pitch, const float* filt, int fh, int fw,
                   float* out_host, long out_pitch, int out_h, int out_w, const ct_config* c,
                   const int* band_rows, int n_bands, void* stream, bool sync) {
  std::lock_guard<std::mutex> lk(g_host_mu);
  int err = CT_OK;
  DeviceState* st = current_state(nullptr, &err);
  if (!st) return err;
  const int in_h = out_h + fh - 1;
  const size_t in_row = sizeof(float) * (size_t)in_pitch;
  const size_t out_row = sizeof(float) * (size_t)out_pitch;
  const size_t in_bytes = in_row * (size_t)in_h;
  const size_t out_bytes = out_row * (size_t)out_h;
  cudaError_t e;
  if (!st->s_in) {
    if ((e = cudaStreamCreateWithFlags(&st->s_in, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&st->s_comp, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&st->s_out, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&st->ev_start, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&st->ev_end, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_status(e);
    for (int q = 0; q < 2; ++q)
      if ((e = cudaEventCreateWithFlags(&st->ev_slot_k[q], cudaEventDisableTiming)) !=
              cudaSuccess ||
          (e = cudaEventCreateWithFlags(&st->ev_slot_out[q], cudaEventDisableTiming)) !=
              cudaSuccess)
        return cuda_status(e);
    st->ev_in.resize(kHostMaxBands);
    st->ev_k.resize(kHostMaxBands);
    for (int b = 0; b < kHostMaxBands; ++b)
      if ((e = cudaEventCreateWithFlags(&st->ev_in[b], cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&st->ev_k[b], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_status(e);
  }
  const int slot = st->host_slot;
  if (st->din_bytes[slot] < in_bytes || st->dout_bytes[slot] < out_bytes) {
    // the set may still be in use by an earlier asynchronous call
    if ((e = cudaStreamSynchronize(st->s_in)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st->s_comp)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st->s_out)) != cudaSuccess)
      return cuda_status(e);
    if (st->din_bytes[slot] < in_bytes) {
      if (st->din[slot]) cudaFree(st->din[slot]);
      st->din[slot] = nullptr;
      st->din_bytes[slot] = 0;
      if ((e = cudaMalloc(&st->din[slot], in_bytes)) != cudaSuccess) return cuda_status(e);
      st->din_bytes[slot] = in_bytes;
    }
    if (st->dout_bytes[slot] < out_bytes) {
      if (st->dout[slot]) cudaFree(st->dout[slot]);
      st->dout[slot] = nullptr;
      st->dout_bytes[slot] = 0;
      if ((e = cudaMalloc(&st->dout[slot], out_bytes)) != cudaSuccess) return cuda_status(e);
      st->dout_bytes[slot] = out_bytes;
    }
  }
  st->host_slot ^= 1;
  float* const din = st->din[slot];
  float* const dout = st->dout[slot];
  // The input rows of band b travel in while band b-1 computes and band
  // b-2's outputs travel back (host <-> device copies run both ways at
  // once).  Input chunk b holds only the rows band b needs beyond the earlier
  // chunks; each output is computed exactly as in one launch.  (One stream
  // per stage: spreading the bands over two streams per stage, so that two
  // copies of one direction run at once, measured slower.)  Across calls
  // the two buffer sets alternate: this call's copies in wait only for the
  // kernels of the call before last (which read the same input buffer), its
  // kernels for that call's copies out (which read the same output buffer).
  int rc = CT_OK;
  auto fail = [&](int code) {
    cudaStreamSynchronize(st->s_in);
    cudaStreamSynchronize(st->s_comp);
    cudaStreamSynchronize(st->s_out);
    return code;
  };
  // start after the caller's earlier work on `stream`
  if (sync && ((e = cudaEventRecord(st->ev_start, (cudaStream_t)stream)) != cudaSuccess ||
               (e = cudaStreamWaitEvent(st->s_in, st->ev_start, 0)) != cudaSuccess))
    return fail(cuda_status(e));
  if ((e = cudaStreamWaitEvent(st->s_in, st->ev_slot_k[slot], 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(st->s_comp, st->ev_slot_out[slot], 0)) != cudaSuccess)
    return fail(cuda_status(e));
  int in_done = 0;  // input rows already sent
  int y0 = 0;
  for (int b = 0; b < n_bands; ++b) {
    const int rb = band_rows[b];
    const int need = y0 + rb + fh - 1;  // input rows band b reads (> in_done: rb >= 1)
    e = cudaMemcpyAsync(reinterpret_cast<char*>(din) + in_row * in_done,
                        reinterpret_cast<const char*>(in_host) + in_row * in_done,
                        in_row * (size_t)(need - in_done), cudaMemcpyHostToDevice, st->s_in);
    if (e != cudaSuccess) return fail(cuda_status(e));
    in_done = need;
    if ((e = cudaEventRecord(st->ev_in[b], st->s_in)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st->s_comp, st->ev_in[b], 0)) != cudaSuccess)
      return fail(cuda_status(e));
    ct_problem p;
    p.in = din + (size_t)y0 * in_pitch;
    p.in_pitch = in_pitch;
    p.filt = filt;
    p.fh = fh;
    p.fw = fw;
    p.out = dout + (size_t)y0 * out_pitch;
    p.out_pitch = out_pitch;
    p.out_h = rb;
    p.out_w = out_w;
    if ((rc = ct_conv2d_run(&p, c, st->s_comp)) != CT_OK) return fail(rc);
    if ((e = cudaEventRecord(st->ev_k[b], st->s_comp)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(st->s_out, st->ev_k[b], 0)) != cudaSuccess)
      return fail(cuda_status(e));
    // the caller's padding columns (out_w .. out_pitch) are left untouched
    if (out_pitch == out_w)
      e = cudaMemcpyAsync(reinterpret_cast<char*>(out_host) + out_row * y0,
                          reinterpret_cast<const char*>(dout) + out_row * y0,
                          out_row * (size_t)rb, cudaMemcpyDeviceToHost, st->s_out);
    else
      e = cudaMemcpy2DAsync(reinterpret_cast<char*>(out_host) + out_row * y0, out_row,
                            reinterpret_cast<const char*>(dout) + out_row * y0, out_row,
                            sizeof(float) * (size_t)out_w, rb, cudaMemcpyDeviceToHost,
                            st->s_out);
    if (e != cudaSuccess) return fail(cuda_status(e));
    y0 += rb;
  }
  if ((e = cudaEventRecord(st->ev_slot_k[slot], st->s_comp)) != cudaSuccess ||
      (e = cudaEventRecord(st->ev_slot_out[slot], st->s_out)) != cudaSuccess)
    return fail(cuda_status(e));
  if (!sync) return CT_OK;
  if ((e = cudaEventRecord(st->ev_end, st->s_out)) != cudaSuccess ||
      (e = cudaStreamWaitEvent((cudaStream_t)stream, st->ev_end, 0)) != cudaSuccess)
    return fail(cuda_status(e));
  return cuda_status(cudaStreamSynchronize(st->s_out));
}

int host_args_check(const float* in_host, long in_pitch, const float* filt, int fh, int fw,
                    float* out_host, long out_pitch, int out_h, int out_w, const ct_config* c) {
  if (!c || !filt) return CT_EINVAL;
  if (out_h < 0 || out_w < 0 || fh < 1 || fw < 1) return CT_EINVAL;
  if (out_h == 0 || out_w == 0) return CT_OK;
  if (!in_host || !out_host) return CT_EINVAL;
  if (in_pitch < (long)out_w + fw - 1 || out_pitch < out_w) return CT_EINVAL;
  return CT_OK;
}

}  // namespace

extern "C" {

int ct_conv2d_run_host(const float* in_host, long in_pitch, const float* filt, int fh, int fw,
                       float* out_host, long out_pitch, int out_h, int out_w, const ct_config* c,
                       void* stream) {
  int rc = host_args_check(in_host, in_pitch, filt, fh, fw, out_host, out_pitch, out_h, out_w, c);
  if (rc != CT_OK || out_h == 0 || out_w == 0) return rc;
  const std::vector<int> rows = default_host_bands(out_h);
  return run_host_bands(in_host, in_pitch, filt, fh, fw, out_host, out_pitch, out_h, out_w, c,
                        rows.data(), (int)rows.size(), stream, true);
}

int ct_conv2d_run_host_async(const float* in_host, long in_pitch, const float* filt, int fh,
                             int fw, float* out_host, long out_pitch, int out_h, int out_w,
                             const ct_config* c) {
  int rc = host_args_check(in_host, in_pitch, filt, fh, fw, out_host, out_pitch, out_h, out_w, c);
  if (rc != CT_OK || out_h == 0 || out_w == 0) return rc;
  // two row bands (one below 512 rows): back-to-back calls overlap one
  // another, so fewer, larger copies than the synchronous split are best
  // (GB300, 4096^2 / 17 x 17, calls back to back: 1 band 0.471 ms per call,
  // 2 bands 0.427, 4 bands 0.492, 8 bands 0.517)
  std::vector<int> rows;
  if (out_h >= 512) rows = {out_h - out_h / 2, out_h / 2};
  else rows = {out_h};
  return run_host_bands(in_host, in_pitch, filt, fh, fw, out_host, out_pitch, out_h, out_w, c,
                        rows.data(), (int)rows.size(), nullptr, false);
}

int ct_conv2d_host_wait(void) {
  std::lock_guard<std::mutex> lk(g_host_mu);
  int err = CT_OK;
  DeviceState* st = current_state(nullptr, &err);
  if (!st) return err;
  if (!st->s_out) return CT_OK;  // no host-buffer call yet
  return cuda_status(cudaStreamSynchronize(st->s_out));
}

int ct_conv2d_run_host_bands(const float* in_host, long in_pitch, const float* filt, int fh,
                             int fw, float* out_host, long out_pitch, int out_h, int out_w,
                             const ct_config* c, const int* band_rows, int n_bands,
                             void* stream) {
  int rc = host_args_check(in_host, in_pitch, filt, fh, fw, out_host, out_pitch, out_h, out_w, c);
  if (rc != CT_OK) return rc;
  if (!band_rows || n_bands < 1 || n_bands > kHostMaxBands) return CT_EINVAL;
  long long total = 0;
  for (int b = 0; b < n_bands; ++b) {
    if (band_rows[b] < 1) return CT_EINVAL;
    total += band_rows[b];
  }
  if (total != out_h) return CT_EINVAL;
  if (out_w == 0) return CT_OK;
  return run_host_bands(in_host, in_pitch, filt, fh, fw, out_host, out_pitch, out_h, out_w, c,
                        band_rows, n_bands, stream, true);
}

int ct_conv2d_host_bands_default(int out_h, int* band_rows, int cap, int* n_bands) {
  if (out_h < 1 || !n_bands) return CT_EINVAL;
  const std::vector<int> rows = default_host_bands(out_h);
  *n_bands = (int)rows.size();
  if (cap < (int)rows.size() || !band_rows) return CT_ENOMEM;
  for (size_t b = 0; b < rows.size(); ++b) band_rows[b] = rows[b];
  return CT_OK;
}

int ct_status_read(unsigned* bits, int clear) {
  if (!bits) return CT_EINVAL;
  int err = CT_OK;
  unsigned* st = device_status_word(&err);
  if (!st) return err;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(bits, st, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(st, 0, sizeof(unsigned));
  return cuda_status(e);
}

int ct_device_info_get(ct_device_info* out) {
  if (!out) return CT_EINVAL;
  memset(out, 0, sizeof(*out));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_status(e);
  out->sm_count = prop.multiProcessorCount;
  out->cc_major = prop.major;
  out->cc_minor = prop.minor;
  out->max_smem_optin_bytes = (int)prop.sharedMemPerBlockOptin;
  out->l2_bytes = prop.l2CacheSize;
  snprintf(out->name, sizeof(out->name), "%.*s", (int)sizeof(out->name) - 1, prop.name);
  int khz = 0;
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) == cudaSuccess)
    out->sm_clock_max_mhz = khz / 1000.0;
  else
    cudaGetLastError();
  return CT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Self-test of the bounded device wait used by TMA staging: one CTA waits on
// an mbarrier phase that nothing completes, gives up after spin_limit polls
// per thread and reports through the device status word, leaving the context
// usable.
// ---------------------------------------------------------------------------
namespace convtune {
namespace {

__global__ void wait_timeout_selftest_kernel(unsigned* status, unsigned spin_limit) {
  __shared__ __align__(8) uint64_t bar;
  const unsigned addr = static_cast<unsigned>(__cvta_generic_to_shared(&bar));
  if (threadIdx.x == 0) {
    // expects one arrival that never comes
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(addr));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  unsigned done = 0;
  for (unsigned it = 0; it < spin_limit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(0u)
        : "memory");
  }
  if (__syncthreads_or(!done) && threadIdx.x == 0) atomicOr(status, kStatusTmaTimeout);
}

}  // namespace
}  // namespace convtune

extern "C" int ct_selftest_wait_timeout(unsigned spin_limit, void* stream) {
  if (spin_limit == 0 || spin_limit > (1u << 24)) return CT_EINVAL;
  int err = CT_OK;
  unsigned* status = device_status_word(&err);
  if (!status) return err;
  wait_timeout_selftest_kernel<<<1, 64, 0, (cudaStream_t)stream>>>(status, spin_limit);
  return cuda_status(cudaGetLastError());
}
