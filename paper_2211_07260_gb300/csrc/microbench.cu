// Microbenchmarks that load the GPU for the power-model fit, and the
// model-steered search (Section IV-E: "run a kernel that fully loads the GPU
// for a range of clock frequencies", fit Eq. powercurve, then tune with a
// fine clock sampling around the predicted optimum).
//
//   FMA-dense: every thread runs 8 independent fmaf chains in registers, no
//              memory traffic; ~1e9 FMAs per launch (exact count reported).
//   stream copy: 1 GiB float4 copy, 2 GiB moved per launch.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <vector>

#include "measure.h"
#include "platform.h"
#include "runtime.h"

namespace convtune {

int tune_impl(const ct_problem& p, const ct_config* space, int n_space, const int* clocks,
              int n_clocks, const ct_tune_options& opt, cudaStream_t stream, ct_record* records,
              int cap, int* n_records, int* best_index);

namespace {

constexpr int kChains = 8;
constexpr int kFmaThreads = 256;
constexpr double kFmaTarget = 1e9;
constexpr size_t kCopyBytes = size_t(1) << 30;

__global__ void __launch_bounds__(kFmaThreads) fma_dense_kernel(float* out, int iters) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 0.5f + 1e-3f * (float)((tid + c) & 255);
  const float a = 0.9999995f, b = 5e-7f;  // fixed point 1: no overflow, no denormals
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[tid] = s;
}

__global__ void copy_kernel(const float4* __restrict__ src, float4* __restrict__ dst, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    dst[i] = src[i];
}

struct Scratch {
  float* fma_out = nullptr;
  int fma_blocks = 0, fma_iters = 0;
  float* copy_src = nullptr;
  float* copy_dst = nullptr;
  int sms = 0;
  ~Scratch() {
    // released at unload; the context may already be gone, so errors are ignored
    if (fma_out) cudaFree(fma_out);
    if (copy_src) cudaFree(copy_src);
    if (copy_dst) cudaFree(copy_dst);
  }
};

std::mutex g_mu;
Scratch g_scratch;

int ensure_scratch(int which) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaError_t e;
  if (!g_scratch.sms) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaDeviceGetAttribute(&g_scratch.sms, cudaDevAttrMultiProcessorCount, dev)) !=
        cudaSuccess)
      return cuda_status(e);
  }
  if (which == CT_UNIT_FMA && !g_scratch.fma_out) {
    g_scratch.fma_blocks = 4 * g_scratch.sms;
    const double per_iter = (double)g_scratch.fma_blocks * kFmaThreads * kChains;
    g_scratch.fma_iters = (int)ceil(kFmaTarget / per_iter);
    e = cudaMalloc(&g_scratch.fma_out, sizeof(float) * g_scratch.fma_blocks * kFmaThreads);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (which == CT_UNIT_COPY && !g_scratch.copy_src) {
    if ((e = cudaMalloc(&g_scratch.copy_src, kCopyBytes)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMalloc(&g_scratch.copy_dst, kCopyBytes)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemset(g_scratch.copy_src, 0, kCopyBytes)) != cudaSuccess) return cuda_status(e);
  }
  return CT_OK;
}

double bench_work(int which) {
  if (which == CT_UNIT_FMA)
    return 2.0 * g_scratch.fma_blocks * (double)kFmaThreads * kChains * g_scratch.fma_iters;
  return 2.0 * (double)kCopyBytes;
}

int launch_bench(int which, cudaStream_t s) {
  if (which == CT_UNIT_FMA) {
    fma_dense_kernel<<<g_scratch.fma_blocks, kFmaThreads, 0, s>>>(g_scratch.fma_out,
                                                                 g_scratch.fma_iters);
  } else {
    copy_kernel<<<8 * g_scratch.sms, 512, 0, s>>>(
        reinterpret_cast<const float4*>(g_scratch.copy_src),
        reinterpret_cast<float4*>(g_scratch.copy_dst), kCopyBytes / sizeof(float4));
  }
  return cuda_status(cudaGetLastError());
}

int measure_bench(int which, const ct_measure_options& o, const ct_platform_ops& ops,
                  cudaStream_t stream, int clock, ct_record* r) {
  MeasureUnit u;
  u.kind = which;
  if (ops.run_launches) {
    u.work = which == CT_UNIT_FMA ? 2.0 * kFmaTarget : 2.0 * (double)kCopyBytes;
  } else {
    const int rc = ensure_scratch(which);
    if (rc != CT_OK) return rc;
    u.work = bench_work(which);
    u.launch = [which](cudaStream_t s) { return launch_bench(which, s); };
  }
  return measure_unit(u, o, ops, stream, clock, r);
}

// Samples (clock, power, throttled) for the fit; one per requested clock.
int power_samples(int which, const int* clocks, int n_clocks, const ct_measure_options& o,
                  const ct_platform_ops& ops, cudaStream_t stream, double* f_meas, double* p_w,
                  int* throttled, ct_record* recs) {
  const int n = n_clocks > 0 ? n_clocks : 1;
  for (int i = 0; i < n; ++i) {
    const int clock = n_clocks > 0 ? clocks[i] : 0;
    ClockLock lock(ops, clock);
    if (clock > 0 && !lock.locked()) return lock.status() == CT_OK ? CT_EPERM : lock.status();
    ct_record r;
    const int rc = measure_bench(which, o, ops, stream, clock, &r);
    if (rc != CT_OK) return rc;
    bool thr = (r.flags & CT_REC_THROTTLED) != 0;
    if (clock > 0 && r.clock_mhz_meas < clock - 8) thr = true;
    if (f_meas) f_meas[i] = r.clock_mhz_meas;
    if (p_w) p_w[i] = isnan(r.power_w_mean) ? r.power_w_median : r.power_w_mean;
    if (throttled) throttled[i] = thr ? 1 : 0;
    if (recs) recs[i] = r;
  }
  return CT_OK;
}

}  // namespace

}  // namespace convtune

using namespace convtune;

extern "C" {

int ct_microbench_launch(int which, void* stream, double* work) {
  if (which != CT_UNIT_FMA && which != CT_UNIT_COPY) return CT_EINVAL;
  int rc = ensure_scratch(which);
  if (rc != CT_OK) return rc;
  if (work) *work = bench_work(which);
  return launch_bench(which, (cudaStream_t)stream);
}

int ct_measure_microbench(int which, const ct_measure_options* opt, void* stream,
                          ct_record* out) {
  if ((which != CT_UNIT_FMA && which != CT_UNIT_COPY) || !out) return CT_EINVAL;
  return measure_bench(which, resolve_options(opt), platform_ops(), (cudaStream_t)stream, 0, out);
}

int ct_measure_power_samples(int which, const int* clocks_mhz, int n_clocks,
                             const ct_measure_options* opt, void* stream, double* f_meas_mhz,
                             double* p_w, int* throttled, ct_record* recs_or_null) {
  if (which != CT_UNIT_FMA && which != CT_UNIT_COPY) return CT_EINVAL;
  if (n_clocks < 0 || (n_clocks > 0 && !clocks_mhz)) return CT_EINVAL;
  return power_samples(which, clocks_mhz, n_clocks, resolve_options(opt), platform_ops(),
                       (cudaStream_t)stream, f_meas_mhz, p_w, throttled, recs_or_null);
}

int ct_microbench_release(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaError_t e = cudaSuccess;
  if (g_scratch.fma_out) e = cudaFree(g_scratch.fma_out);
  if (g_scratch.copy_src) e = cudaFree(g_scratch.copy_src);
  if (g_scratch.copy_dst) e = cudaFree(g_scratch.copy_dst);
  g_scratch.fma_out = g_scratch.copy_src = g_scratch.copy_dst = nullptr;
  return cuda_status(e);
}

int ct_tune_steered(const ct_problem* p, const ct_config* space, int n_space,
                    const int* fit_clocks, int n_fit_clocks, const int* supported,
                    int n_supported, double rel_halfwidth, int which_bench,
                    const ct_tune_options* opt, void* stream, ct_steer_result* res,
                    int* range_out, int range_cap, ct_record* records, int cap, int* n_records,
                    int* best_index) {
  if (!p || !opt || !res || !n_records || !best_index || !fit_clocks || n_fit_clocks < 3)
    return CT_EINVAL;
  if (which_bench != CT_UNIT_FMA && which_bench != CT_UNIT_COPY && which_bench != CT_STEER_UNION)
    return CT_EINVAL;
  memset(res, 0, sizeof(*res));
  const ct_platform_ops ops = platform_ops();
  const ct_measure_options mo = resolve_options(&opt->measure);
  const double t0 = platform_now(ops);
  std::vector<int> sup;
  if (supported && n_supported > 0) {
    sup.assign(supported, supported + n_supported);
  } else {
    if (!ops.supported_sm_clocks) return CT_ENOTSUP;
    sup.resize(1024);
    int ns = 0;
    const int rc = ops.supported_sm_clocks(ops.ctx, sup.data(), (int)sup.size(), &ns);
    if (rc != CT_OK) return rc;
    sup.resize(ns);
  }
  // the fits use the requested (locked) clocks as f; the measured clock
  // decides only whether a sample throttled
  const std::vector<double> freq(fit_clocks, fit_clocks + n_fit_clocks);
  std::vector<double> f(n_fit_clocks), pw(n_fit_clocks), ts(n_fit_clocks);
  std::vector<int> thr(n_fit_clocks);
  std::vector<ct_record> recs(n_fit_clocks);
  std::vector<int> range_c, range_m;
  int rc = CT_OK;
  if (which_bench == CT_UNIT_FMA || which_bench == CT_STEER_UNION) {
    // compute-bound model (Section IV-E): P*(f)/f on the FMA-dense sweep
    rc = power_samples(CT_UNIT_FMA, fit_clocks, n_fit_clocks, mo, ops, (cudaStream_t)stream,
                       f.data(), pw.data(), thr.data(), nullptr);
    if (rc != CT_OK) return rc;
    rc = ct_fit_power_model(freq.data(), pw.data(), nullptr, thr.data(), n_fit_clocks, 0.0,
                            &res->model);
    if (rc != CT_OK) return rc;
    range_c.resize(sup.size());
    int nr = 0;
    rc = ct_pick_clock_range(&res->model, sup.data(), (int)sup.size(), rel_halfwidth, 0,
                             range_c.data(), (int)range_c.size(), &nr, &res->center_mhz);
    if (rc != CT_OK) return rc;
    range_c.resize(nr);
  }
  if (which_bench == CT_UNIT_COPY || which_bench == CT_STEER_UNION) {
    // memory-aware model: P*(f) t(f) on the stream-copy sweep
    rc = power_samples(CT_UNIT_COPY, fit_clocks, n_fit_clocks, mo, ops, (cudaStream_t)stream,
                       f.data(), pw.data(), thr.data(), recs.data());
    if (rc != CT_OK) return rc;
    for (int i = 0; i < n_fit_clocks; ++i) ts[i] = recs[i].t_s;
    rc = ct_fit_power_model(freq.data(), pw.data(), nullptr, thr.data(), n_fit_clocks, 0.0,
                            &res->model_mem);
    if (rc != CT_OK) return rc;
    rc = ct_fit_time_model(freq.data(), ts.data(), thr.data(), n_fit_clocks, &res->time_mem);
    if (rc != CT_OK) return rc;
    rc = ct_memory_aware_optimum(&res->model_mem, &res->time_mem, &res->center_mem_mhz, nullptr);
    if (rc != CT_OK) return rc;
    range_m.resize(sup.size());
    int nr = 0;
    rc = ct_clock_range(res->center_mem_mhz, sup.data(), (int)sup.size(), rel_halfwidth,
                        range_m.data(), (int)range_m.size(), &nr);
    if (rc != CT_OK) return rc;
    range_m.resize(nr);
    if (which_bench == CT_UNIT_COPY) {
      res->model = res->model_mem;
      res->center_mhz = res->center_mem_mhz;
    }
  }
  res->n_range_compute = (int)range_c.size();
  res->n_range_memory = (int)range_m.size();
  std::vector<int> range = range_c;
  range.insert(range.end(), range_m.begin(), range_m.end());
  std::sort(range.begin(), range.end());
  range.erase(std::unique(range.begin(), range.end()), range.end());
  const int nr = (int)range.size();
  res->n_range = nr;
  if (range_out) {
    if (nr > range_cap) return CT_ENOMEM;
    memcpy(range_out, range.data(), sizeof(int) * nr);
  }
  res->fit_wall_s = platform_now(ops) - t0;
  const double t1 = platform_now(ops);
  rc = tune_impl(*p, space, n_space, range.data(), nr, *opt, (cudaStream_t)stream, records, cap,
                 n_records, best_index);
  res->tune_wall_s = platform_now(ops) - t1;
  return rc;
}

}  // extern "C"
