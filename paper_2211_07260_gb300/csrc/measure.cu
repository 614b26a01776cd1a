// Measurement window of one tuning point (Section III-A/B of the paper:
// energy = mean power x elapsed time; the observer runs the kernel
// repeatedly for about a second because the device's power readings refresh
// at only ~10 Hz).
//
// Here the kernel is captured G times into a CUDA graph and the graph is
// replayed back to back with a bounded number of replays in flight, so the
// device never idles.  The energy window opens at an update of the total-
// energy counter (the second one after the load starts, so that the counter
// has integrated load only) and closes at the first update at least
// window_s later; mean power over the window is the counter difference over
// the host-timed distance of the two updates.  Energy per launch = mean
// power x the event-timed device time per launch of the same span.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "measure.h"
#include "runtime.h"

namespace convtune {

namespace {

class Driver {
 public:
  virtual ~Driver() {}
  virtual int replay() = 0;                      // enqueue / run one replay
  virtual int outstanding() = 0;                 // replays still in flight
  virtual int begin_span() = 0;
  virtual int end_span(double* ms) = 0;          // synchronises
  virtual bool synchronous() const { return false; }  // replay() runs to completion
  int per_replay = 1;                            // launches per replay
};

// Real device: a graph of G launches on a private stream.
class GraphDriver : public Driver {
 public:
  ~GraphDriver() override {
    if (exec_) cudaGraphExecDestroy(exec_);
    for (auto e : ring_) cudaEventDestroy(e);
    if (ev0_) cudaEventDestroy(ev0_);
    if (ev1_) cudaEventDestroy(ev1_);
    if (s_) {
      cudaStreamSynchronize(s_);
      cudaStreamDestroy(s_);
    }
  }

  int init(const MeasureUnit& u, cudaStream_t order_after, double graph_ms, int ring) {
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&s_, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_status(e);
    if ((e = cudaEventCreate(&ev0_)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaEventCreate(&ev1_)) != cudaSuccess) return cuda_status(e);
    // order after the caller's stream (its inputs may still be in flight)
    if ((e = cudaEventRecord(ev0_, order_after)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaStreamWaitEvent(s_, ev0_, 0)) != cudaSuccess) return cuda_status(e);
    // size the graph from a few single launches
    int rc = u.launch(s_);
    if (rc != CT_OK) return rc;
    if ((e = cudaEventRecord(ev0_, s_)) != cudaSuccess) return cuda_status(e);
    for (int i = 0; i < 3; ++i)
      if ((rc = u.launch(s_)) != CT_OK) return rc;
    if ((e = cudaEventRecord(ev1_, s_)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaEventSynchronize(ev1_)) != cudaSuccess) return cuda_status(e);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0_, ev1_);
    const double t1 = std::max(1e-4, ms / 3.0);
    per_replay = (int)std::min(4096.0, std::max(1.0, ceil(graph_ms / t1)));
    if (u.eager) {
      // host launches each replay: what a caller issuing one launch per call pays
      eager_ = &u.launch;
    } else {
      if ((rc = capture(u)) != CT_OK) return rc;
    }
    ring_.resize(ring);
    for (auto& ev : ring_)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_status(e);
    return CT_OK;
  }

  int capture(const MeasureUnit& u) {
    cudaError_t e;
    int rc = CT_OK;
    // capture
    if ((e = cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_status(e);
    for (int i = 0; i < per_replay; ++i) {
      rc = u.launch(s_);
      if (rc != CT_OK) break;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s_, &g);
    if (rc != CT_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaGraphInstantiate(&exec_, g, 0);
    cudaGraphDestroy(g);
    return cuda_status(e);
  }

  int replay() override {
    cudaError_t e = cudaSuccess;
    if (eager_) {
      for (int i = 0; i < per_replay; ++i) {
        const int rc = (*eager_)(s_);
        if (rc != CT_OK) return rc;
      }
    } else {
      e = cudaGraphLaunch(exec_, s_);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ring_[tail_ % ring_.size()], s_);
    if (e != cudaSuccess) return cuda_status(e);
    ++tail_;
    return CT_OK;
  }

  int outstanding() override {
    while (head_ < tail_) {
      cudaError_t e = cudaEventQuery(ring_[head_ % ring_.size()]);
      if (e == cudaErrorNotReady) break;
      if (e != cudaSuccess) return -1;
      ++head_;
    }
    return (int)(tail_ - head_);
  }

  int begin_span() override { return cuda_status(cudaEventRecord(ev0_, s_)); }

  int end_span(double* ms) override {
    cudaError_t e = cudaEventRecord(ev1_, s_);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1_);
    if (e != cudaSuccess) return cuda_status(e);
    float f = 0.f;
    e = cudaEventElapsedTime(&f, ev0_, ev1_);
    head_ = tail_;
    *ms = f;
    return cuda_status(e);
  }

 private:
  cudaStream_t s_ = nullptr;
  cudaGraphExec_t exec_ = nullptr;
  const std::function<int(cudaStream_t)>* eager_ = nullptr;
  cudaEvent_t ev0_ = nullptr, ev1_ = nullptr;
  std::vector<cudaEvent_t> ring_;
  long long head_ = 0, tail_ = 0;
};

// Simulation: the platform table's run_launches hook runs synchronously.
class SimDriver : public Driver {
 public:
  SimDriver(const ct_platform_ops& ops, int kind, const ct_config* cfg, double graph_ms)
      : ops_(ops), kind_(kind), cfg_(cfg), graph_ms_(graph_ms) {}
  int init() {
    double ms = 0;
    const int rc = ops_.run_launches(ops_.ctx, kind_, cfg_, 1, &ms);
    if (rc != CT_OK) return rc;
    per_replay = (int)std::min(4096.0, std::max(1.0, ceil(graph_ms_ / std::max(1e-4, ms))));
    return CT_OK;
  }
  int replay() override {
    double ms = 0;
    const int rc = ops_.run_launches(ops_.ctx, kind_, cfg_, per_replay, &ms);
    acc_ += ms;
    return rc;
  }
  int outstanding() override { return 0; }
  bool synchronous() const override { return true; }
  int begin_span() override {
    acc_ = 0;
    return CT_OK;
  }
  int end_span(double* ms) override {
    *ms = acc_;
    return CT_OK;
  }

 private:
  ct_platform_ops ops_;
  int kind_;
  const ct_config* cfg_;
  double graph_ms_;
  double acc_ = 0;
};

double median(std::vector<double> v) {
  if (v.empty()) return NAN;
  std::sort(v.begin(), v.end());
  const size_t n = v.size();
  return n % 2 ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

// Keep replays in flight; returns the replays enqueued by this call.
int top_up(Driver& d, int queue, long long* n, int* rc) {
  const int out = d.outstanding();
  if (out < 0) {
    *rc = CT_ECUDA;
    return 0;
  }
  if (d.synchronous()) queue = out + 1;  // one replay per poll of the sensors
  int k = 0;
  for (; out + k < queue; ++k) {
    if ((*rc = d.replay()) != CT_OK) return k;
    ++*n;
  }
  return k;
}

int run_window(Driver& d, const ct_measure_options& opt, const ct_platform_ops& ops,
               double graph_ms_est, ct_record* r) {
  const int queue = std::max(4, (int)ceil(50.0 / std::max(0.01, graph_ms_est)));
  int rc = CT_OK;
  long long n = 0;
  const double t_begin = platform_now(ops);

  if (opt.time_only) {
    // warm up, then time a fixed number of replays enqueued back to back
    if ((rc = d.begin_span()) != CT_OK) return rc;
    while (platform_now(ops) - t_begin < opt.warmup_s || n < 2) {
      top_up(d, queue, &n, &rc);
      if (rc != CT_OK) return rc;
    }
    double ms = 0;
    if ((rc = d.end_span(&ms)) != CT_OK) return rc;
    if ((rc = d.begin_span()) != CT_OK) return rc;
    for (int i = 0; i < opt.time_reps; ++i)
      if ((rc = d.replay()) != CT_OK) return rc;
    if ((rc = d.end_span(&ms)) != CT_OK) return rc;
    r->n_launches = opt.time_reps * d.per_replay;
    r->t_s = ms / 1e3 / r->n_launches;
    r->flags |= CT_REC_NO_ENERGY;
    r->energy_j = r->power_w_mean = r->power_w_median = r->energy_j_median_power = NAN;
    r->clock_mhz_meas = r->temp_c = NAN;
    unsigned mhz = 0;
    if (ops.sm_clock_mhz && ops.sm_clock_mhz(ops.ctx, &mhz) == CT_OK) r->clock_mhz_meas = mhz;
    return CT_OK;
  }

  unsigned long long e_prev = 0, e_a = 0, e_b = 0;
  bool have_energy = ops.energy_mj && ops.energy_mj(ops.ctx, &e_prev) == CT_OK;
  int edges = 0;  // counter updates seen after the warm-up
  double t_a = 0, t_b = 0, t_last = t_begin, max_gap = 0;
  std::vector<double> pw, clk;
  double temp_max = NAN;
  unsigned long long reasons = 0;
  const double deadline = t_begin + opt.warmup_s + opt.window_s + 3.0;
  if ((rc = d.begin_span()) != CT_OK) return rc;
  for (;;) {
    top_up(d, queue, &n, &rc);
    if (rc != CT_OK) {
      double ms;
      d.end_span(&ms);
      return rc;
    }
    const double t = platform_now(ops);
    max_gap = std::max(max_gap, t - t_last);
    t_last = t;
    const bool warm = t - t_begin >= opt.warmup_s;
    // sensors are sampled inside the energy window (after the warm-up
    // when there is no counter)
    if (have_energy ? edges >= 2 : warm) {
      unsigned v = 0;
      unsigned long long bits = 0;
      if (ops.power_mw && ops.power_mw(ops.ctx, &v) == CT_OK) pw.push_back(v / 1000.0);
      if (ops.sm_clock_mhz && ops.sm_clock_mhz(ops.ctx, &v) == CT_OK) clk.push_back(v);
      if (ops.throttle_reasons && ops.throttle_reasons(ops.ctx, &bits) == CT_OK) reasons |= bits;
      if (ops.temperature_c && ops.temperature_c(ops.ctx, &v) == CT_OK)
        temp_max = isnan(temp_max) ? v : std::max(temp_max, (double)v);
    }
    if (have_energy) {
      unsigned long long e = 0;
      if (ops.energy_mj(ops.ctx, &e) != CT_OK) {
        have_energy = false;
      } else if (e != e_prev) {
        e_prev = e;
        if (warm) {
          ++edges;
          // the first update after the warm-up may still integrate idle
          // time before the load; the window opens at the second
          if (edges == 2) {
            e_a = e;
            t_a = t;
          } else if (edges > 2 && t - t_a >= opt.window_s) {
            e_b = e;
            t_b = t;
            break;
          }
        }
      }
    } else if (warm && t - t_begin >= opt.warmup_s + opt.window_s) {
      edges = 2;
      t_a = t_begin + opt.warmup_s;
      t_b = t;
      break;
    }
    if (t > deadline) {
      have_energy = false;
      if (t_a == 0) t_a = t_begin + opt.warmup_s;
      t_b = t;
      break;
    }
  }
  double ms = 0;
  if ((rc = d.end_span(&ms)) != CT_OK) return rc;
  r->n_launches = (int)(n * d.per_replay);
  r->t_s = ms / 1e3 / std::max(1LL, n * d.per_replay);
  r->power_w_median = median(pw);
  r->clock_mhz_meas = median(clk);
  r->temp_c = temp_max;
  const unsigned long long throttle_mask = CT_THR_SW_POWER_CAP | CT_THR_HW_SLOWDOWN |
                                           CT_THR_SW_THERMAL | CT_THR_HW_THERMAL |
                                           CT_THR_HW_POWER_BRAKE;
  if (reasons & throttle_mask) r->flags |= CT_REC_THROTTLED;
  // the queue held >= 50 ms of work; a longer host stall may have drained it
  if (max_gap * 1e3 > queue * graph_ms_est) r->flags |= CT_REC_IDLE_GAPS;
  if (have_energy && e_b > e_a && t_b > t_a) {
    r->power_w_mean = (double)(e_b - e_a) / 1e3 / (t_b - t_a);
    r->energy_j = r->power_w_mean * r->t_s;
  } else {
    r->flags |= CT_REC_NO_ENERGY;
    r->power_w_mean = NAN;
    r->energy_j = r->power_w_median * r->t_s;
  }
  r->energy_j_median_power = r->power_w_median * r->t_s;
  return CT_OK;
}

}  // namespace

ct_measure_options resolve_options(const ct_measure_options* opt) {
  ct_measure_options o;
  memset(&o, 0, sizeof(o));
  if (opt) o = *opt;
  if (!(o.window_s > 0)) o.window_s = 1.0;
  if (!(o.warmup_s >= 0)) o.warmup_s = 0.2;
  if (!(o.graph_ms > 0)) o.graph_ms = 2.0;
  if (o.time_reps <= 0) o.time_reps = 5;
  return o;
}

int measure_unit(const MeasureUnit& u, const ct_measure_options& opt, const ct_platform_ops& ops,
                 cudaStream_t order_after, int clock_req, ct_record* out) {
  ct_record r;
  memset(&r, 0, sizeof(r));
  if (u.cfg) r.cfg = *u.cfg;
  r.clock_mhz_req = clock_req;
  const double t0 = platform_now(ops);
  int others = 0;
  if (ops.other_processes && ops.other_processes(ops.ctx, &others) == CT_OK && others > 0)
    r.flags |= CT_REC_COTENANT;
  int rc;
  if (ops.run_launches) {
    SimDriver d(ops, u.kind, u.cfg, opt.graph_ms);
    if ((rc = d.init()) != CT_OK) return rc;
    rc = run_window(d, opt, ops, opt.graph_ms, &r);
  } else {
    GraphDriver d;
    const int ring = 8 + (int)ceil(50.0 / std::max(0.01, opt.graph_ms));
    if ((rc = d.init(u, order_after, opt.graph_ms, std::max(64, ring))) != CT_OK) return rc;
    rc = run_window(d, opt, ops, opt.graph_ms, &r);
  }
  if (rc != CT_OK) return rc;
  if (ops.other_processes && ops.other_processes(ops.ctx, &others) == CT_OK && others > 0)
    r.flags |= CT_REC_COTENANT;
  r.gflops = u.work / 1e9 / r.t_s;
  r.gflops_per_j = (r.energy_j > 0) ? u.work / 1e9 / r.energy_j : NAN;
  r.wall_s = platform_now(ops) - t0;
  *out = r;
  return CT_OK;
}

}  // namespace convtune

using namespace convtune;

extern "C" int ct_measure_conv(const ct_problem* p, const ct_config* c,
                               const ct_measure_options* opt, void* stream, ct_record* out) {
  if (!p || !c || !out) return CT_EINVAL;
  memset(out, 0, sizeof(*out));
  out->cfg = *c;
  const ct_platform_ops ops = platform_ops();
  ConvPlan plan;
  int rc = plan_conv(*p, *c, &plan, nullptr, ops.run_launches == nullptr);
  if (rc == CT_ECONFIG) out->flags = CT_REC_INVALID;
  if (rc != CT_OK) return rc;
  if (plan.empty) return CT_EINVAL;
  MeasureUnit u;
  u.kind = CT_UNIT_CONV;
  u.cfg = c;
  u.work = conv_flop(*p);
  u.launch = [&plan](cudaStream_t s) { return launch_plan(plan, s); };
  const ct_measure_options o = resolve_options(opt);
  return measure_unit(u, o, ops, (cudaStream_t)stream, 0, out);
}
