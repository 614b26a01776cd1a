// Exhaustive energy-aware search over configurations x SM clocks
// (Sections III-C and IV of the paper: tunable kernel parameters plus the
// nvml_gr_clock tunable, objectives time / energy / GFLOPs per watt), with a
// JSON-lines results cache so that an interrupted sweep resumes.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "measure.h"
#include "platform.h"
#include "runtime.h"

namespace convtune {

namespace {

std::mutex g_tune_mu;  // tuning and clock control are process-global

void fill_space(int which, std::vector<ct_config>* out) {
  const int bxs[] = {16, 32, 64, 128}, bys[] = {1, 2, 4, 8}, ts[] = {1, 2, 4};
  const int st_basic[] = {CT_STAGE_DIRECT, CT_STAGE_SMEM};
  const int st_full[] = {CT_STAGE_DIRECT, CT_STAGE_SMEM, CT_STAGE_TMA};
  const int fm_basic[] = {CT_FILTER_CONST}, fm_full[] = {CT_FILTER_SHARED, CT_FILTER_CONST};
  const int vw_basic[] = {4}, vw_full[] = {1, 2, 4};
  const bool full = which == CT_SPACE_FULL;
  const int* st = full ? st_full : st_basic;
  const int nst = full ? 3 : 2;
  const int* fm = full ? fm_full : fm_basic;
  const int nfm = full ? 2 : 1;
  const int* vw = full ? vw_full : vw_basic;
  const int nvw = full ? 3 : 1;
  for (int bx : bxs)
    for (int by : bys)
      for (int tx : ts)
        for (int ty : ts)
          for (int a = 0; a < nst; ++a)
            for (int b = 0; b < nfm; ++b)
              for (int v = 0; v < nvw; ++v) out->push_back({bx, by, tx, ty, st[a], fm[b], vw[v]});
}

std::string device_tag(bool simulated) {
  if (simulated) return "simulated";
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  char uuid[40];
  for (int i = 0; i < 16; ++i) snprintf(uuid + 2 * i, 3, "%02x", (unsigned char)prop.uuid.bytes[i]);
  return std::string(prop.name) + "/" + uuid;
}

std::string point_key(const std::string& dev, const ct_problem& p, const ct_config& c, int clock,
                      int limit_mw, const ct_measure_options& m) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|%dx%d|k%dx%d|pitch%ld,%ld|cfg%d,%d,%d,%d,%d,%d,%d|clk%d|w%.4g|t%d",
           dev.c_str(), p.out_h, p.out_w, p.fh, p.fw, p.in_pitch, p.out_pitch, c.block_x,
           c.block_y, c.tile_x, c.tile_y, c.staging, c.filter_mem, c.vec_width, clock, m.window_s,
           m.time_only);
  std::string k = buf;
  if (limit_mw > 0) k += "|pl" + std::to_string(limit_mw);  // (clock keys stay as they were)
  return k;
}

// ---- JSON-lines cache (flat objects written and read by this file) -------
void put_num(std::string* s, const char* k, double v) {
  char b[96];
  if (isfinite(v))
    snprintf(b, sizeof(b), ",\"%s\":%.17g", k, v);
  else
    snprintf(b, sizeof(b), ",\"%s\":null", k);
  *s += b;
}

std::string record_json(const std::string& key, const ct_record& r) {
  std::string s = "{\"key\":\"" + key + "\"";
  put_num(&s, "clock_mhz_req", r.clock_mhz_req);
  put_num(&s, "clock_mhz_meas", r.clock_mhz_meas);
  put_num(&s, "t_s", r.t_s);
  put_num(&s, "energy_j", r.energy_j);
  put_num(&s, "power_w_mean", r.power_w_mean);
  put_num(&s, "power_w_median", r.power_w_median);
  put_num(&s, "energy_j_median_power", r.energy_j_median_power);
  put_num(&s, "gflops", r.gflops);
  put_num(&s, "gflops_per_j", r.gflops_per_j);
  put_num(&s, "temp_c", r.temp_c);
  put_num(&s, "wall_s", r.wall_s);
  put_num(&s, "n_launches", r.n_launches);
  put_num(&s, "flags", r.flags);
  put_num(&s, "power_limit_w", r.power_limit_w);
  return s + "}\n";
}

bool get_num(const std::string& line, const char* k, double* v) {
  const std::string pat = std::string("\"") + k + "\":";
  const size_t pos = line.find(pat);
  if (pos == std::string::npos) return false;
  const char* p = line.c_str() + pos + pat.size();
  if (strncmp(p, "null", 4) == 0) {
    *v = NAN;
    return true;
  }
  char* end = nullptr;
  *v = strtod(p, &end);
  return end != p;
}

int load_cache(const char* path, std::map<std::string, ct_record>* out) {
  FILE* f = fopen(path, "r");
  if (!f) return CT_OK;  // no cache yet
  char* buf = nullptr;
  size_t cap = 0;
  ssize_t len;
  while ((len = getline(&buf, &cap, f)) > 0) {
    std::string line(buf, (size_t)len);
    const std::string kpat = "{\"key\":\"";
    if (line.compare(0, kpat.size(), kpat) != 0) continue;
    const size_t kend = line.find('"', kpat.size());
    if (kend == std::string::npos) continue;
    const std::string key = line.substr(kpat.size(), kend - kpat.size());
    ct_record r;
    memset(&r, 0, sizeof(r));
    double v;
    bool ok = true;
    auto num = [&](const char* k, double* dst) {
      if (get_num(line, k, &v)) *dst = v;
      else ok = false;
    };
    double clk = 0, nl = 0, fl = 0;
    num("clock_mhz_req", &clk);
    num("clock_mhz_meas", &r.clock_mhz_meas);
    num("t_s", &r.t_s);
    num("energy_j", &r.energy_j);
    num("power_w_mean", &r.power_w_mean);
    num("power_w_median", &r.power_w_median);
    num("energy_j_median_power", &r.energy_j_median_power);
    num("gflops", &r.gflops);
    num("gflops_per_j", &r.gflops_per_j);
    num("temp_c", &r.temp_c);
    num("wall_s", &r.wall_s);
    num("n_launches", &nl);
    num("flags", &fl);
    if (!ok) continue;
    if (!get_num(line, "power_limit_w", &r.power_limit_w)) r.power_limit_w = 0;
    r.clock_mhz_req = (int)clk;
    r.n_launches = (int)nl;
    r.flags = (int)fl;
    (*out)[key] = r;
  }
  free(buf);
  fclose(f);
  return CT_OK;
}

double key_energy(const ct_record& r) { return isnan(r.energy_j) ? INFINITY : r.energy_j; }

}  // namespace

// The selection order of the tuner (ties: shorter time, lower clock,
// lexicographically smaller configuration).
bool record_better(const ct_record& a, const ct_record& b, int objective) {
  auto cfg = [](const ct_record& r) {
    return std::make_tuple(r.cfg.block_x, r.cfg.block_y, r.cfg.tile_x, r.cfg.tile_y,
                           r.cfg.staging, r.cfg.filter_mem, r.cfg.vec_width);
  };
  if (objective == CT_OBJ_TIME)
    return std::make_tuple(a.t_s, key_energy(a), a.clock_mhz_req, cfg(a)) <
           std::make_tuple(b.t_s, key_energy(b), b.clock_mhz_req, cfg(b));
  if (objective == CT_OBJ_GFLOPS_PER_W) {
    const double ga = isnan(a.gflops_per_j) ? -INFINITY : a.gflops_per_j;
    const double gb = isnan(b.gflops_per_j) ? -INFINITY : b.gflops_per_j;
    return std::make_tuple(-ga, a.t_s, a.clock_mhz_req, cfg(a)) <
           std::make_tuple(-gb, b.t_s, b.clock_mhz_req, cfg(b));
  }
  return std::make_tuple(key_energy(a), a.t_s, a.clock_mhz_req, cfg(a)) <
         std::make_tuple(key_energy(b), b.t_s, b.clock_mhz_req, cfg(b));
}

int select_best(const ct_record* recs, int n, int objective, const int* clocks, int n_clocks) {
  int best = -1;
  for (int i = 0; i < n; ++i) {
    const ct_record& r = recs[i];
    if (r.flags & CT_REC_INVALID) continue;
    if (!(r.t_s > 0)) continue;
    if (n_clocks > 0) {
      bool in = false;
      for (int k = 0; k < n_clocks; ++k) in |= clocks[k] == r.clock_mhz_req;
      if (!in) continue;
    }
    if (best < 0 || record_better(r, recs[best], objective)) best = i;
  }
  return best;
}

namespace {

// The exhaustive sweep over configurations x one device setting: SM clocks
// (power_axis = false; 0 = default clocks) or board power limits in mW
// (power_axis = true), setting-major so each setting is applied once and
// undone before the next.
int tune_axis(const ct_problem& p, const ct_config* space, int n_space, bool power_axis,
              const int* settings, int n_settings, const ct_tune_options& opt,
              cudaStream_t stream, ct_record* records, int cap, int* n_records,
              int* best_index) {
  std::vector<ct_config> builtin;
  if (!space) {
    fill_space(CT_SPACE_BASIC, &builtin);
    space = builtin.data();
    n_space = (int)builtin.size();
  }
  if (n_space <= 0) return CT_EINVAL;
  std::vector<int> clk;
  if (settings && n_settings > 0) clk.assign(settings, settings + n_settings);
  else clk.push_back(0);
  const long long needed = (long long)n_space * (long long)clk.size();
  *n_records = (int)needed;
  *best_index = -1;
  if (needed > cap || !records) return CT_ENOMEM;

  const ct_platform_ops ops = platform_ops();
  const bool simulated = ops.run_launches != nullptr;
  const ct_measure_options mopt = resolve_options(&opt.measure);
  std::map<std::string, ct_record> cache;
  FILE* cf = nullptr;
  if (opt.cache_path && opt.cache_path[0]) {
    load_cache(opt.cache_path, &cache);
    cf = fopen(opt.cache_path, "a");
    if (!cf) return CT_EIO;
  }
  const std::string dev = device_tag(simulated);
  const double flop = conv_flop(p);
  int written = 0;
  int rc = CT_OK;
  bool default_clock_fallback = false;
  for (size_t ci = 0; ci < clk.size() && rc == CT_OK; ++ci) {
    const int setting = clk[ci];
    const int clock = power_axis ? 0 : setting;
    const int limit = power_axis ? setting : 0;
    ClockLock lock(ops, default_clock_fallback ? 0 : clock);
    PowerLimit plim(ops, default_clock_fallback ? 0 : limit);
    const bool applied = power_axis ? plim.set() : lock.locked();
    if (setting > 0 && !applied) {
      if (!opt.fallback_default_clocks) {
        const int st = power_axis ? plim.status() : lock.status();
        rc = st == CT_OK ? CT_EPERM : st;
        break;
      }
      default_clock_fallback = true;
    }
    if (applied && opt.settle_s > 0)
      std::this_thread::sleep_for(std::chrono::duration<double>(opt.settle_s));
    for (int i = 0; i < n_space; ++i) {
      ct_record& r = records[written];
      memset(&r, 0, sizeof(r));
      r.cfg = space[i];
      r.clock_mhz_req = clock;
      r.power_limit_w = limit / 1000.0;
      if (default_clock_fallback) r.flags |= CT_REC_DEFAULT_CLOCKS;
      const int rec_clock = default_clock_fallback ? 0 : clock;
      const int rec_limit = default_clock_fallback ? 0 : limit;
      const std::string key = point_key(dev, p, space[i], rec_clock, rec_limit, mopt);
      auto hit = cache.find(key);
      if (hit != cache.end()) {
        const int keep = r.flags;
        r = hit->second;
        r.cfg = space[i];
        r.clock_mhz_req = clock;
        r.power_limit_w = limit / 1000.0;
        r.flags |= CT_REC_CACHED | keep;
        ++written;
        continue;
      }
      ConvPlan plan;
      const int prc = plan_conv(p, space[i], &plan, nullptr, !simulated);
      if (prc == CT_ECONFIG || (prc == CT_OK && plan.empty)) {
        r.flags |= CT_REC_INVALID;
        r.t_s = NAN;
        r.energy_j = NAN;
        ++written;
        continue;
      }
      if (prc != CT_OK) {
        rc = prc;
        break;
      }
      MeasureUnit u;
      u.kind = CT_UNIT_CONV;
      u.cfg = &space[i];
      u.work = flop;
      u.launch = [&plan](cudaStream_t s) { return launch_plan(plan, s); };
      ct_record m;
      const int mrc = measure_unit(u, mopt, ops, stream, clock, &m);
      if (mrc == CT_ECONFIG) {  // launch refused (resources): prune
        r.flags |= CT_REC_INVALID;
        r.t_s = NAN;
        r.energy_j = NAN;
        ++written;
        continue;
      }
      if (mrc != CT_OK) {
        rc = mrc;
        break;
      }
      m.flags |= r.flags;
      if (lock.locked()) {
        // a locked clock that the device did not hold is throttling
        if (m.clock_mhz_meas < clock - 8) m.flags |= CT_REC_THROTTLED;
      }
      r = m;
      r.clock_mhz_req = clock;
      r.power_limit_w = limit / 1000.0;
      if (cf) {
        const std::string line = record_json(key, r);
        fputs(line.c_str(), cf);
        fflush(cf);
      }
      ++written;
    }
    if (default_clock_fallback) break;  // one pass is all default clocks give
  }
  if (cf) fclose(cf);
  *n_records = written;
  if (rc == CT_OK) *best_index = select_best(records, written, opt.objective, nullptr, 0);
  (void)flop;
  return rc;
}

}  // namespace

int tune_impl(const ct_problem& p, const ct_config* space, int n_space, const int* clocks,
              int n_clocks, const ct_tune_options& opt, cudaStream_t stream, ct_record* records,
              int cap, int* n_records, int* best_index) {
  return tune_axis(p, space, n_space, false, clocks, n_clocks, opt, stream, records, cap,
                   n_records, best_index);
}

int tune_power_impl(const ct_problem& p, const ct_config* space, int n_space, const int* limits_mw,
                    int n_limits, const ct_tune_options& opt, cudaStream_t stream,
                    ct_record* records, int cap, int* n_records, int* best_index) {
  return tune_axis(p, space, n_space, true, limits_mw, n_limits, opt, stream, records, cap,
                   n_records, best_index);
}

}  // namespace convtune

using namespace convtune;

extern "C" {

int ct_space(int which, ct_config* out, int cap, int* n) {
  if (!n || (which != CT_SPACE_BASIC && which != CT_SPACE_FULL)) return CT_EINVAL;
  std::vector<ct_config> v;
  fill_space(which, &v);
  *n = (int)v.size();
  if (!out || cap < (int)v.size()) return CT_ENOMEM;
  memcpy(out, v.data(), sizeof(ct_config) * v.size());
  return CT_OK;
}

int ct_select_best(const ct_record* recs, int n, int objective, const int* clocks, int n_clocks,
                   int* best_index) {
  if (!recs || n < 0 || !best_index || (n_clocks > 0 && !clocks)) return CT_EINVAL;
  *best_index = select_best(recs, n, objective, clocks, n_clocks);
  return CT_OK;
}

int ct_tune_power_limits(const ct_problem* p, const ct_config* space, int n_space,
                         const int* limits_mw, int n_limits, const ct_tune_options* opt,
                         void* stream, ct_record* records, int cap, int* n_records,
                         int* best_index) {
  if (!p || !opt || !n_records || !best_index) return CT_EINVAL;
  if (opt->objective < CT_OBJ_TIME || opt->objective > CT_OBJ_GFLOPS_PER_W) return CT_EINVAL;
  if (n_limits < 0 || (n_limits > 0 && !limits_mw)) return CT_EINVAL;
  for (int i = 0; i < n_limits; ++i)
    if (limits_mw[i] <= 0) return CT_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return tune_power_impl(*p, space, n_space, limits_mw, n_limits, *opt, (cudaStream_t)stream,
                         records, cap, n_records, best_index);
}

int ct_tune(const ct_problem* p, const ct_config* space, int n_space, const int* clocks_mhz,
            int n_clocks, const ct_tune_options* opt, void* stream, ct_record* records, int cap,
            int* n_records, int* best_index) {
  if (!p || !opt || !n_records || !best_index) return CT_EINVAL;
  if (opt->objective < CT_OBJ_TIME || opt->objective > CT_OBJ_GFLOPS_PER_W) return CT_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return tune_impl(*p, space, n_space, clocks_mhz, n_clocks, *opt, (cudaStream_t)stream, records,
                   cap, n_records, best_index);
}

}  // extern "C"
