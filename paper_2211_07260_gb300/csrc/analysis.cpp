// Analyses over tuning records (Section IV-A and IV-B of the paper): the
// five tuning methods compared in Fig. 3, the Pareto front of speed versus
// energy efficiency (Fig. 4) and the proportion of PageRank centrality of
// good local minima in the fitness flow graph (Fig. 5).
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <functional>
#include <map>
#include <numeric>
#include <vector>

#include "../../include/convtune.h"

namespace convtune {
bool record_better(const ct_record& a, const ct_record& b, int objective);
}  // namespace convtune

using namespace convtune;

namespace {

bool usable(const ct_record& r) { return !(r.flags & CT_REC_INVALID) && r.t_s > 0; }

int best_where(const ct_record* recs, int n, int objective,
               const std::function<bool(const ct_record&)>& keep) {
  int best = -1;
  for (int i = 0; i < n; ++i) {
    if (!usable(recs[i]) || !keep(recs[i])) continue;
    if (best < 0 || record_better(recs[i], recs[best], objective)) best = i;
  }
  return best;
}

bool same_cfg(const ct_config& a, const ct_config& b) { return memcmp(&a, &b, sizeof(a)) == 0; }

// the 8 parameters of a point: the configuration and the requested clock
void params(const ct_record& r, int p[8]) {
  p[0] = r.cfg.block_x;
  p[1] = r.cfg.block_y;
  p[2] = r.cfg.tile_x;
  p[3] = r.cfg.tile_y;
  p[4] = r.cfg.staging;
  p[5] = r.cfg.filter_mem;
  p[6] = r.cfg.vec_width;
  p[7] = r.clock_mhz_req;
}

}  // namespace

extern "C" {

int ct_tuning_methods(const ct_record* recs, int n, int base_clock_mhz, int out[5]) {
  if (!recs || n <= 0 || !out) return CT_EINVAL;
  int cmax = INT_MIN;
  int cbase = 0;
  double dbest = INFINITY;
  for (int i = 0; i < n; ++i) {
    if (!usable(recs[i])) continue;
    cmax = std::max(cmax, recs[i].clock_mhz_req);
  }
  if (cmax == INT_MIN) return CT_EINVAL;
  for (int i = 0; i < n; ++i) {  // sampled clock nearest the base clock (ties lower)
    if (!usable(recs[i])) continue;
    const int c = recs[i].clock_mhz_req;
    const double d = fabs((double)c - base_clock_mhz);
    if (d < dbest || (d == dbest && c < cbase)) {
      dbest = d;
      cbase = c;
    }
  }
  auto any = [](const ct_record&) { return true; };
  auto at = [](int c) { return [c](const ct_record& r) { return r.clock_mhz_req == c; }; };
  out[0] = best_where(recs, n, CT_OBJ_TIME, any);                   // race-to-idle
  out[1] = best_where(recs, n, CT_OBJ_ENERGY, at(cmax));            // energy at max clock
  const int fast = best_where(recs, n, CT_OBJ_TIME, at(cmax));
  const ct_config cf = recs[fast].cfg;
  out[2] = best_where(recs, n, CT_OBJ_ENERGY,
                      [&](const ct_record& r) { return same_cfg(r.cfg, cf); });  // + clocks
  const int eff = best_where(recs, n, CT_OBJ_ENERGY, at(cbase));
  const ct_config ce = recs[eff].cfg;
  out[3] = best_where(recs, n, CT_OBJ_ENERGY,
                      [&](const ct_record& r) { return same_cfg(r.cfg, ce); });  // + clocks
  out[4] = best_where(recs, n, CT_OBJ_ENERGY, any);                 // global energy
  return CT_OK;
}

int ct_pareto_front(const ct_record* recs, int n, int* out_idx, int cap, int* n_out) {
  if (!recs || n < 0 || !n_out) return CT_EINVAL;
  std::vector<int> idx;
  for (int i = 0; i < n; ++i)
    if (usable(recs[i]) && !isnan(recs[i].gflops_per_j)) idx.push_back(i);
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    if (recs[a].gflops != recs[b].gflops) return recs[a].gflops > recs[b].gflops;
    if (recs[a].gflops_per_j != recs[b].gflops_per_j)
      return recs[a].gflops_per_j > recs[b].gflops_per_j;
    return a < b;
  });
  // a group of equal speed is on the front with its best efficiency only if
  // that efficiency beats every strictly faster point
  std::vector<int> front;
  double best_prev = -INFINITY;
  for (size_t s = 0; s < idx.size();) {
    size_t e = s;
    while (e < idx.size() && recs[idx[e]].gflops == recs[idx[s]].gflops) ++e;
    const double gmax = recs[idx[s]].gflops_per_j;
    if (gmax > best_prev)
      for (size_t q = s; q < e && recs[idx[q]].gflops_per_j == gmax; ++q) front.push_back(idx[q]);
    best_prev = std::max(best_prev, gmax);
    s = e;
  }
  *n_out = (int)front.size();
  if ((int)front.size() > cap || (!out_idx && cap > 0)) return CT_ENOMEM;
  for (size_t q = 0; q < front.size(); ++q) out_idx[q] = front[q];
  return CT_OK;
}

int ct_centrality(const ct_record* recs, int n, int objective, double damping, const double* ps,
                  int n_p, double* out_prop) {
  if (!recs || n <= 0 || !ps || n_p <= 0 || !out_prop) return CT_EINVAL;
  if (!(damping >= 0 && damping < 1)) return CT_EINVAL;
  if (objective != CT_OBJ_TIME && objective != CT_OBJ_ENERGY) return CT_EINVAL;
  std::vector<int> node;  // usable records
  for (int i = 0; i < n; ++i)
    if (usable(recs[i]) && (objective == CT_OBJ_TIME || !isnan(recs[i].energy_j))) node.push_back(i);
  const int m = (int)node.size();
  if (m == 0) return CT_EINVAL;
  std::vector<double> fit(m);
  std::vector<std::array<int, 8>> par(m);
  for (int a = 0; a < m; ++a) {
    const ct_record& r = recs[node[a]];
    fit[a] = objective == CT_OBJ_TIME ? r.t_s : r.energy_j;
    int p[8];
    params(r, p);
    for (int d = 0; d < 8; ++d) par[a][d] = p[d];
  }
  // neighbours differ in exactly one parameter: group by the other seven
  std::vector<std::vector<int>> adj(m);
  for (int d = 0; d < 8; ++d) {
    std::map<std::array<int, 8>, std::vector<int>> groups;
    for (int a = 0; a < m; ++a) {
      std::array<int, 8> key = par[a];
      key[d] = 0;
      groups[key].push_back(a);
    }
    for (auto& kv : groups) {
      const std::vector<int>& g = kv.second;
      for (int a : g)
        for (int b : g)
          if (par[a][d] != par[b][d] && fit[b] < fit[a]) adj[a].push_back(b);
    }
  }
  // PageRank: power iteration, minima (no out-edges) restart uniformly
  std::vector<double> pr(m, 1.0 / m), nx(m);
  for (int it = 0; it < 10000; ++it) {
    double dangling = 0;
    for (int a = 0; a < m; ++a)
      if (adj[a].empty()) dangling += pr[a];
    const double base = (1.0 - damping) / m + damping * dangling / m;
    std::fill(nx.begin(), nx.end(), base);
    for (int a = 0; a < m; ++a) {
      if (adj[a].empty()) continue;
      const double share = damping * pr[a] / adj[a].size();
      for (int b : adj[a]) nx[b] += share;
    }
    double delta = 0;
    for (int a = 0; a < m; ++a) delta += fabs(nx[a] - pr[a]);
    pr.swap(nx);
    if (delta < 1e-14) break;
  }
  const double fopt = *std::min_element(fit.begin(), fit.end());
  double total = 0;
  for (int a = 0; a < m; ++a)
    if (adj[a].empty()) total += pr[a];
  for (int q = 0; q < n_p; ++q) {
    double good = 0;
    for (int a = 0; a < m; ++a)
      if (adj[a].empty() && fit[a] <= ps[q] * fopt) good += pr[a];
    out_prop[q] = good / total;
  }
  return CT_OK;
}

}  // extern "C"
