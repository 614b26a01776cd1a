// GPU power model of Section IV-E (Eq. powercurve) -- host FP64.
//
//   P*(f) = min(P_max, P_idle + alpha * f * v(f)^2)
//   v(f)  = measured core voltage, or the estimate 1 + beta * max(0, f - tau)
//
// Fit: the paper fits Eq. powercurve by non-linear least squares with the
// Levenberg-Marquardt method (More 1978), using samples up to the highest
// clock before throttling.  tau is a kink, not a smooth parameter, so it runs
// over the integer-MHz grid between the lowest and highest kept sample (a
// grid point needs two kept samples strictly above it); at each grid point
// LM fits (P_idle, alpha, beta >= 0) from four starts (beta = 0 and beta in
// {0.1, 1, 10} per GHz, with P_idle and alpha the linear least-squares
// solution at that beta), then Gauss-Newton steps polish the minimum while
// they contract.  The least residual wins; a relative difference
// of 1e-12 or less is a tie and keeps the smaller tau.  Frequencies are in
// GHz inside the solver.  P_max is the caller's value, else the largest
// measured power; it enters only the prediction.
//
// Optimum: P*(f)/f is proportional to energy per clock cycle (a kernel's
// time scales as 1/f); its minimiser over [lowest kept, highest kept]
// sample clock is the predicted most energy-efficient clock.  Range: the
// supported clocks within +-rel of it (+-10 % in the paper).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/convtune.h"

namespace {

constexpr int kMaxIter = 500;
constexpr double kStepTol = 1e-15;
constexpr double kTieRel = 1e-12;

// p ~= a + b x in the least-squares sense.
void line_fit(const std::vector<double>& x, const std::vector<double>& p, double* a, double* b) {
  const size_t n = x.size();
  double xm = 0, pm = 0;
  for (size_t i = 0; i < n; ++i) {
    xm += x[i];
    pm += p[i];
  }
  xm /= n;
  pm /= n;
  double sxx = 0, sxp = 0;
  for (size_t i = 0; i < n; ++i) {
    sxx += (x[i] - xm) * (x[i] - xm);
    sxp += (x[i] - xm) * (p[i] - pm);
  }
  *b = sxx > 0 ? sxp / sxx : 0.0;
  *a = pm - *b * xm;
}

struct Samples {
  std::vector<double> f, d, p;  // GHz, GHz above tau, W
};

double residual_sq(const Samples& s, const double th[3]) {
  double acc = 0;
  for (size_t i = 0; i < s.f.size(); ++i) {
    const double v = 1.0 + th[2] * s.d[i];
    const double r = s.p[i] - (th[0] + th[1] * s.f[i] * v * v);
    acc += r * r;
  }
  return acc;
}

// Solve the 3x3 system m y = g by Gaussian elimination with partial pivoting.
bool solve3(double m[3][3], double g[3], double y[3]) {
  int idx[3] = {0, 1, 2};
  for (int c = 0; c < 3; ++c) {
    int piv = c;
    for (int r = c + 1; r < 3; ++r)
      if (fabs(m[idx[r]][c]) > fabs(m[idx[piv]][c])) piv = r;
    std::swap(idx[c], idx[piv]);
    const double dgl = m[idx[c]][c];
    if (dgl == 0.0 || !isfinite(dgl)) return false;
    for (int r = c + 1; r < 3; ++r) {
      const double fct = m[idx[r]][c] / dgl;
      for (int k = c; k < 3; ++k) m[idx[r]][k] -= fct * m[idx[c]][k];
      g[idx[r]] -= fct * g[idx[c]];
    }
  }
  for (int c = 2; c >= 0; --c) {
    double acc = g[idx[c]];
    for (int k = c + 1; k < 3; ++k) acc -= m[idx[c]][k] * y[k];
    y[c] = acc / m[idx[c]][c];
  }
  return isfinite(y[0]) && isfinite(y[1]) && isfinite(y[2]);
}

// Projected Levenberg-Marquardt on (P_idle, alpha, beta >= 0) at fixed tau.
double lm_fit(const Samples& s, double th[3]) {
  th[2] = std::max(th[2], 0.0);
  double cur = residual_sq(s, th);
  double lambda = 1e-3;
  const size_t n = s.f.size();
  for (int it = 0; it < kMaxIter; ++it) {
    // normal equations J^T J and J^T r of the model's Jacobian
    double a[3][3] = {{0}}, g[3] = {0};
    for (size_t i = 0; i < n; ++i) {
      const double v = 1.0 + th[2] * s.d[i];
      const double j[3] = {1.0, s.f[i] * v * v, 2.0 * th[1] * s.f[i] * v * s.d[i]};
      const double r = s.p[i] - (th[0] + th[1] * s.f[i] * v * v);
      for (int q = 0; q < 3; ++q) {
        g[q] += j[q] * r;
        for (int k = 0; k < 3; ++k) a[q][k] += j[q] * j[k];
      }
    }
    bool accepted = false;
    double cand[3], cand_s = 0;
    while (lambda <= 1e16) {
      double m[3][3], rhs[3], step[3];
      for (int q = 0; q < 3; ++q) {
        for (int k = 0; k < 3; ++k) m[q][k] = a[q][k];
        m[q][q] += lambda * std::max(a[q][q], 1e-300);
        rhs[q] = g[q];
      }
      if (!solve3(m, rhs, step)) {
        lambda *= 10.0;
        continue;
      }
      for (int q = 0; q < 3; ++q) cand[q] = th[q] + step[q];
      cand[2] = std::max(cand[2], 0.0);
      cand_s = residual_sq(s, cand);
      if (cand_s < cur) {
        accepted = true;
        break;
      }
      lambda *= 10.0;
    }
    if (!accepted) break;
    double step2 = 0, scale2 = 0;
    for (int q = 0; q < 3; ++q) {
      step2 += (cand[q] - th[q]) * (cand[q] - th[q]);
      scale2 += th[q] * th[q];
      th[q] = cand[q];
    }
    cur = cand_s;
    lambda = std::max(lambda / 10.0, 1e-300);
    if (sqrt(step2) <= kStepTol * std::max(sqrt(scale2), 1e-300)) break;
  }
  return cur;
}

// After LM: Gauss-Newton steps (lambda = 0) while they contract.  LM's test
// "the residual decreased" cannot see changes below the residual's rounding,
// which leaves the parameters at ~sqrt(eps) relative accuracy; the
// Gauss-Newton step follows the gradient J^T r and converges to the
// stationary point.  beta stays at 0 when its bound is active.
double gn_polish(const Samples& s, double th[3]) {
  const size_t n = s.f.size();
  double last = INFINITY;
  for (int it = 0; it < 100; ++it) {
    const bool beta_free = th[2] != 0.0;
    const int nf = beta_free ? 3 : 2;
    double a[3][3] = {{0}}, g[3] = {0};
    for (size_t i = 0; i < n; ++i) {
      const double v = 1.0 + th[2] * s.d[i];
      const double j[3] = {1.0, s.f[i] * v * v, 2.0 * th[1] * s.f[i] * v * s.d[i]};
      const double r = s.p[i] - (th[0] + th[1] * s.f[i] * v * v);
      for (int q = 0; q < nf; ++q) {
        g[q] += j[q] * r;
        for (int k = 0; k < nf; ++k) a[q][k] += j[q] * j[k];
      }
    }
    double step[3] = {0, 0, 0};
    if (nf == 3) {
      if (!solve3(a, g, step)) break;
    } else {
      const double det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
      if (det == 0.0 || !isfinite(det)) break;
      step[0] = (g[0] * a[1][1] - a[0][1] * g[1]) / det;
      step[1] = (a[0][0] * g[1] - a[1][0] * g[0]) / det;
    }
    const double size = sqrt(step[0] * step[0] + step[1] * step[1] + step[2] * step[2]);
    if (!(size < last)) break;
    if (th[2] + step[2] < 0.0) break;
    double scale2 = 0;
    for (int q = 0; q < 3; ++q) {
      th[q] += step[q];
      scale2 += th[q] * th[q];
    }
    last = size;
    if (size <= kStepTol * std::max(sqrt(scale2), 1e-300)) break;
  }
  return residual_sq(s, th);
}

double model_q(const ct_power_model& m, double f_ghz) {
  const double tau = m.tau_mhz / 1000.0;
  const double v = 1.0 + m.beta * std::max(0.0, f_ghz - tau);
  return m.p_idle_w + m.alpha * f_ghz * v * v;
}

double energy_per_cycle(const ct_power_model& m, double f_ghz) {
  return std::min(m.p_max_w, model_q(m, f_ghz)) / f_ghz;
}

// Roots of fn on [lo, hi]: sign changes on a uniform scan, refined by
// bisection down to adjacent doubles.
template <class F>
void scan_roots(F fn, double lo, double hi, std::vector<double>* out) {
  if (!(hi > lo)) return;
  const int n = 4096;
  double x0 = lo, y0 = fn(lo);
  if (y0 == 0.0) out->push_back(lo);
  for (int k = 1; k <= n; ++k) {
    const double x1 = k == n ? hi : lo + (hi - lo) * k / n;
    const double y1 = fn(x1);
    if (y1 == 0.0) {
      out->push_back(x1);
    } else if ((y0 < 0) != (y1 < 0) && y0 != 0.0) {
      double a = x0, b = x1, ya = y0;
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (a + b);
        if (mid <= a || mid >= b) break;
        const double ym = fn(mid);
        if (ym == 0.0) {
          a = b = mid;
          break;
        }
        if ((ym < 0) == (ya < 0)) {
          a = mid;
          ya = ym;
        } else {
          b = mid;
        }
      }
      out->push_back(0.5 * (a + b));
    }
    x0 = x1;
    y0 = y1;
  }
}

double optimum_estimated(const ct_power_model& m) {
  const double lo = m.f_lo_mhz / 1000.0, hi = m.f_thr_mhz / 1000.0;
  const double tau = m.tau_mhz / 1000.0;
  std::vector<double> cand = {lo, hi};
  if (tau >= lo && tau <= hi) cand.push_back(tau);
  // stationary points of Q(f)/f above tau: P_idle = 2 alpha beta f^2 v(f)
  const double a = m.alpha, b = m.beta, p0 = m.p_idle_w;
  scan_roots([&](double f) { return 2.0 * a * b * f * f * (1.0 + b * (f - tau)) - p0; },
             std::max(lo, tau), hi, &cand);
  // where the P_max cap starts or ends
  scan_roots([&](double f) { return model_q(m, f) - m.p_max_w; }, lo, hi, &cand);
  std::sort(cand.begin(), cand.end());
  double best = cand[0], best_h = energy_per_cycle(m, cand[0]);
  for (double c : cand) {
    const double h = energy_per_cycle(m, c);
    if (h < best_h) {
      best_h = h;
      best = c;
    }
  }
  return best * 1000.0;
}

}  // namespace

extern "C" {

int ct_fit_power_model(const double* f_mhz, const double* p_w, const double* v_or_null,
                       const int* throttled_or_null, int n, double p_max_w, ct_power_model* out) {
  if (!f_mhz || !p_w || !out || n < 0) return CT_EINVAL;
  memset(out, 0, sizeof(*out));
  std::vector<double> fk, pk, vk;
  double pmax_seen = -INFINITY;
  for (int i = 0; i < n; ++i) {
    if (!isfinite(f_mhz[i]) || !isfinite(p_w[i]) || f_mhz[i] <= 0) return CT_EINVAL;
    pmax_seen = std::max(pmax_seen, p_w[i]);
    if (throttled_or_null && throttled_or_null[i]) continue;
    fk.push_back(f_mhz[i]);
    pk.push_back(p_w[i]);
    if (v_or_null) vk.push_back(v_or_null[i]);
  }
  if (fk.size() < 3) return CT_EINVAL;
  out->p_max_w = p_max_w > 0 ? p_max_w : pmax_seen;
  out->n_used = (int)fk.size();
  out->f_lo_mhz = *std::min_element(fk.begin(), fk.end());
  out->f_thr_mhz = *std::max_element(fk.begin(), fk.end());

  if (v_or_null) {
    std::vector<double> x(fk.size());
    for (size_t i = 0; i < fk.size(); ++i) x[i] = fk[i] / 1000.0 * vk[i] * vk[i];
    double a, b;
    line_fit(x, pk, &a, &b);
    double s = 0;
    for (size_t i = 0; i < x.size(); ++i) s += (pk[i] - a - b * x[i]) * (pk[i] - a - b * x[i]);
    out->p_idle_w = a;
    out->alpha = b;
    out->has_voltage = 1;
    out->sse = s;
    // optimum over the kept sample clocks (ties: lower clock)
    double best_h = INFINITY, best_f = 0;
    for (size_t i = 0; i < x.size(); ++i) {
      const double h = std::min(out->p_max_w, a + b * x[i]) / fk[i];
      if (h < best_h || (h == best_h && fk[i] < best_f)) {
        best_h = h;
        best_f = fk[i];
      }
    }
    out->f_opt_mhz = best_f;
    return CT_OK;
  }

  Samples s;
  s.f.resize(fk.size());
  s.d.resize(fk.size());
  s.p = pk;
  for (size_t i = 0; i < fk.size(); ++i) s.f[i] = fk[i] / 1000.0;
  const int lo = (int)ceil(out->f_lo_mhz), hi = (int)floor(out->f_thr_mhz);
  bool have = false;
  double best_s = INFINITY, best_th[3] = {0, 0, 0};
  int best_tau = 0;
  std::vector<double> x(fk.size());
  for (int tau = lo; tau <= hi; ++tau) {
    int above = 0;
    for (double f : fk) above += f > tau;
    if (above < 2) continue;
    for (size_t i = 0; i < fk.size(); ++i) s.d[i] = std::max(0.0, fk[i] - tau) / 1000.0;
    double tau_best_s = INFINITY, tau_best[3] = {0, 0, 0};
    const double beta0[4] = {0.0, 0.1, 1.0, 10.0};
    for (double b0 : beta0) {
      for (size_t i = 0; i < fk.size(); ++i) {
        const double v = 1.0 + b0 * s.d[i];
        x[i] = s.f[i] * v * v;
      }
      double th[3];
      line_fit(x, pk, &th[0], &th[1]);
      th[2] = b0;
      lm_fit(s, th);
      const double r = gn_polish(s, th);
      if (r < tau_best_s) {
        tau_best_s = r;
        memcpy(tau_best, th, sizeof(th));
      }
    }
    if (!have || tau_best_s < best_s - kTieRel * best_s) {
      have = true;
      best_s = tau_best_s;
      best_tau = tau;
      memcpy(best_th, tau_best, sizeof(best_th));
    }
  }
  if (!have) return CT_EINVAL;
  out->p_idle_w = best_th[0];
  out->alpha = best_th[1];
  out->beta = best_th[2];
  out->tau_mhz = best_tau;
  out->sse = best_s;
  out->has_voltage = 0;
  out->f_opt_mhz = optimum_estimated(*out);
  return CT_OK;
}

int ct_model_power(const ct_power_model* m, const double* f_mhz, int n, double* p_w) {
  if (!m || !f_mhz || !p_w || n < 0 || m->has_voltage) return CT_EINVAL;
  for (int i = 0; i < n; ++i) p_w[i] = std::min(m->p_max_w, model_q(*m, f_mhz[i] / 1000.0));
  return CT_OK;
}

int ct_optimal_clock(const ct_power_model* m, double* f_opt_mhz) {
  if (!m || !f_opt_mhz) return CT_EINVAL;
  if (m->has_voltage) {
    *f_opt_mhz = m->f_opt_mhz;
    return CT_OK;
  }
  if (!(m->f_thr_mhz >= m->f_lo_mhz) || m->f_lo_mhz <= 0) return CT_EINVAL;
  *f_opt_mhz = optimum_estimated(*m);
  return CT_OK;
}

int ct_pick_clock_range(const ct_power_model* m, const int* supported_mhz, int n_supported,
                        double rel_halfwidth, int center, int* out_mhz, int cap, int* n_out,
                        double* center_mhz) {
  if (!m || !supported_mhz || n_supported <= 0 || !n_out || rel_halfwidth < 0) return CT_EINVAL;
  double c0;
  if (center == 1) {
    c0 = m->tau_mhz;
  } else {
    const int rc = ct_optimal_clock(m, &c0);
    if (rc != CT_OK) return rc;
  }
  if (center_mhz) *center_mhz = c0;
  std::vector<int> sup(supported_mhz, supported_mhz + n_supported);
  std::sort(sup.begin(), sup.end());
  const double lo = (1.0 - rel_halfwidth) * c0, hi = (1.0 + rel_halfwidth) * c0;
  std::vector<int> sel;
  for (int c : sup)
    if (c >= lo && c <= hi) sel.push_back(c);
  if (sel.empty()) {
    int best = sup[0];
    for (int c : sup)
      if (fabs(c - c0) < fabs(best - c0)) best = c;
    sel.push_back(best);
  }
  *n_out = (int)sel.size();
  if ((int)sel.size() > cap || (!out_mhz && cap > 0)) return CT_ENOMEM;
  for (size_t i = 0; i < sel.size(); ++i) out_mhz[i] = sel[i];
  return CT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Memory-aware energy model (Sections II and IV-F): t(f) = t_mem + c_core / f
// by non-negative least squares in (1, 1/f), E(f) = P*(f) t(f), minimised over
// the integer-MHz clocks both fits cover.
// ---------------------------------------------------------------------------
namespace {

double time_sse(const std::vector<double>& u, const std::vector<double>& t, double a, double b) {
  double acc = 0;
  for (size_t i = 0; i < u.size(); ++i) {
    const double r = t[i] - (a + b * u[i]);
    acc += r * r;
  }
  return acc;
}

double model_time_at(const ct_time_model& tm, double f_mhz) {
  return tm.t_mem_s + tm.c_core_s_ghz / (f_mhz / 1000.0);
}

double model_energy_at(const ct_power_model& pm, const ct_time_model& tm, double f_mhz) {
  return std::min(pm.p_max_w, model_q(pm, f_mhz / 1000.0)) * model_time_at(tm, f_mhz);
}

}  // namespace

extern "C" {

int ct_fit_time_model(const double* f_mhz, const double* t_s, const int* throttled_or_null,
                      int n, ct_time_model* out) {
  if (!f_mhz || !t_s || !out || n < 0) return CT_EINVAL;
  memset(out, 0, sizeof(*out));
  std::vector<double> u, t, fk;
  for (int i = 0; i < n; ++i) {
    if (!isfinite(f_mhz[i]) || f_mhz[i] <= 0 || !isfinite(t_s[i])) return CT_EINVAL;
    if (throttled_or_null && throttled_or_null[i]) continue;
    fk.push_back(f_mhz[i]);
    u.push_back(1000.0 / f_mhz[i]);
    t.push_back(t_s[i]);
  }
  if (fk.size() < 2) return CT_EINVAL;
  const size_t m = u.size();
  double um = 0, tmn = 0;
  for (size_t i = 0; i < m; ++i) {
    um += u[i];
    tmn += t[i];
  }
  um /= m;
  tmn /= m;
  double suu = 0, sut = 0, tu = 0, uu = 0;
  for (size_t i = 0; i < m; ++i) {
    suu += (u[i] - um) * (u[i] - um);
    sut += (u[i] - um) * (t[i] - tmn);
    tu += t[i] * u[i];
    uu += u[i] * u[i];
  }
  // candidates: the unconstrained solution if feasible, then the faces
  // t_mem = 0 and c_core = 0 (first least residual wins)
  double cand[3][2];
  int nc = 0;
  if (suu > 0) {
    const double b = sut / suu, a = tmn - b * um;
    if (a >= 0 && b >= 0) {
      cand[nc][0] = a;
      cand[nc][1] = b;
      ++nc;
    }
  }
  cand[nc][0] = 0.0;
  cand[nc][1] = std::max(0.0, tu / uu);
  ++nc;
  cand[nc][0] = std::max(0.0, tmn);
  cand[nc][1] = 0.0;
  ++nc;
  int best = 0;
  double best_s = time_sse(u, t, cand[0][0], cand[0][1]);
  for (int c = 1; c < nc; ++c) {
    const double sc = time_sse(u, t, cand[c][0], cand[c][1]);
    if (sc < best_s) {
      best_s = sc;
      best = c;
    }
  }
  out->t_mem_s = cand[best][0];
  out->c_core_s_ghz = cand[best][1];
  out->sse = best_s;
  out->n_used = (int)m;
  out->f_lo_mhz = *std::min_element(fk.begin(), fk.end());
  out->f_thr_mhz = *std::max_element(fk.begin(), fk.end());
  return CT_OK;
}

int ct_model_time(const ct_time_model* tm, const double* f_mhz, int n, double* t_s) {
  if (!tm || !f_mhz || !t_s || n < 0) return CT_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!(f_mhz[i] > 0)) return CT_EINVAL;
    t_s[i] = model_time_at(*tm, f_mhz[i]);
  }
  return CT_OK;
}

int ct_memory_aware_optimum(const ct_power_model* pm, const ct_time_model* tm,
                            double* f_opt_mhz, double* e_opt_j) {
  if (!pm || !tm || !f_opt_mhz || pm->has_voltage) return CT_EINVAL;
  const double lo = std::max(pm->f_lo_mhz, tm->f_lo_mhz);
  const double hi = std::min(pm->f_thr_mhz, tm->f_thr_mhz);
  const long glo = (long)ceil(lo), ghi = (long)floor(hi);
  if (!(glo > 0) || ghi < glo) return CT_EINVAL;
  double best_f = (double)glo, best_e = model_energy_at(*pm, *tm, (double)glo);
  for (long f = glo + 1; f <= ghi; ++f) {
    const double e = model_energy_at(*pm, *tm, (double)f);
    if (e < best_e) {  // strict: ties keep the lower clock
      best_e = e;
      best_f = (double)f;
    }
  }
  *f_opt_mhz = best_f;
  if (e_opt_j) *e_opt_j = best_e;
  return CT_OK;
}

int ct_clock_range(double center_mhz, const int* supported_mhz, int n_supported,
                   double rel_halfwidth, int* out_mhz, int cap, int* n_out) {
  if (!supported_mhz || n_supported <= 0 || !n_out || rel_halfwidth < 0 ||
      !isfinite(center_mhz))
    return CT_EINVAL;
  std::vector<int> sup(supported_mhz, supported_mhz + n_supported);
  std::sort(sup.begin(), sup.end());
  const double lo = (1.0 - rel_halfwidth) * center_mhz, hi = (1.0 + rel_halfwidth) * center_mhz;
  std::vector<int> sel;
  for (int c : sup)
    if (c >= lo && c <= hi) sel.push_back(c);
  if (sel.empty()) {
    int best = sup[0];
    for (int c : sup)
      if (fabs(c - center_mhz) < fabs(best - center_mhz)) best = c;
    sel.push_back(best);
  }
  *n_out = (int)sel.size();
  if ((int)sel.size() > cap || (!out_mhz && cap > 0)) return CT_ENOMEM;
  for (size_t i = 0; i < sel.size(); ++i) out_mhz[i] = sel[i];
  return CT_OK;
}

}  // extern "C"
