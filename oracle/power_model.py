"""Oracle: FP64 power-curve fit, energy-optimal clock and steered clock range.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product library
never imports this module, and this module imports nothing from the product.

What the paper fixes (Section IV-E, "Model-steered frequency tuning"):

* Eq. (powercurve): the estimated load power is
  ``P*_load = min(P_max, P*_idle + alpha * f * v**2)``.
* Eq. (powersum) motivates it: dynamic power ~ f * V**2 on top of static power.
* For GPUs without a voltage readout, v is replaced by an estimate that is 1
  below a threshold frequency tau and rises with rate beta above it
  ("Estimating GPU core voltage").
* The model is fitted by non-linear least squares with the
  Levenberg-Marquardt method (Section III-A, citing More 1978), using only
  samples up to the highest clock before throttling ("Fitting the model").
* Estimated energy is proportional to P*_load(f) / f; its minimiser is the
  predicted most energy-efficient clock; tuning is then run over a range of
  +-10 % around it (last paragraph of Section IV-E).

Readings taken where the paper is silent or garbled:

* The printed voltage estimate gives v = beta*(f - tau) for f >= tau, which is
  0 at f = tau and drops the power to P_idle at the knee, contradicting the
  text (voltage "unchanged" up to the ridge point, then increasing).  It is
  read as the continuous ``v(f) = 1 + beta * max(0, f - tau)``.
* tau is not a smooth parameter (the residual has kinks at the samples), so it
  is searched over the integer-MHz grid between the lowest and highest kept
  sample; for each grid tau, LM fits (P_idle, alpha, beta) with beta >= 0
  (projected), from four starts: the beta = 0 closed form and
  beta0 in {0.1, 1, 10} per GHz with (P_idle, alpha) the linear least-squares
  solution at that beta0.  LM stops when the relative step is below 1e-15 or
  after 500 iterations, or when no step lowers the residual; Gauss-Newton
  steps (LM with lambda = 0) then continue while they contract, because the
  residual's last bits cannot resolve the parameters beyond ~sqrt(eps).
  The tau with the least residual wins; residuals within 1e-12 relative
  count as a tie and the smaller tau is kept.  A tau needs at
  least two kept samples strictly above it.
* P_max is not fitted: the caller's value, else the largest measured power
  over all samples (throttled ones included), used only in prediction.
* Frequencies are in GHz inside the solver (beta per GHz, alpha in W/GHz with
  the estimated v, W/(GHz V^2) with a measured v) and in MHz at the interface.
* With measured voltage the model is linear in (P_idle, alpha) with
  x = f * v**2 and is solved in closed form; the optimum is then taken over the
  kept sample clocks (ties: lower clock).
* The +-10 % window is centred on the model optimum (the closing paragraph);
  Table II's caption centres it on the ridge point instead, available here as
  ``center="ridge"`` (tau).
* A sample is "throttled" when the caller flags it (clock below the request or
  a throttle reason set).
"""
from __future__ import annotations

import math

import numpy as np

LM_MAX_ITER = 500
LM_STEP_TOL = 1e-15
TAU_TIE_REL = 1e-12
BETA_STARTS = (0.1, 1.0, 10.0)


def _linear_fit(x, p):
    """Least-squares line p = a + b*x (closed form); returns (a, b)."""
    xm = x.mean()
    pm = p.mean()
    sxx = float(((x - xm) ** 2).sum())
    if sxx == 0.0:
        return float(pm), 0.0
    b = float(((x - xm) * (p - pm)).sum()) / sxx
    return float(pm - b * xm), b


def _model(theta, f, d):
    p_idle, alpha, beta = theta
    v = 1.0 + beta * d
    return p_idle + alpha * f * v * v


def _jacobian(theta, f, d):
    _, alpha, beta = theta
    v = 1.0 + beta * d
    return np.stack([np.ones_like(f), f * v * v, 2.0 * alpha * f * v * d], axis=1)


def _levenberg_marquardt(theta0, f, d, p):
    """Projected Levenberg-Marquardt (More 1978 scaling) for one fixed tau.

    Minimises S = sum (p_i - m(f_i))^2 over theta = (P_idle, alpha, beta),
    beta >= 0.  Returns (theta, S).
    """
    theta = np.array(theta0, dtype=np.float64)
    theta[2] = max(theta[2], 0.0)
    r = p - _model(theta, f, d)
    s = float(r @ r)
    lam = 1e-3
    for _ in range(LM_MAX_ITER):
        jac = _jacobian(theta, f, d)
        a = jac.T @ jac
        g = jac.T @ r
        dscale = np.maximum(np.diag(a), 1e-300)
        accepted = False
        while lam <= 1e16:
            m = a + lam * np.diag(dscale)
            try:
                delta = np.linalg.solve(m, g)
            except np.linalg.LinAlgError:
                lam *= 10.0
                continue
            cand = theta + delta
            cand[2] = max(cand[2], 0.0)
            rc = p - _model(cand, f, d)
            sc = float(rc @ rc)
            if sc < s:
                accepted = True
                break
            lam *= 10.0
        if not accepted:
            break
        step = float(np.linalg.norm(cand - theta))
        scale = float(np.linalg.norm(theta))
        theta, r, s = cand, rc, sc
        lam = max(lam / 10.0, 1e-300)
        if step <= LM_STEP_TOL * max(scale, 1e-300):
            break
    return theta, s


def _gauss_newton_polish(theta, f, d, p):
    """Continue the iteration with lambda = 0 while the steps contract.

    Near the minimum the residual sum S changes by less than its rounding
    error long before the parameters settle (S - S* ~ step^2), so the
    LM acceptance test (S must decrease) stops at ~sqrt(eps) relative
    accuracy.  Gauss-Newton steps are driven by the gradient J^T r, which
    stays accurate; iterating them while they shrink converges to the
    stationary point.  beta stays at 0 when the bound is active.
    """
    theta = np.array(theta, dtype=np.float64)
    last = np.inf
    for _ in range(100):
        r = p - _model(theta, f, d)
        jac = _jacobian(theta, f, d)
        free = [0, 1] if theta[2] == 0.0 else [0, 1, 2]
        jf = jac[:, free]
        try:
            delta = np.linalg.solve(jf.T @ jf, jf.T @ r)
        except np.linalg.LinAlgError:
            break
        size = float(np.linalg.norm(delta))
        if not size < last:
            break
        cand = theta.copy()
        cand[free] += delta
        if cand[2] < 0.0:
            break
        theta, last = cand, size
        if size <= LM_STEP_TOL * max(float(np.linalg.norm(theta)), 1e-300):
            break
    r = p - _model(theta, f, d)
    return theta, float(r @ r)


def _fit_fixed_tau(f, d, p):
    best = None
    starts = []
    a0, b0 = _linear_fit(f, p)
    starts.append((a0, b0, 0.0))
    for beta0 in BETA_STARTS:
        x = f * (1.0 + beta0 * d) ** 2
        a, b = _linear_fit(x, p)
        starts.append((a, b, beta0))
    for st in starts:
        theta, s = _levenberg_marquardt(st, f, d, p)
        theta, s = _gauss_newton_polish(theta, f, d, p)
        if best is None or s < best[1]:
            best = (theta, s)
    return best


def fit_power_model(f_mhz, p_w, v=None, throttled=None, p_max_w=0.0) -> dict:
    """Fit Eq. (powercurve) to (clock, power[, voltage]) samples.

    Returns a dict with p_idle_w, alpha, beta, tau_mhz, p_max_w, has_voltage,
    sse, n_used, f_lo_mhz, f_thr_mhz and f_opt_mhz (the energy-optimal clock
    of ``optimal_clock``).
    """
    f_mhz = np.asarray(f_mhz, dtype=np.float64)
    p_w = np.asarray(p_w, dtype=np.float64)
    if f_mhz.shape != p_w.shape or f_mhz.ndim != 1:
        raise ValueError("f and p must be 1-D of equal length")
    thr = (np.zeros(f_mhz.shape, dtype=bool) if throttled is None
           else np.asarray(throttled).astype(bool))
    pmax = float(p_max_w) if p_max_w and p_max_w > 0 else float(p_w.max())
    keep = ~thr
    fk, pk = f_mhz[keep], p_w[keep]
    if fk.size < 3:
        raise ValueError("need at least 3 unthrottled samples")
    res = dict(p_max_w=pmax, n_used=int(fk.size), f_lo_mhz=float(fk.min()),
               f_thr_mhz=float(fk.max()))
    fg = fk / 1000.0

    if v is not None:
        vk = np.asarray(v, dtype=np.float64)[keep]
        x = fg * vk * vk
        p_idle, alpha = _linear_fit(x, pk)
        r = pk - (p_idle + alpha * x)
        res.update(p_idle_w=p_idle, alpha=alpha, beta=0.0, tau_mhz=0.0, has_voltage=1,
                   sse=float(r @ r))
        pstar = np.minimum(pmax, p_idle + alpha * x)
        h = pstar / fk
        order = np.lexsort((fk, h))  # smallest h, ties -> lower clock
        res["f_opt_mhz"] = float(fk[order[0]])
        return res

    lo = int(math.ceil(fk.min()))
    hi = int(math.floor(fk.max()))
    best = None
    for tau in range(lo, hi + 1):
        if int((fk > tau).sum()) < 2:
            continue
        d = np.maximum(0.0, fk - tau) / 1000.0
        theta, s = _fit_fixed_tau(fg, d, pk)
        if best is None or s < best[2] - TAU_TIE_REL * best[2]:
            best = (tau, theta, s)
    if best is None:
        raise ValueError("no threshold has two samples above it")
    tau, theta, s = best
    res.update(p_idle_w=float(theta[0]), alpha=float(theta[1]), beta=float(theta[2]),
               tau_mhz=float(tau), has_voltage=0, sse=float(s))
    res["f_opt_mhz"] = optimal_clock(res)
    return res


def voltage_estimate(model: dict, f_mhz):
    """v(f) = 1 + beta * max(0, f - tau), f in MHz, beta per GHz."""
    f = np.asarray(f_mhz, dtype=np.float64)
    return 1.0 + model["beta"] * np.maximum(0.0, f - model["tau_mhz"]) / 1000.0


def model_power(model: dict, f_mhz):
    """P*_load(f) of Eq. (powercurve) with the estimated voltage."""
    f = np.asarray(f_mhz, dtype=np.float64)
    v = voltage_estimate(model, f)
    return np.minimum(model["p_max_w"], model["p_idle_w"] + model["alpha"] * (f / 1000.0) * v * v)


def energy_per_cycle(model: dict, f_mhz):
    """Estimated energy up to a constant: P*_load(f) / f (J per Mcycle)."""
    f = np.asarray(f_mhz, dtype=np.float64)
    return model_power(model, f) / f


def _real_roots(coeffs, lo, hi):
    c = np.trim_zeros(np.asarray(coeffs, dtype=np.float64), "f")
    if c.size <= 1:
        return []
    out = []
    for z in np.roots(c):
        if abs(z.imag) <= 1e-9 * max(1.0, abs(z.real)) and lo <= z.real <= hi:
            out.append(float(z.real))
    return out


def optimal_clock(model: dict) -> float:
    """argmin of P*_load(f)/f over [f_lo, f_thr] (estimated-voltage model).

    The minimum of a piecewise-smooth function on an interval lies at an end
    point, at a kink (tau, or where the P_max cap starts) or at a stationary
    point.  Above tau, d/df [Q(f)/f] = 0 with Q = P_idle + alpha f v^2 reads
    2 alpha beta^2 f^3 + 2 alpha beta (1 - beta tau) f^2 - P_idle = 0 (f, tau
    in GHz); below tau, Q/f = P_idle/f + alpha has no stationary point unless
    P_idle = 0.  Ties go to the lower clock.
    """
    lo, hi = model["f_lo_mhz"] / 1000.0, model["f_thr_mhz"] / 1000.0
    p0, a, b = model["p_idle_w"], model["alpha"], model["beta"]
    tau = model["tau_mhz"] / 1000.0
    pmax = model["p_max_w"]
    cand = [lo, hi]
    if lo <= tau <= hi:
        cand.append(tau)
    # stationary points above tau
    cand += [z for z in _real_roots([2 * a * b * b, 2 * a * b * (1 - b * tau), 0.0, -p0],
                                    max(lo, tau), hi)]
    # where Q(f) = P_max: below tau a*f + p0 = pmax; above tau
    # a f (1 + b (f - tau))^2 = pmax - p0, i.e. a b^2 f^3 + 2 a b (1 - b tau) f^2
    # + a (1 - b tau)^2 f - (pmax - p0) = 0
    cand += [z for z in _real_roots([a, p0 - pmax], lo, min(hi, tau))]
    cand += [z for z in _real_roots([a * b * b, 2 * a * b * (1 - b * tau),
                                     a * (1 - b * tau) ** 2, p0 - pmax], max(lo, tau), hi)]
    cand = sorted(set(cand))
    hv = [float(energy_per_cycle(model, c * 1000.0)) for c in cand]
    best = min(range(len(cand)), key=lambda k: (hv[k], cand[k]))
    return cand[best] * 1000.0


def pick_clock_range(model: dict, supported_mhz, rel_halfwidth=0.10, center="optimum"):
    """Supported clocks within +-rel_halfwidth of the centre clock.

    centre = the model optimum (``f_opt_mhz``) or, with ``center="ridge"``,
    tau.  An empty window falls back to the nearest supported clock (ties:
    lower).  Returns (sorted list of clocks, centre).
    """
    sup = sorted(float(c) for c in supported_mhz)
    if not sup:
        raise ValueError("no supported clocks")
    c0 = float(model["tau_mhz"]) if center == "ridge" else float(model["f_opt_mhz"])
    lo, hi = (1.0 - rel_halfwidth) * c0, (1.0 + rel_halfwidth) * c0
    sel = [c for c in sup if lo <= c <= hi]
    if not sel:
        sel = [min(sup, key=lambda c: (abs(c - c0), c))]
    return sel, c0
