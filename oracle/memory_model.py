"""Oracle: the memory-aware energy model (time model of a unit whose run time
is only partly clock-bound), its energy-optimal clock and clock ranges.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product library
never imports this module, and this module imports nothing from the product.

What the paper fixes and what it leaves open:

* Section IV-E estimates energy as P*_load(f) / f: a kernel's run time is
  taken to scale as 1/f, which holds for compute-bound kernels (the paper
  fits on one full-load kernel).
* Section IV-F closes by planning to extend the model with memory-dependent
  terms, because the estimated optimum sometimes misses the measured one;
  Section II recalls the roofline energy model of Choi et al., where memory
  traffic costs energy that compute cannot hide.

Reading taken here (the paper gives no formula for the extension):

* Run time of one unit of work at SM clock f (GHz) has a clock-independent
  memory part and a clock-bound part, ``t(f) = t_mem + c_core / f`` with
  ``t_mem >= 0`` and ``c_core >= 0``: a pure copy has c_core ~ 0, the FMA
  kernel t_mem ~ 0.  The two coefficients come from (clock, time) samples of
  the unit by non-negative linear least squares in the regressors (1, 1/f)
  (throttled samples dropped, as for the power fit).
* Energy per unit is ``E(f) = P*_load(f) * t(f)``, P*_load of Eq. (powercurve)
  fitted on the same unit's power samples (``power_model.fit_power_model``).
  With t_mem = 0 this is c_core * P*/f, the paper's estimate.
* Its minimiser is taken over the integer-MHz clocks of the range both fits
  cover, [max of the two lowest kept clocks, min of the two highest]; ties
  go to the lower clock.
* A range is the supported clocks within +-rel of a centre (the +-10 % rule
  of Section IV-E); a kernel of unknown boundness can be tuned over the union
  of the compute-bound and the memory-aware ranges.
"""
from __future__ import annotations

import math

import numpy as np


def _sse(t, a, b, u):
    r = t - (a + b * u)
    return float(r @ r)


def fit_time_model(f_mhz, t_s, throttled=None) -> dict:
    """Non-negative least squares of t = t_mem + c_core / f (f in GHz).

    Two unknowns: the solution is the unconstrained one when it is
    non-negative, else the best of the solutions with one or both
    coefficients held at zero (the faces of the feasible quadrant).
    Returns t_mem_s, c_core_s_ghz, sse, n_used, f_lo_mhz, f_thr_mhz.
    """
    f_mhz = np.asarray(f_mhz, dtype=np.float64)
    t_s = np.asarray(t_s, dtype=np.float64)
    if f_mhz.shape != t_s.shape or f_mhz.ndim != 1:
        raise ValueError("f and t must be 1-D of equal length")
    if np.any(~np.isfinite(f_mhz)) or np.any(f_mhz <= 0) or np.any(~np.isfinite(t_s)):
        raise ValueError("clocks must be positive and times finite")
    thr = (np.zeros(f_mhz.shape, dtype=bool) if throttled is None
           else np.asarray(throttled).astype(bool))
    fk, tk = f_mhz[~thr], t_s[~thr]
    if fk.size < 2:
        raise ValueError("need at least 2 unthrottled samples")
    u = 1000.0 / fk  # 1 / f in 1/GHz
    cands = []
    um, tm = u.mean(), tk.mean()
    suu = float(((u - um) ** 2).sum())
    if suu > 0.0:
        b = float(((u - um) * (tk - tm)).sum()) / suu
        a = float(tm - b * um)
        if a >= 0.0 and b >= 0.0:
            cands.append((a, b))
    # faces: a = 0 (time purely clock-bound), b = 0 (clock-independent)
    b0 = max(0.0, float(tk @ u) / float(u @ u))
    cands.append((0.0, b0))
    cands.append((max(0.0, float(tm)), 0.0))
    best = min(cands, key=lambda ab: _sse(tk, ab[0], ab[1], u))
    return dict(t_mem_s=best[0], c_core_s_ghz=best[1], sse=_sse(tk, best[0], best[1], u),
                n_used=int(fk.size), f_lo_mhz=float(fk.min()), f_thr_mhz=float(fk.max()))


def model_time(tm: dict, f_mhz):
    f = np.asarray(f_mhz, dtype=np.float64)
    return tm["t_mem_s"] + tm["c_core_s_ghz"] / (f / 1000.0)


def model_power(pm: dict, f_mhz):
    """P*_load(f) of Eq. (powercurve), written out here (estimated voltage)."""
    fg = np.asarray(f_mhz, dtype=np.float64) / 1000.0
    v = 1.0 + pm["beta"] * np.maximum(0.0, fg - pm["tau_mhz"] / 1000.0)
    return np.minimum(pm["p_max_w"], pm["p_idle_w"] + pm["alpha"] * fg * v * v)


def model_energy(pm: dict, tm: dict, f_mhz):
    """E(f) = P*_load(f) * t(f) (J per unit of work)."""
    return model_power(pm, f_mhz) * model_time(tm, f_mhz)


def energy_optimum(pm: dict, tm: dict) -> dict:
    """argmin of E(f) over the integer-MHz clocks both fits cover (ties:
    lower clock).  Returns f_opt_mhz, e_opt_j, f_lo_mhz, f_hi_mhz."""
    if pm.get("has_voltage"):
        raise ValueError("the memory-aware optimum needs the estimated-voltage power model")
    lo = max(pm["f_lo_mhz"], tm["f_lo_mhz"])
    hi = min(pm["f_thr_mhz"], tm["f_thr_mhz"])
    glo, ghi = int(math.ceil(lo)), int(math.floor(hi))
    if ghi < glo:
        raise ValueError("the two fits share no integer clock")
    grid = np.arange(glo, ghi + 1, dtype=np.float64)
    e = model_energy(pm, tm, grid)
    k = int(np.argmin(e))  # first minimum: the lower clock on ties
    return dict(f_opt_mhz=float(grid[k]), e_opt_j=float(e[k]), f_lo_mhz=float(glo),
                f_hi_mhz=float(ghi))


def clock_range(center_mhz, supported_mhz, rel_halfwidth=0.10):
    """Supported clocks within +-rel of the centre; an empty window falls back
    to the nearest supported clock (ties: lower)."""
    sup = sorted(int(c) for c in supported_mhz)
    if not sup:
        raise ValueError("no supported clocks")
    c0 = float(center_mhz)
    lo, hi = (1.0 - rel_halfwidth) * c0, (1.0 + rel_halfwidth) * c0
    sel = [c for c in sup if lo <= c <= hi]
    if not sel:
        sel = [min(sup, key=lambda c: (abs(c - c0), c))]
    return sel


def union_range(a, b):
    """Sorted union of two clock ranges."""
    return sorted(set(int(c) for c in a) | set(int(c) for c in b))
