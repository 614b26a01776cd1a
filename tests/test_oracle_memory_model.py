"""Pins of the oracle's memory-aware energy model (oracle/memory_model.py)
against facts that do not come from the oracle itself: exact recovery of a
noiseless time curve, SciPy's NNLS, a closed-form optimum, the reduction to
the paper's compute-bound estimate (Section IV-E) and a monotonicity bound,
and brute force on a fine continuous grid."""
import math

import numpy as np
import pytest

from oracle import memory_model as mm
from oracle import power_model as pmod

CLOCKS = np.array([900, 1050, 1200, 1350, 1500, 1650, 1800, 1950, 2070], dtype=np.float64)


def _pm(p0=180.0, alpha=420.0, beta=0.9, tau=1380.0, lo=900.0, hi=2070.0, pmax=1e9):
    return dict(p_idle_w=p0, alpha=alpha, beta=beta, tau_mhz=tau, p_max_w=pmax, has_voltage=0,
                f_lo_mhz=lo, f_thr_mhz=hi)


def _tm(a, b, lo=900.0, hi=2070.0):
    return dict(t_mem_s=a, c_core_s_ghz=b, f_lo_mhz=lo, f_thr_mhz=hi)


@pytest.mark.parametrize("a,b", [(4e-4, 1e-4), (0.0, 3e-3), (2.5e-3, 0.0), (1e-3, 1e-3)])
def test_noiseless_time_curve_is_recovered(a, b):
    t = a + b / (CLOCKS / 1000.0)
    tm = mm.fit_time_model(CLOCKS, t)
    assert tm["t_mem_s"] == pytest.approx(a, rel=1e-12, abs=1e-18)
    assert tm["c_core_s_ghz"] == pytest.approx(b, rel=1e-12, abs=1e-18)
    assert tm["sse"] <= 1e-30
    assert tm["n_used"] == CLOCKS.size


@pytest.mark.parametrize("seed", range(12))
def test_fit_equals_scipy_nnls(seed):
    nnls = pytest.importorskip("scipy.optimize").nnls
    rng = np.random.default_rng(seed)
    f = np.sort(rng.uniform(600, 2100, size=rng.integers(2, 12)))
    a, b = rng.uniform(-1e-3, 2e-3), rng.uniform(-1e-3, 2e-3)  # some infeasible truths
    t = a + b / (f / 1000.0) + rng.normal(0, 2e-4, size=f.size)
    tm = mm.fit_time_model(f, t)
    x, rnorm = nnls(np.column_stack([np.ones_like(f), 1000.0 / f]), t)
    assert tm["t_mem_s"] == pytest.approx(x[0], rel=1e-9, abs=1e-13)
    assert tm["c_core_s_ghz"] == pytest.approx(x[1], rel=1e-9, abs=1e-13)
    assert tm["sse"] == pytest.approx(rnorm ** 2, rel=1e-9, abs=1e-20)


def test_time_rising_with_clock_clamps_the_clock_term():
    # t grows with f: no non-negative c_core fits better than 0
    t = 1e-3 + 1e-7 * CLOCKS
    tm = mm.fit_time_model(CLOCKS, t)
    assert tm["c_core_s_ghz"] == 0.0
    assert tm["t_mem_s"] == pytest.approx(t.mean(), rel=1e-14)


def test_throttled_samples_are_ignored():
    t = 4e-4 + 1e-4 / (CLOCKS / 1000.0)
    bad = t.copy()
    bad[-2:] *= 3.0
    thr = np.zeros(CLOCKS.size, dtype=bool)
    thr[-2:] = True
    a = mm.fit_time_model(CLOCKS, t)
    b = mm.fit_time_model(CLOCKS, bad, throttled=thr)
    assert b["t_mem_s"] == pytest.approx(a["t_mem_s"], rel=1e-12)
    assert b["c_core_s_ghz"] == pytest.approx(a["c_core_s_ghz"], rel=1e-12)
    assert b["f_thr_mhz"] == CLOCKS[-3]


@pytest.mark.parametrize("p0,alpha,a,b", [(180.0, 420.0, 1e-3, 2e-3), (55.0, 150.0, 5e-4, 4e-3),
                                          (30.0, 70.0, 1e-3, 1.2e-3)])
def test_optimum_below_the_ridge_has_a_closed_form(p0, alpha, a, b):
    # below tau: E(f) = (P0 + alpha f)(a + b/f), dE/df = alpha a - P0 b / f^2,
    # so the minimiser is f* = sqrt(P0 b / (alpha a)) (GHz)
    fstar = math.sqrt(p0 * b / (alpha * a)) * 1000.0
    tau = 2000.0
    assert 600.0 < fstar < tau
    res = mm.energy_optimum(_pm(p0, alpha, 0.9, tau, 500.0, 2070.0), _tm(a, b, 500.0, 2070.0))
    assert abs(res["f_opt_mhz"] - fstar) <= 0.5 + 1e-9


def test_clock_independent_time_picks_the_lowest_clock():
    # t_mem only: E = t_mem P*(f), and P* rises with f
    res = mm.energy_optimum(_pm(), _tm(2e-3, 0.0))
    assert res["f_opt_mhz"] == 900.0


@pytest.mark.parametrize("beta,tau,pmax", [(0.9, 1380.0, 1e9), (1.2, 1025.0, 1e9),
                                           (0.5, 1500.0, 700.0), (0.0, 1000.0, 1e9)])
def test_clock_bound_time_reduces_to_the_papers_estimate(beta, tau, pmax):
    # t_mem = 0: E = c P*(f)/f, the compute-bound estimate of Section IV-E
    pm = _pm(beta=beta, tau=tau, pmax=pmax)
    res = mm.energy_optimum(pm, _tm(0.0, 1.7e-3))
    f_paper = pmod.optimal_clock(pm)
    assert abs(res["f_opt_mhz"] - f_paper) <= 1.0


@pytest.mark.parametrize("a", [1e-5, 1e-4, 1e-3, 1e-2])
def test_a_memory_term_never_raises_the_optimum(a):
    # E = b P/f + a P with P rising in f: for f above argmin P/f both terms
    # are no smaller, so the optimum cannot move up (1 MHz: grid vs exact)
    pm = _pm()
    f_paper = pmod.optimal_clock(pm)
    res = mm.energy_optimum(pm, _tm(a, 1e-3))
    assert res["f_opt_mhz"] <= f_paper + 1.0


@pytest.mark.parametrize("seed", range(8))
def test_grid_optimum_matches_a_fine_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    pm = _pm(p0=rng.uniform(30, 250), alpha=rng.uniform(50, 500), beta=rng.uniform(0.0, 2.0),
             tau=rng.uniform(1000, 1800), pmax=rng.choice([1e9, rng.uniform(400, 900)]))
    tm = _tm(rng.uniform(0, 3e-3), rng.uniform(0, 3e-3))
    res = mm.energy_optimum(pm, tm)
    fine = np.arange(900.0, 2070.0 + 1e-9, 0.01)
    # the same product written out independently of model_energy
    fg = fine / 1000.0
    v = 1.0 + pm["beta"] * np.clip(fg - pm["tau_mhz"] / 1000.0, 0.0, None)
    e = np.minimum(pm["p_max_w"], pm["p_idle_w"] + pm["alpha"] * fg * v ** 2) * \
        (tm["t_mem_s"] + tm["c_core_s_ghz"] / fg)
    f_bf = fine[int(np.argmin(e))]
    e_grid_best = e.min()
    # the integer grid's pick is within 1 MHz of the fine minimiser, or (flat
    # minimum) its energy is within rounding of the fine minimum
    assert abs(res["f_opt_mhz"] - f_bf) <= 1.0 or res["e_opt_j"] <= e_grid_best * (1 + 1e-9)
    assert res["e_opt_j"] >= e_grid_best * (1 - 1e-12)


def test_ranges_and_union():
    sup = list(range(900, 2071, 15))
    r = mm.clock_range(1400.0, sup, 0.10)
    assert r == [c for c in sup if 1260.0 <= c <= 1540.0]
    assert mm.clock_range(5000.0, sup, 0.10) == [2070]
    assert mm.clock_range(100.0, sup, 0.10) == [900]
    u = mm.union_range([900, 915], [915, 930, 2070])
    assert u == [900, 915, 930, 2070]
