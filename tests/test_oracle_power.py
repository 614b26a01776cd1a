"""Pins of the FP64 power-model oracle (Section IV-E of the paper).

Checked against: exact recovery of known parameters from noiseless samples of
the power curve, a library least-squares solver (numpy lstsq for the linear
voltage case, MINPACK's Levenberg-Marquardt through scipy for the estimated
voltage case), the closed-form stationary point of P/f, a brute-force grid
minimum, the model's qualitative properties stated in the paper (energy falls
with f below the ridge point, so the optimum is not below it) and the
+-10 % window of the paper's printed example.
"""
import json
import os

import numpy as np
import pytest
import scipy.optimize

from oracle import power_model as pm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_steering.json")


def curve(f_mhz, p_idle, alpha, beta, tau_mhz):
    """Power of Eq. (powercurve) with the continuous voltage estimate."""
    f = np.asarray(f_mhz, float)
    v = 1.0 + beta * np.maximum(0.0, f - tau_mhz) / 1000.0
    return p_idle + alpha * (f / 1000.0) * v ** 2


CASES = [
    # p_idle W, alpha W/GHz, beta /GHz, tau MHz, clock grid
    (180.0, 400.0, 0.8, 1230, np.arange(990, 1651, 30.0)),
    (95.0, 60.0, 2.5, 1402, np.arange(1200.0, 1801.0, 25.0)),
    (250.0, 700.0, 0.35, 1515, np.arange(1300.0, 2071.0, 40.0)),
]


@pytest.mark.parametrize("case", CASES, ids=["a", "b", "c"])
def test_noiseless_recovery(case):
    p0, a, b, tau, f = case
    p = curve(f, p0, a, b, tau)
    m = pm.fit_power_model(f, p, p_max_w=2000.0)
    assert m["has_voltage"] == 0
    assert m["tau_mhz"] == tau
    for got, want in ((m["p_idle_w"], p0), (m["alpha"], a), (m["beta"], b)):
        assert abs(got - want) <= 1e-9 * abs(want)
    assert m["sse"] < 1e-12
    assert m["f_lo_mhz"] == f.min() and m["f_thr_mhz"] == f.max()


def test_order_invariance_and_throttled_samples_ignored():
    p0, a, b, tau, f = CASES[0]
    rng = np.random.default_rng(1)
    p = curve(f, p0, a, b, tau) + rng.normal(0, 2.0, f.size)
    ref = pm.fit_power_model(f, p, p_max_w=1500.0)
    perm = rng.permutation(f.size)
    m2 = pm.fit_power_model(f[perm], p[perm], p_max_w=1500.0)
    for k in ("p_idle_w", "alpha", "beta", "tau_mhz"):
        assert m2[k] == pytest.approx(ref[k], rel=1e-9, abs=1e-9)
    # throttled samples (clock could not be held) must not move the fit
    f3 = np.concatenate([f, [1700.0, 1800.0]])
    p3 = np.concatenate([p, [5000.0, 1.0]])
    thr = np.concatenate([np.zeros(f.size, bool), [True, True]])
    m3 = pm.fit_power_model(f3, p3, throttled=thr, p_max_w=1500.0)
    for k in ("p_idle_w", "alpha", "beta", "tau_mhz", "sse"):
        assert m3[k] == ref[k]
    # with P_max unset it is the largest measured power, throttled included
    m4 = pm.fit_power_model(f3, p3, throttled=thr)
    assert m4["p_max_w"] == 5000.0


def test_noisy_fit_agrees_with_minpack_lm_at_chosen_tau():
    p0, a, b, tau, f = CASES[1]
    rng = np.random.default_rng(2)
    p = curve(f, p0, a, b, tau) + rng.normal(0, 0.5, f.size)
    m = pm.fit_power_model(f, p, p_max_w=1500.0)
    fg = f / 1000.0
    d = np.maximum(0.0, f - m["tau_mhz"]) / 1000.0
    res = scipy.optimize.least_squares(
        lambda th: th[0] + th[1] * fg * (1 + th[2] * d) ** 2 - p,
        x0=[m["p_idle_w"] * 1.01, m["alpha"] * 0.99, m["beta"] * 1.02],
        method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    assert res.x[2] >= 0
    np.testing.assert_allclose(res.x, [m["p_idle_w"], m["alpha"], m["beta"]], rtol=1e-8)
    # the chosen tau is the least-residual one among its neighbours
    def sse_at(t):
        dd = np.maximum(0.0, f - t) / 1000.0
        best = np.inf
        for b0 in (0.1, 1.0, 10.0):
            r = scipy.optimize.least_squares(
                lambda th: th[0] + th[1] * fg * (1 + th[2] * dd) ** 2 - p,
                x0=[p0, a, b0], bounds=([-np.inf, -np.inf, 0], np.inf),
                xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
            best = min(best, 2 * r.cost)
        return best
    s0 = m["sse"]
    for t in (m["tau_mhz"] - 7, m["tau_mhz"] + 7, m["tau_mhz"] - 40, m["tau_mhz"] + 40):
        assert sse_at(t) >= s0 * (1 - 1e-7)


def test_measured_voltage_is_linear_least_squares():
    rng = np.random.default_rng(3)
    f = np.arange(800.0, 1801.0, 50.0)
    v = 0.7 + 0.25 * np.maximum(0, f - 1100) / 700
    p = 150 + 300 * (f / 1000) * v ** 2 + rng.normal(0, 1.0, f.size)
    m = pm.fit_power_model(f, p, v=v, p_max_w=1000.0)
    x = (f / 1000) * v ** 2
    coef, *_ = np.linalg.lstsq(np.stack([np.ones_like(x), x], 1), p, rcond=None)
    assert m["has_voltage"] == 1
    assert m["p_idle_w"] == pytest.approx(coef[0], rel=1e-10)
    assert m["alpha"] == pytest.approx(coef[1], rel=1e-10)
    h = np.minimum(1000.0, coef[0] + coef[1] * x) / f
    assert m["f_opt_mhz"] == f[np.argmin(h)]


def _model(p0, a, b, tau, lo, hi, pmax=1e9):
    return dict(p_idle_w=p0, alpha=a, beta=b, tau_mhz=tau, p_max_w=pmax,
                f_lo_mhz=lo, f_thr_mhz=hi, has_voltage=0)


def test_optimum_closed_form():
    # tau = 0: d/df (P/f) = 0 <=> 2 a b^2 f^3 + 2 a b f^2 = P_idle;
    # a = b = 1, P_idle = 4 gives f = 1 GHz exactly.
    m = _model(4.0, 1.0, 1.0, 0.0, 200.0, 3000.0)
    assert pm.optimal_clock(m) == pytest.approx(1000.0, rel=1e-12)


def test_optimum_matches_brute_force_grid():
    rng = np.random.default_rng(4)
    for _ in range(40):
        m = _model(rng.uniform(50, 300), rng.uniform(50, 800), rng.uniform(0, 4),
                   rng.uniform(800, 1600), 600.0, 2070.0,
                   pmax=rng.choice([1e9, rng.uniform(400, 1400)]))
        grid = np.arange(600.0, 2070.0 + 1e-9, 0.01)
        brute = grid[np.argmin(pm.energy_per_cycle(m, grid))]
        f_opt = pm.optimal_clock(m)
        assert abs(f_opt - brute) <= 1.0
        assert pm.energy_per_cycle(m, f_opt) <= pm.energy_per_cycle(m, brute) * (1 + 1e-12)


def test_optimum_not_below_ridge_and_energy_falls_below_it():
    # Section IV-E: below the ridge point v is constant, so P/f = P_idle/f + alpha
    # falls with f for P_idle > 0; the optimum is at or above tau.
    rng = np.random.default_rng(5)
    for _ in range(40):
        m = _model(rng.uniform(20, 300), rng.uniform(50, 800), rng.uniform(0.01, 4),
                   rng.uniform(800, 1600), 600.0, 2070.0)
        assert pm.optimal_clock(m) >= m["tau_mhz"] - 1e-9
        below = np.linspace(600.0, m["tau_mhz"], 50)
        assert np.all(np.diff(pm.energy_per_cycle(m, below)) < 0)


def test_constant_voltage_prefers_highest_unthrottled_clock():
    m = _model(120.0, 300.0, 0.0, 1000.0, 600.0, 1900.0)
    assert pm.optimal_clock(m) == 1900.0


def test_fit_reports_optimum_of_fitted_curve():
    p0, a, b, tau, f = CASES[2]
    m = pm.fit_power_model(f, curve(f, p0, a, b, tau), p_max_w=3000.0)
    assert m["f_opt_mhz"] == pytest.approx(pm.optimal_clock(m))
    assert m["f_opt_mhz"] >= m["tau_mhz"]


def test_range_window_paper_example():
    g = json.load(open(GOLDEN))
    hw = g["halfwidth"]
    supported = np.arange(210.0, 1411.0, 15.0)  # a 15 MHz clock grid
    m = dict(f_opt_mhz=float(g["a100_model_optimum_mhz"]), tau_mhz=float(g["a100_ridge_mhz"]))
    sel, c0 = pm.pick_clock_range(m, supported, hw)
    assert c0 == 985.0
    assert min(sel) >= 0.9 * 985 and max(sel) <= 1.1 * 985
    assert [c for c in supported if 0.9 * 985 <= c <= 1.1 * 985] == sel
    # the paper's observed ridge point and Table II's tuned A100 clock lie inside
    assert 0.9 * 985 <= g["a100_ridge_mhz"] <= 1.1 * 985
    for c in g["a100_table2_tuned_mhz"]:
        assert min(sel) <= c <= max(sel)
    sel_r, c_r = pm.pick_clock_range(m, supported, hw, center="ridge")
    assert c_r == 1025.0 and min(sel_r) >= 922.5 and max(sel_r) <= 1127.5


def test_range_empty_window_falls_back_to_nearest():
    m = dict(f_opt_mhz=1000.0, tau_mhz=900.0)
    sel, _ = pm.pick_clock_range(m, [500.0, 1200.0, 1300.0], 0.10)
    assert sel == [1200.0]
    sel, _ = pm.pick_clock_range(m, [800.0, 1200.0], 0.10)  # tie -> lower
    assert sel == [800.0]


def test_rejects_too_few_samples():
    with pytest.raises(ValueError):
        pm.fit_power_model([1000.0, 1100.0], [100.0, 120.0])


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_noisy_fit_equals_variable_projection_to_1e_9(seed):
    # An algorithm unrelated to Levenberg-Marquardt: at the oracle's tau the
    # model is linear in (P_idle, alpha) once beta is fixed, so the least-
    # squares residual is a function of beta alone (closed-form inner solve);
    # its minimiser is bracketed on a grid and refined by Brent's method to
    # the last bits.  The oracle's coefficients must agree to 1e-9 relative.
    p0, a, b, tau, f = CASES[1]
    rng = np.random.default_rng(seed)
    p = curve(f, p0, a, b, tau) + rng.normal(0, 0.5, f.size)
    m = pm.fit_power_model(f, p, p_max_w=1500.0)
    fg = f / 1000.0
    d = np.maximum(0.0, f - m["tau_mhz"]) / 1000.0

    def inner(beta):
        x = fg * (1.0 + beta * d) ** 2
        xm, pm_ = x.mean(), p.mean()
        alpha = float(((x - xm) * (p - pm_)).sum() / ((x - xm) ** 2).sum())
        p_idle = float(pm_ - alpha * xm)
        r = p - p_idle - alpha * x
        return float(r @ r), p_idle, alpha

    grid = np.linspace(0.0, 20.0, 4001)
    k = int(np.argmin([inner(g)[0] for g in grid]))
    lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, grid.size - 1)]
    br = scipy.optimize.minimize_scalar(lambda bb: inner(bb)[0], bounds=(lo, hi),
                                        method="bounded", options={"xatol": 1e-15})
    s, p_idle, alpha = inner(br.x)
    np.testing.assert_allclose([p_idle, alpha, br.x], [m["p_idle_w"], m["alpha"], m["beta"]],
                               rtol=1e-9)
    assert m["sse"] == pytest.approx(s, rel=1e-9)
