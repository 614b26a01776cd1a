"""Pins of the bookkeeping / selection oracle on hand-made tables."""
import itertools

import pytest

from oracle import selection as sel


def test_flop_count_and_metrics():
    # 1024 x 1024 output, 7 x 7 filter: 2 * 49 * 2^20 operations
    assert sel.conv2d_flop(7, 7, 1024, 1024) == 102_760_448
    assert sel.conv2d_flop(17, 17, 4096, 4096) == 9_697_230_848
    m = sel.window_metrics(2e9, n_launches=100, elapsed_ms=50.0, e0_mj=1000, e1_mj=21000,
                           power_w_samples=[390.0, 400.0, 410.0])
    assert m["t_s"] == pytest.approx(5e-4)
    assert m["energy_j"] == pytest.approx(0.2)
    assert m["gflops"] == pytest.approx(4000.0)
    assert m["gflops_per_j"] == pytest.approx(10.0)
    assert m["power_w_median"] == 400.0
    assert m["energy_j_median_power"] == pytest.approx(0.2)


def _table():
    rows = []
    for cfg, clk in itertools.product([(16, 1), (32, 2), (64, 4)], [900, 1000, 1100]):
        t = 1.0 / clk * (1 + 0.1 * cfg[1])
        e = t * (100 + 0.0003 * clk ** 2)
        rows.append(dict(cfg=cfg, clock=clk, t_s=t, energy_j=e, gflops_per_j=1 / e))
    return rows


def test_best_row_by_objective():
    rows = _table()
    e = sel.best_row(rows, "energy")
    assert all(rows[e]["energy_j"] <= r["energy_j"] for r in rows)
    t = sel.best_row(rows, "time")
    assert all(rows[t]["t_s"] <= r["t_s"] for r in rows)
    assert rows[t]["clock"] == 1100
    g = sel.best_row(rows, "gflops_per_j")
    assert g == e


def test_ties_break_on_time_then_clock_then_config():
    rows = [dict(cfg=(2,), clock=1000, t_s=1.0, energy_j=5.0, gflops_per_j=0.2),
            dict(cfg=(1,), clock=1000, t_s=1.0, energy_j=5.0, gflops_per_j=0.2),
            dict(cfg=(0,), clock=1100, t_s=1.0, energy_j=5.0, gflops_per_j=0.2),
            dict(cfg=(3,), clock=900, t_s=2.0, energy_j=5.0, gflops_per_j=0.2)]
    assert sel.best_row(rows) == 1


def test_steering_score():
    rows = _table()
    full = sel.steering_score(rows, [900, 1000, 1100])
    assert full["match"] and full["energy_gap"] == 0.0
    off = sel.steering_score(rows, [1100])
    ex, st = rows[off["exhaustive"]], rows[off["steered"]]
    assert st["clock"] == 1100
    assert off["energy_gap"] == pytest.approx(st["energy_j"] / ex["energy_j"] - 1)
    assert off["match"] == (ex["clock"] == 1100)
    assert sel.tuning_time_fraction(10.0, 100.0, 5.0) == pytest.approx(0.15)
