"""Oracle: energy / metric bookkeeping and exhaustive-vs-steered selection.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Bookkeeping (Section III-A and III-C of the paper):

* Energy is the integral of power over the run; the paper approximates it by
  the median power reading times the elapsed time.  Here the headline energy
  is the difference of the device's total-energy counter over a window of N
  launches (millijoules), divided by N; the paper's median-power product is
  kept beside it.
* Compute performance is GFLOP/s and energy efficiency GFLOPs/W = GFLOP/J
  (Section III-C, user-defined metrics).
* A 2-D correlation of an H x W output with an fh x fw filter is
  2 * fh * fw * H * W floating-point operations (one multiply and one add per
  tap).

Selection (Section IV-A tuning methods; Section IV-E model steering):

* The energy optimum of an exhaustive table is the row with the least energy
  per launch; ties go to the shorter time, then the lower clock, then the
  lexicographically smaller configuration tuple.
* The steered optimum is the same choice restricted to the clocks of the
  steered range.
"""
from __future__ import annotations

import statistics


def conv2d_flop(fh, fw, out_h, out_w) -> int:
    return 2 * int(fh) * int(fw) * int(out_h) * int(out_w)


def window_metrics(flop_per_launch, n_launches, elapsed_ms, e0_mj, e1_mj, power_w_samples=()):
    """Per-launch time, energy and the two user metrics of one window."""
    t_s = elapsed_ms / 1000.0 / n_launches
    energy_j = (e1_mj - e0_mj) / 1000.0 / n_launches
    gflop = flop_per_launch / 1e9
    out = dict(t_s=t_s, energy_j=energy_j, gflops=gflop / t_s,
               gflops_per_j=(gflop / energy_j) if energy_j > 0 else float("nan"))
    if power_w_samples:
        pmed = statistics.median(power_w_samples)
        out["power_w_median"] = pmed
        out["energy_j_median_power"] = pmed * t_s
    return out


def _key(row, objective):
    cfg = tuple(row["cfg"])
    if objective == "time":
        return (row["t_s"], row["energy_j"], row["clock"], cfg)
    if objective == "gflops_per_j":
        return (-row["gflops_per_j"], row["t_s"], row["clock"], cfg)
    return (row["energy_j"], row["t_s"], row["clock"], cfg)


def best_row(rows, objective="energy", clocks=None):
    """Index of the optimal row (optionally restricted to ``clocks``)."""
    idx = [k for k, r in enumerate(rows) if clocks is None or r["clock"] in clocks]
    if not idx:
        raise ValueError("no rows to choose from")
    return min(idx, key=lambda k: _key(rows[k], objective))


def steering_score(rows, range_clocks, objective="energy"):
    """Steered vs exhaustive: relative energy gap and whether they match."""
    ex = best_row(rows, objective)
    st = best_row(rows, objective, clocks=set(range_clocks))
    gap = rows[st]["energy_j"] / rows[ex]["energy_j"] - 1.0
    same = (rows[st]["clock"] == rows[ex]["clock"]
            and tuple(rows[st]["cfg"]) == tuple(rows[ex]["cfg"]))
    return dict(exhaustive=ex, steered=st, energy_gap=gap, match=same)


def tuning_time_fraction(steered_wall_s, exhaustive_wall_s, fit_wall_s=0.0):
    """Fraction of exhaustive tuning time spent by the steered search."""
    return (steered_wall_s + fit_wall_s) / exhaustive_wall_s
