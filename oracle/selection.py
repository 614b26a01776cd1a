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

import numpy as np


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


# ---- Section IV-A: the five tuning methods and the Pareto front ------------
#
# Rows carry "cfg" (tuple), "clock" (MHz), "t_s", "energy_j" and "gflops",
# "gflops_per_j".  Methods (Section IV-A):
#   race_to_idle            fastest point over all configurations and clocks
#   energy_maxclock         least energy among the points at the highest clock
#   race_to_idle_clocks     the fastest configuration at the highest clock,
#                           then its least-energy clock
#   energy_clocks           the least-energy configuration at the base clock,
#                           then its least-energy clock
#   global_energy           least energy over all configurations and clocks
# Ties as best_row.  The base clock is the caller's (the sampled clock
# nearest to it).

def _at_clock(rows, clock):
    return [k for k, r in enumerate(rows) if r["clock"] == clock]


def _best_of(rows, idx, objective):
    return min(idx, key=lambda k: _key(rows[k], objective))


def tuning_methods(rows, base_clock):
    clocks = sorted({r["clock"] for r in rows})
    cmax = clocks[-1]
    cbase = min(clocks, key=lambda c: (abs(c - base_clock), c))
    every = list(range(len(rows)))
    out = {}
    out["race_to_idle"] = _best_of(rows, every, "time")
    out["energy_maxclock"] = _best_of(rows, _at_clock(rows, cmax), "energy")
    fast = rows[_best_of(rows, _at_clock(rows, cmax), "time")]["cfg"]
    out["race_to_idle_clocks"] = _best_of(
        rows, [k for k in every if rows[k]["cfg"] == fast], "energy")
    eff = rows[_best_of(rows, _at_clock(rows, cbase), "energy")]["cfg"]
    out["energy_clocks"] = _best_of(rows, [k for k in every if rows[k]["cfg"] == eff], "energy")
    out["global_energy"] = _best_of(rows, every, "energy")
    return out


def pareto_front(rows):
    """Indices of the points not dominated in (GFLOP/s, GFLOPs/W), both
    maximised: no other point is at least as good in both and better in one.
    Sorted by GFLOP/s descending (ties: GFLOP/J descending, index)."""
    front = []
    for k, r in enumerate(rows):
        dominated = False
        for q, s in enumerate(rows):
            if q == k:
                continue
            if (s["gflops"] >= r["gflops"] and s["gflops_per_j"] >= r["gflops_per_j"]
                    and (s["gflops"] > r["gflops"] or s["gflops_per_j"] > r["gflops_per_j"])):
                dominated = True
                break
        if not dominated:
            front.append(k)
    return sorted(front, key=lambda k: (-rows[k]["gflops"], -rows[k]["gflops_per_j"], k))


# ---- Section IV-B: fitness flow graph and proportion of centrality ---------
#
# Nodes are the points of the space (configuration plus clock).  Reading of
# the neighbourhood (the paper defers to its reference): two points are
# neighbours when they differ in exactly one tunable parameter (the clock
# counts as a parameter).  A directed edge goes from a point to each
# neighbour with strictly better fitness; local minima have no out-edges.
# Centrality is PageRank with damping 0.85 in which a walker at a minimum
# (no out-edge) restarts uniformly; the proportion of centrality for p >= 1 is
# the centrality of minima with fitness <= p * f_optimal over that of all
# minima.

def _params(r):
    return tuple(r["cfg"]) + (r["clock"],)


def fitness_flow_graph(rows, objective="energy"):
    """Adjacency lists (better neighbours) of the fitness flow graph."""
    fit = [r["t_s"] if objective == "time" else r["energy_j"] for r in rows]
    pts = [_params(r) for r in rows]
    out = [[] for _ in rows]
    for a in range(len(rows)):
        for b in range(len(rows)):
            if a == b:
                continue
            diff = sum(1 for x, y in zip(pts[a], pts[b]) if x != y)
            if diff == 1 and fit[b] < fit[a]:
                out[a].append(b)
    return out, fit


def pagerank(adj, damping=0.85, tol=1e-14, max_iter=10000):
    """Power iteration of PageRank on adjacency lists (uniform split over
    out-edges; nodes without out-edges spread their rank uniformly)."""
    n = len(adj)
    pr = np.full(n, 1.0 / n)
    for _ in range(max_iter):
        new = np.full(n, (1.0 - damping) / n)
        dangling = sum(pr[a] for a in range(n) if not adj[a])
        new += damping * dangling / n
        for a in range(n):
            if adj[a]:
                share = damping * pr[a] / len(adj[a])
                for b in adj[a]:
                    new[b] += share
        if np.abs(new - pr).sum() < tol:
            return new
        pr = new
    return pr


def proportion_of_centrality(rows, objective="energy", ps=(1.0, 1.05, 1.1, 1.25, 1.5, 2.0),
                             damping=0.85):
    adj, fit = fitness_flow_graph(rows, objective)
    pr = pagerank(adj, damping)
    minima = [a for a in range(len(rows)) if not adj[a]]
    fopt = min(fit)
    total = sum(pr[m] for m in minima)
    return {p: sum(pr[m] for m in minima if fit[m] <= p * fopt) / total for p in ps}
