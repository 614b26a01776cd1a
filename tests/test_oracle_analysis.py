"""Pins of the tuning-method selection, Pareto front and fitness-flow-graph
centrality (Sections IV-A, IV-B) on hand-built tables and against networkx's
PageRank."""
import itertools

import numpy as np
import pytest

from oracle import selection as sel


def row(cfg, clock, t, e):
    flop = 1.0
    return dict(cfg=tuple(cfg), clock=clock, t_s=t, energy_j=e, gflops=flop / t,
                gflops_per_j=flop / e)


def test_five_methods_on_a_constructed_table():
    rows = [
        row((1,), 2000, 1.00, 10.0),  # 0 fastest overall, max clock
        row((1,), 1500, 1.30, 8.0),   # 1 config 1 at a lower clock: its energy optimum
        row((2,), 2000, 1.20, 9.0),   # 2 least energy at the max clock
        row((2,), 1500, 1.50, 7.5),   # 3
        row((3,), 2000, 1.40, 9.5),   # 4
        row((3,), 1000, 2.00, 7.0),   # 5 global least energy
        row((4,), 1000, 2.20, 7.2),   # 6 least energy at the base clock 1000
        row((4,), 1500, 1.70, 7.1),   # 7 config 4's energy optimum
        row((4,), 2000, 1.50, 11.0),  # 8
    ]
    m = sel.tuning_methods(rows, base_clock=1000)
    assert m == dict(race_to_idle=0, energy_maxclock=2, race_to_idle_clocks=1,
                     energy_clocks=5, global_energy=5)
    # base clock 1000 is nearest to 1200 too
    assert sel.tuning_methods(rows, base_clock=1200)["energy_clocks"] == 5
    rows[5]["energy_j"] = 7.3  # now config 4 wins at the base clock
    m = sel.tuning_methods(rows, base_clock=1000)
    assert m["energy_clocks"] == 7 and m["global_energy"] == 7


def test_pareto_front_of_a_concave_trade_off():
    # points on a concave front plus dominated interior points
    front = [(100.0, 10.0), (90.0, 14.0), (70.0, 17.0), (40.0, 19.0)]
    inner = [(95.0, 9.0), (80.0, 13.0), (60.0, 16.0), (30.0, 18.0), (70.0, 16.9)]
    rows = [dict(cfg=(i,), clock=0, t_s=1 / g, energy_j=1 / e, gflops=g, gflops_per_j=e)
            for i, (g, e) in enumerate(front + inner)]
    assert sel.pareto_front(rows) == [0, 1, 2, 3]
    # a duplicate of a front point is not dominated either
    rows.append(dict(cfg=(99,), clock=0, t_s=0, energy_j=0, gflops=90.0, gflops_per_j=14.0))
    assert sel.pareto_front(rows) == [0, 1, 9, 2, 3]


def test_pagerank_matches_networkx():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(0)
    for n in (5, 17, 40):
        adj = [sorted(set(int(x) for x in rng.choice(n, rng.integers(0, 4)) if x != a))
               for a in range(n)]
        g = nx.DiGraph()
        g.add_nodes_from(range(n))
        for a, outs in enumerate(adj):
            for b in outs:
                g.add_edge(a, b)
        want = nx.pagerank(g, alpha=0.85, tol=1e-14, max_iter=10000)
        got = sel.pagerank(adj, 0.85)
        np.testing.assert_allclose(got, [want[i] for i in range(n)], atol=1e-10)


def test_centrality_single_basin_and_two_basins():
    # a line of points differing in one parameter, fitness falling to one end:
    # every walk ends in the one minimum
    rows = [row((i,), 1000, 1.0, 10.0 - i) for i in range(6)]
    adj, _ = sel.fitness_flow_graph(rows)
    assert [len(a) for a in adj] == [5, 4, 3, 2, 1, 0]  # complete graph on one parameter
    assert sel.proportion_of_centrality(rows, ps=(1.0,))[1.0] == pytest.approx(1.0)
    # two parameters: a 2 x 2 grid whose diagonal corners are minima of
    # fitness 1 (global) and 1.2 (each off-diagonal point has both as neighbours)
    fit = {(0, 0): 1.0, (0, 1): 5.0, (1, 0): 6.0, (1, 1): 1.2}
    rows = [row(k, 1000, 1.0, v) for k, v in fit.items()]
    adj, f = sel.fitness_flow_graph(rows)
    minima = [a for a in range(len(rows)) if not adj[a]]
    assert sorted(f[m] for m in minima) == [1.0, 1.2]
    prop = sel.proportion_of_centrality(rows, ps=(1.0, 1.1, 1.25))
    assert 0.0 < prop[1.0] < 1.0 and prop[1.1] == prop[1.0] and prop[1.25] == pytest.approx(1.0)
    # closed form of this graph (damping 0.85, uniform restart), solved directly
    n = len(rows)
    m = np.zeros((n, n))
    for a in range(n):
        if adj[a]:
            for b in adj[a]:
                m[b, a] += 1.0 / len(adj[a])
        else:
            m[:, a] += 1.0 / n
    pr = np.linalg.solve(np.eye(n) - 0.85 * m, np.full(n, 0.15 / n))
    g = minima[int(np.argmin([f[x] for x in minima]))]
    assert prop[1.0] == pytest.approx(pr[g] / sum(pr[x] for x in minima), rel=1e-10)
