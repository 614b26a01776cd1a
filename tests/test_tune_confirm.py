"""The tuner CLI's confirmation stage (host logic, no GPU): near-tied top
points are re-measured and the best median wins."""
import math

from paper_2211_07260_gb300 import api
from paper_2211_07260_gb300.tune import confirm_best


def rec(cfg, e, t=1e-4, flags=0):
    return dict(cfg=list(cfg), energy_j=e, t_s=t, gflops=1.0 / t, gflops_per_j=1.0 / e,
                power_w_mean=e / t, flags=flags, clock_mhz_meas=2070.0)


A, B, C, D = (16, 8, 4, 4, 2, 1, 4), (32, 4, 4, 4, 2, 1, 4), (128, 8, 4, 2, 2, 1, 4), (64, 2, 4, 4, 2, 1, 4)


def test_median_of_repeats_decides_a_near_tie():
    # one window ranks C first by 0.1 %; its true energy is higher, which
    # the repeats show (each round measures A, B, C once, in that order)
    recs = [rec(C, 0.1000), rec(A, 0.1001), rec(B, 0.1002), rec(D, 0.2000),
            rec((1, 1, 1, 1, 0, 1, 4), float("nan"), flags=api.REC_INVALID)]
    truth = {A: 0.0995, B: 0.1003, C: 0.1010}
    rounds = []

    def measure(cfgs):
        keys = [next(k for k in truth if k[0] == c.block_x and k[1] == c.block_y) for c in cfgs]
        rounds.append(keys)
        return [rec(k, truth[k]) for k in keys]

    best, summ = confirm_best(measure, recs, "energy", confirm=3, repeats=2)
    assert len(rounds) == 2 and all(sorted(r) == sorted([A, B, C]) for r in rounds)
    assert tuple(best["cfg"]) == A and summ["pick"] == list(A)
    assert summ["single_window_pick"] == list(C)
    # medians over 1 + 2 measurements
    assert math.isclose(best["energy_j"], 0.0995)
    assert math.isclose(summ["medians"][",".join(map(str, C))]["energy_j"], 0.1010)


def test_larger_is_better_objective_and_invalid_repeats():
    recs = [rec(A, 0.10), rec(B, 0.11), rec(C, 0.12)]

    def measure(cfgs):
        out = []
        for c in cfgs:
            k = next(k for k in (A, B, C) if k[0] == c.block_x and k[1] == c.block_y)
            # B's repeats are invalid (ignored); A's come out worse in GFLOP/J
            out.append(rec(k, 0.2 if k == A else 0.11, flags=api.REC_INVALID if k == B else 0))
        return out

    best, summ = confirm_best(measure, recs, "gflops_per_w", confirm=2, repeats=3)
    # top 2 by GFLOP/J: A (10.0), B (9.09); A's median over [10, 5, 5, 5] is 5
    assert tuple(best["cfg"]) == B and math.isclose(best["gflops_per_j"], 1 / 0.11)
