"""The library's tuning-method selection, Pareto front and centrality
reproduce the oracle (host code, no GPU), on tables from the simulated
platform and on random tables."""
import itertools

import numpy as np
import pytest

from oracle import selection as sel
from paper_2211_07260_gb300 import api
from paper_2211_07260_gb300 import build as pkg_build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg_build.build()
    api.lib()


def random_records(seed, n_cfg=24, clocks=(900, 1200, 1500, 1800, 2070)):
    rng = np.random.default_rng(seed)
    cfgs = list(itertools.product((16, 32, 64), (1, 2), (2, 4), (1, 2)))[:n_cfg]
    recs = []
    for c in cfgs:
        speed = rng.uniform(0.5, 1.5)
        for f in clocks:
            t = 1e-3 / speed * 2070 / f * rng.uniform(0.98, 1.02)
            p = 180 + 450 * (f / 1000) * (1 + 0.9 * max(0, f - 1400) / 1000) ** 2 * rng.uniform(0.8, 1.0)
            e = p * t
            recs.append(dict(cfg=(c[0], c[1], c[2], c[3], 1, 1, 4), clock_mhz_req=f,
                             clock_mhz_meas=float(f), t_s=t, energy_j=e, power_w_mean=p,
                             power_w_median=p, energy_j_median_power=e, gflops=1.0 / t,
                             gflops_per_j=1.0 / e, temp_c=50.0, wall_s=0.5, n_launches=100,
                             flags=0))
    return recs


def rows_of(recs):
    return [dict(cfg=tuple(r["cfg"]), clock=r["clock_mhz_req"], t_s=r["t_s"],
                 energy_j=r["energy_j"], gflops=r["gflops"], gflops_per_j=r["gflops_per_j"])
            for r in recs]


@pytest.mark.parametrize("seed", range(6))
def test_methods_and_front_match_oracle(seed):
    recs = random_records(seed)
    rows = rows_of(recs)
    got = api.tuning_methods(recs, base_clock_mhz=1400)
    want = sel.tuning_methods(rows, base_clock=1400)
    assert got == want
    assert api.pareto_front(recs) == sel.pareto_front(rows)


@pytest.mark.parametrize("seed", range(3))
def test_centrality_matches_oracle(seed):
    recs = random_records(seed, n_cfg=12, clocks=(1200, 1600, 2070))
    rows = rows_of(recs)
    for objective in ("energy", "time"):
        got = api.centrality(recs, objective)
        want = sel.proportion_of_centrality(rows, objective)
        for p in want:
            assert got[p] == pytest.approx(want[p], rel=1e-9, abs=1e-12)
        assert got[max(want)] <= 1.0 + 1e-12


def test_invalid_records_are_ignored():
    recs = random_records(9, n_cfg=4)
    bad = dict(recs[0])
    bad["flags"] = api.REC_INVALID
    bad["t_s"] = float("nan")
    got = api.tuning_methods([bad] + recs, 1400)
    want = api.tuning_methods(recs, 1400)
    assert {k: v - 1 for k, v in got.items()} == want
