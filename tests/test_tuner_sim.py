"""The measurement window, exhaustive tuner, results cache, clock handling
and model-steered search, run against a simulated GPU (CPU only)."""
import itertools
import math

import numpy as np
import pytest

from oracle import power_model as opm
from oracle import selection as osel
from paper_2211_07260_gb300 import api
from paper_2211_07260_gb300 import build as pkg_build
from sim_platform import FakeBuffers, SimGPU


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg_build.build()
    api.lib()
    yield
    SimGPU.uninstall()


@pytest.fixture
def buf():
    return FakeBuffers()


def small_space():
    cfgs = []
    for bx, ty, st in itertools.product((16, 32, 64), (1, 2), (api.STAGE_DIRECT, api.STAGE_SMEM)):
        cfgs.append(api.Config(bx, 4, 2, ty, st, api.FILTER_CONST, 4))
    return cfgs


def kw(b):
    return dict(in_pitch=b.in_pitch, out_pitch=b.out_pitch)


def test_window_energy_matches_the_simulated_truth(buf):
    sim = SimGPU().install()
    cfg = api.Config(32, 4, 4, 2, api.STAGE_SMEM, api.FILTER_CONST, 4)
    r = api.measure_conv(*buf.args(), cfg, api.measure_options(window_s=1.0), **kw(buf))
    want_t = sim.t_base(api.CT_UNIT_CONV, cfg.to_c())
    want_e = sim.energy_per_launch(api.CT_UNIT_CONV, cfg.to_c(), sim.f_max)
    assert r["t_s"] == pytest.approx(want_t, rel=1e-9)
    assert r["energy_j"] == pytest.approx(want_e, rel=5e-3)
    assert r["power_w_mean"] == pytest.approx(sim.power_at(sim.f_max, sim.util(0, cfg.to_c())),
                                              rel=5e-3)
    assert r["energy_j_median_power"] == pytest.approx(want_e, rel=1e-2)
    assert r["flags"] == 0
    flop = osel.conv2d_flop(buf.k, buf.k, buf.out_h, buf.out_w)
    assert r["gflops"] == pytest.approx(flop / 1e9 / r["t_s"], rel=1e-12)
    assert r["gflops_per_j"] == pytest.approx(flop / 1e9 / r["energy_j"], rel=1e-12)
    # the window spans >= 1 s of load after warm-up and the second counter update
    assert sim.t >= 1.2


def test_time_only_has_no_energy(buf):
    SimGPU().install()
    r = api.measure_conv(*buf.args(), api.Config(), api.measure_options(time_only=True), **kw(buf))
    assert r["flags"] & api.REC_NO_ENERGY and math.isnan(r["energy_j"])
    assert r["t_s"] > 0


def test_flags_throttle_cotenant_and_missing_counter(buf):
    SimGPU(reasons=0x4, others=1).install()
    r = api.measure_conv(*buf.args(), api.Config(), api.measure_options(window_s=0.3), **kw(buf))
    assert r["flags"] & api.REC_THROTTLED and r["flags"] & api.REC_COTENANT
    sim = SimGPU(energy_status=api.CT_ENOTSUP).install()
    r = api.measure_conv(*buf.args(), api.Config(), api.measure_options(window_s=0.3), **kw(buf))
    assert r["flags"] & api.REC_NO_ENERGY
    want = sim.energy_per_launch(api.CT_UNIT_CONV, api.Config().to_c(), sim.f_max)
    assert r["energy_j"] == pytest.approx(want, rel=1e-6)  # median power x time


def _rows(records):
    return [dict(cfg=r["cfg"], clock=r["clock_mhz_req"], t_s=r["t_s"], energy_j=r["energy_j"],
                 gflops_per_j=r["gflops_per_j"]) for r in records
            if not r["flags"] & api.REC_INVALID]


@pytest.mark.parametrize("objective", ["energy", "time", "gflops_per_w"])
def test_exhaustive_tune_selects_like_the_oracle(buf, objective):
    sim = SimGPU().install()
    clocks = [1200, 1400, 1600, 1800, 2070]
    cfgs = small_space()
    recs, best = api.tune(*buf.args(), cfgs, clocks,
                          api.tune_options(objective, window_s=0.3, warmup_s=0.05), **kw(buf))
    assert len(recs) == len(cfgs) * len(clocks)
    # clock-major sweep, every lock undone
    assert [r["clock_mhz_req"] for r in recs[::len(cfgs)]] == clocks
    assert sim.lock_calls == clocks and sim.reset_calls == len(clocks) and sim.locked is None
    rows = _rows(recs)
    obj = {"energy": "energy", "time": "time", "gflops_per_w": "gflops_per_j"}[objective]
    assert best == osel.best_row(rows, obj)
    assert api.select_best(recs, objective) == best
    # energy per launch follows the simulated truth
    for r in recs:
        c = api.Config(*r["cfg"]).to_c()
        assert r["energy_j"] == pytest.approx(
            sim.energy_per_launch(0, c, r["clock_mhz_req"]), rel=1e-2)


def test_cache_resumes_an_interrupted_sweep(buf, tmp_path):
    cache = str(tmp_path / "cache.jsonl")
    cfgs = small_space()
    sim = SimGPU().install()
    recs1, best1 = api.tune(*buf.args(), cfgs, [1500, 1800],
                            api.tune_options(window_s=0.3, warmup_s=0.05, cache_path=cache),
                            **kw(buf))
    n_launch = sim.launches
    sim2 = SimGPU().install()
    recs2, best2 = api.tune(*buf.args(), cfgs, [1500, 1800, 2070],
                            api.tune_options(window_s=0.3, warmup_s=0.05, cache_path=cache),
                            **kw(buf))
    cached = [r for r in recs2 if r["flags"] & api.REC_CACHED]
    assert len(cached) == 2 * len(cfgs)
    assert all(not (r["flags"] & api.REC_CACHED) for r in recs2 if r["clock_mhz_req"] == 2070)
    for a, b in zip(recs1, recs2[:len(recs1)]):
        assert a["energy_j"] == b["energy_j"] and a["t_s"] == b["t_s"]
    assert 0 < sim2.launches < n_launch  # only the new clock was measured
    sim3 = SimGPU().install()
    recs3, best3 = api.tune(*buf.args(), cfgs, [1500, 1800, 2070],
                            api.tune_options(window_s=0.3, warmup_s=0.05, cache_path=cache),
                            **kw(buf))
    assert sim3.launches == 0 and best3 == best2
    assert len(open(cache).read().splitlines()) == 3 * len(cfgs)


def test_refused_lock_fails_or_falls_back(buf):
    cfgs = small_space()[:3]
    sim = SimGPU(lock_status=api.CT_EPERM).install()
    with pytest.raises(api.ConvTuneError) as e:
        api.tune(*buf.args(), cfgs, [1500, 1800],
                 api.tune_options(window_s=0.3, fallback_default_clocks=False), **kw(buf))
    assert e.value.status == api.CT_EPERM and sim.reset_calls == 0
    recs, best = api.tune(*buf.args(), cfgs, [1500, 1800],
                          api.tune_options(window_s=0.3, fallback_default_clocks=True), **kw(buf))
    assert len(recs) == 3 and all(r["flags"] & api.REC_DEFAULT_CLOCKS for r in recs)
    assert best >= 0


def test_unheld_clock_is_flagged_throttled(buf):
    SimGPU(throttle_above=1700).install()
    recs, _ = api.tune(*buf.args(), small_space()[:2], [1600, 1900],
                       api.tune_options(window_s=0.3, warmup_s=0.05), **kw(buf))
    assert all(not r["flags"] & api.REC_THROTTLED for r in recs if r["clock_mhz_req"] == 1600)
    assert all(r["flags"] & api.REC_THROTTLED for r in recs if r["clock_mhz_req"] == 1900)


def test_invalid_points_are_recorded_not_measured(buf):
    SimGPU().install()
    cfgs = [api.Config(48, 1, 1, 1, 0, 1, 1), api.Config(), api.Config(tile_x=3)]
    recs, best = api.tune(*buf.args(), cfgs, None, api.tune_options(window_s=0.3), **kw(buf))
    assert [bool(r["flags"] & api.REC_INVALID) for r in recs] == [True, False, True]
    assert best == 1


def test_capacity_and_argument_errors(buf):
    SimGPU().install()
    with pytest.raises(api.ConvTuneError) as e:
        api.tune(*buf.args(), small_space(), None, api.tune_options(objective=7), **kw(buf))
    assert e.value.status == api.CT_EINVAL


def test_steered_search_lands_near_the_exhaustive_optimum(buf):
    sim = SimGPU()
    sup = sim.clocks
    fit_clocks = [int(c) for c in np.linspace(min(sup), max(sup), 7).round() // 15 * 15]
    fit_clocks = [c if c in sup else min(sup, key=lambda s: abs(s - c)) for c in fit_clocks]
    cfgs = small_space()
    # exhaustive reference over every supported clock
    sim_ex = SimGPU().install()
    ex_recs, ex_best = api.tune(*buf.args(), cfgs, sup,
                                api.tune_options(window_s=0.3, warmup_s=0.05), **kw(buf))
    ex_wall = sum(r["wall_s"] for r in ex_recs)
    sim_st = SimGPU().install()
    res, rng, st_recs, st_best = api.tune_steered(
        *buf.args(), fit_clocks, cfgs, supported=sup, rel_halfwidth=0.10,
        opts=api.tune_options(window_s=0.3, warmup_s=0.05), **kw(buf))
    m = res["model"]
    # the fit recovers the simulated curve (power read from the counter)
    assert m["tau_mhz"] == pytest.approx(sim.tau, abs=40)
    assert m["p_idle_w"] == pytest.approx(sim.p_idle, rel=0.05)
    # its optimum and range follow the oracle's reading of Section IV-E
    ref = opm.fit_power_model(fit_clocks, _fit_powers(sim, fit_clocks), p_max_w=0.0)
    assert res["center_mhz"] == pytest.approx(ref["f_opt_mhz"], rel=0.03)
    assert rng == sorted(c for c in sup if 0.9 * res["center_mhz"] <= c <= 1.1 * res["center_mhz"])
    assert {r["clock_mhz_req"] for r in st_recs} == set(rng)
    gap = st_recs[st_best]["energy_j"] / ex_recs[ex_best]["energy_j"] - 1
    assert gap <= 0.05
    frac = (res["fit_wall_s"] + res["tune_wall_s"]) / ex_wall
    assert frac <= 0.25, frac
    assert sim_st.locked is None and len(sim_st.lock_calls) == sim_st.reset_calls


def _fit_powers(sim, clocks):
    return [sim.power_at(c, 1.0) for c in clocks]
