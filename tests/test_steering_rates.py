"""Model-steered clock search (Section IV-E) under measurement noise and on
devices the power model does not describe exactly (CPU only, simulated).

The deterministic study (test_steering_study.py) simulates devices whose
power is Eq. (powercurve) itself, without noise, so the fit recovers its own
generator.  Here each comparison of steered search and exhaustive sweep is
repeated over five seeds with power jitter (1.5 % per simulated run of
launches), duration jitter (0.3 %) and a millijoule energy counter, on two
kinds of device: one following Eq. (powercurve), and one whose voltage rises
through a smooth, curved knee and whose static power grows with voltage (the
fit can only approximate it).  Reported per device and truth: the match rate
of the steered (configuration, clock) with the exhaustive one, the energy
gap of the steered pick to the true optimum and to the exhaustive pick, and
the tuning-time fraction (with and without the one-off fit).

A second study runs a workload whose time is 80 % memory-bound: the paper's
compute-bound model (P*(f)/f, fitted on the FMA kernel) is then the wrong
model, and the memory-aware model fitted on the stream-copy kernel (Sections
II and IV-F; ct_tune_steered with CT_UNIT_COPY) or the union of both ranges
is compared against it.
"""
import itertools
import statistics

import pytest

from paper_2211_07260_gb300 import api
from paper_2211_07260_gb300 import build as pkg_build
from sim_platform import FakeBuffers, SimGPU

SEEDS = range(5)
# clocks of the microbenchmark sweep the model is fitted on (equidistant over
# the supported range): one microbenchmark window per clock, ~2 % of the
# exhaustive sweep's cost; with 7 the noisy fits sometimes put the ridge
# point, and with it the range, 10-20 % off
N_FIT = 15
NOISE = dict(sigma_p=0.015, sigma_t=0.003)
TRUTHS = {
    "powercurve": dict(truth="powercurve"),
    "curved": dict(truth="curved", knee=80.0, gamma=1.2, leak=0.35),
}
DEVICES = {
    # name: (p_idle W, alpha W/GHz, beta /GHz, ridge tau MHz, f_max MHz, lowest clock, throttle cap)
    "gb300-like": (180.0, 420.0, 0.9, 1380.0, 2070, 900, None),
    "a100-like": (55.0, 150.0, 1.2, 1025.0, 1410, 510, None),
    "a4000-like": (30.0, 70.0, 1.0, 1290.0, 1845, 600, None),
    "v100-like": (40.0, 160.0, 1.1, 1100.0, 1530, 540, None),
    "titan-rtx-like": (40.0, 150.0, 0.8, 1400.0, 2100, 600, 2000),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg_build.build()
    api.lib()
    yield
    SimGPU.uninstall()


def space():
    return [api.Config(bx, 4, 2, ty, st, api.FILTER_CONST, 4)
            for bx, ty, st in itertools.product((16, 32, 64), (1, 2),
                                                (api.STAGE_DIRECT, api.STAGE_SMEM))]


def _opts():
    # the library's default 2 ms replays: the simulated host sees a counter
    # update only when a replay ends, so much longer replays would bias the
    # measured power (by up to ~5 % with 20 ms replays)
    return api.tune_options(window_s=0.3, warmup_s=0.05)


def compare(name, sim_kw, seed, which_bench=api.CT_UNIT_FMA):
    """One exhaustive sweep and one steered search, each on its own noisy
    measurement of the same simulated device."""
    p_idle, alpha, beta, tau, f_max, f_lo, cap = DEVICES[name]
    clocks = list(range(f_max, f_lo - 1, -15))

    def device(s):
        return SimGPU(p_idle=p_idle, alpha=alpha, beta=beta, tau=tau, f_max=f_max, clocks=clocks,
                      throttle_above=cap, seed=s, **sim_kw)

    buf = FakeBuffers()
    kw = dict(in_pitch=buf.in_pitch, out_pitch=buf.out_pitch)
    truth = device(None)
    device(2 * seed).install()
    ex_recs, ex_best = api.tune(*buf.args(), space(), clocks, _opts(), **kw)
    ex_wall = sum(r["wall_s"] for r in ex_recs)
    fit = sorted({min(clocks, key=lambda c: abs(c - x))
                  for x in (f_lo + (f_max - f_lo) * q / (N_FIT - 1) for q in range(N_FIT))})
    sim = device(2 * seed + 1).install()
    res, rng, st_recs, st_best = api.tune_steered(*buf.args(), fit, space(), supported=clocks,
                                                  rel_halfwidth=0.10, which_bench=which_bench,
                                                  opts=_opts(), **kw)
    assert sim.locked is None and len(sim.lock_calls) == sim.reset_calls

    def e_true(r):
        return truth.energy_per_launch(api.CT_UNIT_CONV, api.Config(*r["cfg"]).to_c(),
                                       r["clock_mhz_req"])

    # the true optimum over the whole space (noise-free)
    e_opt = min(truth.energy_per_launch(api.CT_UNIT_CONV, c.to_c(), f)
                for c in space() for f in clocks)
    ex, st = ex_recs[ex_best], st_recs[st_best]
    return dict(
        match=st["clock_mhz_req"] == ex["clock_mhz_req"] and tuple(st["cfg"]) == tuple(ex["cfg"]),
        same_clock=st["clock_mhz_req"] == ex["clock_mhz_req"],
        gap_meas=st["energy_j"] / ex["energy_j"] - 1.0,
        gap_true=e_true(st) / e_opt - 1.0,
        gap_true_exhaustive=e_true(ex) / e_opt - 1.0,
        time_fraction=(res["fit_wall_s"] + res["tune_wall_s"]) / ex_wall,
        sweep_fraction=res["tune_wall_s"] / ex_wall,
        steered_clock=st["clock_mhz_req"], exhaustive_clock=ex["clock_mhz_req"],
        range=(min(rng), max(rng)))


def _summary(rows):
    gaps = [r["gap_true"] for r in rows]
    return dict(match_rate=sum(r["match"] for r in rows) / len(rows),
                clock_match_rate=sum(r["same_clock"] for r in rows) / len(rows),
                gap_true_median=statistics.median(gaps), gap_true_max=max(gaps),
                gap_meas_max=max(r["gap_meas"] for r in rows),
                gap_true_exhaustive_max=max(r["gap_true_exhaustive"] for r in rows),
                time_fraction_max=max(r["time_fraction"] for r in rows),
                sweep_fraction_max=max(r["sweep_fraction"] for r in rows))


@pytest.mark.parametrize("truth", sorted(TRUTHS))
@pytest.mark.parametrize("name", sorted(DEVICES))
def test_steering_rates_under_noise(name, truth):
    rows = [compare(name, dict(TRUTHS[truth], **NOISE), s) for s in SEEDS]
    summ = _summary(rows)
    print(f"\n{name} {truth}: " + ", ".join(f"{k}={v:.3f}" for k, v in summ.items()))
    for r in rows:
        print("   ", {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()})
    # within 5 % of the true energy optimum, on every repeat.  Tuning time:
    # the +-10 % window spans 0.2 f_opt of a clock axis f_max - f_min long,
    # 21-25 % of the axis on these devices, so the steered sweep takes about
    # a quarter of the exhaustive one (measured 0.19-0.25), and the fit -- a
    # one-off per GPU, Section IV-E fits once and reuses the curve for every
    # kernel -- adds ~2 %
    assert summ["gap_true_max"] <= 0.05, summ
    assert summ["sweep_fraction_max"] <= 0.26, summ
    assert summ["time_fraction_max"] <= 0.28, summ


MEM_WORKLOAD = dict(mem_frac=0.8, copy_mem_frac=0.9, p_mem=25.0)


@pytest.mark.parametrize("name", ["gb300-like", "a100-like"])
def test_memory_bound_workload_wants_the_memory_aware_model(name):
    out = {}
    for label, which in (("compute", api.CT_UNIT_FMA), ("memory", api.CT_UNIT_COPY),
                         ("union", api.CT_STEER_UNION)):
        rows = [compare(name, dict(MEM_WORKLOAD, **NOISE), s, which) for s in SEEDS[:3]]
        out[label] = _summary(rows)
        print(f"\n{name} memory-bound workload, {label} model: "
              + ", ".join(f"{k}={v:.3f}" for k, v in out[label].items()))
    # the memory-aware range (alone or in the union) holds a point within 5 %
    # of the true optimum; the compute-bound model's range does worse
    assert out["memory"]["gap_true_max"] <= 0.05, out
    assert out["union"]["gap_true_max"] <= 0.05, out
    assert out["compute"]["gap_true_median"] > out["memory"]["gap_true_median"], out
