"""Power capping versus clock locking (Section IV-C, Figs. 6-7), on simulated
GPUs (CPU only).

A board power limit is a device setting like a locked clock: on the GB300s
this library is measured on it is not changed (closed on this machine), so the
comparison runs on simulated devices whose DVFS lowers the clock to keep a
load under the limit.  The same configurations are swept over 9 equidistant
power limits (the device's whole range, as the paper's 100-300 W in steps of
25 W) and over 9 equidistant locked clocks; the paper finds that clock
tuning controls power more finely and over a larger, lower range, and
reaches the lower energy.
"""
import itertools

import numpy as np
import pytest

from oracle import selection as osel
from paper_2211_07260_gb300 import api
from paper_2211_07260_gb300 import build as pkg_build
from sim_platform import FakeBuffers, SimGPU

DEVICES = {
    # name: (p_idle W, alpha W/GHz, beta /GHz, ridge tau MHz, f_max MHz, lowest clock)
    "gb300-like": (180.0, 420.0, 0.9, 1380.0, 2070, 900),
    "titan-rtx-like": (40.0, 150.0, 0.8, 1400.0, 2100, 300),
    "a100-like": (55.0, 150.0, 1.2, 1025.0, 1410, 510),
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


def _device(name, **kw):
    p_idle, alpha, beta, tau, f_max, f_lo = DEVICES[name]
    clocks = list(range(f_max, f_lo - 1, -15))
    probe = SimGPU(p_idle=p_idle, alpha=alpha, beta=beta, tau=tau, f_max=f_max, clocks=clocks)
    p_top = probe.power_at(f_max, 1.0)
    # limits from a third of the full-load power up to a little above it
    # (the default: no cap at the top clock)
    plimit = (round(p_top / 3.0), round(p_top * 1.05), round(p_top * 1.05))
    return SimGPU(p_idle=p_idle, alpha=alpha, beta=beta, tau=tau, f_max=f_max, clocks=clocks,
                  plimit=plimit, **kw), clocks


def _opts():
    return api.tune_options(window_s=0.3, warmup_s=0.05)


def _rows(records, axis):
    return [dict(cfg=r["cfg"], clock=r[axis], t_s=r["t_s"], energy_j=r["energy_j"],
                 gflops_per_j=r["gflops_per_j"]) for r in records
            if not r["flags"] & api.REC_INVALID]


@pytest.mark.parametrize("name", sorted(DEVICES))
def test_clock_tuning_beats_power_capping(name):
    buf = FakeBuffers()
    kw = dict(in_pitch=buf.in_pitch, out_pitch=buf.out_pitch)
    sim, clocks = _device(name)
    sim.install()
    lo, hi, de = api.power_limit_range()
    limits = [float(x) for x in np.linspace(lo, hi, 9).round()]
    cap_recs, cap_best = api.tune_power_limits(*buf.args(), limits, space(), _opts(), **kw)
    assert len(cap_recs) == len(limits) * len(space())
    # every limit set once, limit-major, and the default restored each time
    assert sim.limit is None and sim.limit_calls == [int(w * 1000) for w in limits]
    assert sim.limit_resets == len(limits)
    assert [r["power_limit_w"] for r in cap_recs[::len(space())]] == limits
    # a limit that lowered the clock shows as power-cap throttling
    assert any(r["flags"] & api.REC_THROTTLED for r in cap_recs)
    assert not any(r["flags"] & api.REC_THROTTLED for r in cap_recs if r["power_limit_w"] == hi)
    # the library's pick over the capped table is the oracle's selection rule
    assert cap_best == osel.best_row(_rows(cap_recs, "power_limit_w"), "energy")

    sim2, _ = _device(name)
    sim2.install()
    sweep = sorted({min(clocks, key=lambda c: abs(c - x))
                    for x in np.linspace(min(clocks), max(clocks), 9)})
    clk_recs, clk_best = api.tune(*buf.args(), space(), sweep, _opts(), **kw)
    e_cap, e_clk = cap_recs[cap_best]["energy_j"], clk_recs[clk_best]["energy_j"]
    p_cap = [r["power_w_mean"] for r in cap_recs]
    p_clk = [r["power_w_mean"] for r in clk_recs]
    print(f"\n{name}: lowest energy capped {e_cap:.4e} J at {cap_recs[cap_best]['power_limit_w']:.0f} W "
          f"({cap_recs[cap_best]['clock_mhz_meas']:.0f} MHz), clock-tuned {e_clk:.4e} J at "
          f"{clk_recs[clk_best]['clock_mhz_req']} MHz ({e_cap / e_clk - 1:+.1%}); power range "
          f"capped {min(p_cap):.0f}-{max(p_cap):.0f} W, clocks {min(p_clk):.0f}-{max(p_clk):.0f} W")
    # Section IV-C: clock tuning reaches the lower energy, over a wider and
    # lower range of power
    assert e_clk <= e_cap * (1 + 1e-3)
    assert min(p_clk) < min(p_cap)
    assert max(p_clk) - min(p_clk) > max(p_cap) - min(p_cap)


def test_refused_power_limit_fails_or_falls_back():
    buf = FakeBuffers()
    kw = dict(in_pitch=buf.in_pitch, out_pitch=buf.out_pitch)
    sim, _ = _device("gb300-like", plimit_status=api.CT_EPERM)
    sim.install()
    opts = api.tune_options(window_s=0.3, warmup_s=0.05, fallback_default_clocks=False)
    with pytest.raises(api.ConvTuneError) as e:
        api.tune_power_limits(*buf.args(), [900.0, 1500.0], space()[:2], opts, **kw)
    assert e.value.status == api.CT_EPERM and sim.limit_resets == 0
    recs, best = api.tune_power_limits(*buf.args(), [900.0, 1500.0], space()[:2], _opts(), **kw)
    assert len(recs) == 2 and all(r["flags"] & api.REC_DEFAULT_CLOCKS for r in recs)
    assert best >= 0


def test_no_power_limit_control():
    # a platform without the power-limit calls (as the GB300 pool's NVML
    # table without CONVTUNE_ALLOW_POWER_CONTROL refuses them)
    buf = FakeBuffers()
    SimGPU().install()
    with pytest.raises(api.ConvTuneError) as e:
        api.power_limit_range()
    assert e.value.status == api.CT_ENOTSUP
    opts = api.tune_options(window_s=0.3, warmup_s=0.05, fallback_default_clocks=False)
    with pytest.raises(api.ConvTuneError) as e:
        api.tune_power_limits(*buf.args(), [900.0], space()[:1], opts,
                              in_pitch=buf.in_pitch, out_pitch=buf.out_pitch)
    assert e.value.status == api.CT_ENOTSUP
