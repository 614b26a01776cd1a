"""Measurement, microbenchmarks and tuning on the real device (GPU).

Clock locking is never attempted here: the NVML table refuses it unless
CONVTUNE_ALLOW_CLOCK_CONTROL=1, and these tests check that refusal.
"""
import math
import os

import numpy as np
import pytest

from gpu_helpers import MAX_REL, max_rel_err, oracle_ref, to_device
from paper_2211_07260_gb300 import api, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _nvml_table():
    api.set_platform_ops(None)
    yield


def test_nvml_and_supported_clocks():
    assert api.nvml_status() == api.CT_OK
    clocks = api.supported_sm_clocks()
    assert len(clocks) > 10 and clocks == sorted(clocks, reverse=True)
    assert 1500 <= clocks[0] <= 3000


def test_clock_control_is_off_by_default():
    assert os.environ.get("CONVTUNE_ALLOW_CLOCK_CONTROL") != "1"
    assert api.lib().ct_lock_sm_clock(1500) == api.CT_EPERM
    assert api.lib().ct_reset_sm_clock() == api.CT_EPERM


def test_measure_conv_energy_window():
    prob = synth.conv_problem(1024, 1024, 7, seed=0)
    d_in, full, d_out = to_device(prob)
    cfg = api.Config(32, 4, 4, 2, api.STAGE_SMEM, api.FILTER_CONST, 4)
    r = api.measure_conv(d_in, prob.filt, d_out, 1024, 1024, cfg,
                         api.measure_options(window_s=0.3))
    assert r["t_s"] > 0 and r["n_launches"] > 100
    assert not r["flags"] & api.REC_NO_ENERGY
    assert 100.0 < r["power_w_mean"] < 1500.0
    assert r["energy_j"] == pytest.approx(r["power_w_mean"] * r["t_s"])
    assert r["gflops"] == pytest.approx(2 * 49 * 1024 * 1024 / 1e9 / r["t_s"])
    # the graph replays computed the right thing
    assert max_rel_err(full.cpu().numpy()[:, :1024], oracle_ref(prob)) <= MAX_REL


def test_microbenchmarks_load_the_gpu():
    info = api.device_info()
    fma = api.measure_microbench(api.CT_UNIT_FMA, api.measure_options(window_s=0.3))
    # the FMA-dense kernel is the empirical check of the derived FP32 peak
    # (SMs x 128 lanes x 2 FLOP x the SM clock measured in its window)
    peak_at_clock = info["sm_count"] * 256 * fma["clock_mhz_meas"] * 1e6 / 1e9
    assert 0.85 * peak_at_clock <= fma["gflops"] <= 1.01 * peak_at_clock
    copy = api.measure_microbench(api.CT_UNIT_COPY, api.measure_options(window_s=0.3))
    assert copy["gflops"] > 3000.0  # "GFLOP" of the copy unit is GB moved
    f, p, thr, recs = api.measure_power_samples(api.CT_UNIT_FMA, None,
                                                api.measure_options(window_s=0.3))
    assert f[0] > 0 and p[0] > 100.0
    api.lib().ct_microbench_release()


def test_tune_at_default_clocks_small_space():
    prob = synth.conv_problem(512, 512, 5, seed=4)
    d_in, full, d_out = to_device(prob)
    cfgs = [api.Config(32, 4, 4, 2, api.STAGE_SMEM, api.FILTER_CONST, 4),
            api.Config(64, 2, 2, 2, api.STAGE_DIRECT, api.FILTER_CONST, 2),
            api.Config(48, 1, 1, 1, 0, 1, 1),  # invalid block_x: pruned
            api.Config(128, 8, 4, 4, api.STAGE_TMA, api.FILTER_SHARED, 4)]
    for objective in ("time", "energy"):
        recs, best = api.tune(d_in, prob.filt, d_out, 512, 512, cfgs, None,
                              api.tune_options(objective, window_s=0.2, warmup_s=0.05,
                                               time_only=(objective == "time")))
        assert len(recs) == 4 and recs[2]["flags"] & api.REC_INVALID
        assert best in (0, 1, 3)
        valid = [r for r in recs if not r["flags"] & api.REC_INVALID]
        key = "t_s" if objective == "time" else "energy_j"
        assert recs[best][key] == min(r[key] for r in valid if not math.isnan(r[key]))
    assert max_rel_err(full.cpu().numpy()[:, :512], oracle_ref(prob)) <= MAX_REL


def test_bounded_device_wait_gives_up_and_reports():
    # a barrier phase that nothing completes: the wait runs out after 1000
    # polls, the kernel returns and says so in the status word
    api.status_read(clear=True)
    assert api.lib().ct_selftest_wait_timeout(1000, None) == api.CT_OK
    assert api.status_read(clear=True) & 1
    assert api.lib().ct_selftest_wait_timeout(0, None) == api.CT_EINVAL
    # the context is still usable afterwards
    prob = synth.conv_problem(64, 80, 9, seed=12)
    d_in, full, d_out = to_device(prob)
    api.conv2d_run(d_in, prob.filt, d_out, 64, 80,
                   api.Config(32, 4, 4, 2, api.STAGE_TMA, api.FILTER_CONST, 4))
    assert max_rel_err(full.cpu().numpy()[:, :80], oracle_ref(prob)) <= MAX_REL
    assert api.status_read(clear=True) == 0
