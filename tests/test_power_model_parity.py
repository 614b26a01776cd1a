"""The library's FP64 power-model fit, optimum and clock range reproduce the
oracle (host code: runs without a GPU)."""
import numpy as np
import pytest

from oracle import power_model as opm
from paper_2211_07260_gb300 import api
from paper_2211_07260_gb300 import build as pkg_build

REL = 1e-9  # parity bar of the fit coefficients


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg_build.build()
    api.lib()


def curve(f, p0, a, b, tau):
    v = 1.0 + b * np.maximum(0.0, f - tau) / 1000.0
    return p0 + a * (f / 1000.0) * v ** 2


DATASETS = [
    # (name, f grid, params, noise sd, n throttled appended)
    ("noiseless_a", np.arange(990.0, 1651.0, 30.0), (180.0, 400.0, 0.8, 1230), 0.0, 0),
    ("noisy_b", np.arange(1200.0, 1801.0, 25.0), (95.0, 60.0, 2.5, 1402), 0.7, 0),
    ("noisy_gb300_like", np.arange(900.0, 2071.0, 97.5), (210.0, 520.0, 0.9, 1545), 4.0, 2),
    ("seven_clocks", np.linspace(900.0, 2070.0, 7).round(), (190.0, 480.0, 1.2, 1290), 2.0, 0),
]


def _same(a, b, rel=REL, abs_=1e-9):
    return abs(a - b) <= max(abs_, rel * max(abs(a), abs(b)))


@pytest.mark.parametrize("ds", DATASETS, ids=[d[0] for d in DATASETS])
def test_fit_matches_oracle(ds):
    name, f, params, sd, n_thr = ds
    rng = np.random.default_rng(abs(hash(name)) % 2**32)
    p = curve(f, *params) + (rng.normal(0, sd, f.size) if sd else 0.0)
    thr = np.zeros(f.size, bool)
    if n_thr:
        f = np.concatenate([f, [2100.0, 2150.0][:n_thr]])
        p = np.concatenate([p, [1500.0, 300.0][:n_thr]])
        thr = np.concatenate([thr, np.ones(n_thr, bool)])
    ref = opm.fit_power_model(f, p, throttled=thr, p_max_w=1400.0)
    got = api.fit_power_model(f, p, throttled=thr, p_max_w=1400.0)
    assert got["tau_mhz"] == ref["tau_mhz"]
    for k in ("p_idle_w", "alpha", "beta", "sse", "f_opt_mhz"):
        assert _same(got[k], ref[k], abs_=1e-9 if k != "sse" else 1e-12), (k, got[k], ref[k])
    assert got["n_used"] == ref["n_used"] and got["f_thr_mhz"] == ref["f_thr_mhz"]
    sup = np.arange(120, 2071, 7).astype(int)
    assert api.pick_clock_range(got, sup)[0] == opm.pick_clock_range(ref, sup)[0]
    assert api.pick_clock_range(got, sup, center="ridge")[0] == \
        opm.pick_clock_range(ref, sup, center="ridge")[0]


def test_voltage_fit_matches_oracle():
    rng = np.random.default_rng(9)
    f = np.arange(700.0, 1801.0, 55.0)
    v = 0.72 + 0.3 * np.maximum(0, f - 1150) / 650
    p = 140 + 330 * (f / 1000) * v ** 2 + rng.normal(0, 1.5, f.size)
    ref = opm.fit_power_model(f, p, v=v, p_max_w=900.0)
    got = api.fit_power_model(f, p, v=v, p_max_w=900.0)
    assert got["has_voltage"] == 1
    for k in ("p_idle_w", "alpha", "sse"):
        assert _same(got[k], ref[k], rel=1e-12), k
    assert got["f_opt_mhz"] == ref["f_opt_mhz"]


def test_optimum_matches_oracle_on_random_models():
    rng = np.random.default_rng(10)
    for _ in range(60):
        m = dict(p_idle_w=rng.uniform(20, 300), alpha=rng.uniform(50, 800),
                 beta=rng.uniform(0, 4), tau_mhz=float(rng.integers(700, 1700)),
                 p_max_w=float(rng.choice([1e9, rng.uniform(300, 1400)])),
                 f_lo_mhz=600.0, f_thr_mhz=2070.0, has_voltage=0)
        assert _same(api.optimal_clock(m), opm.optimal_clock(m), rel=1e-9)
        f = np.linspace(600, 2070, 50)
        np.testing.assert_allclose(api.model_power(m, f), opm.model_power(m, f), rtol=1e-14)


def test_errors():
    with pytest.raises(api.ConvTuneError) as e:
        api.fit_power_model([1000.0, 1100.0], [100.0, 110.0])
    assert e.value.status == api.CT_EINVAL
    with pytest.raises(api.ConvTuneError):
        api.fit_power_model([1000.0, 1100.0, 1200.0], [100.0, 110.0, 120.0],
                            throttled=[1, 0, 0])
    with pytest.raises(api.ConvTuneError):
        api.pick_clock_range(dict(f_opt_mhz=1000.0), [])
