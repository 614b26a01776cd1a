"""The library's memory-aware energy model (time fit, optimum of P*(f) t(f),
clock ranges) reproduces the oracle (host code: runs without a GPU)."""
import numpy as np
import pytest

from oracle import memory_model as omm
from oracle import power_model as opm
from paper_2211_07260_gb300 import api
from paper_2211_07260_gb300 import build as pkg_build

REL = 1e-9  # parity bar of the fitted coefficients


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg_build.build()
    api.lib()


def _close(a, b, rel=REL, abs_=1e-15):
    return abs(a - b) <= max(abs_, rel * max(abs(a), abs(b)))


def _power(f, p0, alpha, beta, tau):
    v = 1.0 + beta * np.maximum(0.0, f - tau) / 1000.0
    return p0 + alpha * (f / 1000.0) * v * v


CASES = [
    # (seed, clocks, power params, t_mem, c_core, time noise sd (rel), throttled tail)
    (0, np.arange(900.0, 2071.0, 97.5), (190.0, 260.0, 0.7, 1450.0), 3.0e-4, 1e-5, 0.01, 0),
    (1, np.linspace(900.0, 2070.0, 7).round(), (210.0, 300.0, 0.9, 1380.0), 2.5e-4, 4e-5, 0.0, 0),
    (2, np.arange(600.0, 1411.0, 45.0), (55.0, 120.0, 1.2, 1025.0), 1e-4, 4e-4, 0.02, 2),
    (3, np.arange(1200.0, 2101.0, 75.0), (40.0, 150.0, 0.8, 1400.0), 0.0, 1.5e-3, 0.005, 1),
    (4, np.arange(900.0, 2071.0, 130.0), (180.0, 420.0, 0.9, 1380.0), 8e-4, 8e-4, 0.03, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[f"case{c[0]}" for c in CASES])
def test_memory_aware_model_matches_oracle(case):
    seed, f, (p0, alpha, beta, tau), a, b, sd, n_thr = case
    rng = np.random.default_rng(seed)
    p = _power(f, p0, alpha, beta, tau) * (1.0 + 0.004 * rng.standard_normal(f.size))
    t = (a + b / (f / 1000.0)) * (1.0 + sd * rng.standard_normal(f.size))
    thr = np.zeros(f.size, dtype=bool)
    if n_thr:
        thr[-n_thr:] = True
        t[-n_thr:] *= 1.5
    # time model
    tm_lib = api.fit_time_model(f, t, thr)
    tm_ora = omm.fit_time_model(f, t, thr)
    for k in ("t_mem_s", "c_core_s_ghz"):
        assert _close(tm_lib[k], tm_ora[k]), (k, tm_lib[k], tm_ora[k])
    assert _close(tm_lib["sse"], tm_ora["sse"], rel=1e-8, abs_=1e-24)
    assert tm_lib["n_used"] == tm_ora["n_used"]
    assert tm_lib["f_lo_mhz"] == tm_ora["f_lo_mhz"] and tm_lib["f_thr_mhz"] == tm_ora["f_thr_mhz"]
    assert np.allclose(api.model_time(tm_lib, f), omm.model_time(tm_ora, f), rtol=1e-12)
    # power model of the same unit (parity of the fit itself is pinned
    # elsewhere), then the memory-aware optimum over the shared clocks
    pm_lib = api.fit_power_model(f, p, throttled=thr)
    pm_ora = opm.fit_power_model(f, p, throttled=thr)
    f_lib, e_lib = api.memory_aware_optimum(pm_lib, tm_lib)
    res = omm.energy_optimum(pm_ora, tm_ora)
    assert f_lib == res["f_opt_mhz"]
    assert _close(e_lib, res["e_opt_j"], rel=1e-8)
    # the library's optimum on the oracle's models is the same clock
    f_lib2, _ = api.memory_aware_optimum(pm_ora, tm_ora)
    assert f_lib2 == res["f_opt_mhz"]
    # range around it
    sup = list(range(int(f.min()), int(f.max()) + 1, 15))
    assert api.clock_range(f_lib, sup, 0.10) == omm.clock_range(res["f_opt_mhz"], sup, 0.10)


def test_range_edges_match_oracle():
    sup = [510, 600, 1005, 1410, 1995]
    for c0 in (0.0, 100.0, 555.0, 1000.0, 1400.0, 1410.0, 3000.0):
        for rel in (0.0, 0.05, 0.10, 0.5):
            assert api.clock_range(c0, sup, rel) == omm.clock_range(c0, sup, rel), (c0, rel)


def test_argument_errors():
    with pytest.raises(api.ConvTuneError):
        api.fit_time_model([1000.0], [1e-3])  # one sample
    with pytest.raises(api.ConvTuneError):
        api.fit_time_model([1000.0, -5.0], [1e-3, 1e-3])
    pm = opm.fit_power_model(np.arange(900.0, 2071.0, 100.0),
                             _power(np.arange(900.0, 2071.0, 100.0), 180.0, 420.0, 0.9, 1380.0))
    tm = omm.fit_time_model([2100.0, 2200.0], [1e-3, 1e-3])
    with pytest.raises(api.ConvTuneError):
        api.memory_aware_optimum(pm, tm)  # no shared clock
    pv = dict(pm, has_voltage=1)
    with pytest.raises(api.ConvTuneError):
        api.memory_aware_optimum(pv, omm.fit_time_model([900.0, 2000.0], [1e-3, 1e-3]))
