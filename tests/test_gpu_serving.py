"""Continuous-batching server: results alone and in the mix are identical,
admission waits for pool memory, plain mode agrees (GPU)."""
import numpy as np
import pytest

from gpu_helpers import MAX_REL, max_rel_err, oracle_ref
from paper_2211_07260_gb300 import api, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _payloads(n, seed, lo=64, hi=600):
    pay = []
    for i, sh in enumerate(synth.request_shapes(n, seed, lo, hi)):
        p = synth.request_problem(seed, i, sh)
        out = np.full((p.out_h, (p.out_w + 3) // 4 * 4), -7.0, np.float32)
        pay.append((p, p.inp, out))
    return pay


def test_each_result_is_the_same_alone_and_in_the_mix():
    mix = _payloads(120, seed=21)
    with api.Server(n_streams=3, max_batch=16, pool_bytes=1 << 30, max_wait_s=50e-6) as sv:
        ids = [sv.submit(inp, p.filt, out, p.out_h, p.out_w) for p, inp, out in mix]
        for i in ids:
            assert sv.wait(i) >= 0.0
        st = sv.stats()
        assert st["completed"] == len(mix) and st["batches"] >= len(mix) // 16
        assert st["mean_batch"] > 1.0  # requests did share launches
        # the same requests, each alone on an idle server
        for p, inp, out in mix[:40]:
            alone = np.full_like(out, -7.0)
            sv.wait(sv.submit(inp, p.filt, alone, p.out_h, p.out_w))
            assert np.array_equal(alone, out)
    for p, inp, out in mix:
        assert np.all(out[:, p.out_w:] == -7.0)
        assert max_rel_err(out[:, :p.out_w], oracle_ref(p)) <= MAX_REL


def test_plain_mode_matches_batched_mode_bitwise():
    mix = _payloads(40, seed=22)
    outs_plain = []
    with api.Server(n_streams=2, max_batch=8, plain=True, pool_bytes=1 << 30) as sv:
        for p, inp, out in mix:
            o = np.full_like(out, -7.0)
            outs_plain.append(o)
            sv.submit(inp, p.filt, o, p.out_h, p.out_w)
        sv.drain()
    with api.Server(n_streams=2, max_batch=8, pool_bytes=1 << 30) as sv:
        for p, inp, out in mix:
            sv.submit(inp, p.filt, out, p.out_h, p.out_w)
        sv.drain()
    for (p, inp, out), o in zip(mix, outs_plain):
        assert np.array_equal(o, out)


def test_admission_waits_for_pool_memory_and_rejects_oversize():
    mix = _payloads(30, seed=23, lo=300, hi=600)
    need = max(4 * (p.in_h * p.in_pitch + p.out_h * out.shape[1]) for p, _, out in mix)
    with api.Server(n_streams=2, max_batch=4, pool_bytes=int(need * 2.5)) as sv:
        for p, inp, out in mix:
            sv.submit(inp, p.filt, out, p.out_h, p.out_w)
        sv.drain()
        st = sv.stats()
        assert st["completed"] == len(mix) and st["pool_used_bytes"] == 0
        big = synth.conv_problem(1400, 1400, 3, seed=1)
        bo = np.zeros((1400, 1400), np.float32)
        with pytest.raises(api.ConvTuneError) as e:
            sv.submit(big.inp, big.filt, bo, 1400, 1400)
        assert e.value.status == api.CT_ENOMEM
    for p, inp, out in mix:
        assert max_rel_err(out[:, :p.out_w], oracle_ref(p)) <= MAX_REL


def test_poisson_driver_reports_latency_and_energy():
    from paper_2211_07260_gb300 import serve
    pay = serve.make_payloads(16, seed=24, lo=128, hi=512)
    for plain in (False, True):
        r = serve.serve_rate(pay, rate=2000.0, seconds=0.5, max_requests=1000, plain=plain,
                             n_streams=2, max_batch=16, pool_bytes=1 << 30, p_idle=150.0)
        assert r["requests"] == 1000
        assert 0 < r["p50_ms"] <= r["p99_ms"]
        assert r["energy_j"] > 0 and r["j_per_req"] > 0


def test_timeline_accounts_for_every_batch():
    mix = _payloads(60, seed=25)
    with api.Server(n_streams=2, max_batch=8, pool_bytes=1 << 30, trace_cap=1000) as sv:
        for p, inp, out in mix:
            sv.submit(inp, p.filt, out, p.out_h, p.out_w)
        sv.drain()
        st = sv.stats()
        tr = sv.trace()
    assert len(tr) == st["batches"] and sum(e["n_requests"] for e in tr) == len(mix)
    for e in tr:
        assert e["t_done"] >= e["t_dispatch"] + e["dispatch_s"] >= e["t_dispatch"]
        assert 0.0 <= e["plan_s"] <= e["dispatch_s"] and e["oldest_wait_s"] >= 0.0
        assert 0 <= e["slot"] < 2 and 0 <= e["busy_slots"] <= 1 and 1 <= e["n_requests"] <= 8
        # device-side split of the batch: copies in, kernels, copies out
        assert e["h2d_ms"] > 0 and e["kernels_ms"] > 0 and e["d2h_ms"] > 0
        assert e["h2d_ms"] + e["kernels_ms"] + e["d2h_ms"] <= (e["t_done"] - e["t_dispatch"]) * 1e3
        assert e["bytes_in"] > 0 and e["bytes_out"] > 0
    with api.Server(n_streams=1, max_batch=4, pool_bytes=1 << 28) as sv:  # no timeline kept
        with pytest.raises(api.ConvTuneError) as e:
            sv.trace()
        assert e.value.status == api.CT_ENOTSUP
    for p, inp, out in mix:
        assert max_rel_err(out[:, :p.out_w], oracle_ref(p)) <= MAX_REL
