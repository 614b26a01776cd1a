"""Serving driver: Poisson-arrival correlation requests through the library's
continuous-batching server (ct_server_*), and the same arrivals served with
one plain kernel per request.

  python -m paper_2211_07260_gb300.serve --rates 100,1000,10000 --seconds 10

Request shapes follow the batched workload's law (sides log-uniform in
[256, 2048], odd filter sides 3..17); a pool of distinct seeded payloads in
pinned host memory is reused cyclically (the arrival process and the shape
of each request come from their own seeded streams).  Reports p50/p99
latency, request throughput, GFLOP/s and joules per request (total and above
the idle power measured just before).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import api, synth


def make_payloads(n, seed=3, lo=256, hi=2048):
    import torch
    shapes = synth.request_shapes(n, seed, lo, hi)
    pay = []
    for i, sh in enumerate(shapes):
        p = synth.request_problem(seed, i, sh)
        inp = torch.from_numpy(p.inp).pin_memory().numpy()
        out = torch.empty((p.out_h, (p.out_w + 3) // 4 * 4), dtype=torch.float32).pin_memory()
        pay.append((p, inp, out.numpy()))
    return pay


def idle_power(seconds=1.0):
    samples = []
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        samples.append(api.read_sensors()["power_w"])
        time.sleep(0.05)
    return float(np.median(samples))


def trace_summary(trace, top=5):
    """Where the slowest batches' time went: waiting before the worker took
    them, enqueueing, device and copies, and pauses of the worker thread."""
    rows = []
    for e in trace:
        dev = e["t_done"] - e["t_dispatch"] - e["dispatch_s"]
        rows.append(dict(latency_ms=(e["oldest_wait_s"] + e["t_done"] - e["t_dispatch"]) * 1e3,
                         wait_ms=e["oldest_wait_s"] * 1e3, enqueue_ms=e["dispatch_s"] * 1e3,
                         plan_ms=e["plan_s"] * 1e3, device_and_copies_ms=dev * 1e3,
                         worker_pause_ms=e["loop_gap_s"] * 1e3, requests=e["n_requests"],
                         queued=e["queued"], busy_slots=e["busy_slots"],
                         h2d_ms=e["h2d_ms"], kernels_ms=e["kernels_ms"], d2h_ms=e["d2h_ms"],
                         h2d_gbs=e["bytes_in"] / max(e["h2d_ms"], 1e-6) / 1e6,
                         d2h_gbs=e["bytes_out"] / max(e["d2h_ms"], 1e-6) / 1e6))
    rows.sort(key=lambda r: -r["latency_ms"])
    gaps = sorted((e["loop_gap_s"] * 1e3 for e in trace), reverse=True)
    return dict(batches=len(trace), slowest=rows[:top],
                worker_pause_ms_max=gaps[0] if gaps else None,
                worker_pauses_over_5ms=sum(g > 5.0 for g in gaps),
                enqueue_ms_max=max((r["enqueue_ms"] for r in rows), default=None))


def serve_rate(payloads, rate, seconds, max_requests, seed=3, plain=False, tiles=None,
               n_streams=4, max_batch=64, max_wait_s=200e-6, pool_bytes=16 << 30, p_idle=None,
               trace_cap=0):
    n = int(min(max_requests, max(1, rate * seconds)))
    arrivals = synth.poisson_arrivals(rate, n, seed)
    with api.Server(n_streams=n_streams, max_batch=max_batch, pool_bytes=pool_bytes,
                    max_wait_s=max_wait_s, plain=plain, tiles=tiles, trace_cap=trace_cap) as sv:
        # warm-up (kernels loaded, pool touched), then a fresh statistics span
        for i in range(min(8, len(payloads))):
            p, inp, out = payloads[i]
            sv.submit(inp, p.filt, out, p.out_h, p.out_w)
        sv.drain()
        sv.stats(reset=True)
        t_warm = max((e["t_dispatch"] for e in sv.trace()), default=0.0) if trace_cap else 0.0
        t0 = time.perf_counter()
        for i in range(n):
            target = t0 + arrivals[i]
            while True:
                now = time.perf_counter()
                if now >= target:
                    break
                if target - now > 2e-3:
                    time.sleep(target - now - 1e-3)
            p, inp, out = payloads[i % len(payloads)]
            sv.submit(inp, p.filt, out, p.out_h, p.out_w)
        submit_lag = time.perf_counter() - (t0 + arrivals[-1])
        sv.drain(timeout_s=600.0)
        st = sv.stats()
        trace = sv.trace() if trace_cap else None
    res = dict(rate_hz=rate, mode="plain" if plain else "batched", requests=st["completed"],
               p50_ms=st["p50_s"] * 1e3, p99_ms=st["p99_s"] * 1e3, max_ms=st["max_s"] * 1e3,
               req_per_s=st["completed"] / st["wall_s"], gflops=st["flop"] / st["wall_s"] / 1e9,
               wall_s=st["wall_s"], mean_batch=st["mean_batch"], batches=st["batches"],
               energy_j=st["energy_j"], j_per_req=st["energy_j"] / max(1, st["completed"]),
               gflop_per_j=st["flop"] / 1e9 / st["energy_j"] if st["energy_j"] > 0 else None,
               submit_lag_s=submit_lag)
    if p_idle is not None:
        above = st["energy_j"] - p_idle * st["wall_s"]
        res["p_idle_w"] = p_idle
        res["j_per_req_above_idle"] = above / max(1, st["completed"])
    if trace is not None:
        # only the batches of the measured span (after the warm-up's last one)
        res["trace"] = trace_summary([e for e in trace if e["t_dispatch"] > t_warm])
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rates", default="100,300,1000,3000,10000,20000")
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--max-requests", type=int, default=20000)
    ap.add_argument("--payloads", type=int, default=256)
    ap.add_argument("--modes", default="batched,plain")
    ap.add_argument("--tiles", default=None,
                    help="JSON file of per-bucket tiles, or a tuned-configuration table "
                         "(its batched_tiles entry for this device)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--trace", type=int, default=0,
                    help="keep a timeline of the last N batches and report the slowest")
    a = ap.parse_args()
    tiles = None
    if a.tiles:
        raw = json.load(open(a.tiles))
        if "batched_tiles" in raw:  # a tuned-configuration table
            raw = raw["batched_tiles"].get(api.device_info()["name"], {})
        tiles = api.tiles_from_json(raw)
    payloads = make_payloads(a.payloads)
    p_idle = idle_power()
    rows = []
    for rate in [float(r) for r in a.rates.split(",")]:
        for mode in a.modes.split(","):
            r = serve_rate(payloads, rate, a.seconds, a.max_requests, plain=(mode == "plain"),
                           tiles=tiles, p_idle=p_idle, trace_cap=a.trace)
            print(json.dumps(r), flush=True)
            rows.append(r)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
