#!/usr/bin/env python
"""Benchmark: FP32 2-D correlation GFLOP/s and GFLOP/J at the tuned
configuration on GB300 (one JSON line on stdout).

Workload (default): a 4096 x 4096 output, 17 x 17 filter, zero-padded input
4112 x 4112 uniform[0, 1) (seed 1), filter uniform[0, 1) normalised to sum 1,
at the configuration the energy-objective tuner picked (tuned_configs.json),
default clocks.  A step is one launch of the correlation; inputs stay
resident in HBM and L2 is flushed (a 256 MiB write) between timed launches.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl convtune|reference]

At N = 1 the same line also carries, each with its own SM-clock record:
  roofline.peak_empirical_fma_kernel  the FMA-dense microbenchmark's TFLOP/s
                                      beside the derived FP32 peak;
  config1_1024x1024_k7                1024 x 1024 / 7 x 7 at its energy-tuned
                                      configuration, graph-replayed and with
                                      L2 flushed, against min(FP32, AI x HBM);
  batched256                          the 256-image batch as one CUDA-graph
                                      launch (the batch's mode: one single-
                                      image kernel per image over 12 graph
                                      branches), the persistent class kernels'
                                      graph, and one host-issued plain launch
                                      per image (GFLOP/s, GFLOP/J, mixed
                                      roofline, FP64 oracle baseline);
  serving                             Poisson requests through the continuous-
                                      batching server vs one plain kernel per
                                      request (p50 / p99, J per request).
(--no-extras leaves them out.)

Under torchrun (N > 1) every rank runs its own replica (no exchange step:
weak scaling); rank 0 prints whole-job throughput.  --impl reference times
the CPU oracle (FP64 direct correlation, OpenMP) on bands of the same
workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "conv2d GFLOP/s & GFLOP/J at tuned config; model-steered vs exhaustive tune time"
WORKLOADS = {
    "4096x4096_k17": dict(h=4096, w=4096, k=17, seed=1),
    "1024x1024_k7": dict(h=1024, w=1024, k=7, seed=0),
    # 256 images, sides log-uniform [256, 2048], odd k 3..17 (seed 2): one
    # persistent CUDA-graph launch vs one plain launch per image
    "batched256": dict(n=256, seed=2),
}
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (4 SMSPs x 32)
FLUSH_BYTES = 256 << 20   # > 129 MiB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="convtune", choices=["convtune", "reference"])
    ap.add_argument("--workload", default="4096x4096_k17", choices=sorted(WORKLOADS))
    ap.add_argument("--config", default=None, help="bx,by,tx,ty,staging,filter,vw")
    ap.add_argument("--energy-window", type=float, default=1.0)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-energy", action="store_true", help="skip the energy window")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline workload only (no 1024^2 / batched / serving / FMA-peak keys)")
    ap.add_argument("--serve-rate", type=float, default=5000.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-payloads", type=int, default=64)
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def all_max(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def tuned_entry(name, wl):
    path = os.path.join(ROOT, "paper_2211_07260_gb300", "tuned_configs.json")
    key = f"{wl['h']}x{wl['w']}_k{wl['k']}"
    if os.path.exists(path):
        table = json.load(open(path))
        for dev, entries in table.get("devices", {}).items():
            if name.startswith(dev) and key in entries:
                return entries[key]
    return None


def tuned_config(api, name, wl, override):
    if override:
        vals = [int(v) for v in override.split(",")]
        return api.Config(*vals), "command line"
    e = tuned_entry(name, wl)
    if e:
        return api.Config(*e["config"]), f"tuned_configs.json ({e.get('objective')})"
    return api.Config(32, 8, 4, 2, api.STAGE_TMA, api.FILTER_CONST, 4), "built-in default"


class ClockSampler:
    """nvidia-smi clocks / power / throttle reasons every 50 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.2)

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), pw=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], cap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        load = [r for r in rows if r["pw"] > 300.0] or rows
        reasons = set()
        for r in load:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("cap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return dict(sm_mhz=statistics.median(r["sm"] for r in load),
                    sm_max_mhz=max(r["smax"] for r in rows),
                    power_w_median=statistics.median(r["pw"] for r in load),
                    samples=len(rows), samples_under_load=len(load), reasons=sorted(reasons))


def cpu_baseline(wl, seconds):
    import oracle
    from oracle import selection
    from paper_2211_07260_gb300 import synth
    prob = synth.conv_problem(wl["h"], wl["w"], wl["k"], seed=wl["seed"])
    flop = selection.conv2d_flop(wl["k"], wl["k"], wl["h"], wl["w"])
    nt = oracle.max_threads()
    oracle.conv2d(prob.inp[:64 + wl["k"]], prob.filt, in_w=prob.in_w)  # warm-up
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.conv2d(prob.inp, prob.filt, in_w=prob.in_w, nthreads=nt)
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return dict(value=reps * flop / dt / 1e9, unit="GFLOP/s", cores=nt, kind="oracle",
                sample=f"full {wl['h']}x{wl['w']} {wl['k']}x{wl['k']} correlation in FP64, "
                       f"{reps} repetition(s), {dt:.1f} s wall, {nt} OpenMP threads")


def run_reference(args, world, rank):
    wl = WORKLOADS[args.workload]
    if rank != 0:
        return
    import oracle
    from oracle import selection
    from paper_2211_07260_gb300 import synth
    prob = synth.conv_problem(wl["h"], wl["w"], wl["k"], seed=wl["seed"])
    k = wl["k"]
    nt = oracle.max_threads()
    # size one step's band of output rows so the whole run takes ~2 minutes
    probe_rows = 64
    t0 = time.perf_counter()
    oracle.conv2d(prob.inp[:probe_rows + k - 1], prob.filt, in_w=prob.in_w, nthreads=nt)
    per_row = (time.perf_counter() - t0) / probe_rows
    rows = int(max(16, min(wl["h"], 120.0 / (args.steps + args.warmup) / per_row)))
    band = prob.inp[:rows + k - 1]
    for _ in range(args.warmup):
        oracle.conv2d(band, prob.filt, in_w=prob.in_w, nthreads=nt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.conv2d(band, prob.filt, in_w=prob.in_w, nthreads=nt)
    dt = time.perf_counter() - t0
    flop = selection.conv2d_flop(k, k, rows, wl["w"])
    value = args.steps * flop / dt / 1e9
    sample = (f"{rows} of {wl['h']} output rows x {wl['w']} columns, {k}x{k}, FP64 "
              f"(band of the {args.workload} workload per step)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample_rows": rows},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": nt, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


def load_tiles(api):
    """Per-bucket batched tiles of this device from tuned_configs.json."""
    path = os.path.join(ROOT, "paper_2211_07260_gb300", "tuned_configs.json")
    if os.path.exists(path):
        t = json.load(open(path)).get("batched_tiles", {}).get(api.device_info()["name"])
        if t:
            return api.tiles_from_json(t), "tuned_configs.json (energy objective per bucket)"
    return None, "default tiles"


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU pool (GB/s), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "MEASURED_PEAKS.json (measured copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def fp32_peak(sm, mhz):
    """FP32 FMA peak (FLOP/s) from the unit counts and an SM clock."""
    return sm * FP32_LANES_PER_SM * 2 * mhz * 1e6


def clocks_summary(c):
    if not c:
        return None
    return {"sm_mhz": c["sm_mhz"], "sm_max_mhz": c["sm_max_mhz"], "reasons": c["reasons"],
            "power_w_median": c["power_w_median"], "samples_under_load": c["samples_under_load"]}


def timed_steps(world, stream, steps, launch, flush=None):
    """Per-step CUDA-event times (s) of `launch` on `stream`, with an optional
    L2 flush before each step outside the timed span."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    barrier(world)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        # ~1 ms of device sleep before the first step (outside every step's
        # events): the host enqueues ahead of the device, so no host-side
        # submission latency of the first launch falls inside its span
        torch.cuda._sleep(2_000_000)
        for s, e in ev:
            if flush is not None:
                flush.zero_()
            s.record(stream)
            launch()
            e.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    return [s.elapsed_time(e) / 1e3 for s, e in ev]


def batched_oracle_baseline(probs, seconds):
    """The FP64 oracle on the batch's images in order, until `seconds` pass."""
    import oracle
    from oracle import selection
    nt = oracle.max_threads()
    t0 = time.perf_counter()
    flop, done = 0.0, 0
    for p in probs:
        oracle.conv2d(p.inp, p.filt, in_w=p.in_w, nthreads=nt)
        flop += selection.conv2d_flop(p.fh, p.fw, p.out_h, p.out_w)
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return dict(value=flop / dt / 1e9, unit="GFLOP/s", cores=nt, kind="oracle",
                sample=f"{done} of {len(probs)} batch images in order (FP64 direct correlation, "
                       f"{flop / 1e9:.1f} GFLOP), {dt:.1f} s wall, {nt} OpenMP threads")


def measure_batched(args, world, local, steps, warmup, cpu_seconds):
    """The 256-image batch: one CUDA-graph launch (the batch's own mode, and
    the persistent class kernels' graph beside it) against one host-issued
    plain launch per image, timed by CUDA events and by the library's energy
    window, with an SM-clock record."""
    import torch

    from paper_2211_07260_gb300 import api, synth
    wl = WORKLOADS["batched256"]
    probs = synth.batch_problems(wl["n"], wl["seed"])
    ents = []
    for p in probs:
        d_in = torch.from_numpy(p.inp).cuda()
        out = torch.empty((p.out_h, (p.out_w + 3) // 4 * 4), dtype=torch.float32, device="cuda")
        ents.append((d_in, p.filt, out, p.out_h, p.out_w))
    tiles, src = load_tiles(api)
    opts = api.measure_options(window_s=args.energy_window)
    info = api.device_info()
    b_hbm, b_src = hbm_peak_gbs()
    stream = torch.cuda.Stream()
    sampler = ClockSampler(local)
    with api.Batch(ents, tiles) as b:
        st = b.info()
        for _ in range(max(3, warmup)):
            b.run(stream)
            b.run(stream, which="persistent")
        b.run_plain(stream)
        torch.cuda.synchronize()
        sampler.start()
        t_graph = all_max(world, sum(timed_steps(world, stream, steps, lambda: b.run(stream))))
        t_pers = all_max(world, sum(timed_steps(
            world, stream, steps, lambda: b.run(stream, which="persistent"))))
        t_plain = all_max(world, sum(timed_steps(world, stream, steps,
                                                 lambda: b.run_plain(stream))))
        rb = b.measure("default", opts)
        rq = b.measure("persistent", opts)
        rp = b.measure("plain", opts)
        clocks = sampler.stop()
    # mixed roofline: per image the slower of its FLOP at the FP32 peak and
    # its bytes at the HBM copy rate
    clk = clocks["sm_max_mhz"] if clocks else 2070.0
    fpk = fp32_peak(info["sm_count"], clk)
    t_roof = 0.0
    for p in probs:
        fl = 2.0 * p.fh * p.fw * p.out_h * p.out_w
        by = 4.0 * (p.in_h * p.in_w + p.out_h * p.out_w + p.fh * p.fw)
        t_roof += max(fl / fpk, by / (b_hbm * 1e9))
    g_graph = st["flop"] * steps / t_graph
    out = {
        "workload": "256 images, sides log-uniform [256, 2048], odd k 3..17, seed 2",
        "images": st["n_images"], "work_items": st["n_items"], "class_launches": st["launches"],
        "persistent_ctas": st["grid"], "tiles_source": src, "gflop": st["flop"] / 1e9,
        "l2": "inputs 0.78 GB > L2 (no flush needed)", "mode": st["mode_name"],
        "graph": {"mode": st["mode_name"], "gflops": g_graph / 1e9,
                  "ms_per_batch": t_graph * 1e3 / steps,
                  "gflops_energy_window": rb["gflops"], "gflop_per_j": rb["gflops_per_j"],
                  "power_w_mean": rb["power_w_mean"], "flags": rb["flags"],
                  "gpu_launches_per_batch": (st["n_images"] if st["mode_name"] == "launches"
                                             else st["launches"])},
        "persistent_graph": {"gflops": st["flop"] * steps / t_pers / 1e9,
                             "ms_per_batch": t_pers * 1e3 / steps,
                             "gflops_energy_window": rq["gflops"],
                             "gflop_per_j": rq["gflops_per_j"],
                             "power_w_mean": rq["power_w_mean"], "flags": rq["flags"],
                             "gpu_launches_per_batch": st["launches"]},
        "plain_per_image": {"gflops": st["flop"] * steps / t_plain / 1e9,
                            "ms_per_batch": t_plain * 1e3 / steps,
                            "gflops_energy_window": rp["gflops"],
                            "gflop_per_j": rp["gflops_per_j"],
                            "power_w_mean": rp["power_w_mean"], "flags": rp["flags"],
                            "idle_gaps": bool(rp["flags"] & api.REC_IDLE_GAPS),
                            "gpu_launches_per_batch": st["n_images"]},
        "roofline": {"bound": "alu (per image max of FP32 and HBM time)",
                     "achieved": g_graph / 1e12, "peak": st["flop"] / t_roof / 1e12,
                     "unit": "TFLOP/s", "frac": t_roof / (t_graph / steps),
                     "peak_basis": f"sum over images of max(FLOP / {fpk / 1e12:.1f} TFLOP/s, "
                                   f"bytes / {b_hbm:.0f} GB/s [{b_src}])"},
        "clocks": clocks_summary(clocks),
        "note": "idle_gaps: the plain leg's energy window saw the device idle between "
                "host-issued launches, so its GFLOP/J includes idle power",
    }
    if cpu_seconds > 0:
        out["cpu_baseline"] = batched_oracle_baseline(probs, cpu_seconds)
    del ents
    torch.cuda.empty_cache()
    return out


def measure_config1(args, world, local, steps, warmup):
    """1024 x 1024 / 7 x 7 at its energy-tuned configuration: back-to-back
    graph replay (the tuner's measurement, L2-resident) and single launches
    with L2 flushed between them."""
    import torch

    from paper_2211_07260_gb300 import api, synth
    wl = WORKLOADS["1024x1024_k7"]
    info = api.device_info()
    cfg, cfg_src = tuned_config(api, info["name"], wl, None)
    prob = synth.conv_problem(wl["h"], wl["w"], wl["k"], seed=wl["seed"])
    flop = 2.0 * wl["k"] ** 2 * wl["h"] * wl["w"]
    alg_bytes = 4.0 * (prob.in_h * prob.in_w + wl["h"] * wl["w"] + wl["k"] ** 2)
    stream = torch.cuda.Stream()
    d_in = torch.from_numpy(prob.inp).cuda()
    d_out = torch.empty((wl["h"], wl["w"]), dtype=torch.float32, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def launch():
        api.conv2d_run(d_in, prob.filt, d_out, wl["h"], wl["w"], cfg, stream=stream)

    for _ in range(max(3, warmup)):
        launch()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    t_flush = all_max(world, sum(timed_steps(world, stream, steps, launch, flush)))
    rec = api.measure_conv(d_in, prob.filt, d_out, wl["h"], wl["w"], cfg,
                           api.measure_options(window_s=args.energy_window), stream=stream)
    clocks = sampler.stop()
    b_hbm, b_src = hbm_peak_gbs()
    clk = clocks["sm_max_mhz"] if clocks else 2070.0
    fpk = fp32_peak(info["sm_count"], clk)
    roof = min(fpk, flop / alg_bytes * b_hbm * 1e9)
    del flush
    torch.cuda.empty_cache()
    return {
        "workload": "1024x1024 output, 7x7 filter, seed 0", "config": list(cfg.as_tuple()),
        "config_source": cfg_src,
        "graph_replay": {"gflops": rec["gflops"], "us_per_launch": rec["t_s"] * 1e6,
                         "gflop_per_j": rec["gflops_per_j"], "power_w_mean": rec["power_w_mean"],
                         "flags": rec["flags"], "l2": "resident (8.4 MB, back-to-back launches)",
                         "frac_of_roofline": rec["gflops"] * 1e9 / roof},
        "l2_flushed": {"gflops": steps * flop / t_flush / 1e9,
                       "us_per_launch": t_flush * 1e6 / steps,
                       "frac_of_roofline": steps * flop / t_flush / roof,
                       "l2": "flushed (256 MiB write) before each timed launch"},
        "roofline": {"bound": "min(FP32 peak, AI x HBM)", "peak": roof / 1e12, "unit": "TFLOP/s",
                     "ai_flop_per_byte": flop / alg_bytes,
                     "peak_basis": f"min({fpk / 1e12:.1f} TFLOP/s, {flop / alg_bytes:.2f} FLOP/B x "
                                   f"{b_hbm:.0f} GB/s [{b_src}])"},
        "clocks": clocks_summary(clocks),
    }


def measure_serving(local, rate, seconds, n_payloads):
    """A short Poisson serving run through the continuous-batching server,
    then the same arrivals served with one plain kernel per request."""
    from paper_2211_07260_gb300 import api, serve
    tiles, src = load_tiles(api)
    payloads = serve.make_payloads(n_payloads)
    p_idle = serve.idle_power(0.5)
    out = {"workload": f"Poisson arrivals at {rate:.0f} req/s for {seconds:.1f} s, shapes of the "
                       f"batched law (seed 3), {n_payloads} pinned host payloads reused",
           "tiles_source": src, "p_idle_w": p_idle}
    for mode in ("batched", "plain"):
        sampler = ClockSampler(local)
        sampler.start()
        r = serve.serve_rate(payloads, rate, seconds, 10 ** 7, plain=(mode == "plain"),
                             tiles=tiles, p_idle=p_idle)
        clocks = sampler.stop()
        out[mode] = {k: r[k] for k in ("requests", "req_per_s", "p50_ms", "p99_ms", "max_ms",
                                       "j_per_req", "j_per_req_above_idle", "gflop_per_j",
                                       "mean_batch", "gflops")}
        out[mode]["clocks"] = clocks_summary(clocks)
    return out


def measure_fp32_peak(local):
    """The FMA-dense microbenchmark: the empirical FP32 ceiling next to the
    peak derived from unit counts and the SM clock it ran at."""
    from paper_2211_07260_gb300 import api
    info = api.device_info()
    sampler = ClockSampler(local)
    sampler.start()
    r = api.measure_microbench(api.CT_UNIT_FMA, api.measure_options(window_s=0.5))
    clocks = sampler.stop()
    clk = r["clock_mhz_meas"] if r["clock_mhz_meas"] > 0 else (clocks or {}).get("sm_mhz", 2070.0)
    return {"tflops": r["gflops"] / 1e3, "sm_mhz": clk,
            "derived_peak_tflops_at_that_clock": fp32_peak(info["sm_count"], clk) / 1e12,
            "frac_of_derived": r["gflops"] * 1e9 / fp32_peak(info["sm_count"], clk),
            "clocks": clocks_summary(clocks)}


def run_batched(args, world, rank, local):
    """--workload batched256: the batched comparison as the headline line."""
    import torch
    torch.cuda.set_device(local)
    b = measure_batched(args, world, local, args.steps, args.warmup,
                        0 if (args.no_cpu or world > 1) else args.cpu_seconds)
    if rank != 0:
        return
    g = b["graph"]
    out = {
        "metric": METRIC, "value": world * g["gflops"], "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": g["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "l2": b["l2"], "parallelism": f"replicas x{world}"},
        "gflop_per_j": g["gflop_per_j"], "batched": b, "roofline": b["roofline"],
        "clocks": b["clocks"], "gpu_launches": args.steps * g["gpu_launches_per_batch"],
    }
    if "cpu_baseline" in b:
        out["cpu_baseline"] = b["cpu_baseline"]
    print(json.dumps(out))


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batched256":
        run_batched(args, world, rank, local)
        return
    import numpy as np
    import torch

    from paper_2211_07260_gb300 import api, synth

    torch.cuda.set_device(local)
    wl = WORKLOADS[args.workload]
    info = api.device_info()
    cfg, cfg_src = tuned_config(api, info["name"], wl, args.config)
    prob = synth.conv_problem(wl["h"], wl["w"], wl["k"], seed=wl["seed"])
    flop = 2.0 * wl["k"] * wl["k"] * wl["h"] * wl["w"]
    in_bytes = prob.inp.nbytes
    out_pitch = (wl["w"] + 3) // 4 * 4
    out_bytes = 4 * wl["h"] * out_pitch
    alg_bytes = 4.0 * (prob.in_h * prob.in_w + wl["h"] * wl["w"] + wl["k"] ** 2)

    stream = torch.cuda.Stream()
    d_in = torch.from_numpy(prob.inp).cuda()
    d_out = torch.empty((wl["h"], out_pitch), dtype=torch.float32, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def launch():
        api.conv2d_run(d_in, prob.filt, d_out, wl["h"], wl["w"], cfg, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            flush.zero_()
            launch()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        # device sleep before the first step (outside every step's events),
        # as in timed_steps: the host enqueues ahead of the device
        torch.cuda._sleep(2_000_000)
        for s, e in ev:
            flush.zero_()          # L2 flush, outside the timed span
            s.record(stream)
            launch()
            e.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    step_ms = [s.elapsed_time(e) for s, e in ev]
    kernel_s = all_max(world, sum(step_ms) / 1e3)
    srt = sorted(step_ms)
    step_stats = dict(min_us=srt[0] * 1e3, median_us=srt[len(srt) // 2] * 1e3,
                      max_us=srt[-1] * 1e3, first_us=step_ms[0] * 1e3)
    # the time-optimal configuration of the same sweep, timed the same way
    time_tuned = None
    te = None if args.config else tuned_entry(info["name"], wl)
    if te and te.get("time_config") and list(te["time_config"]) != list(cfg.as_tuple()):
        tcfg = api.Config(*te["time_config"])
        with torch.cuda.stream(stream):
            for _ in range(3):
                api.conv2d_run(d_in, prob.filt, d_out, wl["h"], wl["w"], tcfg, stream=stream)
            tev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            for s, e in tev:
                flush.zero_()
                s.record(stream)
                api.conv2d_run(d_in, prob.filt, d_out, wl["h"], wl["w"], tcfg, stream=stream)
                e.record(stream)
        torch.cuda.synchronize()
        t_s = sum(s.elapsed_time(e) for s, e in tev) / 1e3 / args.steps
        time_tuned = dict(config=list(tcfg.as_tuple()), gflops=flop / t_s / 1e9,
                          roofline_frac=None, ms_per_step=t_s * 1e3)
    # energy: mean power over >= window of back-to-back launches (NVML energy counter)
    nan = float("nan")
    rec = dict(gflops_per_j=nan, energy_j=nan, power_w_mean=nan, power_w_median=nan,
               energy_j_median_power=nan, gflops=nan, clock_mhz_meas=nan, flags=-1)
    if not args.no_energy:
        rec = api.measure_conv(d_in, prob.filt, d_out, wl["h"], wl["w"], cfg,
                               api.measure_options(window_s=args.energy_window), stream=stream)
    clocks = sampler.stop()
    status_bits = api.status_read(clear=True)

    # end to end through the host-buffer entry point (copies in the timed region)
    # (back-to-back asynchronous calls: each step's copies in,
    # kernels and copies out, with one step's copies in overlapping the
    # previous step's copies out; and, for comparison, the synchronous call)
    e2e_steps = 0 if args.no_e2e else args.e2e_steps
    e2e_s = e2e_sync_s = nan
    if e2e_steps:
        h_in = torch.from_numpy(prob.inp).pin_memory().numpy()
        h_out = torch.empty((wl["h"], out_pitch), dtype=torch.float32).pin_memory().numpy()
        api.conv2d_run_host(h_in, prob.filt, h_out, wl["h"], wl["w"], cfg, stream=stream)
        for _ in range(2):
            api.conv2d_run_host_async(h_in, prob.filt, h_out, wl["h"], wl["w"], cfg)
        api.host_wait()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            api.conv2d_run_host_async(h_in, prob.filt, h_out, wl["h"], wl["w"], cfg)
        api.host_wait()
        e2e_s = all_max(world, time.perf_counter() - t0)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            api.conv2d_run_host(h_in, prob.filt, h_out, wl["h"], wl["w"], cfg, stream=stream)
        e2e_sync_s = all_max(world, time.perf_counter() - t0)

    if rank != 0:
        return
    avg_launch_s = kernel_s / args.steps
    sm = info["sm_count"]
    peak_clock = clocks["sm_max_mhz"] if clocks else 2070.0
    peak = sm * FP32_LANES_PER_SM * 2 * peak_clock * 1e6  # FLOP/s
    achieved = flop / avg_launch_s
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        t = json.load(open(tpath)).get(args.workload)
        if t and tuple(t.get("config", ())) == cfg.as_tuple():
            traffic = t.get("dram_bytes_per_launch")
    out = {
        "metric": METRIC,
        "value": world * args.steps * flop / kernel_s / 1e9,
        "unit": "GFLOP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": kernel_s * 1e3 / args.steps,
        "step_us": step_stats,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "out": [wl["h"], wl["w"]],
                   "filter": [wl["k"], wl["k"]], "seed": wl["seed"],
                   "tuned_config": list(cfg.as_tuple()), "config_source": cfg_src,
                   "clocks": "default (clock locking is a device setting: not changed)",
                   "l2": "flushed (256 MiB write) between timed launches",
                   "parallelism": f"replicas x{world}"},
        "gflop_per_j": rec["gflops_per_j"],
        "energy": {"j_per_launch": rec["energy_j"], "power_w_mean": rec["power_w_mean"],
                   "power_w_median": rec["power_w_median"],
                   "j_per_launch_median_power": rec["energy_j_median_power"],
                   "window_s": args.energy_window, "gflops_in_window": rec["gflops"],
                   "sm_mhz_median": rec["clock_mhz_meas"], "flags": rec["flags"],
                   "source": "NVML total-energy counter, mean power between counter updates"},
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_basis": f"{sm} SMs x {FP32_LANES_PER_SM} FP32 FMA lanes x 2 FLOP x "
                                   f"{peak_clock:.0f} MHz (max SM clock)",
                     "frac_at_measured_clock": (achieved / (sm * FP32_LANES_PER_SM * 2 *
                                                            clocks["sm_mhz"] * 1e6)
                                                if clocks else None),
                     "hbm_gbs_achieved": alg_bytes / avg_launch_s / 1e9},
        "e2e": ({"value": world * e2e_steps * flop / e2e_s / 1e9, "unit": "GFLOP/s",
                 "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": out_bytes,
                 "steps": e2e_steps,
                 "api": "ct_conv2d_run_host_async (pinned host buffers, back-to-back calls, "
                        "ct_conv2d_host_wait after the last)",
                 "sync_value": world * e2e_steps * flop / e2e_sync_s / 1e9,
                 "sync_api": "ct_conv2d_run_host (returns with the result on the host)"}
                if e2e_steps else None),
        "clocks": ({"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                    "reasons": clocks["reasons"], "power_w_median": clocks["power_w_median"],
                    "samples_under_load": clocks["samples_under_load"]} if clocks else None),
        "time_tuned": (dict(time_tuned, roofline_frac=time_tuned["gflops"] * 1e9 / peak)
                       if time_tuned else None),
        "device_status_bits": status_bits,
        "timed_wall_s": wall,
        "steering": "unavailable: clock locking not permitted on this pool (tuning at default "
                    "clocks; the steered-vs-exhaustive comparison runs on the simulated "
                    "platform in the CPU tests)",
    }
    if not args.no_cpu and world == 1:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    if world == 1 and not args.no_extras and args.workload == "4096x4096_k17":
        # the other workloads at N = 1, each under its own SM-clock record
        del flush
        torch.cuda.empty_cache()
        fp = measure_fp32_peak(local)
        out["roofline"]["peak_empirical_fma_kernel"] = fp
        out["config1_1024x1024_k7"] = measure_config1(args, world, local, max(args.steps, 50),
                                                      args.warmup)
        out["batched256"] = measure_batched(args, world, local, max(3, min(args.steps, 10)),
                                            args.warmup, 0 if args.no_cpu else 5.0)
        if args.serve_seconds > 0:
            out["serving"] = measure_serving(local, args.serve_rate, args.serve_seconds,
                                             args.serve_payloads)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
