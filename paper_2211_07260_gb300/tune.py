"""Command-line tuner: run the library's exhaustive search on a seeded
workload at default clocks and record the chosen configuration.

  python -m paper_2211_07260_gb300.tune --workload 1024x1024_k7 --space basic \\
      --objective energy --window 0.3 --out tuned_configs.json

--prefilter N first times every point (time objective, no energy window),
then measures energy only for the N fastest points; without it every point
gets an energy window.  Results are cached (JSON lines) so a sweep resumes.

--confirm C --repeats R (default 8 and 4; --confirm 0 turns it off)
re-measures the C best points of the objective R more times, the C points
one after the other in each round (so that slow drifts of power or
temperature reach all of them alike), and keeps the point with the best
median: near-ties among the top points (GB300, 4096^2 / 17 x 17: the three
most energy-efficient within 0.14 %, below one window's spread) are then
decided on several windows instead of one.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

from . import api, synth

WORKLOADS = {
    "1024x1024_k7": (1024, 1024, 7, 0),
    "4096x4096_k17": (4096, 4096, 17, 1),
}
HERE = os.path.dirname(os.path.abspath(__file__))


# objective -> (record field, True when larger is better)
_METRIC = {"time": ("t_s", False), "energy": ("energy_j", False),
           "gflops_per_w": ("gflops_per_j", True)}


def confirm_best(measure, recs, objective, confirm, repeats):
    """Re-measure the `confirm` best records of the objective `repeats` more
    times (all of them once per round, via measure(configs) -> records) and
    return (record of the point with the best median, summary).  The
    returned record carries the medians of t_s, energy_j, gflops and
    gflops_per_j over its 1 + repeats measurements."""
    import statistics
    key, larger = _METRIC[objective]
    valid = [r for r in recs if not r["flags"] & api.REC_INVALID and r.get(key) is not None
             and not (isinstance(r[key], float) and math.isnan(r[key]))]
    valid.sort(key=lambda r: r[key], reverse=larger)
    top = valid[:confirm]
    samples = {tuple(r["cfg"]): [r] for r in top}
    for _ in range(repeats):
        for r in measure([api.Config(*t) for t in samples]):
            if not r["flags"] & api.REC_INVALID:
                samples[tuple(r["cfg"])].append(r)
    med = {}
    for cfg, rs in samples.items():
        med[cfg] = {f: statistics.median(x[f] for x in rs)
                    for f in ("t_s", "energy_j", "gflops", "gflops_per_j", "power_w_mean")}
    pick = (max if larger else min)(med, key=lambda c: med[c][key])
    best = dict(samples[pick][0])
    best.update(med[pick])
    summary = dict(confirm=confirm, repeats=repeats,
                   single_window_pick=list(top[0]["cfg"]), pick=list(pick),
                   medians={",".join(map(str, c)): {f: v for f, v in m.items()}
                            for c, m in med.items()})
    return best, summary


def run(workload, space="basic", objective="energy", window=0.3, prefilter=0, cache=None,
        out=None, log=print, confirm=0, repeats=0):
    import torch
    h, w, k, seed = WORKLOADS[workload]
    prob = synth.conv_problem(h, w, k, seed=seed)
    d_in = torch.from_numpy(prob.inp).cuda()
    d_out = torch.empty((h, (w + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    cfgs = api.space(api.CT_SPACE_FULL if space == "full" else api.CT_SPACE_BASIC)
    t0 = time.time()
    summary = dict(workload=workload, space=space, n_space=len(cfgs), objective=objective,
                   window_s=window, prefilter=prefilter)
    if prefilter:
        recs, best = api.tune(d_in, prob.filt, d_out, h, w, cfgs, None,
                              api.tune_options("time", window_s=window, warmup_s=0.02,
                                               time_only=True, cache_path=cache))
        valid = [r for r in recs if not r["flags"] & api.REC_INVALID]
        summary["n_valid"] = len(valid)
        summary["time_pass_wall_s"] = time.time() - t0
        valid.sort(key=lambda r: r["t_s"])
        cfgs = [api.Config(*r["cfg"]) for r in valid[:prefilter]]
        summary["time_best"] = dict(cfg=valid[0]["cfg"], t_s=valid[0]["t_s"],
                                    gflops=valid[0]["gflops"])
    recs, best = api.tune(d_in, prob.filt, d_out, h, w, cfgs, None,
                          api.tune_options(objective, window_s=window, warmup_s=0.1,
                                           cache_path=cache))
    valid = [r for r in recs if not r["flags"] & api.REC_INVALID]
    summary.setdefault("n_valid", len(valid))
    b = recs[best]
    if confirm > 1 and repeats > 0:
        def measure(cs):
            rr, _ = api.tune(d_in, prob.filt, d_out, h, w, cs, None,
                             api.tune_options(objective, window_s=window, warmup_s=0.1))
            return rr
        b, summary["confirmation"] = confirm_best(measure, recs, objective, confirm, repeats)
    summary["wall_s"] = time.time() - t0
    summary["best"] = dict(cfg=b["cfg"], t_s=b["t_s"], energy_j=b["energy_j"],
                           gflops=b["gflops"], gflops_per_j=b["gflops_per_j"],
                           power_w_mean=b["power_w_mean"], sm_mhz=b["clock_mhz_meas"],
                           flags=b["flags"])
    tb = api.select_best(recs, "time")
    eb = api.select_best(recs, "energy")
    summary["best_time"] = dict(cfg=recs[tb]["cfg"], t_s=recs[tb]["t_s"],
                                energy_j=recs[tb]["energy_j"])
    summary["best_energy"] = dict(cfg=recs[eb]["cfg"], t_s=recs[eb]["t_s"],
                                  energy_j=recs[eb]["energy_j"])
    summary["same_choice_time_vs_energy"] = recs[tb]["cfg"] == recs[eb]["cfg"]
    log(json.dumps(summary))
    if out:
        table = json.load(open(out)) if os.path.exists(out) else {"devices": {}}
        name = api.device_info()["name"]
        table.setdefault("devices", {}).setdefault(name, {})[workload] = dict(
            config=list(b["cfg"]), objective=objective, space=space, window_s=window,
            prefilter=prefilter, confirm=confirm, repeats=repeats,
            gflops=b["gflops"], gflops_per_j=b["gflops_per_j"],
            clocks="default", time_config=list(summary["time_best"]["cfg"])
            if "time_best" in summary else list(recs[tb]["cfg"]),
            time_gflops=summary["time_best"]["gflops"] if "time_best" in summary
            else recs[tb]["gflops"])
        with open(out, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
            f.write("\n")
    return summary, recs


def tune_batched(objective="energy", window=0.3, out=None, n=256, seed=2, log=print,
                 modes=("persistent", "launches")):
    """Per-bucket tiles of the batched workload into the tuned-configuration
    table: the persistent kernels' tiles (ct_batch_tune) and the launches
    graph's single-image configurations (ct_batch_tune_launches)."""
    import torch
    probs = synth.batch_problems(n, seed)
    ents = []
    for p in probs:
        d_in = torch.from_numpy(p.inp).cuda()
        o = torch.empty((p.out_h, (p.out_w + 3) // 4 * 4), dtype=torch.float32, device="cuda")
        ents.append((d_in, p.filt, o, p.out_h, p.out_w))
    t0 = time.time()
    # start from the device's current table (if any)
    start = None
    if out and os.path.exists(out):
        raw = json.load(open(out)).get("batched_tiles", {}).get(api.device_info()["name"])
        start = api.tiles_from_json(raw) if raw else None
    mo = api.measure_options(window_s=window, warmup_s=0.1)
    tiles, recs = start or {}, []
    if "persistent" in modes:
        tiles, r = api.batch_tune(ents, objective, mo, start=tiles or None)
        recs += r
    if "launches" in modes:
        tiles, r = api.batch_tune_launches(ents, objective, mo, start=tiles or None)
        recs += r
    log(json.dumps(dict(batched_tiles=api.tiles_to_json(tiles), points=len(recs),
                        wall_s=time.time() - t0)))
    if out:
        table = json.load(open(out)) if os.path.exists(out) else {"devices": {}}
        name = api.device_info()["name"]
        table.setdefault("batched_tiles", {})[name] = api.tiles_to_json(tiles)
        with open(out, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
            f.write("\n")
    return tiles, recs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="1024x1024_k7",
                    choices=sorted(WORKLOADS) + ["batched256"])
    ap.add_argument("--space", default="basic", choices=["basic", "full"])
    ap.add_argument("--objective", default="energy", choices=sorted(api.OBJECTIVES))
    ap.add_argument("--window", type=float, default=0.3)
    ap.add_argument("--prefilter", type=int, default=0)
    ap.add_argument("--cache", default=None)
    ap.add_argument("--out", default=os.path.join(HERE, "tuned_configs.json"))
    ap.add_argument("--records", default=None, help="write every record (JSON lines)")
    ap.add_argument("--confirm", type=int, default=8,
                    help="re-measure this many of the best points (with --repeats; 0: off)")
    ap.add_argument("--repeats", type=int, default=4)
    ap.add_argument("--batch-modes", default="persistent,launches",
                    help="batched256: which tables to tune (persistent, launches)")
    a = ap.parse_args()
    if a.workload == "batched256":
        tune_batched(a.objective, a.window, a.out, modes=tuple(a.batch_modes.split(",")))
        return
    summary, recs = run(a.workload, a.space, a.objective, a.window, a.prefilter, a.cache, a.out,
                        confirm=a.confirm, repeats=a.repeats)
    if a.records:
        with open(a.records, "w") as f:
            for r in recs:
                f.write(json.dumps({k: (None if isinstance(v, float) and math.isnan(v) else v)
                                    for k, v in r.items()}) + "\n")


if __name__ == "__main__":
    main()
