"""Analyses of a tuning-record file (JSON lines written by ``tune --records``):
the Pareto front of speed vs energy efficiency, the proportion of PageRank
centrality of good minima for the time and the energy objective, and -- when
the records span several clocks -- the five tuning methods.

  python -m paper_2211_07260_gb300.analyze records.jsonl [--base-clock 1400]
"""
from __future__ import annotations

import argparse
import json
import math

from . import api


def load(path):
    recs = []
    for line in open(path):
        r = json.loads(line)
        for k, v in list(r.items()):
            if v is None:
                r[k] = math.nan
        r["cfg"] = tuple(r["cfg"])
        recs.append(r)
    return recs


def summarise(recs, base_clock=None):
    valid = [r for r in recs if not r["flags"] & api.REC_INVALID and r["t_s"] > 0
             and not math.isnan(r["energy_j"])]
    out = dict(points=len(recs), with_energy=len(valid))
    front = api.pareto_front(valid)
    out["pareto_front"] = [dict(cfg=valid[i]["cfg"], clock=valid[i]["clock_mhz_req"],
                                gflops=valid[i]["gflops"], gflop_per_j=valid[i]["gflops_per_j"])
                           for i in front]
    if len(front) >= 2:
        fast, eff = valid[front[0]], valid[front[-1]]
        out["front_trade_off"] = dict(
            speed_change=eff["gflops"] / fast["gflops"] - 1.0,
            efficiency_change=eff["gflops_per_j"] / fast["gflops_per_j"] - 1.0)
    ps = (1.0, 1.02, 1.05, 1.1, 1.25, 1.5)
    out["centrality_time"] = api.centrality(valid, "time", ps)
    out["centrality_energy"] = api.centrality(valid, "energy", ps)
    clocks = {r["clock_mhz_req"] for r in valid}
    if len(clocks) > 1:
        m = api.tuning_methods(valid, base_clock if base_clock else max(clocks))
        out["methods"] = {k: dict(cfg=valid[i]["cfg"], clock=valid[i]["clock_mhz_req"],
                                  energy_j=valid[i]["energy_j"], t_s=valid[i]["t_s"])
                          for k, i in m.items()}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("records")
    ap.add_argument("--base-clock", type=int, default=None)
    a = ap.parse_args()
    print(json.dumps(summarise(load(a.records), a.base_clock), indent=1))


if __name__ == "__main__":
    main()
