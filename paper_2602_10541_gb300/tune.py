"""Autotuner of the launch shapes: times each candidate on the GPU and records the
fastest in tuning.json next to this module (read by pipeline.tuned()).

Tuned today: the persistent evaluation of the batched inverse problem
(fastlsq_inverse_eval), threads per CTA in {256, 512} x CTAs per SM in {1, 2} x CTAs
per cluster (one instance each) in {1, 2, 4}, on the batched configuration's 256
instances (uneven points and features).
``python -m paper_2602_10541_gb300.tune [--instances N] [--reps R]``.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics

import torch

from . import fastlsq as fl
from . import pipeline as pl
from . import workloads as wl

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
CANDIDATES = [{"threads": t, "ctas_per_sm": c, "cluster": k} for t in (256, 512) for c in (1, 2)
              for k in (1, 2, 4)]


def tune_inverse(n_inst=256, reps=5, device="cuda:0"):
    ctx = fl.Context(0)
    batch = pl.InverseBatch(ctx, [wl.inverse_instance(q) for q in range(n_inst)], device=device)
    batch.observe()
    results = []
    for cand in CANDIDATES:
        batch.launch = dict(cand)
        try:
            batch.eval()                              # attributes, first touch
        except fl.FastLSQError:
            continue                                   # shared memory does not fit this shape
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ctx.stream)
            batch.eval()
            b.record(ctx.stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        results.append((statistics.median(ts), cand))
    batch.close()
    ctx.close()
    best_ms, best = min(results, key=lambda r: r[0])
    return {**best, "ms": best_ms, "instances": n_inst,
            "candidates": [{**c, "ms": ms} for ms, c in results],
            "gpu": torch.cuda.get_device_name(0)}


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2602_10541_gb300.tune")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args(argv)
    table = json.load(open(TABLE)) if os.path.exists(TABLE) else {}
    table["inverse_eval"] = tune_inverse(a.instances, a.reps)
    with open(TABLE, "w") as fh:
        json.dump(table, fh, indent=1)
    print(json.dumps(table["inverse_eval"]))


if __name__ == "__main__":
    main()
