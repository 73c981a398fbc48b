"""Cost of one evaluation against N, reported as pair-interactions/s.

    python -m paper_2103_03348_b300.run_scaling [--sizes 10000,25000,...] [--reps 10]

Workload: the hotspot pattern of the 100,000-event benchmark (2,000 x 2,000 km,
1,500 days, 556 hotspots, log-rates N(0, 0.25)) drawn at each size, so the
density grows with N.  For each size: loglik, loglik + gradient, and loglik +
gradient + Hessian diagonal in FP32C, the last also with exact band skipping, on
space-time tiles
and, up to 50,000 events, in FP64.  CUDA events around each call, L2 flushed
between calls, median of `reps`.  One JSON line per size.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import build, hawkes, synth


def time_call(fn, reps, flush, stream):
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = []
    for i in range(reps + 2):
        flush.zero_()
        ev[0].record(stream)
        fn()
        ev[1].record(stream)
        ev[1].synchronize()
        if i >= 2:
            out.append(ev[0].elapsed_time(ev[1]))
    return float(np.median(out))


def run(sizes=(10_000, 25_000, 50_000, 100_000, 250_000, 500_000, 1_000_000), reps=10, device="cuda"):
    build.build()
    dev = torch.device(device)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)  # 256 MB, larger than the L2
    rows = []
    for n in sizes:
        w = synth.make_large(n=n)
        d = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
        x, y, t, r = d(w.x), d(w.y), d(w.t), d(w.r)
        pairs = n * (n - 1)
        res = {"n": n, "pairs": pairs}
        cases = [("loglik", "fp32c"), ("grad", "fp32c"), ("hess", "fp32c"), ("hess", "fp32c_band"), ("hess", "fp32c_st")]
        if n <= 50_000:
            cases.append(("hess", "fp64"))
        for mode, prec in cases:
            ws = hawkes._workspace(n, hawkes.PRECISIONS[prec], dev)
            out = None

            def fn(mode=mode, prec=prec, ws=ws):
                hawkes._call(mode, x, y, t, r, w.params, prec, stream=stream.cuda_stream, workspace=ws, check=False,
                             out=out)

            ms = time_call(fn, reps if prec != "fp64" else 2, flush, stream)
            res[f"{mode}_{prec}_ms"] = ms
            res[f"{mode}_{prec}_pairs_per_s"] = pairs / (ms * 1e-3)
        rows.append(res)
        print(json.dumps(res), flush=True)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="10000,25000,50000,100000,250000,500000,1000000")
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args()
    run(tuple(int(s) for s in a.sizes.split(",")), a.reps)


if __name__ == "__main__":
    main()
