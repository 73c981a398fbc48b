"""Posterior-predictive simulation, reported as draws/s.

    python -m paper_2103_03348_b300.run_predictive [--samples 4096] [--horizon 30] [--reps 5]

Workload: the 23,422-event synthetic history with 1,610 free log-rates; the
parameter settings are the generating values plus N(0, 0.02^2) in sampler
coordinates (standing in for posterior draws); each setting simulates the
next `horizon` days exactly (one block per setting).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import build, predictive, synth


def run(samples=4096, horizon=30.0, reps=5, capacity=8192, seed=1000, device="cuda"):
    build.build()
    w = synth.make("ebola_like")
    rng = np.random.default_rng(77)
    q0 = np.concatenate([np.log(w.params), w.r[w.sequenced]])
    q = torch.tensor(q0[None, :] + 0.02 * rng.standard_normal((samples, q0.size)), dtype=torch.float64,
                     device=device)
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device=device)  # noqa: E731
    x, y, t, r = d(w.x), d(w.y), d(w.t), d(w.r)
    seq = torch.tensor(w.sequenced, dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream(device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    times, out = [], None
    for i in range(reps + 1):
        ev[0].record(stream)
        out = predictive.simulate(x, y, t, r, seq, q, horizon, seed + i, capacity)
        ev[1].record(stream)
        ev[1].synchronize()
        if i > 0:
            times.append(ev[0].elapsed_time(ev[1]))
    ms = float(np.mean(times))
    counts = out["count"].cpu().numpy()
    status = out["status"].cpu().numpy()
    return {"workload": f"{w.name}: {w.n} past events, {len(w.sequenced)} free log-rates, {horizon:g} days ahead",
            "samples": samples, "ms_per_batch": ms, "samples_per_s": samples / (ms * 1e-3),
            "events_per_s": float(counts.sum()) / (ms * 1e-3), "mean_events_per_sample": float(counts.mean()),
            "past_event_terms_per_s": 2.0 * w.n * samples / (ms * 1e-3),
            "overflowed_samples": int((status == 1).sum()), "capacity": capacity,
            "rng": "Philox4x32-10, counter = (item, draw, stage, sample)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=4096)
    ap.add_argument("--horizon", type=float, default=30.0)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    print(json.dumps(run(a.samples, a.horizon, a.reps)), flush=True)


if __name__ == "__main__":
    main()
