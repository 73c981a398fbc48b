"""Surrogate-trajectory HMC over the six globals, reported against exact HMC.

    python -m paper_2103_03348_b300.run_surrogate [--n 500000] [--pairs 20000] [--iters 500]
                                                 [--exact-iters 50] [--steps 20]

Workload: the surrogate pattern (uniform background plus 500 hotspots,
offspring weight 0.6, [0,2000]^2 km x [0,1500] d; log-rates fixed at 0), the
six globals on the log scale.  Exact HMC warm-up (step size by dual averaging,
mass from the Hessian diagonal) records `--pairs` (q, gradient) pairs; the MLP
is trained on them by the library's kernels; then `--iters` surrogate
iterations (exact accept) and `--exact-iters` exact iterations run from the
same state with the same mass and step size.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import build, hmc, surrogate, synth


def run(n=500_000, pairs=20_000, iters=500, exact_iters=50, n_steps=20, seed=0, device="cuda", eps0=0.02,
        precision="fp32c_band"):
    build.build()
    w = synth.make_surrogate(n=n)
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device=device)  # noqa: E731
    post = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), torch.zeros(0, dtype=torch.int32, device=device),
                         torch.zeros(0, dtype=torch.float64, device=device), hmc.prior_km_days(), precision)
    q0 = d(np.log(w.params))
    t0 = time.perf_counter()
    qp, gp, warm = surrogate.collect_pairs(post, q0, n_pairs=pairs, n_steps=n_steps, eps0=eps0, seed=seed)
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - t0
    sur, fit_rep = surrogate.fit(qp, gp, seed=seed)
    ch_s = surrogate.sample(post, sur, warm.last_q, warm.mass_t, warm.eps, iters, n_steps=n_steps, seed=seed + 1)
    ess_s = hmc.ess_all(ch_s.draws)
    post.calls = {"grad": 0, "hess": 0}
    ch_e = hmc.sample(post, warm.last_q, n_iter=exact_iters, n_warmup=0, n_steps=n_steps, eps0=warm.eps,
                      seed=seed + 2, mass_every=10 ** 9)
    ess_e = hmc.ess_all(ch_e.draws)

    def summ(e):
        return {"min": float(np.min(e)), "median": float(np.median(e)), "max": float(np.max(e))}

    return {
        "workload": w.name, "n_events": w.n, "precision": precision, "pairs_pair_interactions": w.n * (w.n - 1), "leapfrog_steps": n_steps,
        "warmup": {"pairs": int(qp.shape[0]), "seconds": t_warm, "step_size": warm.eps},
        "training": fit_rep,
        "surrogate_hmc": {"iters": iters, "accept_rate": float(ch_s.accept.mean()), "seconds": ch_s.seconds,
                          "exact_loglik_calls": ch_s.exact_loglik_calls, "fell_back": ch_s.fell_back,
                          "monitor_rel_errors": ch_s.monitor_errors, "ess": summ(ess_s),
                          "ess_per_s": {k: v / ch_s.seconds for k, v in summ(ess_s).items()}},
        "exact_hmc": {"iters": exact_iters, "accept_rate": float(ch_e.accept.mean()), "seconds": ch_e.seconds,
                      "exact_gradient_calls": ch_e.grad_calls, "ess": summ(ess_e),
                      "ess_per_s": {k: v / ch_e.seconds for k, v in summ(ess_e).items()}},
        "gain_ess_per_s_min": (float(np.min(ess_s)) / ch_s.seconds) / max(float(np.min(ess_e)) / ch_e.seconds, 1e-300),
        "gain_ess_per_exact_pass_min": (float(np.min(ess_s)) / ch_s.exact_loglik_calls)
                                        / max(float(np.min(ess_e)) / max(ch_e.grad_calls + ch_e.hess_calls, 1), 1e-300),
        "posterior_mean_globals": np.exp(ch_s.draws.mean(0)).tolist(),
        "generating_globals": [float(v) for v in w.params],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=500_000)
    ap.add_argument("--pairs", type=int, default=20_000)
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--exact-iters", type=int, default=50)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precision", default="fp32c_band", choices=["fp32c", "fp32c_band", "fp32c_st", "fp64"])
    a = ap.parse_args()
    print(json.dumps(run(a.n, a.pairs, a.iters, a.exact_iters, a.steps, a.seed, precision=a.precision)), flush=True)


if __name__ == "__main__":
    main()
