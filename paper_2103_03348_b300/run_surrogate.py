"""Surrogate-trajectory HMC over the six globals, reported against exact HMC.

    python -m paper_2103_03348_b300.run_surrogate [--n 500000] [--pairs 20000] [--iters 2000]
                                                 [--exact-iters 500] [--steps 20] [--precision fp32c_st]

Workload: the surrogate pattern (uniform background plus 500 hotspots,
offspring weight 0.6, [0,2000]^2 km x [0,1500] d; log-rates fixed at 0), the
six globals on the log scale.  Exact HMC warm-up (step size by dual averaging,
a dense mass over the six globals from central differences of the gradient, or
with --mass diag the Hessian diagonal) records `--pairs` (q, gradient) pairs; the MLP
is trained on them by the library's kernels; then `--iters` surrogate
iterations (exact accept) and `--exact-iters` exact iterations run from the
same state with the same mass and step size.  Prints one JSON line: the
acceptance rates, the surrogate's gradient error as the exact kernel measures
it along the chain, ESS and ESS/s (min / median / max over the six globals) of
both chains, the gains, and the cost of the warm-up and the training.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import build, hmc, surrogate, synth


def run(n=500_000, pairs=20_000, iters=2000, exact_iters=500, n_steps=20, seed=0, device="cuda", eps0=0.02,
        precision="fp32c_st", mass="dense", jitter=0.2):
    build.build()
    w = synth.make_surrogate(n=n)
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device=device)  # noqa: E731
    post = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), torch.zeros(0, dtype=torch.int32, device=device),
                         torch.zeros(0, dtype=torch.float64, device=device), hmc.prior_km_days(), precision)
    q0 = d(np.log(w.params))
    t0 = time.perf_counter()
    qp, gp, warm = surrogate.collect_pairs(post, q0, n_pairs=pairs, n_steps=n_steps, eps0=eps0, seed=seed, mass=mass,
                                           jitter=jitter)
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - t0
    sur, fit_rep = surrogate.fit(qp, gp, seed=seed)
    ch_s = surrogate.sample(post, sur, warm.last_q, warm.mass_t, warm.eps, iters, n_steps=n_steps, seed=seed + 1,
                            jitter=jitter)
    ess_s = hmc.ess_all(ch_s.draws)
    post.calls = {"grad": 0, "hess": 0}
    ch_e = hmc.sample(post, warm.last_q, n_iter=exact_iters, n_warmup=0, n_steps=n_steps, eps0=warm.eps,
                      seed=seed + 2, mass_every=10 ** 9, mass0=warm.mass_t, mass=mass, jitter=jitter)
    ess_e = hmc.ess_all(ch_e.draws)

    def summ(e):
        return {"min": float(np.min(e)), "median": float(np.median(e)), "max": float(np.max(e))}

    return {
        "workload": w.name, "n_events": w.n, "precision": precision, "mass": mass, "step_jitter": jitter, "pairs_pair_interactions": w.n * (w.n - 1), "leapfrog_steps": n_steps,
        "warmup": {"pairs": int(qp.shape[0]), "seconds": t_warm, "step_size": warm.eps,
                   "ms_per_exact_gradient": 1e3 * t_warm / max(warm.grad_calls + warm.hess_calls, 1)},
        "training": fit_rep,
        "surrogate_hmc": {"iters": iters, "accept_rate": float(ch_s.accept.mean()), "seconds": ch_s.seconds,
                          "exact_loglik_calls": ch_s.exact_loglik_calls, "fell_back": ch_s.fell_back,
                          "monitor_rel_errors": ch_s.monitor_errors,
                          "monitor_rel_error_max": float(max(ch_s.monitor_errors)) if ch_s.monitor_errors else None,
                          "ms_per_iteration": 1e3 * ch_s.seconds / max(iters, 1), "ess": summ(ess_s),
                          "ess_per_s": {k: v / ch_s.seconds for k, v in summ(ess_s).items()}},
        "ess_each_global": {"surrogate": dict(zip(NAMES, map(float, ess_s))),
                            "exact": dict(zip(NAMES, map(float, ess_e)))},
        "exact_hmc": {"iters": exact_iters, "accept_rate": float(ch_e.accept.mean()), "seconds": ch_e.seconds,
                      "ms_per_iteration": 1e3 * ch_e.seconds / max(exact_iters, 1),
                      "exact_gradient_calls": ch_e.grad_calls, "ess": summ(ess_e),
                      "ess_per_s": {k: v / ch_e.seconds for k, v in summ(ess_e).items()}},
        "gain_ess_per_s_min": (float(np.min(ess_s)) / ch_s.seconds) / max(float(np.min(ess_e)) / ch_e.seconds, 1e-300),
        "gain_ess_per_exact_pass_min": (float(np.min(ess_s)) / ch_s.exact_loglik_calls)
                                        / max(float(np.min(ess_e)) / max(ch_e.grad_calls + ch_e.hess_calls, 1), 1e-300),
        "posterior_mean_globals": np.exp(ch_s.draws.mean(0)).tolist(),
        "posterior_mean_globals_exact": np.exp(ch_e.draws.mean(0)).tolist(),
        "means_within_mcse": means_agree(ch_s.draws, ess_s, ch_e.draws, ess_e),
        "generating_globals": [float(v) for v in w.params],
    }


NAMES = ("mu0", "tau_x", "tau_t", "theta0", "omega", "h")


def means_agree(a, ea, b, eb, k=4.5):
    """Largest gap between the two chains' means of the log-globals, in units of
    their combined Monte Carlo standard error (equal accuracy: below k)."""
    mcse = np.sqrt(a.var(0) / np.maximum(ea, 1.0) + b.var(0) / np.maximum(eb, 1.0))
    gap = np.abs(a.mean(0) - b.mean(0)) / np.maximum(mcse, 1e-300)
    return {"max_gap_in_mcse": float(gap.max()), "ok": bool(gap.max() <= k)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=500_000)
    ap.add_argument("--pairs", type=int, default=20_000)
    ap.add_argument("--iters", type=int, default=2000)
    ap.add_argument("--exact-iters", type=int, default=500)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precision", default="fp32c_st", choices=["fp32c", "fp32c_band", "fp32c_st", "fp64"])
    ap.add_argument("--mass", default="dense", choices=["dense", "diag"],
                    help="dense mass over the six globals (default) or the diagonal mass of Section 2.3.2")
    ap.add_argument("--jitter", type=float, default=0.2, help="step-size jitter (0 for a fixed step)")
    a = ap.parse_args()
    print(json.dumps(run(a.n, a.pairs, a.iters, a.exact_iters, a.steps, a.seed, precision=a.precision, mass=a.mass,
                         jitter=a.jitter)), flush=True)


if __name__ == "__main__":
    main()
