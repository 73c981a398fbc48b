"""Preconditioned HMC over the phylogenetic Hawkes posterior, reported as ESS/s.

    python -m paper_2103_03348_b300.run_hmc [--precision fp32c_st|fp32c_band|fp32c|fp64] [--iters 2000]
                                            [--warmup 200]
                                            [--prior tree|dense] [--mass diag|tree]
                                            [--checkpoint PATH [--every K]] [--resume PATH]

Workload: the 23,422-event synthetic pattern with 1,610 sequenced events whose
log-rates are free (the phylogenetic prior on the generator's coalescent tree,
sigma^2 = 1, root variance 0, applied in O(M) on the tree, or through its dense
precision matrix with --prior dense), the six globals on the log scale, 20 leapfrog steps per iteration,
mass matrix refreshed every 100 iterations from the Hessian diagonal (Section
2.3.2), start at the generating values.  With --mass tree the rate block's
mass is instead diag(d) + (sigma^2 V)^-1, d the likelihood's curvature from the
same Hessian diagonal: the phylogenetic prior's correlations are then
preconditioned exactly (tree prior only); --mass tree_joint adds a dense
block for the six globals and its coupling to the rates, from central
differences of the gradient along the globals.  Prints one JSON line with the
acceptance rate, sampling time, and min/median/max ESS and ESS/s for the six
globals and for the 1,610 log-rates.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import build, hmc, synth, tree


def run(precision="fp32c_st", iters=2000, warmup=200, n_steps=20, mass_every=100, eps0=0.05, seed=0, n=23422,
        m_seq=1610, device="cuda", prior="tree", checkpoint=None, checkpoint_every=0, resume=None, mass="diag"):
    build.build()
    w = synth.make_ebola_like(n=n, m_seq=m_seq)
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device=device)  # noqa: E731
    seq = torch.tensor(w.sequenced, device=device)
    if prior == "tree":
        tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0, device=device)
        post = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), seq, None, hmc.prior_km_days(), precision, tree=tp)
    else:
        prec = np.linalg.inv(w.tree_cov)
        post = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), seq, d(prec), hmc.prior_km_days(), precision)
    q0 = d(np.concatenate([np.log(w.params), w.r[w.sequenced]]))
    # untimed: a 4-iteration chain, so that one-off costs of a fresh process
    # (first use of each kernel, graph set-up) stay out of the timed chain
    if resume is None:
        hmc.sample(post, q0, n_iter=2, n_warmup=2, n_steps=n_steps, eps0=eps0, mass_every=mass_every, seed=seed + 1,
                   mass=mass)
        post.calls.update({k: 0 for k in post.calls})  # count the timed chain's evaluations only
    t0 = time.perf_counter()
    ch = hmc.sample(post, q0, n_iter=iters, n_warmup=warmup, n_steps=n_steps, eps0=eps0, mass_every=mass_every,
                    seed=seed, checkpoint=checkpoint, checkpoint_every=checkpoint_every, resume=resume, mass=mass)
    total = time.perf_counter() - t0
    ess = hmc.ess_all(ch.draws)
    eg, er = ess[:6], ess[6:]

    def summ(e):
        return {"min": float(np.min(e)), "median": float(np.median(e)), "max": float(np.max(e))}

    calls = ch.grad_calls + ch.hess_calls
    return {
        "workload": w.name, "n_events": w.n, "n_rates": int(len(w.sequenced)), "precision": precision,
        "phylogenetic_prior": prior, "mass": mass,
        "iters": iters, "warmup": warmup, "leapfrog_steps": n_steps, "mass_every": mass_every,
        "step_size": ch.eps, "accept_rate": float(ch.accept.mean()),
        "sampling_seconds": ch.seconds, "warmup_seconds": ch.warmup_seconds, "total_seconds": total,
        "ms_per_gradient": 1e3 * total / max(calls, 1), "gradient_calls": ch.grad_calls, "hessian_calls": ch.hess_calls,
        "ess_globals": summ(eg), "ess_rates": summ(er),
        "ess_each_global": dict(zip(("mu0", "tau_x", "tau_t", "theta0", "omega", "h"), map(float, eg))),
        "ess_per_s_globals": {k: v / ch.seconds for k, v in summ(eg).items()},
        "ess_per_s_rates": {k: v / ch.seconds for k, v in summ(er).items()},
        "posterior_mean_globals": np.exp(ch.draws[:, :6].mean(0)).tolist(),
        "generating_globals": [float(v) for v in w.params],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="fp32c_st", choices=["fp32c_st", "fp32c_band", "fp32c", "fp64"])
    ap.add_argument("--iters", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--prior", default="tree", choices=["tree", "dense"])
    ap.add_argument("--mass", default="diag", choices=["diag", "tree", "tree_joint"],
                    help="diagonal mass (Section 2.3.2), the tree-structured one on the rates, or that one with "
                         "the globals' dense block coupled to the rates")
    ap.add_argument("--checkpoint", default=None, help="write the sampler state here every --every iterations")
    ap.add_argument("--every", type=int, default=200)
    ap.add_argument("--resume", default=None, help="continue the chain from this checkpoint")
    a = ap.parse_args()
    print(json.dumps(run(a.precision, a.iters, a.warmup, a.steps, seed=a.seed, prior=a.prior, checkpoint=a.checkpoint,
                         checkpoint_every=a.every if a.checkpoint else 0, resume=a.resume, mass=a.mass)), flush=True)


if __name__ == "__main__":
    main()
