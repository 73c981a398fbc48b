"""Writes the golden fixtures in this folder from the oracle alone.

    python tests/golden/make_golden.py            # the small JSON fixtures
    python tests/golden/make_golden.py --large    # large_N100000.npz (minutes, all host cores)

Each small fixture stores its inputs literally (so it does not depend on a
random generator's version) and the oracle's FP64 outputs, with the passage of
the paper that defines them.  The large fixture is the full FP64 evaluation of
the 100,000-event benchmark workload; it stores a SHA-256 digest of that
workload's inputs instead of the 3.2 MB of inputs, so a reader regenerates them
with the seeded generator and checks the digest.  Run it again, and commit the diff with the passage
that justifies it, only when the oracle's arithmetic changes.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import hmc_oracle, tree_oracle  # noqa: E402

LIKELIHOOD_SOURCE = ("Section 2.1: intensity lambda_n (background Gaussian kernel over other locations plus "
                     "rate-weighted exponential-decay excitation by strictly earlier events), log-likelihood Eq. 1 "
                     "with the integral term of Appendix A; gradient in (mu0, tau_x, tau_t, theta0, omega, h, "
                     "r_1..r_N) (Eq. 4 times theta_m for the log-rates) and Hessian diagonal (Eq. 5, in r)")


def lst(a):
    return [float(v) for v in np.asarray(a, float).ravel()]


def write(name, obj):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(obj, f, indent=1)
        f.write("\n")


def hand_events():
    """Seven events chosen by hand: a simultaneous pair, a repeated location,
    a far outlier and unequal rates; parameters in the ebola-like units."""
    x = np.array([0.0, 3.0, 3.0, -2.0, 1.5, 40.0, 2.5])
    y = np.array([0.0, 1.0, 1.0, 4.0, -1.0, 35.0, 0.5])
    t = np.array([0.5, 2.0, 2.0, 3.5, 6.0, 6.5, 9.0])
    r = np.array([0.3, -0.4, 0.0, 1.1, -0.7, 0.2, 0.5])
    params = np.array([0.5, 20.0, 30.0, 0.5, 0.1, 5.0])
    return x, y, t, r, params


def uniform_events(n=96, seed=2103):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 50.0, n)
    y = rng.uniform(0, 50.0, n)
    t = np.sort(rng.uniform(0, 30.0, n))
    r = rng.normal(0.0, 0.5, n)
    params = np.array([0.8, 6.0, 4.0, 0.6, 0.5, 3.0])
    return x, y, t, r, params


def likelihood_fixture(name, x, y, t, r, params, note):
    o = oracle.evaluate(x, y, t, r, params, want=2)
    write(name, {"source": LIKELIHOOD_SOURCE, "note": note,
                 "inputs": {"x": lst(x), "y": lst(y), "t": lst(t), "r": lst(r), "params": lst(params)},
                 "expected": {"loglik": float(o["loglik"]), "Lambda": float(o["Lambda"]), "lam": lst(o["lam"]),
                              "grad": lst(o["grad"]), "hdiag": lst(o["hdiag"])}})


def tree9():
    """A nine-tip rooted binary tree written by hand (internal nodes 9..16, root 16)."""
    parent = np.array([9, 9, 10, 11, 11, 12, 13, 13, 15, 10, 14, 12, 14, 15, 16, 16, -1])
    length = np.array([0.3, 0.5, 1.2, 0.2, 0.25, 0.9, 0.1, 0.15, 2.0, 0.4, 0.3, 0.6, 0.2, 0.7, 0.5, 0.35, 0.0])
    return parent, length


def tree_fixture():
    parent, length = tree9()
    z = np.array([0.4, 0.1, -0.8, 1.3, 1.1, -0.2, 0.6, 0.7, -1.5])
    tau0, s2 = 0.25, 1.8
    ld, pz, pd = tree_oracle.tree_prior(z, parent, length, tau0, s2)  # long double dense algebra
    write("tree_prior_m9.json", {
        "source": "Section 2.2, Eq. 2: z ~ N(0, sigma^2 V), V_ij = root variance + shared root-path length",
        "inputs": {"parent": [int(v) for v in parent], "length": lst(length), "z": lst(z), "root_var": tau0,
                   "sigma2": s2},
        "expected": {"logdens": float(ld), "pz": lst(pz), "pdiag": lst(pd),
                     "V": [lst(row) for row in tree_oracle.tree_cov(parent, length, tau0)]}})


def posterior_fixture():
    x, y, t, r, params = uniform_events(n=48, seed=7)
    parent, length = tree9()
    seq = np.array([1, 4, 9, 13, 20, 26, 31, 40, 45])
    prec = tree_oracle.precision_matrix(parent, length)
    # the Section 3.2 priors in km and days (kinds 0 = gamma(shape, rate), 1 = inverse gamma(shape, scale))
    kind = [0, 1, 1, 0, 0, 1]
    a = [2.0, 1.0, 2.0, 1.0, 2.0, 2.0]
    b = [2.0, 1112.0, 182.625, 0.001, 182.625, 55.6]
    q = np.concatenate([np.log(params), r[seq] + 0.1])
    lp, g, h = hmc_oracle.log_posterior(x, y, t, r, seq, prec, (np.array(kind), np.array(a), np.array(b)), q)
    write("posterior_n48_m9.json", {
        "source": "Section 2.3, Eq. 3: log posterior in sampler coordinates q = (log globals, sequenced log-rates): "
                  "likelihood (Section 2.1) + gamma / inverse-gamma priors on the globals (Section 3.2) + "
                  "log-transform Jacobian + the phylogenetic Brownian prior (Eq. 2, sigma^2 = 1, root variance 0)",
        "inputs": {"x": lst(x), "y": lst(y), "t": lst(t), "r": lst(r), "seq": [int(v) for v in seq],
                   "tree_parent": [int(v) for v in parent], "tree_length": lst(length),
                   "prior_kind": kind, "prior_a": a, "prior_b": b, "q": lst(q)},
        "expected": {"logpost": float(lp), "grad": lst(g), "hdiag": lst(h)}})


def input_digest(w) -> str:
    import hashlib
    h = hashlib.sha256()
    for a in (w.x, w.y, w.t, w.r, np.asarray(w.params, float)):
        h.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    return h.hexdigest()


def large_fixture():
    """Full FP64 oracle evaluation (loglik, gradient[6+N], Hessian diagonal[6+N],
    and the intensities lambda[N]) of the 100,000-event workload that the
    benchmark times."""
    import time
    from paper_2103_03348_b300 import synth
    w = synth.make("large")
    t0 = time.perf_counter()
    o = oracle.evaluate(w.x, w.y, w.t, w.r, w.params, want=2)
    dt = time.perf_counter() - t0
    np.savez_compressed(os.path.join(HERE, "large_N100000.npz"), loglik=np.float64(o["loglik"]),
                        Lambda=np.float64(o["Lambda"]), grad=o["grad"], hdiag=o["hdiag"], lam=o["lam"],
                        input_sha256=np.array(input_digest(w)), source=np.array(LIKELIHOOD_SOURCE),
                        workload=np.array(w.name), params=np.asarray(w.params, float))
    print(f"large_N100000.npz: loglik {o['loglik']:.12e}, {dt:.0f} s on {oracle.max_threads()} threads")


def main():
    if "--large" in sys.argv:
        large_fixture()
        return
    likelihood_fixture("loglik_hand_n7.json", *hand_events(),
                       note="events 1 and 2 are simultaneous at one location: no excitation and no background "
                            "between them; event 5 is far from the rest")
    likelihood_fixture("loglik_uniform_n96.json", *uniform_events(),
                       note="96 events uniform on [0,50]^2 km x [0,30] d, r ~ N(0, 0.5^2)")
    tree_fixture()
    posterior_fixture()


if __name__ == "__main__":
    main()
