"""FP64 NumPy oracle of the HMC pieces (Section 2.3): the log posterior in
sampler coordinates, one leapfrog trajectory, the Metropolis accept step that
closes it, and the effective sample size.

TEST INFRASTRUCTURE: used only by the tests and the bench's CPU legs.

Sampler coordinates q = (log mu0, log tau_x, log tau_t, log theta0, log omega,
log h, r_{s_1..s_M}).  log pi(q) = l(p, r) + sum_k [log prior_k(p_k) + q_k]
- 1/2 r_S^T P r_S with p = exp(q[:6]), priors Gamma(shape a, rate b) or
inverse-Gamma(shape a, scale b) on each p_k (kind 0 / 1), and P the precision
of the phylogenetic Brownian prior (Eq. 2).  The likelihood and its
derivatives come from the C oracle.
"""
from __future__ import annotations

import numpy as np

from . import evaluate

GAMMA, INVGAMMA = 0, 1


def log_prior_terms(p, kind, a, b):
    """log density (up to constants), first and second derivative, per parameter."""
    p, a, b = np.asarray(p, float), np.asarray(a, float), np.asarray(b, float)
    kind = np.asarray(kind)
    lp = np.where(kind == GAMMA, (a - 1) * np.log(p) - b * p, -(a + 1) * np.log(p) - b / p)
    d1 = np.where(kind == GAMMA, (a - 1) / p - b, -(a + 1) / p + b / p ** 2)
    d2 = np.where(kind == GAMMA, -(a - 1) / p ** 2, (a + 1) / p ** 2 - 2 * b / p ** 3)
    return lp, d1, d2


def log_posterior(x, y, t, r_base, seq, prec, prior, q, want_hess=True, trend=None, beta_var=1.0):
    """(log pi, grad_q, hdiag_q or None) at q, with the likelihood from the oracle.

    Without a trend q = (log p[6], z[M]) and the sequenced log-rates are r = z.
    With trend = F ([M, K], the fixed trend features f(t) of the sequenced
    events, Section 2.2) q = (log p[6], z[M], beta[K]), r_seq = z + F beta and
    beta ~ N(0, beta_var I).  The beta entries of hdiag_q are the
    preconditioner sum_j F_jk^2 d2l/dr_j^2 - 1/beta_var: the cross terms
    d2l/dr_i dr_j (i != j) of the exact second derivative are not formed."""
    q = np.asarray(q, float)
    p = np.exp(q[:6])
    r = np.array(r_base, float)
    seq = np.asarray(seq, np.int64)
    m = len(seq)
    zs = q[6:6 + m]
    beta = q[6 + m:]
    F = np.zeros((m, 0)) if trend is None else np.asarray(trend, float).reshape(m, -1)
    r[seq] = zs + F @ beta
    o = evaluate(x, y, t, r, p, want=2 if want_hess else 1)
    lp, d1, d2 = log_prior_terms(p, *prior)
    Pz = prec @ zs if m else np.zeros(0)
    logpost = o["loglik"] + np.sum(lp + q[:6]) - 0.5 * float(zs @ Pz) - 0.5 * float(beta @ beta) / beta_var
    gr = o["grad"][6 + seq]
    g = np.empty(q.size)
    g[:6] = p * (o["grad"][:6] + d1) + 1.0
    g[6:6 + m] = gr - Pz
    g[6 + m:] = F.T @ gr - beta / beta_var
    h = None
    if want_hess:
        hr = o["hdiag"][6 + seq]
        h = np.empty(q.size)
        h[:6] = p * (o["grad"][:6] + d1) + p ** 2 * (o["hdiag"][:6] + d2)
        h[6:6 + m] = hr - np.diag(prec)
        h[6 + m:] = (F ** 2).T @ hr - 1.0 / beta_var
    return logpost, g, h


def velocity(p, minv):
    """M^-1 p for a diagonal inverse mass (a vector) or a dense one (a matrix)."""
    minv = np.asarray(minv, float)
    return minv @ p if minv.ndim == 2 else minv * p


def kinetic(p, minv):
    """The kinetic energy 1/2 p^T M^-1 p (diagonal or dense inverse mass)."""
    p = np.asarray(p, float)
    return 0.5 * float(p @ velocity(p, minv))


def leapfrog(q, p, eps, n_steps, minv, grad_fn):
    """Leapfrog integration of Hamilton's equations, H = -log pi(q) + 1/2 p^T M^-1 p,
    with a diagonal inverse mass (minv a vector) or a dense one (minv a matrix).

    grad_fn(q) -> (log pi, grad).  Returns (q, p, log pi, grad) at the end.
    """
    q = np.array(q, float)
    p = np.array(p, float)
    lp, g = grad_fn(q)
    p = p + 0.5 * eps * g
    for step in range(n_steps):
        q = q + eps * velocity(p, minv)
        lp, g = grad_fn(q)
        p = p + (eps if step < n_steps - 1 else 0.5 * eps) * g
    return q, p, lp, g


def accept_probability(lp0, k0, lp1, k1, ok=True):
    """Metropolis acceptance of an HMC proposal (Section 2.3: the trajectory's end
    point is a proposal corrected by an accept/reject step).  With the energy
    H = -log pi(q) + K(p), the proposal is accepted with probability
    min(1, exp(H0 - H1)).  A proposal whose log posterior or energy is not finite,
    or whose likelihood evaluation reported an error (ok false), has probability 0."""
    h0 = -float(lp0) + float(k0)
    h1 = -float(lp1) + float(k1)
    if not ok or not np.isfinite(lp1) or not np.isfinite(h1):
        return 0.0
    return min(1.0, float(np.exp(min(0.0, h0 - h1))))


def metropolis_step(q0, lp0, g0, k0, q1, lp1, g1, k1, u, ok=True):
    """One accept/reject decision with the uniform draw u in [0, 1): the proposal
    (q1, lp1, g1) replaces the current state iff u < a.  Returns
    (q, lp, g, accepted, a)."""
    a = accept_probability(lp0, k0, lp1, k1, ok)
    if u < a:
        return np.array(q1, float), float(lp1), np.array(g1, float), True, a
    return np.array(q0, float), float(lp0), np.array(g0, float), False, a


def ess_geyer(x):
    """Effective sample size by Geyer's initial monotone sequence estimator.

    tau = -1 + 2 sum_m Gamma_m with Gamma_m = rho_{2m} + rho_{2m+1}, summed while
    positive and made non-increasing; ESS = n / tau with tau floored at
    1/log10(n) (an antithetic chain's ESS is capped at n log10(n)).  Autocovariances by direct
    sums (O(n^2)), which is fine for the chain lengths used in tests.
    """
    x = np.asarray(x, float)
    n = len(x)
    if n < 4 or np.var(x) == 0:
        return float(n)
    xc = x - x.mean()
    acov = np.array([np.dot(xc[: n - k], xc[k:]) / n for k in range(n)])
    rho = acov / acov[0]
    gam = []
    for m in range(n // 2):
        gm = rho[2 * m] + rho[2 * m + 1]
        if gm <= 0:
            break
        if gam and gm > gam[-1]:
            gm = gam[-1]
        gam.append(gm)
    tau = -1.0 + 2.0 * sum(gam)
    return float(n / max(tau, 1.0 / np.log10(n)))
