"""Pins of the oracle's sampled entry points and of the surrogate's
de-standardisation.

oracle.rows (lambda_n and the per-row derivative sums of a listed subset of
rows) and oracle.rate_terms (the log-rate gradient and Hessian entries of Eqs.
4-5 for listed sources, given lambda) are the checkers of the GPU path at the
sizes where the full oracle is too slow.  They have their own loops, their own
t_N and their own integral-term share d Lambda / d r_m, so they are pinned
here on their own:

- on a 200-event pattern with simultaneous events and repeated locations, for
  tau_t finite and infinite, every row and every source reproduce the full
  evaluation's lambda, global sums and log-rate entries bit for bit (the
  same per-pair arithmetic in the same order; the full evaluation is pinned by
  quadrature, finite differences and the identities of test_oracle_pins.py);
- independently of that code, the sampled outputs satisfy the exact identity
  sum_m dl/dr_m = theta0 dl/dtheta0 (Eqs. 4-5 against the row sums);
- slips planted in copies of their C source (a dropped rate in the integral
  share, the wrong end of the window, a missing -sum w^2, the background
  self-exclusion lost) each fail one of these pins.

mlp_oracle.surrogate_gradient (mean_g + A (q - mean_q) + sd_g MLP((q -
mean_q) / sd_q)) is pinned by a case worked by hand and by two exact
reparametrisations of the network that must leave it unchanged; planted slips
in a copy of the module fail them.
"""
import inspect
import math
import types

import numpy as np
import pytest

import oracle
from oracle import mlp_oracle
from paper_2103_03348_b300 import synth

P_MU0, P_TAUX, P_TAUT, P_THETA0, P_OMEGA, P_H = range(6)


def tied_pattern(tau_t, n=200, seed=17):
    """n uniform events with runs of simultaneous events and repeated locations."""
    w = synth.make_uniform(seed, n, box=1.0, t_max=2.0, r_sd=0.6, params=(0.7, 0.15, tau_t, 0.6, 3.0, 0.08))
    t, x, y = w.t.copy(), w.x.copy(), w.y.copy()
    for k in range(5, n - 3, 23):          # three events at one time
        t[k + 1] = t[k + 2] = t[k]
    for k in range(11, n - 1, 31):          # a later event at an earlier event's place
        x[k + 1], y[k + 1] = x[k], y[k]
    return x, y, t, w.r.copy(), np.array(w.params, float)


def sampled(x, y, t, r, p, lib=None):
    idx = np.arange(len(t))
    lam, d1, d2 = oracle.rows(x, y, t, r, p, idx, lib=lib)
    full = oracle.evaluate(x, y, t, r, p, want=2)
    g, h = oracle.rate_terms(x, y, t, r, p, full["lam"], idx, lib=lib)
    return lam, d1, d2, g, h, full


def row_global_sums(lam, d1, d2, k):
    """sum_n d1/lam and sum_n (d2/lam - (d1/lam)^2), sequentially in n."""
    g = hh = 0.0
    for n in range(len(lam)):
        q1 = d1[n, k] / lam[n]
        g += q1
        hh += d2[n, k] / lam[n] - q1 * q1
    return g, hh


def integral_share(t, r, p):
    """d Lambda / d p_k for the six globals, from the Appendix A Claim (numpy)."""
    mu0, tt, th0, om = p[P_MU0], p[P_TAUT], p[P_THETA0], p[P_OMEGA]
    a = t.max() - t
    th, dec = np.exp(r), np.exp(-om * a)
    from scipy import stats
    d = np.zeros(6)
    d[P_MU0] = (stats.norm.cdf(a / tt) - stats.norm.cdf(-t / tt)).sum() if math.isfinite(tt) else len(t) * t.max()
    d[P_THETA0] = (th * (1 - dec)).sum()
    d[P_OMEGA] = (th0 * th * a * dec).sum()
    if math.isfinite(tt):
        d[P_TAUT] = mu0 * (-(a / tt ** 2) * stats.norm.pdf(a / tt) - (t / tt ** 2) * stats.norm.pdf(-t / tt)).sum()
    return d


def agree_with_full(x, y, t, r, p, lib=None):
    """The sampled entry points reproduce the full evaluation (lambda and rate
    entries bit for bit; the global sums exactly where the integral term has no
    share, to 1e-12 through the integral share where it has)."""
    lam, d1, d2, g, h, full = sampled(x, y, t, r, p, lib)
    if not np.array_equal(lam, full["lam"]):
        return False
    if not (np.array_equal(g, full["grad"][6:]) and np.array_equal(h, full["hdiag"][6:])):
        return False
    share = integral_share(t, r, p)
    for k in range(6):
        if k == P_TAUT and not math.isfinite(p[P_TAUT]):
            continue
        gs, hs = row_global_sums(lam, d1, d2, k)
        if k in (P_TAUX, P_H):                       # Lambda does not depend on tau_x, h
            if gs != full["grad"][k] or hs != full["hdiag"][k]:
                return False
        elif abs(gs - share[k] - full["grad"][k]) > 1e-12 * (abs(gs) + abs(share[k])):
            return False
        if k in (P_MU0, P_THETA0) and hs != full["hdiag"][k]:   # Lambda is linear in mu0, theta0
            return False
    return True


def rate_identity(x, y, t, r, p, lib=None):
    """sum_m dl/dr_m = theta0 dl/dtheta0, from rate_terms and rows alone: the
    excitation depends on theta0 and the rates only through theta0 theta_m."""
    idx = np.arange(len(t))
    lam, d1, _ = oracle.rows(x, y, t, r, p, idx, lib=lib)
    g, _ = oracle.rate_terms(x, y, t, r, p, lam, idx, lib=lib)
    a = t.max() - t
    g_theta0 = np.sum(d1[:, P_THETA0] / lam) - np.sum(np.exp(r) * (1 - np.exp(-p[P_OMEGA] * a)))
    return abs(g.sum() - p[P_THETA0] * g_theta0) <= 1e-11 * (np.abs(g).sum() + 1.0)


@pytest.mark.parametrize("tau_t", [0.2, math.inf])
def test_rows_and_rate_terms_reproduce_full_evaluation(tau_t):
    x, y, t, r, p = tied_pattern(tau_t)
    assert len(np.unique(t)) < len(t) and len({(a, b) for a, b in zip(x, y)}) < len(t)
    assert agree_with_full(x, y, t, r, p)


@pytest.mark.parametrize("tau_t", [0.2, math.inf])
def test_rate_terms_satisfy_the_rate_theta0_identity(tau_t):
    x, y, t, r, p = tied_pattern(tau_t)
    assert rate_identity(x, y, t, r, p)


def test_sampled_subsets_equal_the_full_lists():
    """Any subset of rows or sources gives the entries of the full lists (the
    checker samples scattered rows and sources, early ones included)."""
    x, y, t, r, p = tied_pattern(0.2)
    idx = np.array([0, 3, 7, 50, 51, 52, 120, 199])
    lam_all, d1_all, d2_all, g_all, h_all, full = sampled(x, y, t, r, p)
    lam, d1, d2 = oracle.rows(x, y, t, r, p, idx)
    g, h = oracle.rate_terms(x, y, t, r, p, full["lam"], idx)
    assert np.array_equal(lam, lam_all[idx]) and np.array_equal(d1, d1_all[idx]) and np.array_equal(d2, d2_all[idx])
    assert np.array_equal(g, g_all[idx]) and np.array_equal(h, h_all[idx])


C_MUTATIONS = {
    "integral share without the rate": ("dl = params[P_THETA0] * exp(r[m]) * (1.0",
                                        "dl = params[P_THETA0] * (1.0"),
    "integral share over [0, t_m]": ("(1.0 - exp(-params[P_OMEGA] * (tN - t[m])));",
                                     "(1.0 - exp(-params[P_OMEGA] * (t[m])));"),
    "rate Hessian without -sum w^2": ("h[q] = s1 - s2 - dl;", "h[q] = s1 - dl;"),
    "rate gradient without the integral share": ("g[q] = s1 - dl;", "g[q] = s1;"),
    "rows keep the self background": (
        "s += source_term(x[i], y[i], t[i], x[j], y[j], t[j], r[j], params, 1, NULL, p1, p2);",
        "s += source_term(x[i], y[i], t[i], x[j], y[j], t[j], r[j], params, 0, NULL, p1, p2);"),
}


@pytest.mark.parametrize("name", sorted(C_MUTATIONS))
def test_planted_slips_in_sampled_entry_points_are_caught(name, tmp_path):
    old, new = C_MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, name
    lib = oracle.load_variant(src.replace(old, new), str(tmp_path))
    x, y, t, r, p = tied_pattern(0.2, n=60)
    assert not (agree_with_full(x, y, t, r, p, lib=lib) and rate_identity(x, y, t, r, p, lib=lib)), name


# ---------------------------------------------------------------------------
# mlp_oracle.surrogate_gradient
# ---------------------------------------------------------------------------
def only_output_bias(b3):
    w = np.zeros(mlp_oracle.PARAM_COUNT)
    w[-6:] = b3
    return w


def hand_case(mod):
    """W = 0 but b3, so the network's output is b3 whatever q:
    g = mean_g + A (q - mean_q) + sd_g * b3, worked out by hand below."""
    b3 = np.array([1.0, -2.0, 0.5, 0.0, 3.0, -1.0])
    mean_q = np.array([0.5, 0.0, -1.0, 2.0, 0.0, 1.0])
    sd_q = np.array([2.0, 1.0, 0.5, 4.0, 1.0, 3.0])
    mean_g = np.array([10.0, 20.0, 30.0, 40.0, 50.0, 60.0])
    sd_g = np.array([2.0, 0.5, 4.0, 1.0, 10.0, 3.0])
    A = np.zeros((6, 6))
    A[0, 1], A[1, 0], A[2, 2], A[5, 3] = 3.0, -1.0, 2.0, 0.25
    q = np.array([1.5, 2.0, -2.0, 6.0, 0.0, 1.0])       # q - mean_q = (1, 2, -1, 4, 0, 0)
    norm = np.concatenate([mean_q, sd_q, mean_g, sd_g, A.ravel()])
    # rows: 10 + 3*2 + 2*1 = 18;  20 - 1*1 - 2*0.5 = 18;  30 + 2*(-1) + 4*0.5 = 30;
    #       40 + 0 + 1*0 = 40;    50 + 0 + 10*3 = 80;     60 + 0.25*4 - 3*1 = 58
    expect = np.array([18.0, 18.0, 30.0, 40.0, 80.0, 58.0])
    return np.array_equal(mod.surrogate_gradient(only_output_bias(b3), q, norm), expect)


def random_net(seed):
    rng = np.random.default_rng(seed)
    w = rng.normal(0, 0.3, mlp_oracle.PARAM_COUNT)
    norm = np.concatenate([rng.normal(size=6), rng.uniform(0.5, 3, 6), rng.normal(size=6) * 5,
                           rng.uniform(0.5, 4, 6), rng.normal(size=36)])
    return w, norm, rng.normal(size=6)


def input_standardisation_folded(mod):
    """Folding the input standardisation into layer 1 (W1' = W1 / sd_q by
    column, b1' = b1 - W1' mean_q) with mean_q = 0, sd_q = 1 and the linear
    part's offset moved into mean_g leaves the surrogate gradient unchanged."""
    w, norm, q = random_net(3)
    mq, sq, mg, A = norm[0:6], norm[6:12], norm[12:18], norm[24:60].reshape(6, 6)
    u = mlp_oracle.unpack(w)
    W1 = u["W1"] / sq[None, :]
    b1 = u["b1"] - W1 @ mq
    w2 = w.copy()
    w2[:768], w2[768:896] = W1.ravel(), b1
    norm2 = np.concatenate([np.zeros(6), np.ones(6), mg - A @ mq, norm[18:24], A.ravel()])
    a, b = mod.surrogate_gradient(w, q, norm), mod.surrogate_gradient(w2, q, norm2)
    return np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())


def output_scale_folded(mod):
    """Doubling sd_g and halving the last layer (W3, b3) leaves it unchanged."""
    w, norm, q = random_net(4)
    w2, norm2 = w.copy(), norm.copy()
    w2[17408:] *= 0.5
    norm2[18:24] *= 2.0
    a, b = mod.surrogate_gradient(w, q, norm), mod.surrogate_gradient(w2, q, norm2)
    return np.allclose(a, b, rtol=1e-13, atol=1e-13 * np.abs(a).max())


def test_surrogate_gradient_hand_case():
    assert hand_case(mlp_oracle)


def test_surrogate_gradient_reparametrisations():
    assert input_standardisation_folded(mlp_oracle)
    assert output_scale_folded(mlp_oracle)


PY_MUTATIONS = {
    "sd_g dropped": ("+ norm[18:24] * y[0]", "+ y[0]"),
    "input scaled by sd_q": ("(dq / norm[6:12])", "(dq * norm[6:12])"),
    "linear part transposed": ("norm[24:60].reshape(MI, MI) @ dq", "norm[24:60].reshape(MI, MI).T @ dq"),
    "linear part about 0": ("norm[24:60].reshape(MI, MI) @ dq", "norm[24:60].reshape(MI, MI) @ np.asarray(q)[:MI]"),
    "mean_g dropped": ("return norm[12:18] + ", "return 0.0 + "),
}


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_planted_slips_in_surrogate_gradient_are_caught(name):
    old, new = PY_MUTATIONS[name]
    src = inspect.getsource(mlp_oracle)
    assert src.count(old) == 1, name
    mod = types.ModuleType("mlp_oracle_mutant")
    mod.__file__ = mlp_oracle.__file__
    exec(compile(src.replace(old, new), mlp_oracle.__file__, "exec"), mod.__dict__)
    assert not (hand_case(mod) and input_standardisation_folded(mod) and output_scale_folded(mod)), name
