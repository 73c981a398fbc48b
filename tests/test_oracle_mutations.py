"""The oracle's pins have teeth: plausible mistakes planted in copies of the
oracle's C source (on the CPU) are each caught by at least one fast pin.

Each mutation below is a one-line slip a careful implementer could make; the
pins re-run here in compact form (a hand-computed N=2 case, the theta0 -> 0
background-only likelihood from scipy, finite differences of the gradient and
Hessian diagonal, simultaneous events not exciting each other, and the
homogeneity identity).
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2103_03348_b300 import synth

MUTATIONS = {
    "background normalisation": ("/ (TWO_PI * tx * tx);", "/ (TWO_PI * tx);"),
    "sign of d/domega": ("d1[P_OMEGA] += e * (1.0 / om - dt);", "d1[P_OMEGA] += e * (1.0 / om + dt);"),
    "non-strict excitation": ("if (ts < tq) {", "if (ts <= tq) {"),
    "rate missing from Lambda": ("ex += th * (1.0 - decay);", "ex += (1.0 - decay);"),
    "Hessian coefficient in h": ("d2[P_H] += e * (c * c - 3.0", "d2[P_H] += e * (c * c - 2.0"),
    "rate Hessian without -sum w^2": ("hdiag[NPAR + i] = c1[i] - c2[i] - dLr[i];", "hdiag[NPAR + i] = c1[i] - dLr[i];"),
    "integral lower limit": ("bg += std_normal_cdf(za) - std_normal_cdf(zb);", "bg += std_normal_cdf(za);"),
}


def check_two_events(lib):
    p = np.array([0.9, 0.4, 0.3, 0.5, 3.0, 0.25])
    x, y, t, r = np.array([0.1, 0.3]), np.array([0.2, -0.1]), np.array([0.2, 0.5]), np.array([0.4, -0.2])
    mu0, tx, tt, th0, om, h = p
    nx = stats.norm.pdf
    bg = mu0 * nx(x[1], x[0], tx) * nx(y[1], y[0], tx) * nx(t[1], t[0], tt)
    lam2 = bg + th0 * math.exp(r[0]) * om * math.exp(-om * 0.3) * nx(x[1], x[0], h) * nx(y[1], y[0], h)
    Lam = mu0 * sum(stats.norm.cdf(t[1], tk, tt) - stats.norm.cdf(0.0, tk, tt) for tk in t)
    Lam += th0 * sum(math.exp(rk) * (1 - math.exp(-om * (t[1] - tk))) for tk, rk in zip(t, r))
    ll = math.log(bg) + math.log(lam2) - Lam
    return abs(oracle.evaluate(x, y, t, r, p, want=0, lib=lib)["loglik"] - ll) <= 1e-12 * abs(ll)


def check_finite_differences(lib):
    w = synth.make_uniform(7, 12, box=1.0, t_max=2.0, r_sd=0.5, params=(0.7, 0.3, 0.25, 0.6, 2.0, 0.2))
    p0 = np.array(w.params)
    base = oracle.evaluate(w.x, w.y, w.t, w.r, p0, want=2, lib=lib)

    def ev(p, r):
        return oracle.evaluate(w.x, w.y, w.t, r, p, want=1, lib=lib)

    for k in range(6 + w.n):
        def at(v, k=k):
            p, r = p0.copy(), w.r.copy()
            if k < 6:
                p[k] = v
            else:
                r[k - 6] = v
            return ev(p, r)
        v0 = p0[k] if k < 6 else w.r[k - 6]
        hh = 1e-4 * (abs(v0) if k < 6 else 1.0)
        a, b = at(v0 + hh), at(v0 - hh)
        g_fd = (a["loglik"] - b["loglik"]) / (2 * hh)
        h_fd = (a["grad"][k] - b["grad"][k]) / (2 * hh)
        if abs(base["grad"][k] - g_fd) > 1e-5 * max(1.0, abs(g_fd)):
            return False
        if abs(base["hdiag"][k] - h_fd) > 1e-4 * max(1.0, abs(h_fd)):
            return False
    return True


def check_simultaneous(lib):
    p = np.array([0.7, 0.3, 0.25, 0.6, 2.0, 0.2])
    x = np.array([0.1, 0.4, 0.2]); y = np.array([0.1, 0.3, 0.2]); t = np.array([0.5, 0.5, 0.9])
    a = oracle.evaluate(x, y, t, np.zeros(3), p, want=0, lib=lib)["lam"]
    q = p.copy(); q[3] = 1e-300
    b = oracle.evaluate(x, y, t, np.zeros(3), q, want=0, lib=lib)["lam"]
    return np.allclose(a[:2], b[:2], rtol=1e-14)


def check_homogeneity(lib):
    w = synth.make_uniform(21, 80, r_sd=0.7, params=(0.5, 0.1, 0.05, 0.3, 10.0, 0.02))
    o = oracle.evaluate(w.x, w.y, w.t, w.r, w.params, want=1, lib=lib)
    g = o["grad"]
    ok1 = abs(w.params[0] * g[0] + w.params[3] * g[3] - (w.n - o["Lambda"])) <= 1e-9 * w.n
    ok2 = abs(np.sum(g[6:]) - w.params[3] * g[3]) <= 1e-9 * max(1.0, abs(g[3]))
    return ok1 and ok2


def check_theta0_zero(lib):
    w = synth.make_uniform(3, 15, box=1.0, t_max=2.0, r_sd=0.5, params=(0.7, 0.3, 0.25, 0.0, 2.0, 0.2))
    mu0, tx, tt = w.params[:3]
    ll = 0.0
    for n in range(w.n):
        s = sum(stats.norm.pdf(w.x[n], w.x[j], tx) * stats.norm.pdf(w.y[n], w.y[j], tx)
                * stats.norm.pdf(w.t[n], w.t[j], tt) for j in range(w.n) if j != n)
        ll += math.log(mu0 * s)
    ll -= mu0 * np.sum(stats.norm.cdf(w.t.max(), w.t, tt) - stats.norm.cdf(0.0, w.t, tt))
    return abs(oracle.evaluate(w.x, w.y, w.t, w.r, w.params, want=0, lib=lib)["loglik"] - ll) <= 1e-11 * abs(ll)


CHECKS = [check_two_events, check_finite_differences, check_simultaneous, check_homogeneity, check_theta0_zero]


def test_unmodified_oracle_passes_every_check():
    for chk in CHECKS:
        assert chk(None), chk.__name__


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, name
    lib = oracle.load_variant(src.replace(old, new), str(tmp_path))
    failed = [chk.__name__ for chk in CHECKS if not chk(lib)]
    assert failed, f"no pin caught: {name}"
