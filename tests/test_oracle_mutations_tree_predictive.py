"""The pins of the tree-prior and posterior-predictive oracles have teeth:
plausible one-line slips planted in copies of their sources (on the CPU) are
each caught by at least one pin, re-run here in compact form."""
import math
import types

import numpy as np
import pytest
from scipy import stats

from oracle import predictive_oracle, tree_oracle
from paper_2103_03348_b300 import synth

# ------------------------------------------------------------------ tree prior

TREE_MUTATIONS = {
    "root variance dropped": ("const ld s = (ld)root_var + tr[mrca(parent, depth, i, j)];",
                              "const ld s = tr[mrca(parent, depth, i, j)];"),
    "log determinant doubled": ("logdet_half += logl(a[i * m + i]);", "logdet_half += 2.0L * logl(a[i * m + i]);"),
    "sigma^2 missing from V^-1 z": ("pz[i] = (double)(w[i] / s2);", "pz[i] = (double)w[i];"),
    "common ancestor one level too high": ("    return a;\n}", "    return parent[a] >= 0 ? parent[a] : a;\n}"),
    "diagonal of V^-1 without its first term": ("for (int64_t k = c; k < m; ++k) s += li[k * m + c] * li[k * m + c];",
                                                "for (int64_t k = c + 1; k < m; ++k) s += li[k * m + c] * li[k * m + c];"),
}


def tree_two_tips(lib):
    a, b, tau0, s2 = 0.8, 1.5, 0.6, 2.5
    z = np.array([0.3, -1.1])
    ld, pz, pd = tree_oracle.tree_prior(z, [2, 2, -1], [a, b, 0.0], tau0, s2, lib=lib)
    det = s2 * s2 * ((tau0 + a) * (tau0 + b) - tau0 * tau0)
    inv = np.array([[tau0 + b, -tau0], [-tau0, tau0 + a]]) * s2 / det
    want = -np.log(2 * np.pi) - 0.5 * np.log(det) - 0.5 * z @ inv @ z
    return (abs(ld - want) <= 1e-12 * abs(want) and np.allclose(pz, inv @ z, rtol=1e-12)
            and np.allclose(pd, np.diag(inv), rtol=1e-12))


def tree_against_scipy(lib):
    w = synth.make_ebola_like(seed=9, n=600, m_seq=60, box=120.0, t_max=120.0, n_hot=4)
    tau0, s2 = 0.25, 0.8
    z = np.random.default_rng(2).normal(size=60)
    ld, pz, pd = tree_oracle.tree_prior(z, w.tree_parent, w.tree_length, tau0, s2, lib=lib)
    cov = s2 * (tau0 + w.tree_cov)
    prec = np.linalg.inv(cov)
    return (abs(ld - stats.multivariate_normal(np.zeros(60), cov).logpdf(z)) <= 1e-9 * abs(ld)
            and np.allclose(pz, prec @ z, rtol=1e-6, atol=1e-9) and np.allclose(pd, np.diag(prec), rtol=1e-6))


TREE_CHECKS = [tree_two_tips, tree_against_scipy]


def test_unmodified_tree_oracle_passes():
    for chk in TREE_CHECKS:
        assert chk(None), chk.__name__


@pytest.mark.parametrize("name", sorted(TREE_MUTATIONS))
def test_tree_mistake_is_caught(name, tmp_path):
    old, new = TREE_MUTATIONS[name]
    src = tree_oracle.source_text()
    assert src.count(old) == 1, name
    lib = tree_oracle.load_variant(src.replace(old, new), str(tmp_path))
    failed = []
    for chk in TREE_CHECKS:
        try:
            ok = chk(lib)
        except np.linalg.LinAlgError:  # a mistake may also make V indefinite: the oracle refuses
            ok = False
        if not ok:
            failed.append(chk.__name__)
    assert failed, f"no pin caught: {name}"


# ------------------------------------------------------ predictive simulation

PRED_MUTATIONS = {
    "past events' children not restarted at T0": ("tf = lambda u: t0 - math.log1p(-u * one_m_h) / om  # noqa: E731",
                                                  "tf = lambda u, i=i: t[i] - math.log1p(-u * one_m_h) / om  # noqa: E731"),
    "rate theta_n missing from the children's mean": ("lam = th0 * math.exp(r[i] - om * (t0 - t[i])) * one_m_h",
                                                      "lam = th0 * math.exp(-om * (t0 - t[i])) * one_m_h"),
    "background placed with the excitation bandwidth": ("e = child(i, k, 0, x[i], y[i], tf, tx)",
                                                         "e = child(i, k, 0, x[i], y[i], tf, h)"),
    "new events' children not truncated at the horizon": ("one_m = -math.expm1(-om * span)",
                                                          "one_m = -math.expm1(-om * horizon)"),
    "Poisson shortcut too generous": ("if u <= 1.0 - lam:  # P(K = 0) = e^-lam > 1 - lam",
                                      "if u <= 1.0 - 0.5 * lam:  # P(K = 0) = e^-lam > 1 - lam"),
    "Philox key schedule frozen": ("k0 = (k0 + PHILOX_W0) & MASK32", "k0 = k0"),
    "background mass not truncated at the horizon": ("lam = mu0 * (qa - qb)", "lam = mu0 * qa"),
}


def _history():
    w = synth.make_ebola_like(seed=5, n=400, m_seq=30, box=120.0, t_max=120.0, n_hot=4)
    r = w.r.copy()
    r[np.argsort(w.t)[-60:]] = 1.0  # recent, contagious events: the children's mean depends on theta
    q = np.concatenate([np.log(w.params), r[w.sequenced]])
    return w, r, q


def _runs(po, samples=200, horizon=10.0):
    w, r, q = _history()
    return w, r, q, [po.simulate(w.x, w.y, w.t, r, w.sequenced, q, horizon, 11, s, 100000) for s in range(samples)]


def pred_philox(po):
    return po.philox4x32((0, 0, 0, 0), (0, 0)) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)


def pred_quantiles(po):
    rng = np.random.default_rng(1)
    return all(po.poisson(lam, u) == int(stats.poisson.ppf(u, lam))
               for lam in (0.01, 0.3, 2.0, 40.0) for u in rng.uniform(size=200))


def pred_window_and_mean(po):
    w, r, q, out = _runs(po)
    t0 = w.t.max()
    for ev, src, st in out:
        if st != 0 or len(ev) and not (np.all(ev[:, 2] > t0) and np.all(ev[:, 2] <= t0 + 10.0 + 1e-9)):
            return False
    c = np.array([len(e) for e, _, _ in out])
    expect = predictive_oracle.expected_count(w.t, r, np.exp(q[:6]), 10.0)  # the unmodified pin
    return abs(c.mean() - expect) < 4.0 * c.std() / math.sqrt(c.size)


def pred_displacements(po):
    w, r, q, out = _runs(po, samples=120)
    p = np.exp(q[:6])
    bg, ch = [], []
    for ev, src, _ in out:
        for (x, y, t), s in zip(ev, src):
            if s < 0:
                bg += [(x - w.x[-s - 1]) / p[1], (y - w.y[-s - 1]) / p[1]]
            elif s < w.n:
                ch += [(x - w.x[s]) / p[5], (y - w.y[s]) / p[5]]
    return len(bg) > 100 and len(ch) > 100 and stats.kstest(bg, "norm").pvalue > 1e-3 and \
        stats.kstest(ch, "norm").pvalue > 1e-3


PRED_CHECKS = [pred_philox, pred_quantiles, pred_window_and_mean, pred_displacements]


def _variant(src):
    mod = types.ModuleType("predictive_variant")
    exec(compile(src, "predictive_variant", "exec"), mod.__dict__)
    return mod


def test_unmodified_predictive_oracle_passes():
    for chk in PRED_CHECKS:
        assert chk(predictive_oracle), chk.__name__


@pytest.mark.parametrize("name", sorted(PRED_MUTATIONS))
def test_predictive_mistake_is_caught(name):
    old, new = PRED_MUTATIONS[name]
    with open(predictive_oracle.__file__) as f:
        src = f.read()
    assert src.count(old) == 1, name
    mod = _variant(src.replace(old, new))
    failed = []
    for chk in PRED_CHECKS:
        try:
            ok = chk(mod)
        except Exception:  # a mistake may also break the simulation outright
            ok = False
        if not ok:
            failed.append(chk.__name__)
            break
    assert failed, f"no pin caught: {name}"
