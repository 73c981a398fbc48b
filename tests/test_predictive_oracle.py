"""Pins of the posterior-predictive simulation oracle, on the CPU.

* Philox4x32-10 reproduces the published known-answer vectors (Salmon et al.
  2011, the Random123 distribution's test values).
* The Poisson inversion equals scipy's Poisson quantile function; split means
  keep the Poisson mean and variance.
* The mean number of simulated events matches the closed-form expectation of
  the branching process (m(s) = (1 - theta0 e^{-omega (1 - theta0)(T1 - s)}) /
  (1 - theta0) integrated against the conditional intensity by quadrature),
  for tau_t finite and infinite.
* Children's displacements are N(0, h^2 I) (background: tau_x^2); children's
  delays follow the truncated exponential; background times follow the
  truncated normal (probability integral transform, Kolmogorov-Smirnov).
* Capacity, bad parameters and reproducibility behave as specified.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import predictive_oracle as po
from paper_2103_03348_b300 import synth


def test_philox_known_answers():
    assert po.philox4x32((0, 0, 0, 0), (0, 0)) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)
    assert po.philox4x32((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2) == (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)
    assert po.philox4x32((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0)) == \
        (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)


def test_uniforms_stay_inside_the_open_interval():
    assert po.u53(0, 0) == 2.0 ** -54
    assert po.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -54
    w = [po.philox4x32((i, 0, 0, 0), (7, 9)) for i in range(20000)]
    u = np.array([po.u53(a[0], a[1]) for a in w])
    assert stats.kstest(u, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("lam", [1e-12, 1e-6, 0.01, 0.3, 1.0, 4.5, 37.0, 250.0, 499.0])
def test_poisson_inversion_is_the_quantile_function(lam):
    rng = np.random.default_rng(int(lam * 1000) + 1)
    us = np.concatenate([rng.uniform(size=400), [2.0 ** -54, 0.5, 1.0 - 2.0 ** -20]])
    for u in us:
        assert po.poisson(lam, u) == int(stats.poisson.ppf(u, lam)), (lam, u)


def test_split_poisson_keeps_mean_and_variance():
    lam, key = 1234.5, (3, 4)
    k = np.array([po.poisson_count(lam, key, i, 0, 0, 10 ** 6) for i in range(4000)])
    assert abs(k.mean() - lam) < 4 * math.sqrt(lam / k.size)
    assert abs(k.var() / lam - 1.0) < 0.1
    assert po.poisson_count(5000.0, key, 0, 0, 0, 1000) == 1001  # saturated above 4 x capacity


def history(seed=5, n=400):
    w = synth.make_ebola_like(seed=seed, n=n, m_seq=30, box=120.0, t_max=120.0, n_hot=4)
    q = np.concatenate([np.log(w.params), w.r[w.sequenced]])
    return w, q


def run_many(w, q, horizon, samples, seed=11, capacity=100000):
    out = [po.simulate(w.x, w.y, w.t, w.r, w.sequenced, q, horizon, seed, s, capacity) for s in range(samples)]
    assert all(st == po.STATUS_OK for _, _, st in out)
    return out


@pytest.mark.parametrize("tau_t", [30.0, math.inf])
def test_mean_count_matches_branching_expectation(tau_t):
    w, q = history()
    q = q.copy()
    q[2] = math.log(tau_t)
    if math.isinf(tau_t):
        q[0] = math.log(0.5 / w.n)  # the purely spatial background: mu0 N events per day in all
    r = w.r.copy()
    r[w.sequenced] = q[6:]
    p = np.exp(q[:6])
    out = run_many(w, q, 10.0, 300)
    c = np.array([len(e) for e, _, _ in out])
    expect = po.expected_count(w.t, r, p, 10.0)
    assert abs(c.mean() - expect) < 4.0 * c.std() / math.sqrt(c.size), (c.mean(), expect)


def test_displacements_delays_and_background_times():
    w, q = history()
    p = np.exp(q[:6])
    tx, tt, om, h = p[1], p[2], p[4], p[5]
    out = run_many(w, q, 20.0, 150)
    t0, t1 = w.t.max(), w.t.max() + 20.0
    dx_bg, dx_ch, pit, delays = [], [], [], []
    for ev, src, _ in out:
        for (x, y, t), s in zip(ev, src):
            if s < 0:
                i = -s - 1
                dx_bg += [(x - w.x[i]) / tx, (y - w.y[i]) / tx]
                qa, qb = po.upper_tail((t0 - w.t[i]) / tt), po.upper_tail((t1 - w.t[i]) / tt)
                pit.append((qa - po.upper_tail((t - w.t[i]) / tt)) / (qa - qb))
            elif s < w.n:
                dx_ch += [(x - w.x[s]) / h, (y - w.y[s]) / h]
                delays.append(t - t0)
            else:
                par = ev[s - w.n]
                dx_ch += [(x - par[0]) / h, (y - par[1]) / h]
    for z in (np.array(dx_bg), np.array(dx_ch)):
        assert z.size > 500
        assert stats.kstest(z, "norm").pvalue > 1e-3
    assert stats.kstest(np.array(pit), "uniform").pvalue > 1e-3
    # delays after T0 of past events' children: Exp(omega) truncated to (0, H]
    cdf = lambda d: -np.expm1(-om * d) / -math.expm1(-om * 20.0)  # noqa: E731
    assert stats.kstest(np.array(delays), cdf).pvalue > 1e-3
    assert np.all((np.array(delays) > 0) & (np.array(delays) <= 20.0))


def test_all_times_inside_the_window_and_parents_precede_children():
    w, q = history()
    for ev, src, _ in run_many(w, q, 15.0, 20):
        t0 = w.t.max()
        assert np.all((ev[:, 2] > t0) & (ev[:, 2] <= t0 + 15.0 + 1e-9))
        for k, s in enumerate(src):
            if s >= w.n:
                assert s - w.n < k and ev[s - w.n, 2] < ev[k, 2]


def test_capacity_keeps_the_first_events():
    w, q = history()
    full, fsrc, st = po.simulate(w.x, w.y, w.t, w.r, w.sequenced, q, 10.0, 5, 3, 100000)
    assert st == po.STATUS_OK and len(full) > 10
    part, psrc, st2 = po.simulate(w.x, w.y, w.t, w.r, w.sequenced, q, 10.0, 5, 3, 10)
    assert st2 == po.STATUS_OVERFLOW
    np.testing.assert_array_equal(part, full[:10])
    np.testing.assert_array_equal(psrc, fsrc[:10])


def test_bad_parameters_and_reproducibility():
    w, q = history()
    bad = q.copy()
    bad[4] = math.nan
    ev, src, st = po.simulate(w.x, w.y, w.t, w.r, w.sequenced, bad, 10.0, 5, 0, 1000)
    assert st == po.STATUS_BADPARAM and len(ev) == 0
    a = po.simulate(w.x, w.y, w.t, w.r, w.sequenced, q, 10.0, 5, 0, 1000)
    b = po.simulate(w.x, w.y, w.t, w.r, w.sequenced, q, 10.0, 5, 0, 1000)
    c = po.simulate(w.x, w.y, w.t, w.r, w.sequenced, q, 10.0, 5, 1, 1000)
    np.testing.assert_array_equal(a[0], b[0])
    assert len(a[0]) != len(c[0]) or not np.array_equal(a[0], c[0])
