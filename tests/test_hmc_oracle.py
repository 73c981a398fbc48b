"""Pins of the HMC oracle (Section 2.3) and of the product's ESS estimator."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import hmc_oracle
from paper_2103_03348_b300 import synth


def test_prior_terms_match_scipy_densities():
    kind = np.array([0, 1, 1, 0, 0, 1])
    a = np.array([2.0, 1.0, 2.0, 1.0, 2.0, 2.0])
    b = np.array([2.0, 1112.0, 182.6, 0.001, 182.6, 55.6])
    p1 = np.array([0.5, 20.0, 30.0, 0.5, 0.1, 5.0])
    p2 = p1 * 1.37
    lp1, d1, d2 = hmc_oracle.log_prior_terms(p1, kind, a, b)
    lp2, _, _ = hmc_oracle.log_prior_terms(p2, kind, a, b)

    def scipy_logpdf(p, k):
        if kind[k] == 0:
            return stats.gamma.logpdf(p, a[k], scale=1.0 / b[k])
        return stats.invgamma.logpdf(p, a[k], scale=b[k])

    for k in range(6):
        # densities agree up to the normalising constant: compare differences
        assert abs((lp2[k] - lp1[k]) - (scipy_logpdf(p2[k], k) - scipy_logpdf(p1[k], k))) < 1e-10
        h = 1e-5 * p1[k]
        fd1 = (scipy_logpdf(p1[k] + h, k) - scipy_logpdf(p1[k] - h, k)) / (2 * h)
        h2 = 1e-3 * p1[k]  # a wider step for the second difference (roundoff ~ eps |f| / h^2)
        fd2 = (scipy_logpdf(p1[k] + h2, k) - 2 * scipy_logpdf(p1[k], k) + scipy_logpdf(p1[k] - h2, k)) / h2 ** 2
        assert abs(d1[k] - fd1) <= 1e-6 * max(1.0, abs(fd1))
        assert abs(d2[k] - fd2) <= 1e-4 * abs(d2[k]) + 1e-8 / p1[k] ** 2


def small_problem(n=60, m=8, seed=3):
    w = synth.make_ebola_like(seed=seed, n=n, m_seq=m, box=100.0, t_max=60.0, n_hot=3)
    prec = np.linalg.inv(w.tree_cov)
    prior = (np.array([0, 1, 1, 0, 0, 1]), np.array([2.0, 1.0, 2.0, 1.0, 2.0, 2.0]),
             np.array([2.0, 1112.0, 182.6, 0.001, 182.6, 55.6]))
    q = np.concatenate([np.log(w.params), w.r[w.sequenced]])
    return w, prec, prior, q


def test_log_posterior_finite_differences():
    w, prec, prior, q = small_problem()
    lp, g, h = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, prior, q)

    def f(qq):
        return hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, prior, qq, want_hess=False)

    for k in range(len(q)):
        step = 1e-4

        def dd(hh, k=k):
            qp, qm = q.copy(), q.copy()
            qp[k] += hh
            qm[k] -= hh
            a, b = f(qp), f(qm)
            return (a[0] - b[0]) / (2 * hh), (a[1][k] - b[1][k]) / (2 * hh)

        (g1, h1), (g2, h2) = dd(step), dd(step / 2)
        g_fd, h_fd = (4 * g2 - g1) / 3, (4 * h2 - h1) / 3
        assert abs(g[k] - g_fd) <= 1e-7 * max(1.0, abs(g_fd)), (k, g[k], g_fd)
        assert abs(h[k] - h_fd) <= 1e-6 * max(1.0, abs(h_fd)), (k, h[k], h_fd)


def test_leapfrog_harmonic_oscillator_closed_form():
    # log pi = -q^2/2, unit mass: one leapfrog step is the linear map
    # [[1 - e^2/2, e], [-e (1 - e^2/4), 1 - e^2/2]]
    eps, steps = 0.3, 17
    A = np.array([[1 - eps ** 2 / 2, eps], [-eps * (1 - eps ** 2 / 4), 1 - eps ** 2 / 2]])
    q0, p0 = np.array([0.7]), np.array([-1.1])
    q, p, _, _ = hmc_oracle.leapfrog(q0, p0, eps, steps, np.ones(1), lambda x: (-0.5 * x @ x, -x))
    ref = np.linalg.matrix_power(A, steps) @ np.array([q0[0], p0[0]])
    assert np.allclose([q[0], p[0]], ref, rtol=1e-13, atol=1e-14)


def test_dense_mass_leapfrog_whitened_closed_form():
    """With a dense mass equal to the target's precision P = L L^T, the whitened
    coordinates u = L^T q, v = L^-1 p turn every direction into the unit
    oscillator, so the dense-mass leapfrog is the closed-form map of the
    one-dimensional test applied in those coordinates."""
    rng = np.random.default_rng(3)
    X = rng.normal(size=(6, 6))
    P = X @ X.T + 0.5 * np.eye(6)
    L = np.linalg.cholesky(P)
    eps, steps = 0.27, 13
    A = np.array([[1 - eps ** 2 / 2, eps], [-eps * (1 - eps ** 2 / 4), 1 - eps ** 2 / 2]])
    An = np.linalg.matrix_power(A, steps)
    q0, p0 = rng.normal(size=6), rng.normal(size=6)
    q, p, _, _ = hmc_oracle.leapfrog(q0, p0, eps, steps, np.linalg.inv(P), lambda x: (-0.5 * x @ P @ x, -P @ x))
    u0, v0 = L.T @ q0, np.linalg.solve(L, p0)
    u1, v1 = An[0, 0] * u0 + An[0, 1] * v0, An[1, 0] * u0 + An[1, 1] * v0
    assert np.allclose(L.T @ q, u1, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.linalg.solve(L, p), v1, rtol=1e-12, atol=1e-12)
    # the kinetic energy in whitened coordinates is 1/2 |v|^2
    assert abs(hmc_oracle.kinetic(p0, np.linalg.inv(P)) - 0.5 * v0 @ v0) <= 1e-12 * (v0 @ v0)


def test_dense_leapfrog_with_a_diagonal_matrix_is_the_diagonal_leapfrog():
    rng = np.random.default_rng(4)
    prec = np.diag(rng.uniform(0.5, 4.0, 5))
    minv = rng.uniform(0.3, 2.0, 5)
    q0, p0 = rng.normal(size=5), rng.normal(size=5)
    gf = lambda x: (-0.5 * x @ prec @ x, -prec @ x)  # noqa: E731
    a = hmc_oracle.leapfrog(q0, p0, 0.1, 9, minv, gf)
    b = hmc_oracle.leapfrog(q0, p0, 0.1, 9, np.diag(minv), gf)
    assert np.allclose(a[0], b[0], rtol=1e-14, atol=1e-15) and np.allclose(a[1], b[1], rtol=1e-14, atol=1e-15)


def test_leapfrog_reversible_and_second_order():
    rng = np.random.default_rng(0)
    prec = np.diag(rng.uniform(0.5, 4.0, 5))

    def gf(x):
        return -0.5 * x @ prec @ x, -prec @ x

    q0, p0 = rng.normal(size=5), rng.normal(size=5)
    minv = np.full(5, 0.8)
    q1, p1, _, _ = hmc_oracle.leapfrog(q0, p0, 0.1, 25, minv, gf)
    q2, p2, _, _ = hmc_oracle.leapfrog(q1, -p1, 0.1, 25, minv, gf)
    assert np.allclose(q2, q0, atol=1e-12) and np.allclose(-p2, p0, atol=1e-12)

    def energy_err(eps):
        q, p, lp, _ = hmc_oracle.leapfrog(q0, p0, eps, int(round(1.0 / eps)), minv, gf)
        return abs((-lp + 0.5 * np.sum(minv * p * p)) - (-gf(q0)[0] + 0.5 * np.sum(minv * p0 * p0)))

    e1, e2 = energy_err(0.1), energy_err(0.05)
    assert 3.0 < e1 / e2 < 5.0  # energy error is O(eps^2)


def ar1(rho, n, seed):
    rng = np.random.default_rng(seed)
    x = np.empty(n)
    x[0] = rng.normal() / math.sqrt(1 - rho ** 2)
    e = rng.normal(size=n)
    for i in range(1, n):
        x[i] = rho * x[i - 1] + e[i]
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_ess_of_ar1_chains(rho):
    n = 8000
    x = ar1(rho, n, seed=int(rho * 10))
    ess = hmc_oracle.ess_geyer(x)
    expected = n * (1 - rho) / (1 + rho)  # n / integrated autocorrelation time
    assert abs(ess / expected - 1) < 0.2, (ess, expected)


def test_product_ess_matches_oracle():
    from paper_2103_03348_b300 import hmc
    for rho, seed in ((0.3, 1), (0.95, 2)):
        x = ar1(rho, 3000, seed)
        assert abs(hmc.ess(x) / hmc_oracle.ess_geyer(x) - 1) < 1e-9


def test_log_posterior_with_trend_finite_differences():
    """r_seq = z + F beta (Section 2.2's trend): the gradient in every
    coordinate, including beta, and the Hessian diagonal in the globals and z
    match central differences; the beta entries of the diagonal are the
    stated preconditioner."""
    w, prec, prior, q = small_problem()
    m = len(w.sequenced)
    ts = w.t[w.sequenced]
    F = np.stack([(ts - ts.mean()) / ts.std(), ((ts - ts.mean()) / ts.std()) ** 2 - 1.0], axis=1)
    beta = np.array([0.15, -0.1])
    qt = np.concatenate([q, beta])
    bv = 0.5
    lp, g, h = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, prior, qt, trend=F, beta_var=bv)

    def f(qq):
        return hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, prior, qq, want_hess=False,
                                        trend=F, beta_var=bv)

    for k in range(len(qt)):
        def dd(hh, k=k):
            qp, qm = qt.copy(), qt.copy()
            qp[k] += hh
            qm[k] -= hh
            a, b = f(qp), f(qm)
            return (a[0] - b[0]) / (2 * hh), (a[1][k] - b[1][k]) / (2 * hh)

        (g1, h1), (g2, h2) = dd(1e-4), dd(5e-5)
        g_fd, h_fd = (4 * g2 - g1) / 3, (4 * h2 - h1) / 3
        assert abs(g[k] - g_fd) <= 1e-7 * max(1.0, abs(g_fd)), (k, g[k], g_fd)
        if k < 6 + m:
            assert abs(h[k] - h_fd) <= 1e-6 * max(1.0, abs(h_fd)), (k, h[k], h_fd)
    # the beta preconditioner from the rate diagonal at the same point
    r = w.r.copy()
    r[w.sequenced] = qt[6:6 + m] + F @ beta
    import oracle
    hr = oracle.evaluate(w.x, w.y, w.t, r, np.exp(qt[:6]), want=2)["hdiag"][6 + w.sequenced]
    np.testing.assert_allclose(h[6 + m:], (F ** 2).T @ hr - 1.0 / bv, rtol=1e-13)
    # zero features: the trend only adds its Gaussian prior
    lp0, g0, _ = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, prior, q)
    lpz, gz, _ = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, prior, qt, trend=0 * F, beta_var=bv)
    assert abs(lpz - (lp0 - 0.5 * beta @ beta / bv)) <= 1e-12 * abs(lp0)
    np.testing.assert_allclose(gz[:6 + m], g0, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(gz[6 + m:], -beta / bv, rtol=1e-13)


def test_accept_probability_closed_forms():
    acc = hmc_oracle.accept_probability
    assert acc(-3.0, 1.0, -3.0, 1.0) == 1.0                       # energy conserved
    assert abs(acc(0.0, 0.0, -math.log(4.0), 0.0) - 0.25) < 1e-15  # H1 - H0 = log 4
    assert abs(acc(0.0, 0.5, 0.0, 0.5 + math.log(2.0)) - 0.5) < 1e-15  # the kinetic side enters with H
    assert acc(0.0, 2.0, 0.0, 0.0) == 1.0                          # energy dropped: always accepted
    assert acc(0.0, 0.0, 5.0, 0.0) == 1.0                          # higher log posterior, same kinetic
    for lp1, k1, ok in [(-math.inf, 0.0, True), (math.nan, 0.0, True), (0.0, math.inf, True),
                        (0.0, math.nan, True), (0.0, 0.0, False)]:
        assert acc(0.0, 0.0, lp1, k1, ok) == 0.0


def test_accept_probability_keeps_a_discrete_target_in_detailed_balance():
    # Metropolis with a symmetric proposal: T[i, j] = Q[i, j] a(i -> j) off the diagonal.
    # Detailed balance pi_i T_ij = pi_j T_ji fixes the sign of every term of the energy;
    # a swapped sign or a dropped kinetic term breaks it.
    rng = np.random.default_rng(5)
    pi = rng.uniform(0.1, 1.0, 5)
    pi /= pi.sum()
    k = rng.uniform(0.0, 2.0, 5)  # a kinetic energy per state, with pi_i proportional to exp(lp_i - k_i)
    lp = np.log(pi) + k
    Q = rng.uniform(0.0, 1.0, (5, 5))
    Q = Q + Q.T
    np.fill_diagonal(Q, 0.0)
    Q /= Q.sum(axis=1).max()
    T = np.zeros((5, 5))
    for i in range(5):
        for j in range(5):
            if i != j:
                T[i, j] = Q[i, j] * hmc_oracle.accept_probability(lp[i], k[i], lp[j], k[j])
        T[i, i] = 1.0 - T[i].sum()
    F = pi[:, None] * T
    assert np.allclose(F, F.T, atol=1e-15)
    assert np.allclose(pi @ T, pi, atol=1e-15)


def test_metropolis_step_selects_by_strict_comparison():
    q0, g0, q1, g1 = np.zeros(3), np.ones(3), np.full(3, 2.0), np.full(3, 3.0)
    # a = 0.25 exactly
    lp1 = -math.log(4.0)
    q, lp, g, ok, a = hmc_oracle.metropolis_step(q0, 0.0, g0, 0.0, q1, lp1, g1, 0.0, u=0.2)
    assert ok and a == 0.25 and np.array_equal(q, q1) and lp == lp1 and np.array_equal(g, g1)
    q, lp, g, ok, a = hmc_oracle.metropolis_step(q0, 0.0, g0, 0.0, q1, lp1, g1, 0.0, u=0.25)
    assert not ok and np.array_equal(q, q0) and lp == 0.0 and np.array_equal(g, g0)
    q, lp, g, ok, a = hmc_oracle.metropolis_step(q0, 0.0, g0, 0.0, q1, math.nan, g1, 0.0, u=0.0)
    assert not ok and a == 0.0 and np.array_equal(q, q0)
