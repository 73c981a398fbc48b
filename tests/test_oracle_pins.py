"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's closed forms and compares them to
themselves.  Each check reaches the same quantity by a different route:
numerical integration of the oracle's own intensity (Appendix A Claim), the
paper's pre-simplification interval sum (Appendix A), library pdfs/cdfs for
special cases, finite differences of the log-likelihood (Eqs. 1, 4, 5), exact
identities that tie the row sums to the column sums, and invariances of the
model under rescaling, translation, rotation and relabelling.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2103_03348_b300 import synth

P_MU0, P_TAUX, P_TAUT, P_THETA0, P_OMEGA, P_H = range(6)


def small_pattern(n, seed, params=(0.7, 0.3, 0.25, 0.6, 2.0, 0.2), r_sd=0.5, t_max=2.0):
    w = synth.make_uniform(seed, n, box=1.0, t_max=t_max, r_sd=r_sd, params=params)
    return w


# ---------------------------------------------------------------------------
# Appendix A Claim (with the background integrated exactly): Lambda equals the
# numerical integral of the oracle's own intensity over R^2 x [0, t_N].
# ---------------------------------------------------------------------------
def _quadrature_of_intensity(w, params):
    # space: composite Gauss-Legendre over a box that holds > 8 sigma of every kernel
    lo, hi = -2.7, 3.7
    panels, per = 32, 12
    g, gw = np.polynomial.legendre.leggauss(per)
    edges = np.linspace(lo, hi, panels + 1)
    xs = np.concatenate([(a + b) / 2 + (b - a) / 2 * g for a, b in zip(edges[:-1], edges[1:])])
    ws = np.concatenate([(b - a) / 2 * gw for a, b in zip(edges[:-1], edges[1:])])
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    WXY = np.outer(ws, ws).ravel()
    X, Y = X.ravel(), Y.ravel()
    # time: Gauss-Legendre on every inter-event interval (the intensity jumps at events)
    tg, tw = np.polynomial.legendre.leggauss(16)
    breaks = np.concatenate([[0.0], np.sort(w.t)])
    total = 0.0
    for a, b in zip(breaks[:-1], breaks[1:]):
        if b <= a:
            continue
        for tk, wk in zip((a + b) / 2 + (b - a) / 2 * tg, (b - a) / 2 * tw):
            lam = oracle.intensity(w.x, w.y, w.t, w.r, params, X, Y, np.full_like(X, tk))
            total += wk * np.dot(WXY, lam)
    return total


@pytest.mark.parametrize("tau_t", [0.25, math.inf])
def test_integral_matches_quadrature(tau_t):
    params = np.array([0.7, 0.3, tau_t, 0.6, 2.0, 0.2])
    w = small_pattern(4, seed=11, params=params)
    q = _quadrature_of_intensity(w, params)
    closed = oracle.integral(w.t, w.r, params)
    assert abs(q - closed) <= 1e-9 * abs(closed), (q, closed)
    # and the same Lambda comes back from the full evaluation
    o = oracle.evaluate(w.x, w.y, w.t, w.r, params, want=0)
    assert o["Lambda"] == closed


def test_claim_interval_sum_form():
    """Appendix A: the excitation integral written as the sum over inter-event
    intervals (before the Claim's simplification) equals the closed form."""
    params = np.array([0.7, 0.3, math.inf, 0.6, 2.0, 0.2])
    w = small_pattern(40, seed=5, params=params)
    t, th = w.t, np.exp(w.r)
    th0, om = params[P_THETA0], params[P_OMEGA]
    N = len(t)
    interval_sum = 0.0
    for n in range(N - 1):
        for m in range(n + 1):
            interval_sum += th[m] * (math.exp(-om * (t[n + 1] - t[m])) - math.exp(-om * (t[n] - t[m])))
    excitation_integral = -th0 * interval_sum
    background_integral = params[P_MU0] * N * t[-1]  # every spatial kernel has mass 1
    closed = oracle.integral(w.t, w.r, params)
    assert abs(closed - (background_integral + excitation_integral)) <= 1e-12 * abs(closed)


# ---------------------------------------------------------------------------
# theta0 -> 0: the likelihood reduces to an inhomogeneous Poisson process with
# the background intensity alone, written here with scipy's normal pdf/cdf.
# ---------------------------------------------------------------------------
def _background_poisson_loglik(w, params):
    mu0, tx, tt = params[:3]
    ll = 0.0
    for n in range(w.n):
        s = 0.0
        for j in range(w.n):
            if w.x[j] == w.x[n] and w.y[j] == w.y[n]:
                continue
            s += (stats.norm.pdf(w.x[n], w.x[j], tx) * stats.norm.pdf(w.y[n], w.y[j], tx)
                  * stats.norm.pdf(w.t[n], w.t[j], tt))
        ll += math.log(mu0 * s)
    tN = w.t.max()
    integral = mu0 * np.sum(stats.norm.cdf(tN, w.t, tt) - stats.norm.cdf(0.0, w.t, tt))
    return ll - integral


def _excitation_per_theta0(w, params, n):
    om, h = params[P_OMEGA], params[P_H]
    s = 0.0
    for j in range(w.n):
        if w.t[j] < w.t[n]:
            s += (math.exp(w.r[j]) * om * math.exp(-om * (w.t[n] - w.t[j]))
                  * stats.norm.pdf(w.x[n], w.x[j], h) * stats.norm.pdf(w.y[n], w.y[j], h))
    return s


def test_theta0_zero_limit():
    params = np.array([0.7, 0.3, 0.25, 0.0, 2.0, 0.2])
    w = small_pattern(25, seed=3, params=params)
    o = oracle.evaluate(w.x, w.y, w.t, w.r, params, want=1)
    ref = _background_poisson_loglik(w, params)
    assert abs(o["loglik"] - ref) <= 1e-12 * abs(ref)
    # d l / d theta0 at theta0 = 0: sum_n xi_n/(theta0 mu_n) - sum_n theta_n (1 - exp(-omega (t_N - t_n)))
    lam_bg = o["lam"]
    tN = w.t.max()
    g_ref = sum(_excitation_per_theta0(w, params, n) / lam_bg[n] for n in range(w.n))
    g_ref -= np.sum(np.exp(w.r) * (1.0 - np.exp(-params[P_OMEGA] * (tN - w.t))))
    assert abs(o["grad"][P_THETA0] - g_ref) <= 1e-11 * abs(g_ref)


def test_two_events_by_hand():
    params = np.array([0.9, 0.4, 0.3, 0.5, 3.0, 0.25])
    x, y, t, r = np.array([0.1, 0.3]), np.array([0.2, -0.1]), np.array([0.2, 0.5]), np.array([0.4, -0.2])
    mu0, tx, tt, th0, om, h = params
    nx = stats.norm.pdf
    bg = mu0 * nx(x[1], x[0], tx) * nx(y[1], y[0], tx) * nx(t[1], t[0], tt)  # symmetric in the pair
    lam1 = bg
    lam2 = bg + th0 * math.exp(r[0]) * om * math.exp(-om * (t[1] - t[0])) * nx(x[1], x[0], h) * nx(y[1], y[0], h)
    Lam = mu0 * sum(stats.norm.cdf(t[1], tk, tt) - stats.norm.cdf(0.0, tk, tt) for tk in t)
    Lam += th0 * sum(math.exp(rk) * (1 - math.exp(-om * (t[1] - tk))) for tk, rk in zip(t, r))
    ll = math.log(lam1) + math.log(lam2) - Lam
    o = oracle.evaluate(x, y, t, r, params, want=0)
    assert abs(o["loglik"] - ll) <= 1e-14 * abs(ll) + 1e-15
    np.testing.assert_allclose(o["lam"], [lam1, lam2], rtol=1e-14)


def test_single_event_has_zero_intensity():
    o = oracle.evaluate([0.0], [0.0], [0.5], [0.0], [0.5, 0.1, 0.05, 0.3, 10.0, 0.02], want=0)
    assert o["status"] == 1 and o["loglik"] == -math.inf


def test_isolated_event_underflows_to_zero_intensity():
    # an event 1 unit away from the rest with tau_x = h = 0.01: exp(-5000) == 0 in FP64
    params = np.array([0.5, 0.01, 0.05, 0.3, 10.0, 0.01])
    x = np.array([0.0, 0.001, 1.0])
    y = np.array([0.0, 0.0, 1.0])
    t = np.array([0.1, 0.2, 0.3])
    o = oracle.evaluate(x, y, t, np.zeros(3), params, want=0)
    assert o["status"] == 1 and o["lam"][2] == 0.0 and o["loglik"] == -math.inf


# ---------------------------------------------------------------------------
# Duplicate locations: the background indicator drops sources at the target's
# exact location (not only the event itself); excitation is unaffected.
# ---------------------------------------------------------------------------
def test_duplicate_location_indicator():
    params = np.array([0.7, 0.3, 0.25, 0.6, 2.0, 0.2])
    x = np.array([0.1, 0.1, 0.5, 0.1])
    y = np.array([0.2, 0.2, 0.4, 0.2])
    t = np.array([0.1, 0.4, 0.6, 0.9])
    r = np.array([0.3, -0.1, 0.2, 0.0])
    o = oracle.evaluate(x, y, t, r, params, want=0)
    mu0, tx, tt, th0, om, h = params
    nx = stats.norm.pdf
    for n in range(4):
        bg = sum(mu0 * nx(x[n], x[j], tx) * nx(y[n], y[j], tx) * nx(t[n], t[j], tt)
                 for j in range(4) if not (x[j] == x[n] and y[j] == y[n]))
        ex = sum(th0 * math.exp(r[j]) * om * math.exp(-om * (t[n] - t[j])) * nx(x[n], x[j], h) * nx(y[n], y[j], h)
                 for j in range(4) if t[j] < t[n])
        assert abs(o["lam"][n] - (bg + ex)) <= 1e-14 * (bg + ex)


# ---------------------------------------------------------------------------
# Finite differences (Richardson-extrapolated central differences) pin the
# gradient against the log-likelihood and the Hessian diagonal against the
# gradient, for all 6 + N coordinates.
# ---------------------------------------------------------------------------
def _richardson(f, x0, step):
    def d(hh):
        return (f(x0 + hh) - f(x0 - hh)) / (2 * hh)
    return (4 * d(step / 2) - d(step)) / 3


@pytest.mark.parametrize("tau_t", [0.25, math.inf])
def test_gradient_and_hessian_finite_differences(tau_t):
    params = np.array([0.7, 0.3, tau_t, 0.6, 2.0, 0.2])
    w = small_pattern(30, seed=7, params=params)
    base = oracle.evaluate(w.x, w.y, w.t, w.r, params, want=2)

    def ev(p, r):
        return oracle.evaluate(w.x, w.y, w.t, r, p, want=1)

    for k in range(6):
        if k == P_TAUT and not math.isfinite(tau_t):
            assert base["grad"][k] == 0.0 and base["hdiag"][k] == 0.0
            continue
        step = 1e-3 * params[k]

        def f_ll(v, k=k):
            p = params.copy(); p[k] = v
            return ev(p, w.r)["loglik"]

        def f_g(v, k=k):
            p = params.copy(); p[k] = v
            return ev(p, w.r)["grad"][k]

        g_fd = _richardson(f_ll, params[k], step)
        h_fd = _richardson(f_g, params[k], step)
        assert abs(base["grad"][k] - g_fd) <= 1e-8 * max(abs(g_fd), 1.0), (k, base["grad"][k], g_fd)
        assert abs(base["hdiag"][k] - h_fd) <= 1e-7 * max(abs(h_fd), 1.0), (k, base["hdiag"][k], h_fd)

    for m in range(w.n):
        def f_ll(v, m=m):
            r = w.r.copy(); r[m] = v
            return ev(params, r)["loglik"]

        def f_g(v, m=m):
            r = w.r.copy(); r[m] = v
            return ev(params, r)["grad"][6 + m]

        g_fd = _richardson(f_ll, w.r[m], 1e-3)
        h_fd = _richardson(f_g, w.r[m], 1e-3)
        assert abs(base["grad"][6 + m] - g_fd) <= 1e-8 * max(abs(g_fd), 1.0), (m, base["grad"][6 + m], g_fd)
        assert abs(base["hdiag"][6 + m] - h_fd) <= 1e-7 * max(abs(h_fd), 1.0), (m, base["hdiag"][6 + m], h_fd)


# ---------------------------------------------------------------------------
# Exact identities (all N): homogeneity in (mu0, theta0), and the link between
# the per-rate column sums and the theta0 row sums.
# ---------------------------------------------------------------------------
def test_euler_and_rate_identities_unit_square():
    w = synth.make_unit_square()
    o = oracle.evaluate(w.x, w.y, w.t, w.r, w.params, want=2)
    g, H = o["grad"], o["hdiag"]
    mu0, th0 = w.params[P_MU0], w.params[P_THETA0]
    # lambda_n is 1-homogeneous in (mu0, theta0) and Lambda is linear in them
    lhs = mu0 * g[P_MU0] + th0 * g[P_THETA0]
    assert abs(lhs - (w.n - o["Lambda"])) <= 1e-10 * w.n
    # excitation depends on theta0 and theta_m only through theta0*theta_m
    assert abs(np.sum(g[6:]) - th0 * g[P_THETA0]) <= 1e-10 * max(1.0, abs(th0 * g[P_THETA0]))
    # concavity in mu0, theta0 and each theta_m (d2l/dtheta_m^2 = (H_r - g_r)/theta_m^2)
    assert H[P_MU0] <= 0 and H[P_THETA0] <= 0
    assert np.all(H[6:] - g[6:] <= 1e-12)


def test_euler_identity_with_rates():
    w = synth.make_uniform(21, 300, box=1.0, t_max=1.0, r_sd=0.7, params=(0.5, 0.1, 0.05, 0.3, 10.0, 0.02))
    o = oracle.evaluate(w.x, w.y, w.t, w.r, w.params, want=1)
    g = o["grad"]
    assert abs(w.params[0] * g[0] + w.params[3] * g[3] - (w.n - o["Lambda"])) <= 1e-10 * w.n
    assert abs(np.sum(g[6:]) - w.params[3] * g[3]) <= 1e-10 * max(1.0, abs(w.params[3] * g[3]))


# ---------------------------------------------------------------------------
# Invariances of the model.
# ---------------------------------------------------------------------------
def test_space_and_time_rescaling():
    w = small_pattern(60, seed=9)
    p = np.array([0.7, 0.3, 0.25, 0.6, 2.0, 0.2])
    ll = oracle.evaluate(w.x, w.y, w.t, w.r, p, want=0)["loglik"]
    s = 3.7
    ps = p.copy(); ps[P_TAUX] *= s; ps[P_H] *= s
    lls = oracle.evaluate(w.x * s, w.y * s, w.t, w.r, ps, want=0)["loglik"]
    assert abs(lls - (ll - 2 * w.n * math.log(s))) <= 1e-12 * abs(ll)
    pt = p.copy(); pt[P_TAUT] *= s; pt[P_OMEGA] /= s
    llt = oracle.evaluate(w.x, w.y, w.t * s, w.r, pt, want=0)["loglik"]
    assert abs(llt - (ll - w.n * math.log(s))) <= 1e-12 * abs(ll)


def test_translation_and_rotation():
    w = small_pattern(60, seed=13)
    p = np.array([0.7, 0.3, 0.25, 0.6, 2.0, 0.2])
    ref = oracle.evaluate(w.x, w.y, w.t, w.r, p, want=1)
    tr = oracle.evaluate(w.x + 12.5, w.y - 3.25, w.t, w.r, p, want=1)
    a = 0.83
    xr = math.cos(a) * w.x - math.sin(a) * w.y
    yr = math.sin(a) * w.x + math.cos(a) * w.y
    ro = oracle.evaluate(xr, yr, w.t, w.r, p, want=1)
    for o in (tr, ro):
        assert abs(o["loglik"] - ref["loglik"]) <= 1e-12 * abs(ref["loglik"])
        np.testing.assert_allclose(o["grad"], ref["grad"], rtol=1e-9, atol=1e-9 * np.abs(ref["grad"]).max())


def test_relabelling_simultaneous_events():
    w = small_pattern(50, seed=17)
    t = w.t.copy()
    t[10:15] = t[10]  # five simultaneous events
    t[30:32] = t[30]
    p = np.array([0.7, 0.3, 0.25, 0.6, 2.0, 0.2])
    ref = oracle.evaluate(w.x, w.y, t, w.r, p, want=2)
    perm = np.arange(w.n)
    perm[10:15] = [13, 10, 14, 12, 11]
    perm[30:32] = [31, 30]
    o = oracle.evaluate(w.x[perm], w.y[perm], t[perm], w.r[perm], p, want=2)
    assert abs(o["loglik"] - ref["loglik"]) <= 1e-14 * abs(ref["loglik"])
    np.testing.assert_allclose(o["grad"][:6], ref["grad"][:6], rtol=1e-13)
    np.testing.assert_allclose(o["grad"][6:], ref["grad"][6:][perm], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(o["hdiag"][6:], ref["hdiag"][6:][perm], rtol=1e-13, atol=1e-15)


def test_simultaneous_events_do_not_excite():
    # two events at the same time and place plus a later one: the first two
    # receive no excitation from each other
    p = np.array([0.7, 0.3, 0.25, 0.6, 2.0, 0.2])
    x = np.array([0.1, 0.4, 0.2]); y = np.array([0.1, 0.3, 0.2]); t = np.array([0.5, 0.5, 0.9])
    o = oracle.evaluate(x, y, t, np.zeros(3), p, want=1)
    o_far = oracle.evaluate(x, y, t, np.zeros(3), np.array([0.7, 0.3, 0.25, 1e-300, 2.0, 0.2]), want=0)
    # with theta0 ~ 0 the first two intensities are unchanged: they were background only
    np.testing.assert_allclose(o["lam"][:2], o_far["lam"][:2], rtol=1e-14)


def test_thread_count_does_not_change_result():
    w = synth.make_uniform(23, 500, r_sd=0.3)
    a = oracle.evaluate(w.x, w.y, w.t, w.r, w.params, want=2, threads=1)
    b = oracle.evaluate(w.x, w.y, w.t, w.r, w.params, want=2, threads=4)
    assert a["loglik"] == b["loglik"]
    assert np.array_equal(a["grad"], b["grad"]) and np.array_equal(a["hdiag"], b["hdiag"])
