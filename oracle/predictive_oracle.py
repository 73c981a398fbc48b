"""Oracle of posterior-predictive simulation of the spatiotemporal Hawkes
process (the forward simulation that the paper's Discussion proposes to run
in parallel over posterior parameter settings with counter-based random
numbers, exploiting the exponential temporal trigger).

TEST INFRASTRUCTURE: used only by the tests and the bench's CPU legs.

Given the history (x, y, t, r) of N events, one parameter setting in sampler
coordinates q = (log mu0, log tau_x, log tau_t, log theta0, log omega, log h,
r of the M sequenced events) and a horizon H, it draws the events of
(T0, T0 + H], T0 = max t, from the intensity of Section 2.1 conditioned on
the history, exactly, through the branching (cluster) representation:

  stage 0  each past event n' seeds Poisson(mu0 * m_n') background events,
           m_n' = Phi((T1 - t_n')/tau_t) - Phi((T0 - t_n')/tau_t) (H when
           tau_t is infinite), at times from N(t_n', tau_t^2) truncated to the
           window (uniform when tau_t is infinite) and places
           (x_n', y_n') + tau_x N(0, I);
  stage 1  each past event n has Poisson(theta0 theta_n e^{-omega (T0 - t_n)}
           (1 - e^{-omega H})) children in the window; by the memorylessness
           of the exponential trigger their times are T0 + Exp(omega)
           truncated to (0, H], their places (x_n, y_n) + h N(0, I);
  stage g  each event e of the previous generation (theta = 1: a new case
           has no sequence) has Poisson(theta0 (1 - e^{-omega (T1 - t_e)}))
           children at t_e + Exp(omega) truncated to (0, T1 - t_e] and
           (x_e, y_e) + h N(0, I);
until a generation is empty.  Events are listed stage by stage, parent by
parent, child by child.

Random numbers: Philox4x32-10 (Salmon, Moraes, Dror and Shaw 2011),
key = the 64-bit seed, counter = (item, draw, stage, sample).  Draw 0 of an
item decides its number of children; draws 2k+1 and 2k+2 give child k its time
and place.  A uniform is made from two words as (a 2^26 + b + 1/2) 2^-53 with
a = w0 >> 5, b = w1 >> 6, so it lies strictly inside (0, 1).  A Poisson mean
above 500 is split into ceil(mean / 500) equal parts drawn by inversion from
draws 2^31 + p (a sum of independent Poissons is Poisson); a mean above four
times the capacity saturates the count (the output then holds the first
`capacity` events and reports an overflow, which such a mean makes certain
in all but a vanishing fraction of draws).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

MASK32 = 0xFFFFFFFF
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85

STATUS_OK, STATUS_OVERFLOW, STATUS_BADPARAM = 0, 1, 2
POISSON_PART = 500.0  # largest mean drawn by one inversion (e^-500 is far from underflow)
PART_DRAW = 0x80000000
MAX_CAPACITY = 1 << 24


def philox4x32(ctr, key, rounds=10):
    """Philox4x32 block function: 4 counter words, 2 key words -> 4 words."""
    c0, c1, c2, c3 = (int(v) & MASK32 for v in ctr)
    k0, k1 = (int(v) & MASK32 for v in key)
    for i in range(rounds):
        if i > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def u53(w0, w1):
    return ((w0 >> 5) * 67108864.0 + (w1 >> 6) + 0.5) / 9007199254740992.0


def draws(key, item, draw, stage, sample):
    w = philox4x32((item, draw, stage, sample), key)
    return u53(w[0], w[1]), u53(w[2], w[3])


def poisson(lam, u):
    """Inversion: the smallest k with u <= P(K <= k), K ~ Poisson(lam)."""
    if not lam > 0.0:
        return 0
    if u <= 1.0 - lam:  # P(K = 0) = e^-lam > 1 - lam
        return 0
    p = math.exp(-lam)
    f = p
    k = 0
    while u > f:
        k += 1
        p *= lam / k
        f += p
        if p == 0.0 and k > lam:
            break
    return k


def poisson_count(lam, key, item, stage, sample, capacity):
    if not lam > 0.0:
        return 0
    if lam > 4.0 * capacity:
        return capacity + 1
    if lam <= POISSON_PART:
        return poisson(lam, draws(key, item, 0, stage, sample)[0])
    parts = math.ceil(lam / POISSON_PART)
    sub = lam / parts
    return sum(poisson(sub, draws(key, item, PART_DRAW + j, stage, sample)[0]) for j in range(parts))


def upper_tail(z):
    """Q(z) = P(Z > z) for a standard normal Z."""
    return 0.5 * special.erfc(z / math.sqrt(2.0))


def upper_tail_inv(p):
    return math.sqrt(2.0) * special.erfcinv(2.0 * p)


def simulate(x, y, t, r_base, seq_idx, q, horizon, seed, sample, capacity):
    """(events [K, 3] as (x, y, t), src [K], status) for one parameter setting.

    src: -(n'+1) for background seeded by past event n'; n for a child of past
    event n; N + e for a child of new event e (its row in the output)."""
    x, y, t = (np.asarray(a, float) for a in (x, y, t))
    q = np.asarray(q, float)
    n = t.size
    r = np.array(r_base, float)
    r[np.asarray(seq_idx, np.int64)] = q[6:6 + len(seq_idx)]
    p = np.exp(q[:6])
    mu0, tx, tt, th0, om, h = (float(v) for v in p)
    ok = all(math.isfinite(v) and v > 0 for k, v in enumerate(p) if k != 2) and tt > 0 and not math.isnan(tt)
    if not (ok and horizon > 0) or not 1 <= capacity <= MAX_CAPACITY:
        return np.zeros((0, 3)), np.zeros(0, np.int64), STATUS_BADPARAM
    key = (seed & MASK32, (seed >> 32) & MASK32)
    t0 = float(np.max(t))
    t1 = t0 + horizon
    tt_inf = math.isinf(tt)
    ev, src = [], []

    def child(item, k, stage, px, py, pt_of, sd):
        u1, u2 = draws(key, item, 2 * k + 1, stage, sample)
        u3, _ = draws(key, item, 2 * k + 2, stage, sample)
        rad = math.sqrt(-2.0 * math.log(u2))
        ang = 6.283185307179586 * u3
        return px + sd * rad * math.cos(ang), py + sd * rad * math.sin(ang), pt_of(u1)

    def add(e, s):
        if len(ev) >= capacity:
            return False
        ev.append(e)
        src.append(s)
        return True

    one_m_h = -math.expm1(-om * horizon)
    for stage in (0, 1):
        for i in range(n):
            if stage == 0:
                if tt_inf:
                    lam, qa, qb = mu0 * horizon, 0.0, 0.0
                else:
                    qa, qb = upper_tail((t0 - t[i]) / tt), upper_tail((t1 - t[i]) / tt)
                    lam = mu0 * (qa - qb)
            else:
                lam = th0 * math.exp(r[i] - om * (t0 - t[i])) * one_m_h
            kk = poisson_count(lam, key, i, stage, sample, capacity)
            for k in range(kk):
                if stage == 0:
                    if tt_inf:
                        tf = lambda u: t0 + u * horizon  # noqa: E731
                    else:
                        tf = lambda u, i=i, qa=qa, qb=qb: t[i] + tt * upper_tail_inv(qa - u * (qa - qb))  # noqa: E731
                    e = child(i, k, 0, x[i], y[i], tf, tx)
                    s = -(i + 1)
                else:
                    tf = lambda u: t0 - math.log1p(-u * one_m_h) / om  # noqa: E731
                    e = child(i, k, 1, x[i], y[i], tf, h)
                    s = i
                if not add(e, s):
                    return np.array(ev).reshape(-1, 3), np.array(src, np.int64), STATUS_OVERFLOW
    start, end, stage = 0, len(ev), 2
    while start < end:
        for e_idx in range(start, end):
            ex, ey, et = ev[e_idx]
            span = t1 - et
            one_m = -math.expm1(-om * span)
            lam = th0 * one_m
            kk = poisson_count(lam, key, e_idx, stage, sample, capacity)
            for k in range(kk):
                tf = lambda u, et=et, one_m=one_m: et - math.log1p(-u * one_m) / om  # noqa: E731
                if not add(child(e_idx, k, stage, ex, ey, tf, h), n + e_idx):
                    return np.array(ev).reshape(-1, 3), np.array(src, np.int64), STATUS_OVERFLOW
        start, end, stage = end, len(ev), stage + 1
    return np.array(ev).reshape(-1, 3), np.array(src, np.int64), STATUS_OK


def expected_count(t, r, p, horizon, n_quad=2000):
    """E[number of events in (T0, T0 + H]] under the model, by quadrature.

    A new event at time s has, counting itself, an expected
        m(s) = (1 - theta0 e^{-omega (1 - theta0) (T1 - s)}) / (1 - theta0)
    events in the window (m' = omega (1 - theta0) m - omega, m(T1) = 1), so
        E = int_T0^T1 [mu_b(s) + sum_n theta0 theta_n omega e^{-omega (s - t_n)}] m(s) ds,
    mu_b(s) = mu0 sum_n' phi((s - t_n')/tau_t) / tau_t (mu0 N when tau_t is infinite)."""
    t, r = np.asarray(t, float), np.asarray(r, float)
    mu0, tx, tt, th0, om, h = (float(v) for v in p)
    t0 = float(t.max())
    t1 = t0 + horizon
    xs, ws = np.polynomial.legendre.leggauss(n_quad)
    s = t0 + (xs + 1.0) * 0.5 * horizon
    w = ws * 0.5 * horizon
    m = (1.0 - th0 * np.exp(-om * (1.0 - th0) * (t1 - s))) / (1.0 - th0)
    if math.isinf(tt):
        mub = np.full_like(s, mu0 * t.size)
    else:
        mub = mu0 * np.sum(np.exp(-0.5 * ((s[:, None] - t[None, :]) / tt) ** 2), axis=1) / (tt * math.sqrt(2 * math.pi))
    exc = th0 * om * np.sum(np.exp(r[None, :] - om * (s[:, None] - t[None, :])), axis=1)
    return float(np.sum(w * (mub + exc) * m))
