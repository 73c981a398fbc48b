"""Randomised parity against the oracle: 40 seeded problems with varied sizes
(2 to 700 events, ragged tails), parameters spread over orders of magnitude,
clustered and uniform events, exact ties in time and repeated locations, and
spread log-rates.  FP64 is held to 1e-10, FP32C and its band-skipping form to
the stated FP32C bars; the band form must also equal FP32C bit for bit, and the
space-time form meets the FP32C bars.

Seed 32 has two events whose intensity is about 7e-303 at tau_x = 6e-4: an
extended-precision (60-digit) evaluation of those rows' Hessian terms agrees
with the oracle to 2e-13, so the oracle holds there; the GPU's FP64 path once
took its moments in raw units (G d^4 near 1e-315, deep in FP64's subnormal
range) and was off by 1e-7 on the tau_x entry.  Its moments are now in the
kernels' scaled units and every output is held to 1e-10, that case included."""
import math

import numpy as np
import pytest

import oracle
from parity_util import (FP32C_GNORM_TOL, FP32C_HNORM_TOL, FP32C_LL_TOL, FP64_TOL, norm_rel, rel,
                         scaled_err)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def problem(seed):
    rng = np.random.default_rng(10_000 + seed)
    n = int(rng.choice([2, 3, 17, 128, 129, 255, int(rng.integers(4, 700))]))
    box, t_max = 10.0 ** rng.uniform(-1, 3), 10.0 ** rng.uniform(-1, 3)
    # clustered events around a few centres, plus uniform ones
    k = int(rng.integers(1, 6))
    cx, cy = rng.uniform(0, box, k), rng.uniform(0, box, k)
    which = rng.integers(0, k, n)
    spread = box * 10.0 ** rng.uniform(-3, -0.5)
    x = np.where(rng.uniform(size=n) < 0.7, cx[which] + spread * rng.standard_normal(n), rng.uniform(0, box, n))
    y = np.where(rng.uniform(size=n) < 0.7, cy[which] + spread * rng.standard_normal(n), rng.uniform(0, box, n))
    t = rng.uniform(0, t_max, n)
    if n > 4 and rng.uniform() < 0.5:  # exact ties in time
        idx = rng.choice(n, n // 5, replace=False)
        t[idx] = t[rng.choice(n, len(idx))]
    if n > 4 and rng.uniform() < 0.5:  # repeated locations
        idx = rng.choice(n, n // 6, replace=False)
        src = rng.choice(n, len(idx))
        x[idx], y[idx] = x[src], y[src]
    order = np.argsort(t, kind="stable")
    x, y, t = x[order], y[order], t[order]
    r = rng.normal(0.0, rng.uniform(0.0, 1.0), n)
    # bandwidths relative to the extent; rates relative to the time span
    tx = box * 10.0 ** rng.uniform(-2.5, -0.3)
    h = box * 10.0 ** rng.uniform(-2.5, -0.3)
    tt = math.inf if rng.uniform() < 0.15 else t_max * 10.0 ** rng.uniform(-2, 0)
    om = 10.0 ** rng.uniform(-1, 1.5) / max(t_max / max(n, 1), 1e-6)
    params = np.array([10.0 ** rng.uniform(-2, 1), tx, tt, 10.0 ** rng.uniform(-3, 0), om, h])
    return x, y, t, r, params


def gpu(x, y, t, r, params, prec):
    from paper_2103_03348_b300 import hawkes
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    ll, g, h = hawkes.hess_diag(d(x), d(y), d(t), d(r), params, prec, check=False)
    return ll.item(), g.cpu().numpy(), h.cpu().numpy()


@pytest.mark.parametrize("seed", range(40))
def test_random_problem(seed):
    from paper_2103_03348_b300 import build
    build.build()
    x, y, t, r, params = problem(seed)
    ref = oracle.evaluate(x, y, t, r, params, want=2)
    if not np.isfinite(ref["loglik"]):
        pytest.skip("an event with zero intensity (the status test covers it)")
    ll, g, h = gpu(x, y, t, r, params, "fp64")
    assert rel(ll, ref["loglik"]) <= FP64_TOL
    assert scaled_err(g, ref["grad"]) <= FP64_TOL
    assert scaled_err(h, ref["hdiag"]) <= FP64_TOL, (scaled_err(h, ref["hdiag"]), ref["lam"].min())
    ll, g, h = gpu(x, y, t, r, params, "fp32c")
    assert rel(ll, ref["loglik"]) <= FP32C_LL_TOL, (ll, ref["loglik"], params)
    assert norm_rel(g, ref["grad"]) <= FP32C_GNORM_TOL, (norm_rel(g, ref["grad"]), params)
    assert norm_rel(h, ref["hdiag"]) <= FP32C_HNORM_TOL, (norm_rel(h, ref["hdiag"]), params)
    llb, gb, hb = gpu(x, y, t, r, params, "fp32c_band")
    assert llb == ll and np.array_equal(gb, g) and np.array_equal(hb, h)
    # space-time tiles: the same FP32 terms in another order, with dead group pairs skipped
    ll, g, h = gpu(x, y, t, r, params, "fp32c_st")
    assert rel(ll, ref["loglik"]) <= FP32C_LL_TOL, (ll, ref["loglik"], params)
    assert norm_rel(g, ref["grad"]) <= FP32C_GNORM_TOL, (norm_rel(g, ref["grad"]), params)
    assert norm_rel(h, ref["hdiag"]) <= FP32C_HNORM_TOL, (norm_rel(h, ref["hdiag"]), params)
