"""CUDA path (through the C-ABI) vs the FP64 CPU oracle, element by element."""
import math

import numpy as np
import pytest

import oracle
from paper_2103_03348_b300 import synth
from parity_util import check, error_report, large_reference, rate_condition_scales, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def hawkes_mod():
    from paper_2103_03348_b300 import build, hawkes
    build.build()
    return hawkes


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), dtype=torch.float64, device="cuda")


def gpu_eval(w_or_arrays, params, prec, mode="hess", check_status=True):
    H = hawkes_mod()
    if hasattr(w_or_arrays, "x"):
        x, y, t, r = (dev(w_or_arrays.x), dev(w_or_arrays.y), dev(w_or_arrays.t), dev(w_or_arrays.r))
    else:
        x, y, t, r = (dev(a) for a in w_or_arrays)
    if mode == "loglik":
        return H.loglik(x, y, t, r, params, prec, check=check_status).item(), None, None
    if mode == "grad":
        ll, g = H.grad(x, y, t, r, params, prec, check=check_status)
        return ll.item(), g.cpu().numpy(), None
    ll, g, h = H.hess_diag(x, y, t, r, params, prec, check=check_status)
    return ll.item(), g.cpu().numpy(), h.cpu().numpy()


_ORACLE_CACHE = {}


def oracle_of(w, params=None):
    p = tuple(w.params if params is None else params)
    key = (w.name, w.n, p)
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = oracle.evaluate(w.x, w.y, w.t, w.r, np.array(p), want=2)
    return _ORACLE_CACHE[key]


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_st"])
@pytest.mark.parametrize("name", ["unit_square", "ebola_like"])
def test_workload_parity(name, prec):
    w = synth.make(name)
    ref = oracle_of(w)
    ll, g, h = gpu_eval(w, w.params, prec)
    check(prec, ll, g, h, ref, label=name)


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_st"])
def test_modes_agree(prec):
    w = synth.make("unit_square")
    ll0, _, _ = gpu_eval(w, w.params, prec, "loglik")
    ll1, g1, _ = gpu_eval(w, w.params, prec, "grad")
    ll2, g2, h2 = gpu_eval(w, w.params, prec, "hess")
    assert rel(ll0, ll2) <= 1e-14 and rel(ll1, ll2) <= 1e-14
    np.testing.assert_allclose(g1, g2, rtol=1e-13, atol=1e-13 * np.abs(g2).max())


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_st"])
@pytest.mark.parametrize("n", [2, 3, 127, 128, 129, 255, 257, 1000, 4099])
def test_ragged_sizes(n, prec):
    w = synth.make_uniform(100 + n, n, box=1.0, t_max=1.0, r_sd=0.5, params=(0.5, 0.2, 0.1, 0.3, 5.0, 0.05))
    ref = oracle_of(w)
    ll, g, h = gpu_eval(w, w.params, prec)
    check(prec, ll, g, h, ref, label=f"uniform N={n}")


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_band", "fp32c_st"])
def test_dense_burst_then_sparse_tail(prec):
    """A dense burst (1,000 events in one time unit) followed by a sparse tail
    (200 events over 29 units) under fast decay (omega = 3): time-order tiles
    whose time spans differ by two orders of magnitude, space-time groups that
    mix both parts, and r^ spreads within a tile from about 4 to about 80
    (base-2 units); every output against the oracle at its precision's bars.  (|t~|
    stays below 65 here: much longer spans at this decay put FP32's
    quantisation of t~ itself above the log-rate bar.)"""
    rng = np.random.default_rng(22)
    t = np.sort(np.concatenate([rng.uniform(0.0, 1.0, 1000), rng.uniform(1.0, 30.0, 200)]))
    x, y = rng.uniform(0.0, 1.0, t.size), rng.uniform(0.0, 1.0, t.size)
    r = rng.normal(0.0, 0.5, t.size)
    p = np.array([0.5, 0.2, 0.1, 0.3, 3.0, 0.05])
    spread = (r + 3.0 * t) * 1.4426950408889634
    assert np.ptp(spread[:128]) < 10 and np.ptp(spread[-128:]) > 60
    ref = oracle.evaluate(x, y, t, r, p, want=2)
    ll, g, h = gpu_eval((x, y, t, r), p, prec)
    check(prec, ll, g, h, ref, label=f"burst and tail {prec}")


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_st"])
def test_paper_background_without_temporal_bandwidth(prec):
    w = synth.make("unit_square")
    p = np.array(w.params)
    p[2] = math.inf
    ref = oracle_of(w, p)
    ll, g, h = gpu_eval(w, p, prec)
    assert g[2] == 0.0 and h[2] == 0.0
    check(prec, ll, g, h, ref, label="tau_t=inf")


def tie_and_duplicate_pattern(seed=5, n=700):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, n)
    y = rng.uniform(0, 1, n)
    t = np.round(rng.uniform(0, 1, n), 2)  # heavy ties in time
    src = rng.choice(n, 120, replace=False)
    dst = rng.choice(n, 120, replace=False)
    x[dst], y[dst] = x[src], y[src]  # exact duplicate locations
    x[:5] = 0.25; y[:5] = 0.75  # one location shared by five events
    r = rng.normal(0, 0.5, n)
    o = np.argsort(t, kind="stable")
    return x[o], y[o], t[o], r[o]


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_st"])
def test_ties_and_duplicate_locations(prec):
    x, y, t, r = tie_and_duplicate_pattern()
    p = np.array([0.5, 0.2, 0.1, 0.3, 5.0, 0.05])
    ref = oracle.evaluate(x, y, t, r, p, want=2)
    ll, g, h = gpu_eval((x, y, t, r), p, prec)
    check(prec, ll, g, h, ref, label="ties+duplicates")


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_st"])
@pytest.mark.parametrize("far", [6.0, 9.0])
def test_near_zero_intensity_rows(prec, far):
    # two events far from everything else: their intensities fall to about
    # 2^-85..2^-110 (far=6) or 2^-207..2^-240 (far=9, below FP32's range), both
    # below 2^-60, so the FP32C path recomputes those rows in FP64
    w = synth.make_uniform(77, 500, box=1.0, t_max=1.0, r_sd=0.3, params=(0.5, 0.5, 0.1, 0.3, 5.0, 0.05))
    x = np.append(w.x, [far + 0.5, far + 0.5])
    y = np.append(w.y, [0.5, far + 0.5])  # far from the cluster and from each other
    t = np.append(w.t, [0.3, 0.6])
    r = np.append(w.r, [0.0, 0.1])
    o = np.argsort(t, kind="stable")
    x, y, t, r = x[o], y[o], t[o], r[o]
    ref = oracle.evaluate(x, y, t, r, w.params, want=2)
    assert ref["status"] == 0 and ref["lam"].min() < 2.0 ** -60
    ll, g, h = gpu_eval((x, y, t, r), w.params, prec)
    check(prec, ll, g, h, ref, label=f"isolated far={far}")


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_st"])
def test_zero_intensity_status(prec):
    H = hawkes_mod()
    p = np.array([0.5, 0.01, 0.05, 0.3, 10.0, 0.01])
    x, y, t = np.array([0.0, 0.001, 1.0]), np.array([0.0, 0.0, 1.0]), np.array([0.1, 0.2, 0.3])
    r = np.zeros(3)
    assert oracle.evaluate(x, y, t, r, p, want=0)["status"] == 1
    with pytest.raises(FloatingPointError):
        gpu_eval((x, y, t, r), p, prec)
    ll, g, h = gpu_eval((x, y, t, r), p, prec, check_status=False)
    assert ll == -math.inf and np.all(np.isnan(g)) and np.all(np.isnan(h))
    del H


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_st"])
def test_invalid_data_status(prec):
    w = synth.make_uniform(9, 300, r_sd=0.2)
    t_bad = w.t.copy()
    t_bad[100], t_bad[101] = t_bad[101], t_bad[100] - 1.0
    with pytest.raises(ValueError):
        gpu_eval((w.x, w.y, t_bad, w.r), w.params, prec)
    x_bad = w.x.copy()
    x_bad[7] = np.nan
    with pytest.raises(ValueError):
        gpu_eval((x_bad, w.y, w.t, w.r), w.params, prec)
    ll, g, h = gpu_eval((x_bad, w.y, w.t, w.r), w.params, prec, check_status=False)
    assert math.isnan(ll) and np.all(np.isnan(g))
    # the workspace is reusable after an error
    ref = oracle_of(w)
    ll, g, h = gpu_eval(w, w.params, prec)
    check(prec, ll, g, h, ref, label="after error")


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_st"])
def test_bitwise_deterministic(prec):
    w = synth.make("unit_square")
    a = gpu_eval(w, w.params, prec)
    b = gpu_eval(w, w.params, prec)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


# ---------------------------------------------------------------------------
# Full size (100,000 events, the benchmark's workload and launch configuration)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def large():
    w = synth.make("large")
    ll, g, h = gpu_eval(w, w.params, "fp32c")
    return w, ll, g, h


def test_large_identities(large):
    """Exact identities that hold at any size: 1-homogeneity in (mu0, theta0)
    and the tie between the column sums and the theta0 row sums."""
    w, ll, g, h = large
    mu0, th0 = w.params[0], w.params[3]
    Lam = oracle.integral(w.t, w.r, w.params)
    assert rel(mu0 * g[0] + th0 * g[3], w.n - Lam) <= 1e-6
    assert rel(np.sum(g[6:]), th0 * g[3]) <= 1e-5
    assert h[0] <= 0 and h[3] <= 0 and np.all(h[6:] - g[6:] <= 1e-9)


@pytest.fixture(scope="module")
def large_ref():
    w = synth.make("large")
    return large_reference(w)


@pytest.mark.parametrize("prec", ["fp32c", "fp32c_band", "fp32c_st", "fp64"])
def test_large_full_parity_vs_oracle(large_ref, prec):
    """The benchmark's workload (100,000 events) in the benchmark's launch
    configuration against the full FP64 oracle evaluation stored by
    tests/golden/make_golden.py --large: loglik, the 12 global entries and every
    one of the 2 x 100,000 log-rate entries, early sources included, at the
    stated bars (FP64 1e-10 per entry; FP32C 1e-5 on loglik and the gradient
    norm, 1e-4 per global entry, the log-rate entry guard with its condition
    scale: a few entries of Eq. 4 cancel to 1/200 of their parts here)."""
    w = synth.make("large")
    ll, g, h = gpu_eval(w, w.params, prec)
    rep = error_report(ll, g, h, large_ref)
    print(f"N=100000 {prec} vs oracle: {rep}")
    check(prec, ll, g, h, large_ref, label="N=100000", cond=rate_condition_scales(w.t, w.r, w.params, large_ref))


def test_large_sampled_rates_vs_oracle(large, large_ref):
    """64 log-rate gradient and Hessian entries drawn over the whole range of
    sources (the earliest, whose column sums are the longest, included),
    recomputed one by one by oracle.rate_terms from the stored intensities."""
    w, ll, g, h = large
    rng = np.random.default_rng(4)
    idx = np.sort(np.concatenate([[0, 1, 2], rng.choice(np.arange(3, w.n - 1), 61, replace=False)]))
    g_ref, h_ref = oracle.rate_terms(w.x, w.y, w.t, w.r, w.params, large_ref["lam"], idx)
    scale_g = np.abs(g[6:]).max()
    assert np.max(np.abs(g[6 + idx] - g_ref) / np.maximum(np.abs(g_ref), 1e-3 * scale_g)) <= 2e-3
    assert np.linalg.norm(g[6 + idx] - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    assert np.linalg.norm(h[6 + idx] - h_ref) <= 1e-4 * np.linalg.norm(h_ref)


def test_large_fp32c_vs_fp64_path(large):
    """The FP64 GPU path (pinned to the oracle above at 2,000 and 23,422 events)
    against the FP32C path at full size."""
    w, ll, g, h = large
    ll64, g64, h64 = gpu_eval(w, w.params, "fp64")
    assert rel(ll, ll64) <= 1e-5
    assert np.linalg.norm(g - g64) <= 1e-5 * np.linalg.norm(g64)
    assert np.linalg.norm(h - h64) <= 1e-4 * np.linalg.norm(h64)


@pytest.mark.parametrize("name", ["ebola_like", "large"])
def test_band_skipping_is_bitwise_identical(name):
    """HAWKES_FP32C_BAND skips only tile pairs whose background terms are all
    exactly 0 in FP32, so every output equals HAWKES_FP32C's bit for bit."""
    w = synth.make(name)
    a = gpu_eval(w, w.params, "fp32c")
    b = gpu_eval(w, w.params, "fp32c_band")
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_band_skipping_with_infinite_tau_t():
    w = synth.make("unit_square")
    p = np.array(w.params)
    p[2] = math.inf
    a = gpu_eval(w, p, "fp32c")
    b = gpu_eval(w, p, "fp32c_band")
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_million_events_ragged():
    """1,048,653 events (8,193 tiles, a ragged tail of 77): the same exact
    identities, and 48 sampled log-rate gradient and Hessian entries recomputed
    one by one by the oracle, in both FP32C precisions (which must agree bit
    for bit)."""
    w = synth.make_large(seed=77, n=1_048_653)
    ll, g, h = gpu_eval(w, w.params, "fp32c")
    llb, gb, hb = gpu_eval(w, w.params, "fp32c_band")
    assert ll == llb and np.array_equal(g, gb) and np.array_equal(h, hb)
    assert np.isfinite(ll) and np.all(np.isfinite(g)) and np.all(np.isfinite(h))
    mu0, th0 = w.params[0], w.params[3]
    Lam = oracle.integral(w.t, w.r, w.params)
    assert rel(mu0 * g[0] + th0 * g[3], w.n - Lam) <= 1e-6
    assert rel(np.sum(g[6:]), th0 * g[3]) <= 1e-5
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(np.arange(w.n - 600, w.n - 1), 48, replace=False))
    later = np.arange(idx.min(), w.n)
    lam_later, _, _ = oracle.rows(w.x, w.y, w.t, w.r, w.params, later)
    lam = np.ones(w.n)
    lam[later] = lam_later
    g_ref, h_ref = oracle.rate_terms(w.x, w.y, w.t, w.r, w.params, lam, idx)
    scale_g = np.abs(g[6:]).max()
    assert np.max(np.abs(g[6 + idx] - g_ref) / np.maximum(np.abs(g_ref), 1e-3 * scale_g)) <= 2e-3
    assert np.linalg.norm(g[6 + idx] - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    assert np.linalg.norm(h[6 + idx] - h_ref) <= 1e-4 * np.linalg.norm(h_ref)


def test_four_million_events_spacetime():
    """4,194,305 events (32,769 tiles, a ragged tail of one event; 131,073
    32-event groups) on space-time tiles: every output finite, the exact
    identities, and 32 log-rate gradient and Hessian entries of late sources
    recomputed one by one by the oracle from intensities the oracle computes."""
    w = synth.make_large(seed=78, n=4_194_305)
    ll, g, h = gpu_eval(w, w.params, "fp32c_st")
    assert np.isfinite(ll) and np.all(np.isfinite(g)) and np.all(np.isfinite(h))
    mu0, th0 = w.params[0], w.params[3]
    Lam = oracle.integral(w.t, w.r, w.params)
    assert rel(mu0 * g[0] + th0 * g[3], w.n - Lam) <= 1e-6
    assert rel(np.sum(g[6:]), th0 * g[3]) <= 1e-5
    rng = np.random.default_rng(6)
    idx = np.sort(rng.choice(np.arange(w.n - 300, w.n - 1), 32, replace=False))
    later = np.arange(idx.min(), w.n)
    lam_later, _, _ = oracle.rows(w.x, w.y, w.t, w.r, w.params, later)
    lam = np.ones(w.n)
    lam[later] = lam_later
    g_ref, h_ref = oracle.rate_terms(w.x, w.y, w.t, w.r, w.params, lam, idx)
    scale_g = np.abs(g[6:]).max()
    assert np.max(np.abs(g[6 + idx] - g_ref) / np.maximum(np.abs(g_ref), 1e-3 * scale_g)) <= 2e-3
    assert np.linalg.norm(g[6 + idx] - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    assert np.linalg.norm(h[6 + idx] - h_ref) <= 1e-4 * np.linalg.norm(h_ref)


@pytest.fixture(scope="module")
def surrogate_workload():
    return synth.make("surrogate")


# a point of the posterior the surrogate's sampler explores (bandwidths well below the generating ones)
SURROGATE_POSTERIOR_POINT = (0.86, 6.7, 17.9, 0.144, 0.211, 3.59)


@pytest.mark.parametrize("point", ["generating", "posterior"])
def test_surrogate_configuration_at_full_size(surrogate_workload, point):
    """The learned surrogate's configuration at its full size (500,000 events:
    uniform background plus 500 hotspots, every log-rate 0), in the launch
    configuration its sampler uses (space-time tiles, the six globals read on
    the device as logarithms), at the generating values and at a point of the
    posterior it samples:
      * the globals-only gradient (the exact warm-up's call) and the
        log-likelihood (the accept step's call) agree with the full evaluation
        to rounding order (the same row sums);
      * the log-likelihood and the 12 global entries agree with the time-order
        FP32C path at the FP32C bars (two summation orders of the same terms,
        both pinned to the oracle at 100,000 events);
      * the exact identities: 1-homogeneity in (mu0, theta0) and the column
        sums against the theta0 row sums;
      * 48 log-rate gradient and Hessian entries of late sources, recomputed one
        by one by the oracle from intensities the oracle computes."""
    w = surrogate_workload
    p = np.array(w.params if point == "generating" else SURROGATE_POSTERIOR_POINT)
    H = hawkes_mod()
    x, y, t, r = dev(w.x), dev(w.y), dev(w.t), dev(w.r)
    ll, g, h = (v.cpu().numpy() for v in H.hess_diag(x, y, t, r, p, "fp32c_st"))
    ll = float(ll)
    q = dev(np.log(p))
    og = H._call("grad_globals", x, y, t, r, q, "fp32c_st", log_params=True)
    ol = H._call("loglik", x, y, t, r, q, "fp32c_st", log_params=True)
    assert rel(og["loglik"].item(), ll) <= 1e-14 and rel(ol["loglik"].item(), ll) <= 1e-14
    np.testing.assert_allclose(og["grad"][:6].cpu().numpy(), g[:6], rtol=1e-13, atol=1e-13 * np.abs(g[:6]).max())

    ll_t, g_t, h_t = gpu_eval(w, p, "fp32c")
    assert rel(ll, ll_t) <= 1e-6
    assert np.max(np.abs(g[:6] - g_t[:6]) / np.abs(g_t[:6])) <= 1e-5
    assert np.max(np.abs(h[:6] - h_t[:6]) / np.abs(h_t[:6])) <= 1e-4

    mu0, th0 = p[0], p[3]
    Lam = oracle.integral(w.t, w.r, p)
    assert rel(mu0 * g[0] + th0 * g[3], w.n - Lam) <= 1e-6
    assert rel(np.sum(g[6:]), th0 * g[3]) <= 1e-5

    rng = np.random.default_rng(9)
    idx = np.sort(rng.choice(np.arange(w.n - 600, w.n - 1), 48, replace=False))
    later = np.arange(idx.min(), w.n)
    lam_later, _, _ = oracle.rows(w.x, w.y, w.t, w.r, p, later)
    lam = np.ones(w.n)
    lam[later] = lam_later
    g_ref, h_ref = oracle.rate_terms(w.x, w.y, w.t, w.r, p, lam, idx)
    scale_g = np.abs(g[6:]).max()
    assert np.max(np.abs(g[6 + idx] - g_ref) / np.maximum(np.abs(g_ref), 1e-3 * scale_g)) <= 2e-3
    assert np.linalg.norm(g[6 + idx] - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    assert np.linalg.norm(h[6 + idx] - h_ref) <= 1e-4 * np.linalg.norm(h_ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_st"])
def test_reused_event_preparation(prec):
    """HAWKES_MODE_REUSE_EVENTS: a second call on the same events and workspace
    skips their preparation and gives the same results bit for bit, with new
    log-rates and parameters; a non-finite log-rate is still reported, and so
    is the earlier call's unsorted-time status."""
    H = hawkes_mod()
    w = synth.make_uniform(12, 3001, r_sd=0.4)
    x, y, t, r = dev(w.x), dev(w.y), dev(w.t), dev(w.r)
    ws = torch.empty(H.workspace_size(w.n, prec), dtype=torch.uint8, device="cuda")
    q = torch.tensor(np.log(w.params), dtype=torch.float64, device="cuda")
    H._call("hess", x, y, t, r, q, prec, workspace=ws, log_params=True)
    r2 = dev(w.r + 0.1)
    q2 = q + 0.05
    a = H._call("hess", x, y, t, r2, q2, prec, workspace=ws, log_params=True, reuse_events=True)
    a = {k: v.clone() for k, v in a.items()}
    b = H._call("hess", x, y, t, r2, q2, prec, log_params=True)  # fresh workspace, full preparation
    for k in ("loglik", "grad", "hdiag"):
        assert torch.equal(a[k], b[k]), k
    rn = w.r.copy()
    rn[17] = np.nan
    out = H._call("hess", x, y, t, dev(rn), q2, prec, workspace=ws, log_params=True, reuse_events=True, check=False)
    assert int(out["status"].item()) == H.ENONFINITE
    tu = w.t.copy()
    tu[[5, 6]] = tu[[6, 5]]
    ws2 = torch.empty_like(ws)
    H._call("hess", x, y, dev(tu), r, q, prec, workspace=ws2, log_params=True, check=False)
    out = H._call("hess", x, y, dev(tu), r, q, prec, workspace=ws2, log_params=True, reuse_events=True, check=False)
    assert int(out["status"].item()) == H.EUNSORTED
