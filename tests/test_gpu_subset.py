"""The rate-subset evaluation (hawkes_eval_rates_subset): the rate entries of a
chosen set of sources, with an O(N k) column pass in FP32C.

Checked against the full evaluation on the same inputs and against the oracle:
  * log-likelihood and the six global entries equal the full call's bit for bit
    (the row pass and its epilogue are the same code);
  * FP64 subset entries equal the full call's bit for bit (the FP64 column
    pass covers every source);
  * FP32C subset entries: the same Kahan-compensated FP32 sums, cut into
    chunks at different tile boundaries, so they agree with the full call to
    rounding and with the oracle to the FP32C bars.  Each tile adds up to 64
    packed pair terms in plain FP32 before compensation (relative error up to
    ~64 * 2^-24 = 4e-6 of the tile's sum); the gradient entry is held to 1e-5
    (scaled), the Hessian entry c1 - c2 - dLambda, which cancels by up to an
    order of magnitude, to 1e-4;
  * every other rate entry is left as it was;
  * an index outside [0, n) gives status EINVAL; k = 0 writes no rate entry."""
import numpy as np
import pytest

import oracle
from parity_util import FP32C_GNORM_TOL, FP32C_HNORM_TOL, FP32C_RATE_TOL, norm_rel, scaled_err
from paper_2103_03348_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SENTINEL = 12345.0
G_TOL, H_TOL = 1e-5, 1e-4  # subset against full FP32C call (see above)


def lib():
    from paper_2103_03348_b300 import build, hawkes
    build.build()
    return hawkes


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def run(H, w, prec, mode, idx, params=None):
    n = len(w.t)
    out = {"loglik": torch.empty((), dtype=torch.float64, device="cuda"),
           "grad": torch.full((6 + n,), SENTINEL, dtype=torch.float64, device="cuda"),
           "hdiag": torch.full((6 + n,), SENTINEL, dtype=torch.float64, device="cuda") if mode == "hess" else None,
           "status": torch.empty((), dtype=torch.int32, device="cuda")}
    p = dev(w.params if params is None else params)
    ri = None if idx is None else dev(idx, torch.int32)
    H._call(mode, dev(w.x), dev(w.y), dev(w.t), dev(w.r), p, prec, out=out, rate_idx=ri, check=False)
    g = out["grad"].cpu().numpy()
    h = out["hdiag"].cpu().numpy() if mode == "hess" else None
    return out["loglik"].item(), g, h, int(out["status"].item())


def subset(n, k, seed, sort=True):
    rng = np.random.default_rng(seed)
    idx = rng.choice(n, k, replace=False)
    return np.sort(idx) if sort else idx


@pytest.mark.parametrize("prec", ["fp32c", "fp32c_band", "fp64"])
@pytest.mark.parametrize("mode", ["grad", "hess"])
def test_subset_matches_full_and_oracle(prec, mode):
    H = lib()
    w = synth.make_large(n=3000, seed=4)
    n = len(w.t)
    idx = subset(n, 333, 1, sort=(mode == "hess"))  # ragged: 2 full blocks of 128 and a tail; unsorted for grad
    ll_f, g_f, h_f, st_f = run(H, w, prec, mode, None)
    ll_s, g_s, h_s, st_s = run(H, w, prec, mode, idx)
    assert st_f == 0 and st_s == 0
    assert ll_s == ll_f and np.array_equal(g_s[:6], g_f[:6])
    rest = np.setdiff1d(np.arange(n), idx)
    assert np.all(g_s[6 + rest] == SENTINEL)
    if mode == "hess":
        assert np.array_equal(h_s[:6], h_f[:6]) and np.all(h_s[6 + rest] == SENTINEL)
    pairs = [(g_s, g_f, G_TOL)] + ([(h_s, h_f, H_TOL)] if mode == "hess" else [])
    for a, b, tol in pairs:
        if prec == "fp64":
            assert np.array_equal(a[6 + idx], b[6 + idx])
        else:
            assert scaled_err(a[6 + idx], b[6 + idx]) <= tol
    if prec != "fp64":
        ref = oracle.evaluate(w.x, w.y, w.t, w.r, w.params, want=2 if mode == "hess" else 1)
        assert scaled_err(g_s[6 + idx], ref["grad"][6 + idx]) <= FP32C_RATE_TOL
        assert norm_rel(g_s[6 + idx], ref["grad"][6 + idx]) <= 10 * FP32C_GNORM_TOL
        if mode == "hess":
            assert norm_rel(h_s[6 + idx], ref["hdiag"][6 + idx]) <= FP32C_HNORM_TOL


def test_subset_of_the_sampler_shape():
    """A subset spread over the whole index range (every seventh event) on the
    23,422-event pattern, against the full FP32C call and the oracle."""
    H = lib()
    w = synth.make_ebola_like(m_seq=0)
    n = len(w.t)
    idx = np.arange(3, n, 7)
    ll_f, g_f, h_f, _ = run(H, w, "fp32c", "hess", None)
    ll_s, g_s, h_s, st = run(H, w, "fp32c", "hess", idx)
    assert st == 0 and ll_s == ll_f
    assert scaled_err(g_s[6 + idx], g_f[6 + idx]) <= G_TOL
    assert scaled_err(h_s[6 + idx], h_f[6 + idx]) <= H_TOL
    ref = oracle.evaluate(w.x, w.y, w.t, w.r, w.params, want=2)
    assert scaled_err(g_s[6 + idx], ref["grad"][6 + idx]) <= FP32C_RATE_TOL
    assert norm_rel(h_s[6 + idx], ref["hdiag"][6 + idx]) <= FP32C_HNORM_TOL


def test_subset_edge_cases():
    H = lib()
    w = synth.make_large(n=700, seed=2)
    n = len(w.t)
    ll_f, g_f, h_f, _ = run(H, w, "fp32c", "hess", None)
    # k = 0: no rate entry written
    ll, g, h, st = run(H, w, "fp32c", "hess", np.zeros(0, np.int32))
    assert st == 0 and ll == ll_f and np.array_equal(g[:6], g_f[:6])
    assert np.all(g[6:] == SENTINEL) and np.all(h[6:] == SENTINEL)
    # every source, and the last source alone (no later target: its sum is 0)
    ll, g, h, st = run(H, w, "fp32c", "hess", np.arange(n))
    assert st == 0 and scaled_err(g[6:], g_f[6:]) <= G_TOL and scaled_err(h[6:], h_f[6:]) <= H_TOL
    ll, g, h, st = run(H, w, "fp32c", "hess", np.array([n - 1]))
    assert st == 0 and g[6 + n - 1] == g_f[6 + n - 1] and h[6 + n - 1] == h_f[6 + n - 1]
    # an index outside [0, n): status EINVAL, in both precisions
    from paper_2103_03348_b300.hawkes import EINVAL
    for prec in ("fp32c", "fp64"):
        for bad in (n, -1):
            _, _, _, st = run(H, w, prec, "hess", np.array([0, 5, bad, 9]))
            assert st == EINVAL, (prec, bad, st)
    # the binding refuses a host parameter vector or a globals-only mode
    with pytest.raises(ValueError):
        H._call("hess", dev(w.x), dev(w.y), dev(w.t), dev(w.r), w.params, "fp32c", rate_idx=dev([0], torch.int32))
    with pytest.raises(ValueError):
        H._call("hess_globals", dev(w.x), dev(w.y), dev(w.t), dev(w.r), dev(w.params), "fp32c",
                rate_idx=dev([0], torch.int32))
