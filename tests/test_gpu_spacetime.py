"""HAWKES_FP32C_ST (space-time tiles with group pruning) beyond the parity
suite, which runs it against the oracle on every small workload.

The space-time mode evaluates the same FP32 pair terms as FP32C, in another
order, and skips only group pairs whose terms all underflow to exactly 0; so
at any size it must agree with the FP32C path (itself pinned to the oracle)
to rounding: log-likelihood within 1e-6 relative, gradient within 1e-5 and
Hessian diagonal within 1e-4 (scaled: the Hessian entries are differences
that cancel), and with the oracle to the FP32C bars where the oracle can
follow.  Workloads where pruning removes most of the work (small bandwidths
on a wide domain) check that nothing live is skipped."""
import math

import numpy as np
import pytest

import oracle
from parity_util import (FP32C_GLOBAL_TOL, FP32C_GNORM_TOL, FP32C_HNORM_TOL, FP32C_LL_TOL, FP32C_RATE_TOL, norm_rel,
                         rel, scaled_err)
from paper_2103_03348_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LL_TOL, G_TOL, H_TOL = 1e-6, 1e-5, 1e-4  # FP32C_ST against FP32C (summation order only)


def H():
    from paper_2103_03348_b300 import build, hawkes
    build.build()
    return hawkes


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def evaluate(w, params, prec, mode="hess"):
    h = H()
    x, y, t, r = dev(w.x), dev(w.y), dev(w.t), dev(w.r)
    o = h._call(mode, x, y, t, r, params, prec)
    g = o["grad"].cpu().numpy() if o.get("grad") is not None else None
    hd = o["hdiag"].cpu().numpy() if o.get("hdiag") is not None else None
    return o["loglik"].item(), g, hd


def agree(a, b):
    assert rel(a[0], b[0]) <= LL_TOL, (a[0], b[0])
    assert scaled_err(a[1], b[1]) <= G_TOL, scaled_err(a[1], b[1])
    if a[2] is not None:
        assert scaled_err(a[2], b[2]) <= H_TOL, scaled_err(a[2], b[2])


@pytest.mark.parametrize("name", ["ebola_like", "large"])
def test_agrees_with_fp32c_at_full_size(name):
    w = synth.make(name)
    agree(evaluate(w, w.params, "fp32c_st"), evaluate(w, w.params, "fp32c"))


def test_agrees_with_fp32c_at_a_million_events():
    w = synth.make_large(seed=77, n=1_048_653)
    a = evaluate(w, w.params, "fp32c_st")
    b = evaluate(w, w.params, "fp32c")
    agree(a, b)
    assert np.all(np.isfinite(a[1])) and np.all(np.isfinite(a[2]))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_heavily_pruned_workload_vs_oracle(seed):
    """9,000 events on a 5,000 km square over 3 years with 20 km / 5 km
    bandwidths: almost every group pair is dead.  Against the oracle, the
    log-likelihood and the gradient and Hessian norms meet the FP32C bars; per
    log-rate entry, FP32 coordinates on so wide a domain (5,000 km against a
    5 km bandwidth) cost both FP32C paths the same few 1e-3, so the space-time
    entries are held to the plain FP32C path's own error (and agree with it to
    rounding)."""
    rng = np.random.default_rng(300 + seed)
    n = 9000
    x, y = rng.uniform(0, 5000, n), rng.uniform(0, 5000, n)
    k = rng.integers(0, 40, n)  # a share of the events around 40 centres
    cx, cy = rng.uniform(0, 5000, 40), rng.uniform(0, 5000, 40)
    near = rng.uniform(size=n) < 0.6
    x = np.where(near, cx[k] + rng.normal(0, 15, n), x)
    y = np.where(near, cy[k] + rng.normal(0, 15, n), y)
    t = np.sort(rng.uniform(0, 1100, n))
    r = rng.normal(0, 0.5, n)
    params = np.array([0.5, 20.0, 30.0, 0.5, 0.1, 5.0])
    if seed == 2:
        params[2] = math.inf  # background without a temporal kernel: space alone prunes
    w = synth.Workload(f"pruned_{seed}", x, y, t, r, params, np.arange(n))
    ref = oracle.evaluate(x, y, t, r, params, want=2)
    st = evaluate(w, params, "fp32c_st")
    plain = evaluate(w, params, "fp32c")
    agree(st, plain)
    assert rel(st[0], ref["loglik"]) <= FP32C_LL_TOL
    assert norm_rel(st[1], ref["grad"]) <= FP32C_GNORM_TOL
    assert norm_rel(st[2], ref["hdiag"]) <= FP32C_HNORM_TOL
    for a, b, key in ((st[1], plain[1], "grad"), (st[2], plain[2], "hdiag")):
        assert scaled_err(a[:6], ref[key][:6]) <= FP32C_GLOBAL_TOL
        assert scaled_err(a[6:], ref[key][6:]) <= 1.1 * scaled_err(b[6:], ref[key][6:]) + 1e-6


def test_subset_and_reuse():
    """The rate-subset call and event reuse in the space-time mode."""
    h = H()
    w = synth.make_ebola_like(m_seq=0)
    n = w.n
    x, y, t, r = dev(w.x), dev(w.y), dev(w.t), dev(w.r)
    q = dev(np.log(w.params))
    ws = torch.empty(h.workspace_size(n, "fp32c_st"), dtype=torch.uint8, device="cuda")
    full = h._call("hess", x, y, t, r, q, "fp32c_st", workspace=ws, log_params=True)
    full = {k: v.clone() for k, v in full.items()}
    idx = np.sort(np.random.default_rng(3).choice(n, 1610, replace=False))
    out = {"loglik": torch.empty((), dtype=torch.float64, device="cuda"),
           "grad": torch.full((6 + n,), 7.0, dtype=torch.float64, device="cuda"),
           "hdiag": torch.full((6 + n,), 7.0, dtype=torch.float64, device="cuda"),
           "status": torch.empty((), dtype=torch.int32, device="cuda")}
    h._call("hess", x, y, t, r, q, "fp32c_st", workspace=ws, log_params=True, reuse_events=True, out=out,
            rate_idx=dev(idx, torch.int32))
    g, hd = out["grad"].cpu().numpy(), out["hdiag"].cpu().numpy()
    gf, hf = full["grad"].cpu().numpy(), full["hdiag"].cpu().numpy()
    assert out["loglik"].item() == full["loglik"].item() and np.array_equal(g[:6], gf[:6])
    assert scaled_err(g[6 + idx], gf[6 + idx]) <= G_TOL and scaled_err(hd[6 + idx], hf[6 + idx]) <= H_TOL
    rest = np.setdiff1d(np.arange(n), idx)
    assert np.all(g[6 + rest] == 7.0) and np.all(hd[6 + rest] == 7.0)
    ref = oracle.evaluate(w.x, w.y, w.t, w.r, w.params, want=2)
    assert scaled_err(g[6 + idx], ref["grad"][6 + idx]) <= FP32C_RATE_TOL
    assert norm_rel(hd[6 + idx], ref["hdiag"][6 + idx]) <= FP32C_HNORM_TOL
    # an index outside [0, n) is reported
    bad = dev(np.array([0, n, 5]), torch.int32)
    o2 = h._call("hess", x, y, t, r, q, "fp32c_st", workspace=ws, log_params=True, reuse_events=True, rate_idx=bad,
                 check=False)
    assert int(o2["status"].item()) == h.EINVAL


def test_shards_refuse_spacetime():
    h = H()
    from paper_2103_03348_b300 import shard
    w = synth.make("unit_square")
    with pytest.raises(Exception):
        shard.evaluate(dev(w.x), dev(w.y), dev(w.t), dev(w.r), w.params, "fp32c_st", 2, "hess")
    assert h.workspace_size(w.n, "fp32c_st") > h.workspace_size(w.n, "fp32c")


def test_live_pair_counts():
    """hawkes_st_live_pairs (the roofline count of the space-time passes): with
    bandwidths as wide as the domain nothing is pruned and the row pass's
    background count is every ordered pair (self pairs included, padding
    excluded), n^2; its excitation and column counts cover at least the causal
    pairs; with narrow bandwidths on a wide domain every count shrinks (the
    background's by more than 5x)."""
    from paper_2103_03348_b300 import build, hawkes, synth
    build.build()
    n = 5000
    wide = synth.make_uniform(3, n, box=10.0, t_max=10.0, r_sd=0.3, params=(0.5, 100.0, 1e4, 0.3, 1e-3, 100.0))
    narrow = synth.make_uniform(3, n, box=2000.0, t_max=1e4, r_sd=0.3, params=(0.5, 2.0, 1.0, 0.3, 10.0, 2.0))
    counts = {}
    for name, w in (("wide", wide), ("narrow", narrow)):
        d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
        ws = torch.empty(hawkes.workspace_size(n, "fp32c_st"), dtype=torch.uint8, device="cuda")
        hawkes._call("hess", d(w.x), d(w.y), d(w.t), d(w.r), w.params, "fp32c_st", workspace=ws, check=False)
        counts[name] = hawkes.st_live_pairs(n, ws)
    c = counts["wide"]
    assert c["row_background_pairs"] == n * n
    assert n * (n - 1) // 2 <= c["row_excitation_pairs"] <= n * n
    assert n * (n - 1) // 2 <= c["column_pairs"] <= n * n
    c2 = counts["narrow"]
    # the background prunes by space and time; the excitation and column bounds compare a
    # group's latest source with its earliest target, and a group spans its slab's time range,
    # so inside a slab they prune by space alone
    assert 0 < c2["row_background_pairs"] < c["row_background_pairs"] // 5
    assert 0 < c2["row_excitation_pairs"] < c["row_excitation_pairs"]
    assert 0 <= c2["column_pairs"] < c["column_pairs"]
