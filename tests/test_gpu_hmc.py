"""GPU HMC pieces (posterior assembly, leapfrog kernels, accept step, sampler) vs the oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import hmc_oracle, tree_oracle
from paper_2103_03348_b300 import synth
from parity_util import FP64_TOL, norm_rel, scaled_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def problem(n=600, m=40, seed=11):
    w = synth.make_ebola_like(seed=seed, n=n, m_seq=m, box=120.0, t_max=120.0, n_hot=4)
    prec = tree_oracle.precision_matrix(w.tree_parent, w.tree_length)
    return w, prec


def make_post(w, prec, precision):
    from paper_2103_03348_b300 import build, hmc
    build.build()
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")  # noqa: E731
    post = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), torch.tensor(w.sequenced, device="cuda"),
                         d(prec), hmc.prior_km_days(), precision)
    return post, hmc


@pytest.mark.parametrize("precision", ["fp64", "fp32c", "fp32c_st"])
def test_posterior_parity(precision):
    w, prec = problem()
    post, hmc = make_post(w, prec, precision)
    q = np.concatenate([np.log(w.params), w.r[w.sequenced]])
    q[6:] += np.random.default_rng(0).normal(0, 0.3, len(q) - 6)
    ev = post.evaluate(torch.tensor(q, dtype=torch.float64, device="cuda"), want_hess=True)
    lp, g, h = ev["logpost"].item(), ev["grad"].cpu().numpy(), ev["hdiag"].cpu().numpy()
    ref = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, hmc.prior_km_days().as_tuple(), q)
    if precision == "fp64":
        assert abs(lp - ref[0]) <= FP64_TOL * abs(ref[0])
        assert scaled_err(g, ref[1]) <= FP64_TOL and scaled_err(h, ref[2]) <= FP64_TOL
    else:
        assert abs(lp - ref[0]) <= 1e-5 * abs(ref[0])
        assert norm_rel(g, ref[1]) <= 1e-5 and norm_rel(h, ref[2]) <= 1e-4


def test_leapfrog_trajectory_parity():
    w, prec = problem()
    post, hmc = make_post(w, prec, "fp64")
    prior = hmc.prior_km_days().as_tuple()
    rng = np.random.default_rng(1)
    q0 = np.concatenate([np.log(w.params), w.r[w.sequenced]])
    dim = len(q0)
    _, _, h0 = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, prior, q0)
    minv = 1.0 / np.maximum(-h0, 1e-2)
    p0 = rng.normal(size=dim) / np.sqrt(minv)
    eps, steps = 0.05, 20

    def gf(q):
        lp, g, _ = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, prior, q, want_hess=False)
        return lp, g

    q_ref, p_ref, lp_ref, _ = hmc_oracle.leapfrog(q0, p0, eps, steps, minv, gf)
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    q, p, mi = d(q0), d(p0), d(minv)
    g0 = post.evaluate(q)["grad"].clone()
    scratch = {"logpost": torch.empty((), dtype=torch.float64, device="cuda"),
               "grad": torch.empty(dim, dtype=torch.float64, device="cuda")}
    ev = hmc.leapfrog(post, q, p, g0, eps, steps, mi, scratch)
    assert np.max(np.abs(q.cpu().numpy() - q_ref)) <= 1e-9
    assert np.max(np.abs(p.cpu().numpy() - p_ref) / np.maximum(np.abs(p_ref), 1.0)) <= 1e-8
    assert abs(ev["logpost"].item() - lp_ref) <= 1e-9 * abs(lp_ref)


def test_dense_mass_leapfrog_trajectory_parity():
    """A 20-step trajectory with a dense mass over the 46 coordinates of a small
    Hawkes posterior (FP64 likelihood) against the oracle's dense-mass leapfrog."""
    w, prec = problem()
    post, hmc = make_post(w, prec, "fp64")
    prior = hmc.prior_km_days().as_tuple()
    rng = np.random.default_rng(2)
    q0 = np.concatenate([np.log(w.params), w.r[w.sequenced]])
    dim = len(q0)
    _, _, h0 = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, prior, q0)
    s = np.sqrt(np.maximum(-h0, 1e-2))
    C = rng.normal(size=(dim, dim)) * 0.1
    M = np.outer(s, s) * (np.eye(dim) + 0.5 * (C + C.T) @ (C + C.T).T / dim)  # SPD, dense
    op = hmc.DenseMassOp(dim, "cuda")
    op.set(M)
    minv = np.linalg.inv(op.M)
    p0 = np.linalg.cholesky(op.M) @ rng.normal(size=dim)
    eps, steps = 0.05, 20

    def gf(q):
        lp, g, _ = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, prior, q, want_hess=False)
        return lp, g

    q_ref, p_ref, lp_ref, _ = hmc_oracle.leapfrog(q0, p0, eps, steps, minv, gf)
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    q, p = d(q0), d(p0)
    g0 = post.evaluate(q)["grad"].clone()
    scratch = {"logpost": torch.empty((), dtype=torch.float64, device="cuda"),
               "grad": torch.empty(dim, dtype=torch.float64, device="cuda")}
    ev = hmc.leapfrog(post, q, p, g0, eps, steps, op, scratch)
    assert np.max(np.abs(q.cpu().numpy() - q_ref)) <= 1e-9
    assert np.max(np.abs(p.cpu().numpy() - p_ref) / np.maximum(np.abs(p_ref), 1.0)) <= 1e-8
    assert abs(ev["logpost"].item() - lp_ref) <= 1e-9 * abs(lp_ref)
    k = torch.empty((), dtype=torch.float64, device="cuda")
    hmc.kinetic(p, op, k)
    assert abs(k.item() - hmc_oracle.kinetic(p_ref, minv)) <= 1e-9 * hmc_oracle.kinetic(p_ref, minv)


class GaussPost:
    """A Gaussian target with known moments, in the Posterior interface."""

    def __init__(self, sig):
        self.sig = sig
        self.dim = sig.numel()
        self.calls = {"grad": 0, "hess": 0}

    def evaluate(self, q, want_hess=False, out=None):
        if out is None:
            out = {"logpost": torch.empty((), dtype=torch.float64, device=q.device),
                   "grad": torch.empty_like(q), "hdiag": torch.empty_like(q)}
        out["logpost"].copy_(-0.5 * torch.sum((q / self.sig) ** 2))
        out["grad"].copy_(-q / self.sig ** 2)
        if want_hess:
            out["hdiag"].copy_(-1.0 / self.sig ** 2)
        self.calls["hess" if want_hess else "grad"] += 1
        return out

    def status(self):
        return 0


def test_sampler_recovers_gaussian_moments():
    from paper_2103_03348_b300 import build, hmc
    build.build()
    sig = torch.logspace(-1.5, 1.0, 20, dtype=torch.float64, device="cuda")
    post = GaussPost(sig)
    q0 = torch.zeros(20, dtype=torch.float64, device="cuda") + 0.3 * sig
    ch = hmc.sample(post, q0, n_iter=1500, n_warmup=300, n_steps=10, eps0=0.1, mass_every=50, seed=3)
    s = sig.cpu().numpy()
    ess = hmc.ess_all(ch.draws)
    mean, var = ch.draws.mean(0), ch.draws.var(0)
    assert 0.5 < ch.accept.mean() <= 1.0
    assert np.all(np.abs(mean) <= 5 * s / np.sqrt(ess))
    assert np.all(np.abs(var / s ** 2 - 1) <= 5 * np.sqrt(2 / ess) + 0.05)


class DenseGaussPost(GaussPost):
    """A correlated Gaussian target (precision P) with known moments."""

    def __init__(self, cov):
        self.cov = cov
        self.P = torch.linalg.inv(cov)
        self.dim = cov.shape[0]
        self.calls = {"grad": 0, "hess": 0}

    def evaluate(self, q, want_hess=False, out=None):
        if out is None:
            out = {"logpost": torch.empty((), dtype=torch.float64, device=q.device),
                   "grad": torch.empty_like(q), "hdiag": torch.empty_like(q)}
        Pq = self.P @ q
        out["logpost"].copy_(-0.5 * torch.dot(q, Pq))
        out["grad"].copy_(-Pq)
        if want_hess:
            out["hdiag"].copy_(-torch.diagonal(self.P))
        self.calls["hess" if want_hess else "grad"] += 1
        return out


def test_dense_mass_kernels_vs_numpy():
    """hawkes_hmc_position_dense and hawkes_hmc_kinetic_dense against their
    definitions, q += eps M^-1 p and 1/2 p^T M^-1 p."""
    from paper_2103_03348_b300 import build, hmc
    build.build()
    rng = np.random.default_rng(8)
    for k in (1, 6, 33, 64):
        A = rng.normal(size=(k, k))
        M = A @ A.T + k * np.eye(k)
        op = hmc.DenseMassOp(k, "cuda")
        op.set(M)
        q0, p0 = rng.normal(size=k), rng.normal(size=k)
        q = torch.tensor(q0, device="cuda")
        p = torch.tensor(p0, device="cuda")
        op.position(q, p, 0.37)
        mi = np.linalg.inv(M)
        assert np.allclose(q.cpu().numpy(), q0 + 0.37 * mi @ p0, rtol=1e-12, atol=1e-12)
        out = torch.empty((), dtype=torch.float64, device="cuda")
        op.kinetic(p, out)
        assert abs(out.item() - 0.5 * p0 @ mi @ p0) <= 1e-12 * abs(0.5 * p0 @ mi @ p0)
        # p = chol(M) xi has covariance M
        xi = torch.randn(k, 4000, dtype=torch.float64, device="cuda")
        P = (op.chol @ xi).cpu().numpy()
        assert np.allclose(np.cov(P), M, rtol=0.0, atol=0.12 * np.abs(M).max())


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_dense_mass_sampler_recovers_correlated_gaussian(jitter):
    """mass='dense' (central-difference Hessian, running average) on a 6-D
    Gaussian with correlations up to 0.97 and scales over two decades: means
    and covariances recovered, and the slowest coordinate's ESS above the
    diagonal mass's from the same start (with and without step-size jitter)."""
    from paper_2103_03348_b300 import build, hmc
    build.build()
    rng = np.random.default_rng(12)
    sd = np.array([0.05, 0.2, 1.0, 3.0, 0.5, 0.1])
    C = np.full((6, 6), 0.0)
    C[0, 3] = C[3, 0] = 0.97
    C[1, 2] = C[2, 1] = -0.9
    C[4, 5] = C[5, 4] = 0.8
    C += np.eye(6)
    cov = torch.tensor(C * np.outer(sd, sd), device="cuda")
    post = DenseGaussPost(cov)
    q0 = torch.tensor(0.5 * sd, device="cuda")
    ch = hmc.sample(post, q0, n_iter=1500, n_warmup=300, n_steps=10, eps0=0.1, mass_every=50, seed=4, mass="dense",
                    jitter=jitter)
    ess = hmc.ess_all(ch.draws)
    assert 0.5 < ch.accept.mean() <= 1.0
    s = sd
    assert np.all(np.abs(ch.draws.mean(0)) <= 5 * s / np.sqrt(ess))
    # each covariance entry is the mean of z = (q_i - m_i)(q_j - m_j): held to 5 of its
    # own Monte Carlo standard errors (HMC can be antithetic for the means but not for z)
    xc = ch.draws - ch.draws.mean(0)
    for i in range(6):
        for j in range(i + 1):
            z = xc[:, i] * xc[:, j]
            mcse = z.std() / np.sqrt(min(hmc.ess(z), len(z)))
            assert abs(z.mean() - C[i, j] * s[i] * s[j]) <= 5 * mcse + 1e-3 * s[i] * s[j], (i, j)
    post.calls = {"grad": 0, "hess": 0}
    ch_d = hmc.sample(post, q0, n_iter=1500, n_warmup=300, n_steps=10, eps0=0.1, mass_every=50, seed=4,
                      jitter=jitter)
    assert ess.min() > 1.5 * hmc.ess_all(ch_d.draws).min()


def test_short_chain_on_hawkes_posterior():
    w, prec = problem()
    post, hmc = make_post(w, prec, "fp32c")
    q0 = torch.tensor(np.concatenate([np.log(w.params), w.r[w.sequenced]]), dtype=torch.float64, device="cuda")
    ch = hmc.sample(post, q0, n_iter=150, n_warmup=150, n_steps=20, eps0=0.02, mass_every=50, seed=5)
    assert np.all(np.isfinite(ch.logpost))
    assert 0.4 < ch.accept.mean() <= 1.0
    # divergent warm-up trajectories stop early; one eager trajectory precedes the graph capture
    assert 0.8 * 300 * 20 <= post.calls["grad"] <= 301 * 20


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
@pytest.mark.parametrize("prior_form", ["dense", "tree"])
def test_posterior_with_trend_parity(precision, prior_form):
    """theta_s = exp(z_s + beta^T f(t_s)) (Section 2.2): state (log globals, z, beta)."""
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    w, prec = problem()
    F = hmc.trend_features(w.t[w.sequenced], degree=2)
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")  # noqa: E731
    seq = torch.tensor(w.sequenced, device="cuda")
    kw = dict(trend=d(F), beta_var=0.25)
    if prior_form == "dense":
        post = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), seq, d(prec), hmc.prior_km_days(), precision, **kw)
    else:
        tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0)
        post = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), seq, None, hmc.prior_km_days(), precision, tree=tp,
                             **kw)
    assert post.dim == 6 + len(w.sequenced) + 2
    q = np.concatenate([np.log(w.params), w.r[w.sequenced], [0.2, -0.05]])
    q[6:6 + len(w.sequenced)] += np.random.default_rng(3).normal(0, 0.2, len(w.sequenced))
    ev = post.evaluate(d(q), want_hess=True)
    lp, g, h = ev["logpost"].item(), ev["grad"].cpu().numpy(), ev["hdiag"].cpu().numpy()
    ref = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, hmc.prior_km_days().as_tuple(), q,
                                   trend=F, beta_var=0.25)
    if precision == "fp64":
        assert abs(lp - ref[0]) <= FP64_TOL * abs(ref[0])
        assert scaled_err(g, ref[1]) <= FP64_TOL and scaled_err(h, ref[2]) <= FP64_TOL
    else:
        assert abs(lp - ref[0]) <= 1e-5 * abs(ref[0])
        assert norm_rel(g, ref[1]) <= 1e-5 and norm_rel(h, ref[2]) <= 1e-4
    lp_only = {"logpost": torch.empty((), dtype=torch.float64, device="cuda")}
    post.logpost_only(d(q), lp_only)
    assert abs(lp_only["logpost"].item() - lp) <= 1e-12 * abs(lp)


def test_short_chain_with_trend():
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    w, prec = problem()
    F = hmc.trend_features(w.t[w.sequenced], degree=1)
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")  # noqa: E731
    tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0)
    post = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), torch.tensor(w.sequenced, device="cuda"), None,
                         hmc.prior_km_days(), "fp32c", tree=tp, trend=d(F), beta_var=1.0)
    q0 = d(np.concatenate([np.log(w.params), w.r[w.sequenced], [0.0]]))
    ch = hmc.sample(post, q0, n_iter=60, n_warmup=30, n_steps=10, eps0=0.05, mass_every=20, seed=2)
    assert ch.draws.shape[1] == post.dim
    assert np.all(np.isfinite(ch.draws)) and ch.accept.mean() > 0.3
    assert np.std(ch.draws[:, -1]) > 0  # beta moves


@pytest.mark.parametrize("precision", ["fp32c", "fp32c_st"])
def test_graph_replayed_trajectories_equal_eager_ones(precision):
    """After warm-up each trajectory replays as one captured CUDA graph; the
    kernels and their inputs are the same, so the chain is identical bit for
    bit to the eagerly launched one (same seed)."""
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    w, prec = problem()
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")  # noqa: E731
    tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0)

    def make():
        return hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), torch.tensor(w.sequenced, device="cuda"), None,
                             hmc.prior_km_days(), precision, tree=tp)

    q0 = d(np.concatenate([np.log(w.params), w.r[w.sequenced]]))
    a = hmc.sample(make(), q0, n_iter=40, n_warmup=20, n_steps=8, eps0=0.05, mass_every=15, seed=3, use_graph=False)
    b = hmc.sample(make(), q0, n_iter=40, n_warmup=20, n_steps=8, eps0=0.05, mass_every=15, seed=3, use_graph=True)
    assert np.array_equal(a.draws, b.draws) and np.array_equal(a.accept, b.accept)
    assert b.grad_calls == a.grad_calls + 8  # one eager trajectory before the capture


def test_jittered_graph_trajectories_equal_eager_ones():
    """With step-size jitter each level's trajectory is captured once and
    replayed; the levels are drawn from the chain's own generator, so the
    replayed chain still equals the eagerly launched one bit for bit."""
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    w, prec = problem()
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")  # noqa: E731
    tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0)

    def make():
        return hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), torch.tensor(w.sequenced, device="cuda"), None,
                             hmc.prior_km_days(), "fp32c_st", tree=tp)

    q0 = d(np.concatenate([np.log(w.params), w.r[w.sequenced]]))
    kw = dict(n_iter=40, n_warmup=20, n_steps=8, eps0=0.05, mass_every=15, seed=3, jitter=0.2)
    a = hmc.sample(make(), q0, use_graph=False, **kw)
    b = hmc.sample(make(), q0, use_graph=True, **kw)
    assert np.array_equal(a.draws, b.draws) and np.array_equal(a.accept, b.accept)
    assert b.grad_calls - a.grad_calls in (8, 16, 24, 32, 40)  # one eager trajectory per captured level


def test_checkpoint_resume_equals_uninterrupted_chain(tmp_path):
    """A chain checkpointed in warm-up and again in sampling, then resumed from
    each checkpoint, ends exactly where the uninterrupted chain ends."""
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    w, prec = problem()
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")  # noqa: E731
    tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0)

    def make():
        return hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), torch.tensor(w.sequenced, device="cuda"), None,
                             hmc.prior_km_days(), "fp32c", tree=tp)

    q0 = d(np.concatenate([np.log(w.params), w.r[w.sequenced]]))
    kw = dict(n_iter=15, n_warmup=30, n_steps=6, eps0=0.05, mass_every=12, seed=9)
    full = hmc.sample(make(), q0, **kw)
    for every in (25, 35):  # the last checkpoint falls in warm-up (25), then in sampling (35)
        ck = str(tmp_path / f"ck{every}.pt")
        hmc.sample(make(), q0, checkpoint=ck, checkpoint_every=every, **kw)
        resumed = hmc.sample(make(), q0, resume=ck, **kw)
        assert np.array_equal(resumed.draws, full.draws) and np.array_equal(resumed.accept, full.accept)
        assert resumed.eps == full.eps and np.array_equal(resumed.mass, full.mass)


@pytest.mark.gpu
def test_device_accept_step_matches_oracle():
    """hawkes_hmc_accept against oracle.hmc_oracle.metropolis_step: the decision,
    the resulting state, log posterior and gradient, and the record slots, over
    random energies and the cases that must reject (non-finite proposal,
    likelihood error) or sit on the boundary (u == a rejects)."""
    import ctypes
    from paper_2103_03348_b300 import build, hmc
    build.build()
    L = hmc._lib()
    rng = np.random.default_rng(17)
    dev = "cuda"
    f64 = dict(dtype=torch.float64, device=dev)
    k = 300
    keep = np.array([0, 5, 299, 17, 300])  # the last index is out of range: recorded as NaN
    keep_d = torch.tensor(keep, dtype=torch.int64, device=dev)
    cases = []
    for _ in range(60):
        lp0, k0 = rng.normal(-50.0, 5.0), rng.exponential(5.0)
        lp1, k1 = lp0 + rng.normal(0.0, 1.5), k0 + rng.normal(0.0, 1.5)
        cases.append((lp0, k0, lp1, k1, rng.uniform(), 0))
    cases += [(-1.0, 0.0, -1.0 - math.log(4.0), 0.0, 0.25, 0),  # u == a: rejected
              (-1.0, 0.0, -1.0 - math.log(4.0), 0.0, 0.2499, 0),
              (-1.0, 0.0, math.nan, 0.0, 0.0, 0), (-1.0, 0.0, -math.inf, 0.0, 0.0, 0),
              (-1.0, 0.0, -1.0, math.inf, 0.0, 0), (-1.0, 0.0, 5.0, 0.0, 0.0, 2)]
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for lp0, k0, lp1, k1, u, st in cases:
        q0, g0 = rng.normal(size=k), rng.normal(size=k)
        q1, g1 = rng.normal(size=k), rng.normal(size=k)
        q_d, g_d = torch.tensor(q0, **f64), torch.tensor(g0, **f64)
        lp_d = torch.tensor(lp0, **f64)
        rec_q, rec = torch.full((len(keep),), -7.0, **f64), torch.full((3,), -7.0, **f64)
        args = [torch.tensor(v, **f64) for v in (u, k0, k1, lp1)]
        q1_d, g1_d = torch.tensor(q1, **f64), torch.tensor(g1, **f64)
        st_d = torch.tensor(st, dtype=torch.int32, device=dev)
        rc = L.hawkes_hmc_accept(k, hmc._ptr(args[0]), hmc._ptr(args[1]), hmc._ptr(args[2]), hmc._ptr(args[3]),
                                 hmc._ptr(g1_d), hmc._ptr(q1_d), hmc._ptr(st_d), hmc._ptr(q_d), hmc._ptr(lp_d),
                                 hmc._ptr(g_d), len(keep), hmc._ptr(keep_d), hmc._ptr(rec_q), hmc._ptr(rec), s)
        assert rc == 0
        torch.cuda.synchronize()
        q_r, lp_r, g_r, ok_r, a_r = hmc_oracle.metropolis_step(q0, lp0, g0, k0, q1, lp1, g1, k1, u, ok=st == 0)
        a_d = rec[1].item()
        assert abs(a_d - a_r) <= 4e-16 * max(a_r, 1e-300)
        if abs(u - a_r) > 1e-12 or u == a_r:  # a decision on the boundary is taken the same way only when exact
            assert bool(rec[2].item()) == ok_r
            assert np.array_equal(q_d.cpu().numpy(), q_r) and np.array_equal(g_d.cpu().numpy(), g_r)
            assert lp_d.item() == lp_r and rec[0].item() == lp_r
            want = np.array([q_r[i] if i < k else np.nan for i in keep])
            assert np.array_equal(rec_q.cpu().numpy(), want, equal_nan=True)
    # argument checks: aliasing proposal and state, negative keep count
    rc = L.hawkes_hmc_accept(k, hmc._ptr(args[0]), hmc._ptr(args[1]), hmc._ptr(args[2]), hmc._ptr(args[3]),
                             hmc._ptr(g1_d), hmc._ptr(q_d), None, hmc._ptr(q_d), hmc._ptr(lp_d), hmc._ptr(g_d),
                             0, None, None, None, s)
    assert rc == hmc.hawkes.EINVAL


class _SeparateLaunches:
    """A posterior without scatter_args: leapfrog then takes the separate
    momentum, position and scatter launches."""

    def __init__(self, post):
        self.post = post

    def evaluate(self, q, want_hess=False, out=None):
        return self.post.evaluate(q, want_hess=want_hess, out=out)


@pytest.mark.parametrize("precision", ["fp64", "fp32c_st"])
def test_fused_leapfrog_step_equals_separate_launches(precision):
    """hawkes_hmc_leapfrog_step (momentum, position and rate scatter in one
    launch) gives the trajectory of hawkes_hmc_momentum, hawkes_hmc_position
    and hawkes_hmc_scatter_rates in sequence, bit for bit, including every
    intermediate position seen by record; and its argument checks."""
    w, prec = problem()
    post, hmc = make_post(w, prec, precision)
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")  # noqa: E731
    rng = np.random.default_rng(3)
    q0 = np.concatenate([np.log(w.params), w.r[w.sequenced]])
    p0 = rng.normal(0, 1, q0.size)
    minv = d(rng.uniform(0.02, 0.2, q0.size))
    g0 = post.evaluate(d(q0))["grad"].clone()
    runs = []
    for target in (post, _SeparateLaunches(post)):
        q, p = d(q0), d(p0)
        seen = []
        scratch = {"logpost": torch.empty((), dtype=torch.float64, device="cuda"),
                   "grad": torch.empty(q.numel(), dtype=torch.float64, device="cuda")}
        ev = hmc.leapfrog(target, q, p, g0, 0.05, 6, minv, scratch,
                          record=lambda qq, gg: seen.append((qq.clone(), gg.clone())))
        runs.append((q, p, ev["logpost"].clone(), ev["grad"].clone(), seen))
    (qa, pa, la, ga, sa), (qb, pb, lb, gb, sb) = runs
    assert torch.equal(qa, qb) and torch.equal(pa, pb) and torch.equal(la, lb) and torch.equal(ga, gb)
    assert len(sa) == len(sb) == 6
    assert all(torch.equal(x[0], y[0]) and torch.equal(x[1], y[1]) for x, y in zip(sa, sb))
    L = hmc._lib()
    k, m = q0.size, len(w.sequenced)
    q, p = d(q0), d(p0)
    args = lambda kk, mm, seq, r: L.hawkes_hmc_leapfrog_step(kk, hmc._ptr(q), hmc._ptr(p), hmc._ptr(g0), 0.1,  # noqa: E731
                                                             hmc._ptr(minv), 0.1, mm, seq, r, None)
    seq_p, r_p = hmc._ptr(post.seq), hmc._ptr(post.r)
    assert args(0, 0, None, None) == hmc.hawkes.EINVAL
    assert args(k, k - 5, seq_p, r_p) == hmc.hawkes.EINVAL  # 6 + m > k
    assert args(k, -1, seq_p, r_p) == hmc.hawkes.EINVAL
    assert args(k, m, None, r_p) == hmc.hawkes.EINVAL
