"""Adaptively preconditioned Hamiltonian Monte Carlo over the phylogenetic Hawkes
posterior (Section 2.3).

The state q = (log mu0, log tau_x, log tau_t, log theta0, log omega, log h,
r_{s_1..s_M}) lives on the GPU.  Every leapfrog step runs the library's kernels:
scatter of the sequenced log-rates, the fused likelihood gradient with the
globals read from q on the device (hawkes_eval_device_params), the posterior
assembly (priors, log-transform Jacobian, phylogenetic Brownian prior through
its dense precision matrix or, in O(M), on the tree) and the momentum and
position updates.  Nothing crosses to the host inside a trajectory; each
iteration reads back two energies for the accept step.

Adaptation (Section 2.3.2): a diagonal mass matrix from the running average of
max(-H_qq, floor) over Hessian-diagonal evaluations made every `mass_every`
iterations, and, during warm-up, the step size by dual averaging toward a
target acceptance rate.  The effective sample size uses Geyer's initial
monotone sequence estimator.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import time

import numpy as np
import torch

from . import hawkes

PRIOR_GAMMA, PRIOR_INVGAMMA = 0, 1
KM_PER_DEGREE = 111.2
DAYS_PER_YEAR = 365.25


class _Prior(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int * 6), ("a", ctypes.c_double * 6), ("b", ctypes.c_double * 6)]


@dataclasses.dataclass
class Prior:
    kind: tuple
    a: tuple
    b: tuple

    def as_c(self):
        return _Prior((ctypes.c_int * 6)(*self.kind), (ctypes.c_double * 6)(*self.a), (ctypes.c_double * 6)(*self.b))

    def as_tuple(self):
        return (np.array(self.kind), np.array(self.a, float), np.array(self.b, float))


def prior_km_days() -> Prior:
    """Section 3.2's priors restated in km and days.

    mu0 ~ Gamma(2, rate 2); tau_x ~ IG(1, 10 degrees); h and 1/omega ~ IG(2, 0.5)
    (degrees and years); theta0 ~ Gamma(1, rate 0.001).  The paper's "scale
    0.001 / 2" for theta0 / mu0 is read as a rate: the stated aim is to upweight
    self-excitation, which a scale of 0.001 would do the opposite of.  The paper
    has no tau_t; it gets the same IG(2, 0.5 year) as the other time scale.
    1/omega ~ IG(a, b) is omega ~ Gamma(a, rate b).
    """
    half_year = 0.5 * DAYS_PER_YEAR
    return Prior(kind=(PRIOR_GAMMA, PRIOR_INVGAMMA, PRIOR_INVGAMMA, PRIOR_GAMMA, PRIOR_GAMMA, PRIOR_INVGAMMA),
                 a=(2.0, 1.0, 2.0, 1.0, 2.0, 2.0),
                 b=(2.0, 10.0 * KM_PER_DEGREE, half_year, 0.001, half_year, 0.5 * KM_PER_DEGREE))


def trend_features(t_seq, degree: int = 1, standardise: bool = True) -> np.ndarray:
    """[M, degree] polynomial trend features f(t) of the sequenced events'
    times (Section 2.2).  standardise=False with degree 1 is the paper's
    choice f(t) = t (Section 3.2, with beta ~ N(0, 10^2): beta_var = 100);
    the default uses u = (t - mean) / sd and f_d = u^d, which keeps the
    coefficients on a common scale."""
    t_seq = np.asarray(t_seq, float)
    u = (t_seq - t_seq.mean()) / (t_seq.std() if t_seq.std() > 0 else 1.0) if standardise else t_seq
    return np.stack([u ** d for d in range(1, degree + 1)], axis=1)


def _lib():
    L = hawkes.lib()
    if not getattr(L, "_hmc_typed", False):
        vp, i64, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        L.hawkes_posterior_workspace_size.argtypes = [i64]
        L.hawkes_posterior_workspace_size.restype = ctypes.c_size_t
        L.hawkes_posterior.argtypes = [i64, i64, vp, vp, ctypes.POINTER(_Prior), vp, vp, vp, vp,
                                       vp, ctypes.c_size_t, vp, vp, vp, vp]
        L.hawkes_posterior.restype = ctypes.c_int
        L.hawkes_posterior_tree_workspace_size.argtypes = [i64]
        L.hawkes_posterior_tree_workspace_size.restype = ctypes.c_size_t
        L.hawkes_posterior_tree.argtypes = [i64, i64, vp, vp, vp, d, d, ctypes.POINTER(_Prior), vp, vp, vp, vp,
                                            vp, ctypes.c_size_t, vp, vp, vp, vp]
        L.hawkes_posterior_tree.restype = ctypes.c_int
        L.hawkes_posterior_assemble.argtypes = [i64, i64, vp, vp, vp, ctypes.POINTER(_Prior), vp, vp, vp, vp, vp,
                                                vp, vp, vp]
        L.hawkes_posterior_assemble.restype = ctypes.c_int
        L.hawkes_hmc_scatter_rates.argtypes = [i64, vp, vp, vp, vp]
        L.hawkes_hmc_scatter_rates_trend.argtypes = [i64, ctypes.c_int, vp, vp, vp, vp, vp]
        L.hawkes_hmc_scatter_rates_trend.restype = ctypes.c_int
        L.hawkes_posterior_add_trend.argtypes = [i64, ctypes.c_int, vp, vp, d, vp, vp, vp, vp, vp, vp, vp]
        L.hawkes_posterior_add_trend.restype = ctypes.c_int
        L.hawkes_hmc_momentum.argtypes = [i64, vp, vp, d, vp]
        L.hawkes_hmc_position.argtypes = [i64, vp, vp, vp, d, vp]
        L.hawkes_hmc_kinetic.argtypes = [i64, vp, vp, vp, vp]
        L.hawkes_hmc_position_dense.argtypes = [i64, vp, vp, vp, d, vp]
        L.hawkes_hmc_kinetic_dense.argtypes = [i64, vp, vp, vp, vp]
        L.hawkes_hmc_accept.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp]
        L.hawkes_hmc_leapfrog_step.argtypes = [i64, vp, vp, vp, d, vp, d, i64, vp, vp, vp]
        for f in (L.hawkes_hmc_scatter_rates, L.hawkes_hmc_momentum, L.hawkes_hmc_position, L.hawkes_hmc_kinetic,
                  L.hawkes_hmc_position_dense, L.hawkes_hmc_kinetic_dense, L.hawkes_hmc_accept,
                  L.hawkes_hmc_leapfrog_step):
            f.restype = ctypes.c_int
        L._hmc_typed = True
    return L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check(rc):
    if rc != hawkes.OK:
        raise hawkes.HawkesError(rc, hawkes.strerror(rc))


class Posterior:
    """log pi(q) and its derivatives for fixed events, priors and tree precision."""

    def __init__(self, x, y, t, r_base, seq_idx, prec, prior: Prior, precision="fp32c", tree=None, trend=None,
                 beta_var=1.0):
        """prec: the dense M x M precision (sigma^2 V)^-1 on the device, or None
        with tree: a tree.TreePrior over the same M sequenced events (O(M) per
        evaluation instead of O(M^2)).  trend: optional device [M, K] matrix
        F of trend features f(t_s) (Section 2.2): the state becomes
        (log globals, z[M], beta[K]) with r_s = z_s + F_s beta and
        beta ~ N(0, beta_var I)."""
        self.x, self.y, self.t = x, y, t
        self.r = r_base.clone()
        self.dev = t.device
        self.n = t.numel()
        self.seq = seq_idx.to(torch.int32).contiguous()
        self.m = self.seq.numel()
        self.tree = tree
        self.prec = prec.contiguous() if prec is not None else None
        if (tree is None) == (prec is None):
            raise ValueError("give exactly one of prec and tree")
        if tree is not None and tree.m != self.m:
            raise ValueError("the tree's tips must be the sequenced events")
        self.prior = prior
        self.c_prior = prior.as_c()
        self.precision = precision
        L = _lib()
        ws_bytes = (L.hawkes_posterior_tree_workspace_size(self.m) if tree is not None
                    else L.hawkes_posterior_workspace_size(self.m))
        self.ws = torch.empty(int(ws_bytes), dtype=torch.uint8, device=self.dev)
        f64 = dict(dtype=torch.float64, device=self.dev)
        self.like = {"loglik": torch.empty((), **f64), "grad": torch.empty(6 + self.n, **f64),
                     "hdiag": torch.empty(6 + self.n, **f64), "status": torch.empty((), dtype=torch.int32, device=self.dev)}
        # a workspace of its own: after the first evaluation the events' preparation is reused
        self.like_ws = torch.empty(hawkes.workspace_size(self.n, precision), dtype=torch.uint8, device=self.dev)
        self.prepared = False
        self.trend = trend.to(torch.float64).contiguous() if trend is not None else None
        self.k = int(self.trend.shape[1]) if self.trend is not None else 0
        if self.trend is not None and (self.trend.shape[0] != self.m or self.m == 0):
            raise ValueError("trend must be [M, K] over the M >= 1 sequenced events")
        self.beta_var = float(beta_var)
        self.dim = 6 + self.m + self.k
        if tree is not None:
            # the tree prior runs on a side stream, concurrently with the likelihood
            self.side = torch.cuda.Stream(device=t.device)
            self.fork, self.join = torch.cuda.Event(), torch.cuda.Event()
            self.pz = torch.empty(self.m, dtype=torch.float64, device=t.device)
            self.pd = torch.empty(self.m, dtype=torch.float64, device=t.device)
        self.calls = {"grad": 0, "hess": 0}

    def evaluate(self, q, want_hess=False, out=None, scattered=False):
        """Fill out = {'logpost', 'grad', ['hdiag']} (device tensors) at q; returns out.

        Everything is enqueued on the current stream: the likelihood reads the
        six globals from q on the device (as logarithms), so no value crosses to
        the host.  A q outside the parameter space gives log pi = -inf (or NaN
        through the likelihood's NaN outputs), which the sampler rejects.
        scattered: q's sequenced log-rates are already in the likelihood's rate
        vector (written by hawkes_hmc_leapfrog_step with scatter_args())."""
        L = _lib()
        stream = torch.cuda.current_stream(self.dev).cuda_stream
        if out is None:
            f64 = dict(dtype=torch.float64, device=self.dev)
            out = {"logpost": torch.empty((), **f64), "grad": torch.empty(self.dim, **f64),
                   "hdiag": torch.empty(self.dim, **f64)}
        if not scattered:
            self._scatter(q, stream)
        self._prior_async(q, want_hess)
        # with no free log-rates the column pass is skipped (globals-only modes)
        mode = ("hess" if want_hess else "grad") if self.m > 0 else ("hess_globals" if want_hess else "grad_globals")
        # the rate entries are needed for the sequenced events only: O(N M) column work
        hawkes._call(mode, self.x, self.y, self.t, self.r, q, self.precision, stream=stream, check=False,
                     out=self.like, log_params=True, workspace=self.like_ws, reuse_events=self.prepared,
                     rate_idx=self.seq if self.m > 0 else None)
        self.prepared = True
        self.calls["hess" if want_hess else "grad"] += 1
        self._assemble(q, self.like["grad"], self.like["hdiag"] if want_hess else None, out["logpost"],
                       out["grad"], out["hdiag"] if want_hess else None, stream)
        return out

    def scatter_args(self):
        """(m, seq, r) for hawkes_hmc_leapfrog_step's scatter of the sequenced
        log-rates into the likelihood's rate vector, or None with the trend
        (whose rates are not q's entries themselves)."""
        return None if self.trend is not None else (self.m, self.seq, self.r)

    def _scatter(self, q, stream):
        L = _lib()
        if self.trend is None:
            _check(L.hawkes_hmc_scatter_rates(self.m, _ptr(self.seq), _ptr(q), _ptr(self.r), ctypes.c_void_p(stream)))
        else:
            _check(L.hawkes_hmc_scatter_rates_trend(self.m, self.k, _ptr(self.seq), _ptr(self.trend), _ptr(q),
                                                    _ptr(self.r), ctypes.c_void_p(stream)))

    def _prior_async(self, q, want_diag):
        """Tree prior: (sigma^2 V)^-1 z (and its diagonal) on the side stream,
        forked after the state update; _assemble joins it."""
        if self.tree is None:
            return
        cur = torch.cuda.current_stream(self.dev)
        self.fork.record(cur)
        self.side.wait_event(self.fork)
        with torch.cuda.stream(self.side):
            self.tree.evaluate(q[6:6 + self.m], out={"pz": self.pz, "pdiag": self.pd if want_diag else None})
        self.join.record(self.side)

    def _assemble(self, q, grad, hdiag, logpost, grad_q, hdiag_q, stream):
        """Priors, Jacobian and the phylogenetic prior (dense or on the tree) on the device."""
        L = _lib()
        if self.tree is None:
            _check(L.hawkes_posterior(self.n, self.m, _ptr(self.seq), _ptr(self.prec), ctypes.byref(self.c_prior),
                                      _ptr(q), _ptr(self.like["loglik"]), _ptr(grad), _ptr(hdiag), _ptr(self.ws),
                                      ctypes.c_size_t(self.ws.numel()), _ptr(logpost), _ptr(grad_q), _ptr(hdiag_q),
                                      ctypes.c_void_p(stream)))
        else:
            torch.cuda.current_stream(self.dev).wait_event(self.join)
            _check(L.hawkes_posterior_assemble(self.n, self.m, _ptr(self.seq), _ptr(self.pz),
                                               _ptr(self.pd) if hdiag is not None else None,
                                               ctypes.byref(self.c_prior), _ptr(q), _ptr(self.like["loglik"]),
                                               _ptr(grad), _ptr(hdiag), _ptr(logpost), _ptr(grad_q), _ptr(hdiag_q),
                                               ctypes.c_void_p(stream)))
        if self.trend is not None:
            _check(L.hawkes_posterior_add_trend(self.m, self.k, _ptr(self.seq), _ptr(self.trend), self.beta_var,
                                                _ptr(q), _ptr(grad), _ptr(hdiag), _ptr(logpost), _ptr(grad_q),
                                                _ptr(hdiag_q), ctypes.c_void_p(stream)))

    def logpost_only(self, q, out):
        """out['logpost'] = log pi(q) from a log-likelihood-only pass (the exact
        accept step of surrogate trajectories)."""
        L = _lib()
        stream = torch.cuda.current_stream(self.dev).cuda_stream
        self._scatter(q, stream)
        self._prior_async(q, False)
        hawkes._call("loglik", self.x, self.y, self.t, self.r, q, self.precision, stream=stream, check=False,
                     out=self.like, log_params=True, workspace=self.like_ws, reuse_events=self.prepared)
        self.prepared = True
        self.calls["loglik"] = self.calls.get("loglik", 0) + 1
        self._assemble(q, None, None, out["logpost"], None, None, stream)
        return out

    def status(self):
        return int(self.like["status"].item())


class TreeMassOp:
    """The tree-structured mass matrix (tree.TreeMass: diag(d) + (sigma2 V)^-1 on
    the rate block) with the diagonal inverse mass minv elsewhere, in the
    form leapfrog, kinetic and TrajectoryGraph take in place of minv."""

    def __init__(self, tm, minv):
        self.tm, self.minv = tm, minv

    def position(self, q, p, eps):
        self.tm.velocity(p, self.minv, q=q, eps=eps)

    def kinetic(self, p, out):
        self.tm.velocity(p, self.minv, kinetic=out)


class DenseMassOp:
    """A dense mass matrix M over all dim <= 64 coordinates (a posterior over
    the six globals alone, whose correlations a diagonal mass cannot follow),
    in the form leapfrog, kinetic and TrajectoryGraph take in place of minv.
    M^-1 and the Cholesky factor of M live in device buffers updated in place,
    so captured trajectories see mass updates."""

    def __init__(self, dim, device, floor=1e-2):
        if dim > 64:
            raise ValueError("a dense mass is offered for at most 64 coordinates")
        f64 = dict(dtype=torch.float64, device=device)
        self.dim, self.floor = dim, floor
        self.M = np.eye(dim)
        self.minv = torch.eye(dim, **f64).reshape(-1).contiguous()
        self.chol = torch.eye(dim, **f64)

    def set(self, M):
        """Symmetrise M, clip its eigenvalues at the floor, and refresh M^-1 and chol(M)."""
        M = 0.5 * (np.asarray(M, float) + np.asarray(M, float).T)
        w, V = np.linalg.eigh(M)
        w = np.maximum(w, self.floor)
        self.M = (V * w) @ V.T
        self.minv.copy_(torch.as_tensor(((V / w) @ V.T).ravel()))
        self.chol.copy_(torch.as_tensor(np.linalg.cholesky(self.M)))

    def position(self, q, p, eps):
        s = ctypes.c_void_p(torch.cuda.current_stream(q.device).cuda_stream)
        _check(_lib().hawkes_hmc_position_dense(self.dim, _ptr(q), _ptr(p), _ptr(self.minv), eps, s))

    def kinetic(self, p, out):
        s = ctypes.c_void_p(torch.cuda.current_stream(p.device).cuda_stream)
        _check(_lib().hawkes_hmc_kinetic_dense(self.dim, _ptr(p), _ptr(self.minv), _ptr(out), s))

    def draw(self, xi, p):
        """p = chol(M) xi, so that p ~ N(0, M) for xi ~ N(0, I)."""
        torch.mv(self.chol, xi, out=p)


def leapfrog(post, q, p, g, eps, n_steps, minv, scratch, record=None):
    """n_steps leapfrog steps from (q, p) with gradient g at q; updates q, p in place.

    minv: the diagonal inverse mass (device tensor) or a TreeMassOp.
    record(q, grad), when given, sees every position of the trajectory with its
    gradient (device tensors, valid until the next step).  Returns the
    evaluation dict at the final position.  With a diagonal mass and a
    posterior that offers scatter_args(), each step's momentum update, position
    update and rate scatter are one launch (hawkes_hmc_leapfrog_step), with the
    same results as the separate launches."""
    L = _lib()
    k = q.numel()
    s = ctypes.c_void_p(torch.cuda.current_stream(q.device).cuda_stream)
    sc = post.scatter_args() if isinstance(minv, torch.Tensor) and hasattr(post, "scatter_args") else None
    ev = None
    if sc is not None:
        m, seq, r = sc
        gcur, a = g, 0.5 * eps
        for step in range(n_steps):
            _check(L.hawkes_hmc_leapfrog_step(k, _ptr(q), _ptr(p), _ptr(gcur), a, _ptr(minv), eps, m, _ptr(seq),
                                              _ptr(r), s))
            ev = post.evaluate(q, out=scratch, scattered=True)
            if record is not None:
                record(q, ev["grad"])
            gcur, a = ev["grad"], eps
        _check(L.hawkes_hmc_momentum(k, _ptr(p), _ptr(gcur), 0.5 * eps, s))
        return ev
    _check(L.hawkes_hmc_momentum(k, _ptr(p), _ptr(g), 0.5 * eps, s))
    for step in range(n_steps):
        if isinstance(minv, torch.Tensor):
            _check(L.hawkes_hmc_position(k, _ptr(q), _ptr(p), _ptr(minv), eps, s))
        else:
            minv.position(q, p, eps)
        ev = post.evaluate(q, out=scratch)
        if record is not None:
            record(q, ev["grad"])
        _check(L.hawkes_hmc_momentum(k, _ptr(p), _ptr(ev["grad"]), eps if step < n_steps - 1 else 0.5 * eps, s))
    return ev


def kinetic(p, minv, out):
    """out = p^T M^-1 p / 2 for a diagonal minv tensor or a TreeMassOp."""
    if not isinstance(minv, torch.Tensor):
        minv.kinetic(p, out)
        return out
    L = _lib()
    s = ctypes.c_void_p(torch.cuda.current_stream(p.device).cuda_stream)
    _check(L.hawkes_hmc_kinetic(p.numel(), _ptr(p), _ptr(minv), _ptr(out), s))
    return out


class DualAveraging:
    """Step-size adaptation toward a target acceptance probability (dual averaging)."""

    def __init__(self, eps0, target=0.8, gamma=0.05, t0=10.0, kappa=0.75):
        self.mu = math.log(10.0 * eps0)
        self.target, self.gamma, self.t0, self.kappa = target, gamma, t0, kappa
        self.hbar, self.log_eps_bar, self.t = 0.0, 0.0, 0
        self.eps = eps0

    def update(self, accept_prob):
        self.t += 1
        eta = 1.0 / (self.t + self.t0)
        self.hbar = (1 - eta) * self.hbar + eta * (self.target - accept_prob)
        log_eps = self.mu - math.sqrt(self.t) / self.gamma * self.hbar
        w = self.t ** (-self.kappa)
        self.log_eps_bar = w * log_eps + (1 - w) * self.log_eps_bar
        self.eps = math.exp(log_eps)
        return self.eps

    def final(self):
        return math.exp(self.log_eps_bar)


@dataclasses.dataclass
class Chain:
    draws: np.ndarray          # [n_iter, dim] post-warm-up states
    logpost: np.ndarray        # [n_iter]
    accept: np.ndarray         # [n_iter] accepted?
    accept_prob: np.ndarray    # [n_iter]
    eps: float
    mass: np.ndarray
    seconds: float             # wall time of the post-warm-up iterations
    warmup_seconds: float
    grad_calls: int
    hess_calls: int
    last_q: object = None      # device state at the end
    mass_t: object = None      # device mass matrix at the end


class TrajectoryGraph:
    """One leapfrog trajectory of fixed step size and length, captured once as
    a CUDA graph and replayed per iteration: every kernel of the n_steps
    likelihood evaluations, posterior assemblies and momentum/position
    updates is enqueued by one launch, with no Python or driver overhead per
    kernel.  Works on static buffers: set q, p and g (the gradient at q), then
    replay; the trajectory's end state is in q, p and out, and the kinetic
    energy at the end in k1.  minv is read from device memory at replay, so
    mass updates made in place take effect.  The eager run that precedes the
    capture starts from (q0, p0, g0), a state of the chain: from an arbitrary
    state (all zeros: every global 1 in its unit) the likelihood can take its
    slowest path (rows redone in FP64)."""

    def __init__(self, post, eps, n_steps, minv, q0, p0, g0):
        dev = q0.device
        f64 = dict(dtype=torch.float64, device=dev)
        dim = q0.numel()
        self.post, self.n_steps = post, n_steps
        self.q, self.p, self.g = torch.zeros(dim, **f64), torch.zeros(dim, **f64), torch.zeros(dim, **f64)
        self.out = {"logpost": torch.empty((), **f64), "grad": torch.empty(dim, **f64),
                    "hdiag": torch.empty(dim, **f64)}
        self.k1 = torch.empty((), **f64)
        self.q.copy_(q0)
        self.p.copy_(p0)
        self.g.copy_(g0)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):  # one eager run first, so every lazily made buffer exists
            self._body(eps, minv)
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        calls = dict(post.calls)
        with torch.cuda.graph(self.graph):
            self._body(eps, minv)
        post.calls.update(calls)  # capture enqueues nothing: count replays instead

    def _body(self, eps, minv):
        leapfrog(self.post, self.q, self.p, self.g, eps, self.n_steps, minv, self.out)
        kinetic(self.p, minv, self.k1)

    def replay(self):
        self.graph.replay()
        self.post.calls["grad"] += self.n_steps
        return self.out


def jitter_levels(jitter: float):
    """Step-size factors of a jittered sampler: 1 + jitter * (-1, -1/2, 0, 1/2, 1),
    or [1] without jitter."""
    if not jitter:
        return [1.0]
    if not 0.0 < jitter < 1.0:
        raise ValueError("jitter must lie in [0, 1)")
    return [1.0 + jitter * f for f in (-1.0, -0.5, 0.0, 0.5, 1.0)]


def save_state(path, state: dict):
    """Write a sampler checkpoint atomically (a temporary file, then a rename)."""
    tmp = f"{path}.tmp"
    torch.save(state, tmp)
    os.replace(tmp, path)


def load_state(path) -> dict:
    return torch.load(path, map_location="cpu", weights_only=False)


def sample(post: Posterior, q0, n_iter, n_warmup, n_steps=20, eps0=0.01, mass_every=100, target_accept=0.8,
           mass_floor=1e-2, seed=0, keep=None, record=None, use_graph=True, checkpoint=None, checkpoint_every=0,
           resume=None, mass="diag", fd_step=1e-3, mass0=None, jitter=0.0):
    """Run n_warmup + n_iter HMC iterations from q0 (device tensor); returns a Chain.

    mass: "diag", the diagonal mass of Section 2.3.2 (a running average of
    max(-H_diag, mass_floor)); or "tree", for a posterior with a tree prior:
    the same diagonal outside the rate block and diag(d) + (sigma2 V)^-1 on
    it, d a running average of the likelihood's own curvature
    max(-H_diag - diag((sigma2 V)^-1), 0), so that the prior's tree
    correlations are preconditioned exactly (tree.TreeMass); or
    "dense": a dense mass over all coordinates (at most 64: a posterior over
    the six globals alone), the running average of minus the Hessian taken by
    central differences of the gradient (2 dim extra gradients per update),
    its eigenvalues clipped at mass_floor; or
    "tree_joint": the tree mass on the rates plus a dense block for the six
    globals and its coupling to the rates, [[A, B^T], [B, M_z]], with A and
    B running averages of minus the log posterior's Hessian columns along
    the globals, taken by central differences of the gradient (step fd_step
    in the log scale; 12 extra gradients per mass update).  The coupling is
    switched on at the first mass update from the middle of warm-up on (the
    globals' block is the diagonal mass until then): a mass fitted where the
    chain starts can hold it in a minor mode (seen on the 23,422-event
    posterior, 635 log-units below the main one).

    keep: optional index array of coordinates to store (all by default);
    record: optional callback given every leapfrog position and its gradient;
    use_graph: after warm-up (step size fixed) replay each trajectory as one
    captured CUDA graph (not with record, which needs every position);
    checkpoint, checkpoint_every: write the whole sampler state (position,
    gradient, mass, step size and its adaptation, both random streams, draws so
    far, counters) to `checkpoint` every that many iterations;
    resume: a checkpoint to continue from; the chain then equals the one that
    was never interrupted, bit for bit (the other arguments must match);
    mass0: optional mass to start from instead of the Hessian at q0: a
    diagonal (device tensor [dim]) with mass="diag", another chain's
    DenseMassOp with mass="dense" (e.g. another chain's adapted mass, so that
    two samplers can be compared with the same one);
    jitter: each trajectory's step size is eps times a factor drawn uniformly
    from the five levels 1 + jitter * (-1, -1/2, 0, 1/2, 1), so that a fixed
    trajectory length eps * n_steps cannot sit on a multiple of a half period
    of the dynamics along some direction (one captured graph per level)."""
    dev = q0.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    dim = q0.numel()
    f64 = dict(dtype=torch.float64, device=dev)
    p = torch.empty(dim, **f64)
    keep = np.arange(dim) if keep is None else np.asarray(keep)
    keep_t = torch.as_tensor(keep, device=dev)
    total = n_warmup + n_iter
    da = DualAveraging(eps0, target_accept)
    if mass not in ("diag", "tree", "tree_joint", "dense"):
        raise ValueError("mass must be 'diag', 'tree', 'tree_joint' or 'dense'")
    dm = DenseMassOp(dim, dev, floor=mass_floor) if mass == "dense" else None
    tm = xi = None
    joint = None  # running averages of the coupled blocks A (6 x 6) and B (m x 6)
    if mass in ("tree", "tree_joint"):
        if getattr(post, "tree", None) is None:
            raise ValueError(f"mass='{mass}' needs a posterior with a tree prior")
        from . import tree as tree_mod
        tm = tree_mod.TreeMass(post.tree, dim, z0=6, nc=6 if mass == "tree_joint" else 0)
        xi = torch.empty(tm.n_normals, **f64)

    def hessian_columns(qc, ncols=6):
        """-(d grad / d q_k) for the first ncols coordinates by central differences: (dim x ncols)."""
        cols = np.empty((dim, ncols))
        qp = torch.empty_like(qc)
        for kk in range(ncols):
            qp.copy_(qc)
            qp[kk] += fd_step
            gp = post.evaluate(qp)["grad"].cpu().numpy()
            qp[kk] -= 2 * fd_step
            gm = post.evaluate(qp)["grad"].cpu().numpy()
            cols[:, kk] = -(gp - gm) / (2 * fd_step)
        return cols

    joint_from = max(1, n_warmup // 2)  # first iteration count at which the coupling may start

    def update_joint(qc, diag_mass, it_done):
        """The coupled blocks' running average (counted from the coupling's start)
        and the coupling, or the diagonal mass on the globals before that."""
        nonlocal joint
        if it_done < joint_from:
            tm.set_coupling(np.diag(diag_mass[:6].cpu().numpy()), np.zeros((tm.m, 6)), floor=mass_floor)
            return
        cols = hessian_columns(qc)
        A, B = 0.5 * (cols[:6] + cols[:6].T), cols[6:6 + tm.m]
        if joint is None:
            joint = {"A": A, "B": B, "n": 1}
        else:
            n = joint["n"]
            joint = {"A": (n * joint["A"] + A) / (n + 1), "B": (n * joint["B"] + B) / (n + 1), "n": n + 1}
        tm.set_coupling(joint["A"], joint["B"], floor=mass_floor)

    def rate_curvature(hdiag_q):
        # the log-likelihood's curvature on the rates: the posterior's minus the prior's
        return torch.clamp(-hdiag_q[6:6 + tm.m] - post.pd, min=0.0)
    if resume is None:
        q = q0.clone()
        cur = post.evaluate(q, want_hess=True)
        cur = {k: v.clone() for k, v in cur.items()}
        if mass0 is not None and dm is not None:
            if not isinstance(mass0, DenseMassOp) or mass0.dim != dim:
                raise ValueError("with mass='dense', mass0 is another chain's DenseMassOp over the same coordinates")
            dm.set(mass0.M)
            mass = torch.clamp(-cur["hdiag"], min=mass_floor)
        elif mass0 is not None:
            if tm is not None or not isinstance(mass0, torch.Tensor) or mass0.numel() != dim:
                raise ValueError("mass0 is a diagonal mass over all coordinates (mass='diag')")
            mass = mass0.to(**f64).clone()
        else:
            mass = torch.clamp(-cur["hdiag"], min=mass_floor)
            if dm is not None:
                dm.set(hessian_columns(q, dim))
        n_mass = 1
        minv = 1.0 / mass  # updated in place from here on (a captured trajectory reads it)
        if tm is not None:
            tm.d.copy_(rate_curvature(cur["hdiag"]))
            tm.factor()
            if tm.nc:
                update_joint(q, mass, 0)
        eps = eps0
        draws = np.empty((n_iter, len(keep)))
        lps, acc, aprob = np.empty(n_iter), np.zeros(n_iter, bool), np.empty(n_iter)
        start, spent_warm, spent_samp = 0, 0.0, 0.0
    else:
        st = load_state(resume)
        if (st["n_iter"], st["n_warmup"], st["n_steps"], st["dim"]) != (n_iter, n_warmup, n_steps, dim):
            raise ValueError("the checkpoint belongs to a chain with other settings")
        q = st["q"].to(dev)
        cur = {"logpost": st["logpost"].to(dev), "grad": st["grad"].to(dev)}
        mass, minv = st["mass"].to(dev), st["minv"].to(dev)
        n_mass, eps = st["n_mass"], st["eps"]
        if tm is not None:
            tm.d.copy_(st["tree_d"].to(dev))
            tm.factor()
            if tm.nc:
                joint = st["joint"]
                if joint is None:
                    tm.set_coupling(np.diag(mass[:6].cpu().numpy()), np.zeros((tm.m, 6)), floor=mass_floor)
                else:
                    tm.set_coupling(joint["A"], joint["B"], floor=mass_floor)
        da.__dict__.update(st["dual_averaging"])
        gen.set_state(st["gen_state"])
        rng.bit_generator.state = st["rng_state"]
        draws, lps, acc, aprob = st["draws"], st["lps"], st["acc"], st["aprob"]
        post.calls.update(st["calls"])
        start, spent_warm, spent_samp = st["it"], st["spent_warm"], st["spent_samp"]
    if dm is not None and resume is not None:
        dm.set(st["dense_M"])
    mop = TreeMassOp(tm, minv) if tm is not None else (dm if dm is not None else minv)  # what leapfrog applies
    xi_d = torch.empty(dim, **f64) if dm is not None else None
    levels = jitter_levels(jitter)
    graphs = {}  # one captured trajectory per step-size level
    graph = None
    scratch = {"logpost": torch.empty((), **f64), "grad": torch.empty(dim, **f64), "hdiag": torch.empty(dim, **f64)}
    k0, k1 = torch.empty((), **f64), torch.empty((), **f64)
    # After warm-up the accept step runs on the device (hawkes_hmc_accept) and each
    # iteration's record goes to its own device slot, so that an iteration needs no
    # host round trip; the slots are copied to the host arrays at checkpoints and at
    # the end.  The uniform draws still come from the host stream, in the same order.
    L = _lib()
    stream = lambda: ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)  # noqa: E731
    keep_d = keep_t.to(torch.int64)
    rec_q = torch.empty((n_iter, len(keep)), **f64)
    rec = torch.empty((n_iter, 3), **f64)
    u_pin = torch.empty(max(n_iter, 1), dtype=torch.float64, pin_memory=True)
    u_dev = torch.empty(max(n_iter, 1), **f64)
    status_t = post.like.get("status") if isinstance(getattr(post, "like", None), dict) else None
    first_slot = max(start, n_warmup) - n_warmup  # the first slot this call fills

    def pull(j1):
        """Copy device record slots [first_slot, j1) to the host arrays."""
        if j1 > first_slot:
            draws[first_slot:j1] = rec_q[first_slot:j1].cpu().numpy()
            r = rec[first_slot:j1].cpu().numpy()
            lps[first_slot:j1], aprob[first_slot:j1], acc[first_slot:j1] = r[:, 0], r[:, 1], r[:, 2] != 0.0

    torch.cuda.synchronize()
    t_seg = time.perf_counter()  # start of the current warm-up or sampling segment
    for it in range(start, total):
        if it == n_warmup:
            eps = da.final() if n_warmup > 0 else eps
            torch.cuda.synchronize()
            now = time.perf_counter()
            spent_warm += now - t_seg
            t_seg = now
        if dm is not None:
            torch.randn(dim, generator=gen, out=xi_d, dtype=torch.float64, device=dev)
            dm.draw(xi_d, p)
        elif tm is None:
            torch.randn(dim, generator=gen, out=p, dtype=torch.float64, device=dev)
            p.mul_(torch.sqrt(mass))
        else:
            torch.randn(tm.n_normals, generator=gen, out=xi, dtype=torch.float64, device=dev)
            tm.momentum(minv, xi, p)
        kinetic(p, mop, k0)
        lvl = int(rng.integers(len(levels))) if len(levels) > 1 else 0
        eps_it = eps * levels[lvl]
        if it >= n_warmup:
            j = it - n_warmup
            u_pin[j] = rng.uniform()  # slot j is written once, so the copy may run later
            u_dev[j:j + 1].copy_(u_pin[j:j + 1], non_blocking=True)
        if use_graph and record is None and it >= n_warmup:
            graph = graphs.get(lvl)
            if graph is None:
                graph = graphs[lvl] = TrajectoryGraph(post, eps_it, n_steps, mop, q, p, cur["grad"])
            graph.q.copy_(q)
            graph.p.copy_(p)
            graph.g.copy_(cur["grad"])
            ev = graph.replay()
            qn, k1_t = graph.q, graph.k1
        else:
            qn = q.clone()
            ev = leapfrog(post, qn, p, cur["grad"], eps_it, n_steps, mop, scratch, record)
            kinetic(p, mop, k1)
            k1_t = k1
        if it >= n_warmup:
            _check(L.hawkes_hmc_accept(dim, _ptr(u_dev[j]), _ptr(k0), _ptr(k1_t), _ptr(ev["logpost"]),
                                       _ptr(ev["grad"]), _ptr(qn), _ptr(status_t), _ptr(q), _ptr(cur["logpost"]),
                                       _ptr(cur["grad"]), len(keep), _ptr(keep_d), _ptr(rec_q[j]), _ptr(rec[j]),
                                       stream()))
        else:
            h0 = -cur["logpost"].item() + k0.item()
            lp1 = ev["logpost"].item()
            h1 = -lp1 + k1_t.item()
            ok_num = math.isfinite(lp1) and post.status() == hawkes.OK
            a = min(1.0, math.exp(min(0.0, h0 - h1))) if ok_num and math.isfinite(h1) else 0.0
            if rng.uniform() < a:
                q = qn
                cur["logpost"].copy_(ev["logpost"])
                cur["grad"].copy_(ev["grad"])
            eps = da.update(a)
        if (it + 1) % mass_every == 0 and dm is not None:
            # running average of minus the Hessian by central differences of the gradient
            dm.set((n_mass * dm.M + 0.5 * (lambda c: c + c.T)(hessian_columns(q, dim))) / (n_mass + 1))
            n_mass += 1
        elif (it + 1) % mass_every == 0:
            hd = post.evaluate(q, want_hess=True)
            new = torch.clamp(-hd["hdiag"], min=mass_floor)
            if tm is not None:
                tm.d.mul_(n_mass).add_(rate_curvature(hd["hdiag"])).div_(n_mass + 1)
                tm.factor()  # in place: a captured trajectory reads the new coefficients
            mass = (n_mass * mass + new) / (n_mass + 1)  # running average of the Hessian-based masses
            if tm is not None and tm.nc:
                update_joint(q, mass, it + 1)
            n_mass += 1
            torch.reciprocal(mass, out=minv)
            cur["logpost"].copy_(hd["logpost"])
            cur["grad"].copy_(hd["grad"])
        if checkpoint and checkpoint_every and (it + 1) % checkpoint_every == 0 and it + 1 < total:
            pull(it + 1 - n_warmup)
            torch.cuda.synchronize()
            now = time.perf_counter()
            seg = now - t_seg
            save_state(checkpoint, {
                "it": it + 1, "n_iter": n_iter, "n_warmup": n_warmup, "n_steps": n_steps, "dim": dim,
                "q": q.cpu(), "logpost": cur["logpost"].cpu(), "grad": cur["grad"].cpu(),
                "mass": mass.cpu(), "minv": minv.cpu(), "n_mass": n_mass, "eps": eps,
                "dual_averaging": dict(da.__dict__), "gen_state": gen.get_state(),
                "rng_state": rng.bit_generator.state, "draws": draws, "lps": lps, "acc": acc, "aprob": aprob,
                "calls": dict(post.calls), "tree_d": tm.d.cpu() if tm is not None else None, "joint": joint,
                "dense_M": dm.M.copy() if dm is not None else None,
                "spent_warm": spent_warm + (seg if it < n_warmup else 0.0),
                "spent_samp": spent_samp + (seg if it >= n_warmup else 0.0)})
            # the checkpoint's own cost is left out of both phases
            if it < n_warmup:
                spent_warm += seg
            else:
                spent_samp += seg
            t_seg = time.perf_counter()
    pull(n_iter)
    torch.cuda.synchronize()
    now = time.perf_counter()
    if total > n_warmup and max(start, n_warmup) < total:
        spent_samp += now - t_seg
    else:
        spent_warm += now - t_seg
    if n_iter == 0:  # warm-up only: report the adapted step size
        eps = da.final() if n_warmup > 0 else eps
    if dm is not None:
        return Chain(draws, lps, acc, aprob, eps, dm.M.copy(), spent_samp, spent_warm,
                     post.calls["grad"], post.calls["hess"], q, dm)
    return Chain(draws, lps, acc, aprob, eps, mass.cpu().numpy(), spent_samp, spent_warm,
                 post.calls["grad"], post.calls["hess"], q, mass)


def ess(x) -> float:
    """Geyer's initial monotone sequence estimate of the effective sample size of a 1-D chain.

    Autocovariances through the FFT; tau = -1 + 2 sum_m Gamma_m, Gamma_m =
    rho_2m + rho_2m+1 summed while positive and made non-increasing; tau is kept
    at or above 1/log10(n), so the ESS never exceeds n log10(n)."""
    x = np.asarray(x, float)
    n = len(x)
    if n < 4 or np.var(x) == 0:
        return float(n)
    xc = x - x.mean()
    f = np.fft.rfft(xc, 2 * n)
    acov = np.fft.irfft(f * np.conj(f), 2 * n)[:n] / n
    rho = acov / acov[0]
    tau, prev = -1.0, math.inf
    for m in range(n // 2):
        gm = rho[2 * m] + rho[2 * m + 1]
        if gm <= 0:
            break
        gm = min(gm, prev)
        tau += 2.0 * gm
        prev = gm
    return float(n / max(tau, 1.0 / math.log10(n)))


def ess_all(draws) -> np.ndarray:
    return np.array([ess(draws[:, j]) for j in range(draws.shape[1])])
