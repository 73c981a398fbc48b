"""Learned gradient surrogate for HMC over the six global parameters.

A 6 -> 128 -> 128 -> 6 tanh MLP (BF16 weights, FP32 accumulation, trained by
the library's own forward/backward and Adam kernels) learns the map from the
log-globals q to the gradient of the log posterior, from (q, gradient) pairs
that the exact kernel produces along exact HMC warm-up trajectories.  Sampling
then integrates each leapfrog trajectory with the surrogate gradient (one fused
kernel per step) and accepts with the exact log posterior at the end point
(one log-likelihood pass).  A leapfrog map driven by any smooth vector field
stays volume preserving and reversible, so the exact Metropolis step keeps
the exact posterior invariant.  If the acceptance rate collapses the sampler
falls back to exact gradients.

Inputs and outputs are standardised with the training set's mean and standard
deviation: g(q) = mean_g + sd_g * MLP((q - mean_q) / sd_q).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import time

import numpy as np
import torch

from . import hawkes, hmc

MI, MH, MO = 6, 128, 6


def _lib():
    L = hmc._lib()
    if not getattr(L, "_mlp_typed", False):
        vp, i64, f = ctypes.c_void_p, ctypes.c_int64, ctypes.c_float
        L.hawkes_mlp_param_count.restype = ctypes.c_size_t
        L.hawkes_mlp_workspace_size.argtypes = [i64]
        L.hawkes_mlp_workspace_size.restype = ctypes.c_size_t
        L.hawkes_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
        L.hawkes_mlp_loss_grad.argtypes = [vp, vp, vp, i64, vp, ctypes.c_size_t, vp, vp, vp]
        L.hawkes_mlp_adam.argtypes = [vp, vp, vp, vp, vp, f, f, f, f, ctypes.c_int, vp]
        L.hawkes_mlp_adam_table.argtypes = [f, f, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
        L.hawkes_mlp_adam_device.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.c_int, vp, f, f, f, vp]
        L.hawkes_surrogate_momentum.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp, vp]
        L.hawkes_surrogate_trajectory.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_int, vp]
        L.hawkes_surrogate_trajectory_dense.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_int, vp]
        for fn in (L.hawkes_mlp_forward, L.hawkes_mlp_loss_grad, L.hawkes_mlp_adam, L.hawkes_surrogate_momentum,
                   L.hawkes_surrogate_trajectory, L.hawkes_surrogate_trajectory_dense, L.hawkes_mlp_adam_table,
                   L.hawkes_mlp_adam_device):
            fn.restype = ctypes.c_int
        L._mlp_typed = True
    return L


_p = hmc._ptr
_check = hmc._check


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


class MLP:
    """Weights (FP32 master + BF16 working copy) and Adam state on the device."""

    def __init__(self, device="cuda", seed=0):
        L = _lib()
        self.dev = torch.device(device)
        self.count = int(L.hawkes_mlp_param_count())
        rng = np.random.default_rng(seed)
        w = np.zeros(self.count, np.float32)
        off = 0
        for fan_out, fan_in in ((MH, MI), (MH, MH), (MO, MH)):
            lim = math.sqrt(6.0 / (fan_in + fan_out))  # Glorot uniform, zero biases
            w[off:off + fan_out * fan_in] = rng.uniform(-lim, lim, fan_out * fan_in)
            off += fan_out * fan_in + fan_out
        self.wm = torch.tensor(w, device=self.dev)
        self.wb = self.wm.to(torch.bfloat16)
        self.m = torch.zeros_like(self.wm)
        self.v = torch.zeros_like(self.wm)
        self.grad = torch.zeros_like(self.wm)
        self.loss = torch.zeros((), dtype=torch.float32, device=self.dev)
        self.step = 0

    def loss_grad(self, x, y):
        L = _lib()
        ws = torch.empty(int(L.hawkes_mlp_workspace_size(x.shape[0])), dtype=torch.uint8, device=self.dev)
        _check(L.hawkes_mlp_loss_grad(_p(self.wb), _p(x), _p(y), x.shape[0], _p(ws), ctypes.c_size_t(ws.numel()),
                                      _p(self.grad), _p(self.loss), _stream(self.dev)))
        return self.loss, self.grad

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        _check(_lib().hawkes_mlp_adam(_p(self.wm), _p(self.wb), _p(self.m), _p(self.v), _p(self.grad), lr, beta1,
                                      beta2, eps, self.step, _stream(self.dev)))

    def forward(self, x):
        y = torch.empty(x.shape[0], MO, dtype=torch.float32, device=self.dev)
        _check(_lib().hawkes_mlp_forward(_p(self.wb), _p(x), x.shape[0], _p(y), _stream(self.dev)))
        return y

    def adam_table(self, first_step, steps, beta1=0.9, beta2=0.999):
        """Device table of Adam's bias corrections for steps first_step .. first_step + steps - 1."""
        host = (ctypes.c_float * (2 * (first_step + steps - 1)))()
        _check(_lib().hawkes_mlp_adam_table(beta1, beta2, first_step + steps - 1, host))
        t = torch.tensor(np.frombuffer(host, dtype=np.float32), device=self.dev)
        return t[2 * (first_step - 1):].contiguous()

    def train(self, x, y, epochs=200, batch=256, lr=1e-3, seed=0, use_graph=True):
        """Minibatch Adam on the mean squared error (cosine-decayed learning rate);
        returns the per-epoch mean loss.

        Each minibatch step gathers its rows, runs the loss-gradient kernels and
        a device-step Adam update (step, learning rate and bias corrections read
        from device memory).  With use_graph the first epoch runs eagerly and the
        epoch's steps are then captured once as a CUDA graph and replayed for the
        other epochs (one launch per epoch instead of several per step); the
        weights equal those of eager training bit for bit."""
        n = x.shape[0]
        L = _lib()
        nb = max((n - batch) // batch + 1, 0) if n >= batch else 0
        ws = torch.empty(int(L.hawkes_mlp_workspace_size(batch)), dtype=torch.uint8, device=self.dev)
        gen = torch.Generator(device=self.dev)
        gen.manual_seed(seed)
        perm = torch.empty(n, dtype=torch.int64, device=self.dev)
        xb = torch.empty(batch, x.shape[1], dtype=x.dtype, device=self.dev)
        yb = torch.empty(batch, y.shape[1], dtype=y.dtype, device=self.dev)
        total_steps = epochs * nb
        table = self.adam_table(self.step + 1, max(total_steps, 1))
        step_dev = torch.zeros(1, dtype=torch.int32, device=self.dev)
        lr_dev = torch.empty(1, dtype=torch.float32, device=self.dev)
        tot = torch.zeros((), dtype=torch.float32, device=self.dev)

        def epoch_body():
            s = _stream(self.dev)
            for b in range(nb):
                idx = perm[b * batch:(b + 1) * batch]
                torch.index_select(x, 0, idx, out=xb)
                torch.index_select(y, 0, idx, out=yb)
                _check(L.hawkes_mlp_loss_grad(_p(self.wb), _p(xb), _p(yb), batch, _p(ws), ctypes.c_size_t(ws.numel()),
                                              _p(self.grad), _p(self.loss), s))
                _check(L.hawkes_mlp_adam_device(_p(self.wm), _p(self.wb), _p(self.m), _p(self.v), _p(self.grad),
                                                _p(lr_dev), _p(table), max(total_steps, 1), _p(step_dev), 0.9, 0.999,
                                                1e-8, s))
                tot.add_(self.loss)

        history, graph = [], None
        for ep in range(epochs):
            torch.randperm(n, generator=gen, device=self.dev, out=perm)
            lr_ep = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))  # cosine decay
            lr_dev.fill_(max(lr_ep, 1e-5))
            tot.zero_()
            if graph is not None:
                graph.replay()
            elif use_graph and ep > 0 and nb > 0:
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    epoch_body()
                graph.replay()  # capture records the kernels without running them
            else:
                epoch_body()
            history.append(float(tot.item()) / max(nb, 1))
        self.step += total_steps
        return history


@dataclasses.dataclass
class Surrogate:
    mlp: MLP
    norm: torch.Tensor  # [24] doubles: mean_q, sd_q, mean_g, sd_g

    def gradient(self, q):
        g = torch.empty(MO, dtype=torch.float64, device=q.device)
        _check(_lib().hawkes_surrogate_momentum(_p(self.mlp.wb), _p(q), ctypes.c_void_p(0), 0.0, _p(self.norm),
                                                _p(g), _stream(q.device)))
        return g


def fit(q_pairs, g_pairs, epochs=200, batch=256, lr=1e-3, seed=0, holdout=0.1):
    """Train a surrogate on exact (q, gradient) pairs (device float64 [n, 6]).

    The gradient is modelled as mean_g + A (q - mean_q) (least squares) plus the
    MLP's standardised residual, so the network only learns what the linear
    model misses (near the posterior mode the gradient is close to linear).
    Returns (Surrogate, report); the report's holdout_rel_error is the relative
    RMS error on held-out pairs, sqrt(sum ||pred - exact||^2 / sum ||exact||^2)."""
    n = q_pairs.shape[0]
    gen = torch.Generator(device=q_pairs.device)
    gen.manual_seed(seed + 1)
    perm = torch.randperm(n, generator=gen, device=q_pairs.device)
    n_hold = max(1, int(holdout * n))
    tr, ho = perm[n_hold:], perm[:n_hold]
    qt, gt = q_pairs[tr], g_pairs[tr]
    mq, sq = qt.mean(0), qt.std(0).clamp_min(1e-12)
    mg = gt.mean(0)
    # least-squares linear part (a 6 x 6 solve on the host)
    dq = (qt - mq).cpu().numpy()
    dg = (gt - mg).cpu().numpy()
    A = np.linalg.lstsq(dq, dg, rcond=None)[0].T  # dg ~ dq A^T
    A_t = torch.tensor(A, dtype=torch.float64, device=q_pairs.device)
    resid = lambda q, g: g - mg - (q - mq) @ A_t.T  # noqa: E731
    sg = resid(qt, gt).std(0).clamp_min(1e-12)
    norm = torch.cat([mq, sq, mg, sg, A_t.reshape(-1)]).contiguous()
    xs = ((q_pairs - mq) / sq).float().contiguous()
    ys = (resid(q_pairs, g_pairs) / sg).float().contiguous()
    mlp = MLP(q_pairs.device, seed)
    t0 = time.perf_counter()
    hist = mlp.train(xs[tr].contiguous(), ys[tr].contiguous(), epochs, min(batch, len(tr)), lr, seed)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    sur = Surrogate(mlp, norm)
    qh = q_pairs[ho]
    pred = mg + (qh - mq) @ A_t.T + mlp.forward(xs[ho].contiguous()).double() * sg
    lin = mg + (qh - mq) @ A_t.T
    return sur, {"train_pairs": int(len(tr)), "holdout_pairs": int(n_hold), "epochs": epochs,
                 "train_seconds": train_s, "final_train_loss": hist[-1],
                 "holdout_rel_error": relative_error(pred, g_pairs[ho]),
                 "holdout_median_rel_error": median_rel_error(pred, g_pairs[ho]),
                 "holdout_rel_error_linear_only": relative_error(lin, g_pairs[ho])}


def relative_error(pred, exact):
    """Relative RMS error: sqrt(sum ||pred - exact||^2 / sum ||exact||^2)."""
    num = torch.sum((pred - exact) ** 2)
    den = torch.sum(exact ** 2).clamp_min(1e-300)
    return float(torch.sqrt(num / den).item())


def median_rel_error(pred, exact):
    """Median over pairs of ||pred - exact||, relative to the RMS of ||exact||:
    robust to the few warm-up excursions whose gradients are huge."""
    err = torch.linalg.vector_norm(pred - exact, dim=-1)
    rms = torch.sqrt(torch.mean(torch.sum(exact ** 2, dim=-1))).clamp_min(1e-300)
    return float((torch.median(err) / rms).item())


def collect_pairs(post, q0, n_pairs, n_steps=20, eps0=0.02, mass_every=50, seed=0, target_accept=0.8,
                  burn_iters=100, mass="diag", jitter=0.0):
    """Exact HMC warm-up over the globals that records (q, gradient) at every
    leapfrog step after the first `burn_iters` iterations (which move the chain
    from its start to the posterior); returns (q_pairs, g_pairs, chain state).
    mass: "diag" (Section 2.3.2) or "dense" (hmc.sample); the chain state's
    mass_t is then the diagonal tensor or the DenseMassOp."""
    dev = q0.device
    dim = q0.numel()
    n_iter = int(math.ceil(n_pairs / n_steps))
    qs = torch.empty(n_iter * n_steps, dim, dtype=torch.float64, device=dev)
    gs = torch.empty(n_iter * n_steps, dim, dtype=torch.float64, device=dev)
    counter = [0]
    skip = burn_iters * n_steps

    def record(q, g):
        i = counter[0] - skip
        if 0 <= i < qs.shape[0]:
            qs[i].copy_(q)
            gs[i].copy_(g)
        counter[0] += 1

    ch = hmc.sample(post, q0, n_iter=0, n_warmup=n_iter + burn_iters, n_steps=n_steps, eps0=eps0, mass=mass,
                    jitter=jitter,
                    mass_every=mass_every, seed=seed, target_accept=target_accept, record=record)
    k = min(max(counter[0] - skip, 0), qs.shape[0])
    qs, gs = qs[:k], gs[:k]
    # positions of divergent trajectories (early in the step-size adaptation)
    # carry non-finite or huge gradients: keep finite pairs whose gradient norm
    # is within 50x the median
    ok = torch.isfinite(qs).all(1) & torch.isfinite(gs).all(1)
    qs, gs = qs[ok], gs[ok]
    gn = torch.linalg.vector_norm(gs, dim=1)
    keep = gn <= 50.0 * torch.median(gn)
    qs, gs = qs[keep][:n_pairs], gs[keep][:n_pairs]
    return qs.contiguous(), gs.contiguous(), ch


def surrogate_leapfrog(sur, q, p, eps, n_steps, minv):
    """Leapfrog trajectory over the six globals driven by the surrogate gradient:
    one launch of the fused trajectory kernel.  minv: the diagonal inverse
    mass (device tensor) or an hmc.DenseMassOp."""
    if isinstance(minv, hmc.DenseMassOp):
        _check(_lib().hawkes_surrogate_trajectory_dense(_p(sur.mlp.wb), _p(sur.norm), _p(q), _p(p), _p(minv.minv),
                                                        eps, n_steps, _stream(q.device)))
        return
    _check(_lib().hawkes_surrogate_trajectory(_p(sur.mlp.wb), _p(sur.norm), _p(q), _p(p), _p(minv), eps, n_steps,
                                              _stream(q.device)))


def surrogate_leapfrog_steps(sur, q, p, eps, n_steps, minv):
    """The same trajectory as one surrogate-momentum and one position launch per
    step (the fused kernel's definition; tests compare the two)."""
    L = _lib()
    s = _stream(q.device)
    w, nrm = _p(sur.mlp.wb), _p(sur.norm)
    _check(L.hawkes_surrogate_momentum(w, _p(q), _p(p), 0.5 * eps, nrm, ctypes.c_void_p(0), s))
    for step in range(n_steps):
        if isinstance(minv, hmc.DenseMassOp):
            minv.position(q, p, eps)
        else:
            _check(L.hawkes_hmc_position(q.numel(), _p(q), _p(p), _p(minv), eps, s))
        _check(L.hawkes_surrogate_momentum(w, _p(q), _p(p), eps if step < n_steps - 1 else 0.5 * eps, nrm,
                                           ctypes.c_void_p(0), s))


class _SurrogateIteration:
    """The device part of one surrogate HMC iteration after the momentum draw,
    captured once as a CUDA graph: kinetic energy at the start, the fused
    surrogate trajectory from a copy of q, the exact log posterior at its end
    point (one log-likelihood pass) and the kinetic energy there.  The four
    numbers the accept step needs land in one device vector
    e = [log pi(q), K(p0), log pi(q'), K(p')], read back with one copy."""

    def __init__(self, post, sur, q, p, minv, eps, n_steps, use_graph=True, qn=None, e=None):
        dev = q.device
        f64 = dict(dtype=torch.float64, device=dev)
        self.post, self.sur, self.eps, self.n_steps = post, sur, eps, n_steps
        self.q, self.p, self.minv = q, p, minv
        self.qn = torch.empty_like(q) if qn is None else qn  # buffers that several step sizes' graphs share
        self.e = torch.zeros(4, **f64) if e is None else e
        self.cur = {"logpost": self.e[0]}
        self.cand = {"logpost": self.e[2]}
        self.graph = None
        if use_graph:
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(side):  # one eager run first, so every lazily made buffer exists
                self._body()
            torch.cuda.current_stream(dev).wait_stream(side)
            torch.cuda.synchronize(dev)
            calls = dict(post.calls)
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._body()
            post.calls.update(calls)

    def _body(self):
        hmc.kinetic(self.p, self.minv, self.e[1])
        self.qn.copy_(self.q)
        surrogate_leapfrog(self.sur, self.qn, self.p, self.eps, self.n_steps, self.minv)
        self.post.logpost_only(self.qn, self.cand)
        hmc.kinetic(self.p, self.minv, self.e[3])

    def run(self):
        if self.graph is not None:
            self.graph.replay()
            self.post.calls["loglik"] = self.post.calls.get("loglik", 0) + 1
        else:
            self._body()
        return self.e.cpu().numpy()  # the iteration's one host synchronisation


@dataclasses.dataclass
class SurrogateChain:
    draws: np.ndarray
    accept: np.ndarray
    seconds: float
    exact_loglik_calls: int
    fell_back: bool
    fallback_at: int
    monitor_errors: list


def sample(post, sur, q0, mass, eps, n_iter, n_steps=20, seed=0, monitor_every=100, fallback_window=50,
           fallback_rate=0.2, use_graph=True, jitter=0.0):
    """Surrogate-trajectory HMC with the exact Metropolis accept.  mass: the
    diagonal mass (device tensor) or an hmc.DenseMassOp; jitter: step-size
    levels as in hmc.sample (one captured iteration per level).

    Each iteration draws the momentum, then runs the captured iteration graph
    (fused surrogate trajectory, exact log posterior at the end point, both
    kinetic energies) and reads its four energies back in one copy: one host
    synchronisation per iteration.  The draws stay on the device until the end.
    Every `monitor_every` iterations the exact gradient at the current state
    measures the surrogate's relative error.  If the acceptance rate over the last
    `fallback_window` iterations drops below `fallback_rate`, the remaining
    iterations use exact gradients."""
    dev = q0.device
    dim = q0.numel()
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    f64 = dict(dtype=torch.float64, device=dev)
    q = q0.clone()
    dense = isinstance(mass, hmc.DenseMassOp)
    minv = mass if dense else 1.0 / mass  # what the trajectory and the kinetic energy apply
    sqrt_mass = None if dense else torch.sqrt(mass)
    xi = torch.empty(dim, **f64)
    p = torch.empty(dim, **f64)

    def draw_momentum(g):
        if dense:
            torch.randn(dim, generator=g, out=xi, dtype=torch.float64, device=dev)
            mass.draw(xi, p)
        else:
            torch.randn(dim, generator=g, out=p, dtype=torch.float64, device=dev)
            p.mul_(sqrt_mass)

    warm_gen = torch.Generator(device=dev)
    warm_gen.manual_seed(seed + 1)
    draw_momentum(warm_gen)  # a plausible momentum for the eager run that precedes the capture
    levels = hmc.jitter_levels(jitter)
    its = []
    for f in levels:
        its.append(_SurrogateIteration(post, sur, q, p, minv, eps * f, n_steps, use_graph=use_graph,
                                       qn=its[0].qn if its else None, e=its[0].e if its else None))
        draw_momentum(warm_gen)
    it_dev = its[0]
    post.logpost_only(q, it_dev.cur)  # log pi at the start (the eager runs used e as scratch)
    scratch = {"logpost": torch.empty((), **f64), "grad": torch.empty(dim, **f64), "hdiag": torch.empty(dim, **f64)}
    k1 = torch.empty((), **f64)
    draws_dev = torch.empty(n_iter, dim, **f64)
    acc = np.zeros(n_iter, bool)
    errors, fell_back, fb_at, calls = [], False, -1, 1
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(n_iter):
        draw_momentum(gen)
        lvl = int(rng.integers(len(levels))) if len(levels) > 1 else 0
        if fell_back:
            hmc.kinetic(p, minv, it_dev.e[1])
            qn = q.clone()
            g0 = post.evaluate(q, out=scratch)["grad"].clone()
            ev = hmc.leapfrog(post, qn, p, g0, eps * levels[lvl], n_steps, minv, scratch)
            it_dev.e[2].copy_(ev["logpost"])
            hmc.kinetic(p, minv, k1)
            it_dev.e[3].copy_(k1)
            e = it_dev.e.cpu().numpy()
        else:
            e = its[lvl].run()
            qn = it_dev.qn
            calls += 1
        h0 = -e[0] + e[1]
        h1 = -e[2] + e[3]
        a = min(1.0, math.exp(min(0.0, h0 - h1))) if math.isfinite(e[2]) and math.isfinite(h1) else 0.0
        if rng.uniform() < a:
            q.copy_(qn)
            it_dev.e[0].copy_(it_dev.e[2])
            acc[it] = True
        draws_dev[it].copy_(q)
        if monitor_every and (it + 1) % monitor_every == 0 and not fell_back:
            exact = post.evaluate(q, out=scratch)["grad"][:MO]
            errors.append(relative_error(sur.gradient(q)[None], exact[None]))
        if (not fell_back and it + 1 >= fallback_window
                and acc[it + 1 - fallback_window:it + 1].mean() < fallback_rate):
            fell_back, fb_at = True, it + 1
    draws = draws_dev.cpu().numpy()
    torch.cuda.synchronize()
    return SurrogateChain(draws, acc, time.perf_counter() - t0, calls, fell_back, fb_at, errors)
