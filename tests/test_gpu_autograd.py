"""The differentiable log-likelihood (torch.autograd.Function over the fused
forward + adjoint) against finite differences, at the full 100,000 events."""
import numpy as np
import pytest

from paper_2103_03348_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autograd_function_matches_fused_gradient():
    from paper_2103_03348_b300 import build, hawkes
    build.build()
    w = synth.make_uniform(5, 3000, r_sd=0.4)
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    x, y, t = d(w.x), d(w.y), d(w.t)
    r = d(w.r).requires_grad_(True)
    p = torch.tensor(w.params, dtype=torch.float64, requires_grad=True)
    ll = hawkes.HawkesLogLik.apply(x, y, t, r, p, "fp32c")
    (3.0 * ll).backward()
    _, g = hawkes.grad(x, y, t, d(w.r), w.params, "fp32c")
    g = g.cpu().numpy()
    np.testing.assert_allclose(r.grad.cpu().numpy(), 3.0 * g[6:], rtol=1e-15, atol=0)
    np.testing.assert_allclose(p.grad.numpy(), 3.0 * g[:6], rtol=1e-15, atol=0)


def test_fused_adjoint_vs_finite_differences_at_64_coordinates():
    """Central differences of the FP64 GPU log-likelihood at the six globals and
    58 random log-rates, against the FP32C adjoint returned by backward()."""
    from paper_2103_03348_b300 import build, hawkes
    build.build()
    w = synth.make("large")
    d = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    x, y, t = d(w.x), d(w.y), d(w.t)
    r = d(w.r).requires_grad_(True)
    p = torch.tensor(w.params, dtype=torch.float64, requires_grad=True)
    hawkes.HawkesLogLik.apply(x, y, t, r, p, "fp32c").backward()
    adj = np.concatenate([p.grad.numpy(), r.grad.cpu().numpy()])
    rng = np.random.default_rng(64)
    rates = rng.choice(w.n, 58, replace=False)
    coords = list(range(6)) + [6 + int(m) for m in rates]
    fd = []
    for k in coords:
        if k < 6:
            h = 1e-4 * w.params[k]
            pp, pm = w.params.copy(), w.params.copy()
            pp[k] += h
            pm[k] -= h
            lp = hawkes.loglik(x, y, t, d(w.r), pp, "fp64").item()
            lm = hawkes.loglik(x, y, t, d(w.r), pm, "fp64").item()
        else:
            h = 1e-3
            rp, rm = w.r.copy(), w.r.copy()
            rp[k - 6] += h
            rm[k - 6] -= h
            lp = hawkes.loglik(x, y, t, d(rp), w.params, "fp64").item()
            lm = hawkes.loglik(x, y, t, d(rm), w.params, "fp64").item()
        fd.append((lp - lm) / (2 * h))
    fd = np.array(fd)
    a = adj[coords]
    # central differences carry O(h^2) truncation and ~1e-16 |l| / h roundoff
    scale = np.maximum(np.abs(fd), 1e-2 * np.abs(fd).max())
    assert np.max(np.abs(a - fd) / scale) <= 2e-3, np.max(np.abs(a - fd) / scale)
    assert np.linalg.norm(a - fd) <= 1e-5 * np.linalg.norm(fd) + 1e-4 * np.linalg.norm(fd[6:])
