"""Pins of the surrogate-MLP oracle: finite differences, Adam's first step,
round-to-nearest-even BF16 against torch's conversion."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo


def rand_problem(seed=0, n=9):
    rng = np.random.default_rng(seed)
    w = rng.normal(0, 0.3, mo.PARAM_COUNT)
    x = rng.normal(size=(n, 6))
    t = rng.normal(size=(n, 6))
    return w, x, t


def test_loss_gradient_finite_differences():
    w, x, t = rand_problem()
    loss, g = mo.loss_grad(w, x, t)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(mo.PARAM_COUNT, 60, replace=False), [768, 17280, 18176, 18181]])
    for i in idx:
        h = 1e-5
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mo.loss_grad(wp, x, t)[0] - mo.loss_grad(wm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(g[i]), (i, fd, g[i])


def test_adam_first_step_moves_by_lr_times_sign():
    rng = np.random.default_rng(2)
    w, g = rng.normal(size=50), rng.normal(size=50)
    w1, m1, v1 = mo.adam_step(w, np.zeros(50), np.zeros(50), g, lr=1e-3, b1=0.9, b2=0.999, eps=0.0, step=1)
    np.testing.assert_allclose(w1 - w, -1e-3 * np.sign(g), rtol=1e-12)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)


def test_bf16_rounding_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(size=2000).astype(np.float32),
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 3.0e38, 1e-40], np.float32)])
    ours = mo.bf16_round(x)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours, ref)
    # exact ties go to the even mantissa
    assert mo.bf16_round(np.float32(1 + 2 ** -8)) == np.float32(1.0)
    assert mo.bf16_round(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)
