"""Posterior-predictive simulation on the GPU against the oracle, draw for
draw: both sides use the same Philox4x32-10 counters, so every sample's
event count, parents and statuses must be identical, and times and places
equal up to the last bits of libm-vs-CUDA exp/log/erfc/sin/cos."""
import math

import numpy as np
import pytest

from oracle import predictive_oracle as po
from paper_2103_03348_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def posterior_like(w, s_count, seed, spread=0.05):
    q0 = np.concatenate([np.log(w.params), w.r[w.sequenced]])
    rng = np.random.default_rng(seed)
    return q0[None, :] + spread * rng.standard_normal((s_count, q0.size))


def run_gpu(w, q, horizon, seed, capacity, offset=0):
    from paper_2103_03348_b300 import build, predictive
    build.build()
    return predictive.simulate(dev(w.x), dev(w.y), dev(w.t), dev(w.r), dev(w.sequenced, torch.int32), dev(q),
                               horizon, seed, capacity, sample_offset=offset)


def check_sample(w, out, s, q_row, horizon, seed, capacity, sample_index):
    ev, src, st = po.simulate(w.x, w.y, w.t, w.r, w.sequenced, q_row, horizon, seed, sample_index, capacity)
    k = int(out["count"][s])
    assert int(out["status"][s]) == st, (s, int(out["status"][s]), st)
    assert k == len(ev), (s, k, len(ev))
    np.testing.assert_array_equal(out["src"][s, :k].cpu().numpy(), src)
    for j, name in enumerate("xyt"):
        got = out[name][s, :k].cpu().numpy()
        np.testing.assert_allclose(got, ev[:, j], rtol=1e-12, atol=1e-9)
    return k


def test_parity_small_history():
    w = synth.make_ebola_like(seed=5, n=400, m_seq=30, box=120.0, t_max=120.0, n_hot=4)
    q = posterior_like(w, 24, 1)
    out = run_gpu(w, q, 10.0, 2024, 100000)
    total = sum(check_sample(w, out, s, q[s], 10.0, 2024, 100000, s) for s in range(24))
    assert total > 200


def test_parity_infinite_tau_t_and_sample_offset():
    w = synth.make_ebola_like(seed=6, n=300, m_seq=20, box=100.0, t_max=90.0, n_hot=3)
    q = posterior_like(w, 8, 2)
    q[:, 2] = math.inf
    q[:, 0] = math.log(0.4 / w.n)
    out = run_gpu(w, q, 7.5, 99, 100000, offset=1000)
    for s in range(8):
        check_sample(w, out, s, q[s], 7.5, 99, 100000, 1000 + s)


def test_overflow_bad_parameters_and_split_means():
    w = synth.make_ebola_like(seed=7, n=350, m_seq=25, box=100.0, t_max=100.0, n_hot=3)
    q = posterior_like(w, 6, 3)
    q[1, 4] = math.nan             # sample 1: invalid omega
    q[2, 6 + 24] = 9.0             # sample 2: one sequenced event with theta ~ 8100: a split Poisson mean
    last = int(np.argmax(w.t[w.sequenced]))
    q[3, 6 + last] = 8.0           # sample 3: the latest sequenced event very contagious
    out = run_gpu(w, q, 10.0, 7, 40)   # capacity 40: most samples overflow
    statuses = [int(v) for v in out["status"].cpu()]
    assert statuses[1] == po.STATUS_BADPARAM and int(out["count"][1]) == 0
    assert po.STATUS_OVERFLOW in statuses
    for s in range(6):
        check_sample(w, out, s, q[s], 10.0, 7, 40, s)
    big = run_gpu(w, q[2:4], 10.0, 7, 200000, offset=2)
    for s in range(2):
        check_sample(w, big, s, q[2 + s], 10.0, 7, 200000, 2 + s)


def test_full_size_sampled_parity_and_mean_count():
    """The 23,422-event history with 1,610 free log-rates, 30 days ahead, 512
    posterior-like settings: three samples recomputed by the oracle, and the
    mean count of 2,048 draws at fixed parameters against the branching
    expectation."""
    w = synth.make("ebola_like")
    q = posterior_like(w, 512, 4, spread=0.02)
    out = run_gpu(w, q, 30.0, 31337, 20000)
    assert (out["status"] == 0).all()
    for s in (0, 1, 511):
        check_sample(w, out, s, q[s], 30.0, 31337, 20000, s)
    q0 = np.repeat(np.concatenate([np.log(w.params), w.r[w.sequenced]])[None, :], 2048, axis=0)
    fixed = run_gpu(w, q0, 30.0, 5, 20000)
    c = fixed["count"].cpu().numpy().astype(float)
    expect = po.expected_count(w.t, w.r, w.params, 30.0)
    assert abs(c.mean() - expect) < 4.0 * c.std() / math.sqrt(c.size), (c.mean(), expect)
