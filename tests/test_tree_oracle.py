"""Pins of the tree-prior oracle (Section 2.2, Eq. 2) and of the host-side
traversal plan, on the CPU.

The oracle's V is pinned to: the generator's covariance (built a different way,
from node heights); a two-tip and a three-tip tree worked by hand; the
empirical covariance of Brownian motion simulated down the tree; and scipy's
multivariate normal density.  Its gradient is pinned by finite differences.
"""
import ctypes

import numpy as np
import pytest
from scipy import stats

from oracle import tree_oracle
from paper_2103_03348_b300 import synth


def small_tree():
    # tips 0, 1, 2; node 3 joins 0 and 1; node 4 (root) joins 3 and 2
    parent = np.array([3, 3, 4, 4, -1])
    length = np.array([0.5, 0.7, 1.6, 0.4, 0.0])
    return parent, length


def test_three_tip_tree_by_hand():
    parent, length = small_tree()
    v = tree_oracle.tree_cov(parent, length, root_var=0.3)
    # root-to-tip paths: tip 0 = 0.5 + 0.4, tip 1 = 0.7 + 0.4, tip 2 = 1.6; tips 0, 1 share 0.4
    want = 0.3 + np.array([[0.9, 0.4, 0.0], [0.4, 1.1, 0.0], [0.0, 0.0, 1.6]])
    np.testing.assert_allclose(v, want, rtol=0, atol=1e-15)


def test_two_tip_closed_form():
    parent, length = np.array([2, 2, -1]), np.array([0.8, 1.5, 0.0])
    a, b, tau0, s2 = 0.8, 1.5, 0.6, 2.5
    z = np.array([0.3, -1.1])
    ld, pz, pd = tree_oracle.tree_prior(z, parent, length, tau0, s2)
    det = s2 * s2 * ((tau0 + a) * (tau0 + b) - tau0 * tau0)
    inv = np.array([[tau0 + b, -tau0], [-tau0, tau0 + a]]) * s2 / det
    want = -np.log(2 * np.pi) - 0.5 * np.log(det) - 0.5 * z @ inv @ z
    assert abs(ld - want) <= 1e-14 * abs(want)
    np.testing.assert_allclose(pz, inv @ z, rtol=1e-14)
    np.testing.assert_allclose(pd, np.diag(inv), rtol=1e-14)


def test_matches_generator_covariance():
    w = synth.make_ebola_like(seed=5, n=900, m_seq=150, box=120.0, t_max=120.0, n_hot=4)
    v = tree_oracle.tree_cov(w.tree_parent, w.tree_length, root_var=0.0)
    np.testing.assert_allclose(v, w.tree_cov, rtol=1e-13, atol=1e-13)


def test_simulated_brownian_covariance():
    parent, length = small_tree()
    tau0, s2 = 0.3, 1.7
    draws = tree_oracle.simulate(np.random.default_rng(3), parent, length, tau0, s2, 400_000)
    emp = np.cov(draws.T)
    want = s2 * tree_oracle.tree_cov(parent, length, tau0)
    # standard error of a covariance estimate ~ sqrt((S_ii S_jj + S_ij^2) / n) <~ 0.01 here
    assert np.max(np.abs(emp - want)) < 0.02


def test_density_against_scipy_and_finite_differences():
    w = synth.make_ebola_like(seed=9, n=600, m_seq=60, box=120.0, t_max=120.0, n_hot=4)
    tau0, s2 = 0.25, 0.8
    z = np.random.default_rng(2).normal(size=60)
    ld, pz, pd = tree_oracle.tree_prior(z, w.tree_parent, w.tree_length, tau0, s2)
    cov = s2 * (tau0 + w.tree_cov)
    assert abs(ld - stats.multivariate_normal(np.zeros(60), cov).logpdf(z)) <= 1e-11 * abs(ld)
    h = 1e-5
    for k in range(0, 60, 7):
        e = np.zeros(60)
        e[k] = h
        fd = (tree_oracle.tree_prior(z + e, w.tree_parent, w.tree_length, tau0, s2)[0]
              - tree_oracle.tree_prior(z - e, w.tree_parent, w.tree_length, tau0, s2)[0]) / (2 * h)
        assert abs(-pz[k] - fd) <= 1e-6 * max(1.0, abs(fd))
        # the log density is quadratic, so a wide second difference is exact up to roundoff
        e2 = 0.1 * e / h
        d2 = (tree_oracle.tree_prior(z + e2, w.tree_parent, w.tree_length, tau0, s2)[0] - 2 * ld
              + tree_oracle.tree_prior(z - e2, w.tree_parent, w.tree_length, tau0, s2)[0]) / 0.01
        assert abs(-pd[k] - d2) <= 1e-8 * pd[k]


# ---------------------------------------------------------------- host plan


@pytest.fixture(scope="module")
def tree_mod():
    from paper_2103_03348_b300 import build, tree
    build.build()
    return tree


def check_plan(plan, parent):
    parent = np.asarray(parent)
    nn = parent.size
    m = (nn + 1) // 2
    levels, mm = int(plan[0]), int(plan[1])
    assert mm == m
    p = plan[2:2 + nn]
    ca, cb = plan[2 + nn:2 + 2 * nn], plan[2 + 2 * nn:2 + 3 * nn]
    order = plan[2 + 3 * nn:2 + 3 * nn + m - 1]
    offs = plan[2 + 3 * nn + m - 1:2 + 3 * nn + m - 1 + levels + 1]
    np.testing.assert_array_equal(p, parent)
    assert sorted(order) == list(range(m, nn))
    assert offs[0] == 0 and offs[-1] == m - 1
    level = np.zeros(nn, int)
    for L in range(levels):
        for v in order[offs[L]:offs[L + 1]]:
            assert {ca[v], cb[v]} == set(np.flatnonzero(parent == v))
            assert level[ca[v]] <= L and level[cb[v]] <= L  # children are done before v
            assert max(level[ca[v]], level[cb[v]]) == L  # and v sits at its height
            level[v] = L + 1
    assert order[-1] == int(np.flatnonzero(parent < 0)[0])


def test_plan_of_generated_trees(tree_mod):
    for seed in range(3):
        w = synth.make_ebola_like(seed=seed, n=700, m_seq=200, box=120.0, t_max=120.0, n_hot=4)
        check_plan(tree_mod.plan(w.tree_parent), w.tree_parent)


def test_plan_of_caterpillar_and_cherry(tree_mod):
    m = 50
    parent = np.full(2 * m - 1, -1)
    parent[0] = parent[1] = m
    for k in range(2, m):
        parent[k] = m + k - 1
        parent[m + k - 2] = m + k - 1
    plan = tree_mod.plan(parent)
    assert plan[0] == m - 1
    check_plan(plan, parent)
    check_plan(tree_mod.plan([2, 2, -1]), [2, 2, -1])


@pytest.mark.parametrize("parent", [
    [3, 3, 4, -1, -1],        # two roots
    [3, 3, 3, 4, -1],         # three children
    [3, 3, 4, 4, 0],          # a tip as a parent (and no root)
    [3, 3, 4, 4, 3],          # a cycle, no root
    [4, 3, 4, 4, -1],         # node 3 has one child
    [4, 4, 3, 3, -1],         # node 3 is its own child: a loop off a rooted tree
    [2, 2, 5],                # parent out of range
])
def test_plan_rejects_non_trees(tree_mod, parent):
    from paper_2103_03348_b300 import hawkes
    with pytest.raises(hawkes.HawkesError):
        tree_mod.plan(parent)


def test_plan_size_and_bounds(tree_mod):
    L = tree_mod._lib()
    assert L.hawkes_tree_plan_size(1) == 0
    assert L.hawkes_tree_plan_size(2) > 0
    assert L.hawkes_tree_workspace_size(1) == 0
    par = np.array([2, 2, -1], dtype=np.int64)
    buf = np.zeros(4, dtype=np.int32)
    rc = L.hawkes_tree_plan(2, par.ctypes.data_as(ctypes.c_void_p), buf.ctypes.data_as(ctypes.c_void_p),
                            ctypes.c_size_t(buf.nbytes))
    assert rc == 4  # HAWKES_EWORKSPACE: the plan does not fit
    # bad scalars are rejected before any device pointer is touched
    assert L.hawkes_tree_prior(2, ctypes.c_void_p(8), ctypes.c_void_p(8), 0.0, 0.0, ctypes.c_void_p(8),
                               ctypes.c_void_p(8), ctypes.c_size_t(1 << 20), None, None, None, None) == 1
    assert L.hawkes_tree_prior(1, ctypes.c_void_p(8), ctypes.c_void_p(8), 0.0, 1.0, ctypes.c_void_p(8),
                               ctypes.c_void_p(8), ctypes.c_size_t(1 << 20), None, None, None, None) == 1
