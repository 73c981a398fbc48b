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


# ---------------------------------------------------------------------------
# Tree-structured mass matrix oracle (M_z = diag(d) + (sigma2 V)^-1)
# ---------------------------------------------------------------------------
def random_tree(rng, m, lo=0.2, hi=1.0):
    """A random rooted binary tree on m tips by joining random pairs, with
    branch lengths uniform on [lo, hi] (well conditioned V)."""
    parent = -np.ones(2 * m - 1, np.int64)
    live = list(range(m))
    nxt = m
    while len(live) > 1:
        i, j = rng.choice(len(live), 2, replace=False)
        a, b = live[i], live[j]
        parent[a] = parent[b] = nxt
        live = [v for k, v in enumerate(live) if k not in (i, j)] + [nxt]
        nxt += 1
    length = rng.uniform(lo, hi, 2 * m - 1)
    length[nxt - 1] = 0.0
    return parent, length


def test_mass_velocity_two_tip_closed_form():
    parent, length = np.array([2, 2, -1]), np.array([0.8, 1.5, 0.0])
    a, b, tau0, s2 = 0.8, 1.5, 0.6, 2.5
    d = np.array([1.3, 0.4])
    pz = np.array([0.7, -2.0])
    # (sigma2 V)^-1 by the 2 x 2 adjugate, then diag(d) + P inverted the same way
    det_v = s2 * s2 * ((tau0 + a) * (tau0 + b) - tau0 * tau0)
    P = np.array([[tau0 + b, -tau0], [-tau0, tau0 + a]]) * s2 / det_v
    Mz = np.diag(d) + P
    det_m = Mz[0, 0] * Mz[1, 1] - Mz[0, 1] * Mz[1, 0]
    want = np.array([Mz[1, 1] * pz[0] - Mz[0, 1] * pz[1], -Mz[1, 0] * pz[0] + Mz[0, 0] * pz[1]]) / det_m
    got = tree_oracle.mass_velocity(d, pz, parent, length, tau0, s2)
    np.testing.assert_allclose(got, want, rtol=1e-14)


@pytest.mark.parametrize("root_var", [0.0, 0.4])
def test_mass_velocity_equals_the_plain_solve(root_var):
    rng = np.random.default_rng(41)
    parent, length = random_tree(rng, 24)
    s2 = 1.7
    d = rng.uniform(0.0, 3.0, 24)
    d[::5] = 0.0
    pz = rng.standard_normal(24)
    C = s2 * tree_oracle.tree_cov(parent, length, root_var)
    want = np.linalg.solve(np.diag(d) + np.linalg.inv(C), pz)
    got = tree_oracle.mass_velocity(d, pz, parent, length, root_var, s2)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12 * np.abs(want).max())
    # no curvature: the velocity is the prior covariance times p
    np.testing.assert_allclose(tree_oracle.mass_velocity(-np.ones(24), pz, parent, length, root_var, s2), C @ pz,
                               rtol=1e-13, atol=1e-13 * np.abs(C @ pz).max())


def test_brownian_from_normals_has_the_tree_covariance():
    rng = np.random.default_rng(42)
    parent, length = random_tree(rng, 9)
    tau0, s2 = 0.3, 1.9
    nn = parent.size
    # the map xi -> w is linear: its columns from unit vectors give S with S S^T = Cov(w)
    S = np.stack([tree_oracle.brownian_from_normals(parent, length, tau0, s2, e)[:9] for e in np.eye(nn)], axis=1)
    np.testing.assert_allclose(S @ S.T, s2 * tree_oracle.tree_cov(parent, length, tau0), rtol=1e-13, atol=1e-14)


def test_mass_momentum_covariance_is_the_mass_matrix():
    rng = np.random.default_rng(43)
    m, z0, k = 7, 3, 12
    parent, length = random_tree(rng, m)
    tau0, s2 = 0.2, 0.8
    minv = rng.uniform(0.1, 2.0, k)
    d = rng.uniform(0.0, 2.0, m)
    d[1] = 0.0
    cols = [tree_oracle.mass_momentum(minv, d, e, z0, parent, length, tau0, s2) for e in np.eye(k + parent.size)]
    A = np.stack(cols, axis=1)
    M = np.diag(1.0 / minv)
    M[z0:z0 + m, z0:z0 + m] = np.diag(d) + tree_oracle.precision_matrix(parent, length, tau0, s2)
    np.testing.assert_allclose(A @ A.T, M, rtol=1e-10, atol=1e-12 * np.abs(M).max())
    # and the velocity inverts that same M
    p = rng.standard_normal(k)
    np.testing.assert_allclose(M @ tree_oracle.mass_full_velocity(minv, d, p, z0, parent, length, tau0, s2), p,
                               rtol=1e-10, atol=1e-11)


def joint_case(rng, m=9, nc=3, z0=4, k=16):
    parent, length = random_tree(rng, m)
    G = rng.standard_normal((nc, nc))
    A = G @ G.T + 4.0 * np.eye(nc)
    B = 0.3 * rng.standard_normal((m, nc))
    minv = rng.uniform(0.1, 2.0, k)
    d = rng.uniform(0.0, 2.0, m)
    return parent, length, A, B, minv, d, z0, k


def test_joint_mass_velocity_equals_the_plain_solve():
    rng = np.random.default_rng(44)
    parent, length, A, B, minv, d, z0, k = joint_case(rng)
    tau0, s2 = 0.3, 1.4
    M = tree_oracle.joint_mass_matrix(minv, d, A, B, z0, parent, length, tau0, s2)
    assert np.all(np.linalg.eigvalsh(M) > 0)
    p = rng.standard_normal(k)
    got = tree_oracle.joint_mass_velocity(minv, d, A, B, p, z0, parent, length, tau0, s2)
    np.testing.assert_allclose(got, np.linalg.solve(M, p), rtol=1e-11, atol=1e-12)


def test_joint_mass_momentum_covariance_is_the_mass_matrix():
    rng = np.random.default_rng(45)
    parent, length, A, B, minv, d, z0, k = joint_case(rng)
    tau0, s2 = 0.0, 0.9
    M = tree_oracle.joint_mass_matrix(minv, d, A, B, z0, parent, length, tau0, s2)
    cols = [tree_oracle.joint_mass_momentum(minv, d, A, B, e, z0, parent, length, tau0, s2)
            for e in np.eye(k + parent.size)]
    Am = np.stack(cols, axis=1)
    np.testing.assert_allclose(Am @ Am.T, M, rtol=1e-10, atol=1e-11 * np.abs(M).max())
