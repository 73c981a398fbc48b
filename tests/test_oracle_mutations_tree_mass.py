"""The pins of the tree-structured mass oracle have teeth: plausible one-line
slips planted in a copy of oracle/tree_oracle.py (executed as a module of its
own, on the CPU) are each caught by at least one of its pins, re-run here in
compact form."""
import inspect
import types

import numpy as np
import pytest

from oracle import tree_oracle
from test_tree_oracle import random_tree

SRC = inspect.getsource(tree_oracle)

MUTATIONS = {
    "Woodbury correction added": ("return Cb - C @ (s * np.linalg.solve(K, s * Cb))",
                                  "return Cb + C @ (s * np.linalg.solve(K, s * Cb))"),
    "curvature not square-rooted": ("    s = np.sqrt(dd)\n", "    s = dd\n"),
    "refinement residual sign": ("v = v + woodbury(p_z - dd * v - pv)", "v = v + woodbury(p_z - dd * v + pv)"),
    "Brownian root term dropped": ("base = np.sqrt(sigma2 * root_var) * xi[root]", "base = 0.0"),
    "Brownian branch without sigma^2": ("np.sqrt(sigma2 * length[e]) * xi[e]", "np.sqrt(length[e]) * xi[e]"),
    "momentum without sqrt(d)": ("p[z0:z0 + m] = np.sqrt(np.maximum(np.asarray(d, float), 0.0)) * xi[z0:z0 + m] + pw",
                                 "p[z0:z0 + m] = np.maximum(np.asarray(d, float), 0.0) * xi[z0:z0 + m] + pw"),
    "momentum scaled by minv": ("p = xi[:k] / np.sqrt(minv)", "p = xi[:k] * np.sqrt(minv)"),
    "Schur complement sign": ("S = A - B.T @ U", "S = A + B.T @ U"),
    "rate block correction sign": ("x[z0:z0 + m] = y - U @ xg", "x[z0:z0 + m] = y + U @ xg"),
    "coupled momentum mean dropped": ("p[:nc] = U.T @ p[z0:z0 + m] + np.linalg.cholesky",
                                      "p[:nc] = 0.0 * p[:nc] + np.linalg.cholesky"),
}


def mutated(old, new):
    assert SRC.count(old) >= 1, old
    mod = types.ModuleType("tree_oracle_mutant")
    mod.__file__ = tree_oracle.__file__
    exec(compile(SRC.replace(old, new, 1), tree_oracle.__file__, "exec"), mod.__dict__)
    return mod


def two_tip(mod):
    a, b, tau0, s2 = 0.8, 1.5, 0.6, 2.5
    d, pz = np.array([1.3, 0.4]), np.array([0.7, -2.0])
    det_v = s2 * s2 * ((tau0 + a) * (tau0 + b) - tau0 * tau0)
    Mz = np.diag(d) + np.array([[tau0 + b, -tau0], [-tau0, tau0 + a]]) * s2 / det_v
    got = mod.mass_velocity(d, pz, np.array([2, 2, -1]), np.array([a, b, 0.0]), tau0, s2)
    return np.allclose(got, np.linalg.solve(Mz, pz), rtol=1e-13)


def plain_solve(mod):
    rng = np.random.default_rng(41)
    parent, length = random_tree(rng, 12)
    d = rng.uniform(0.0, 3.0, 12)
    pz = rng.standard_normal(12)
    C = 1.7 * tree_oracle.tree_cov(parent, length, 0.4)
    got = mod.mass_velocity(d, pz, parent, length, 0.4, 1.7)
    return np.allclose(got, np.linalg.solve(np.diag(d) + np.linalg.inv(C), pz), rtol=1e-10, atol=1e-12)


def brownian_covariance(mod):
    rng = np.random.default_rng(42)
    parent, length = random_tree(rng, 6)
    S = np.stack([mod.brownian_from_normals(parent, length, 0.3, 1.9, e)[:6] for e in np.eye(parent.size)], axis=1)
    return np.allclose(S @ S.T, 1.9 * tree_oracle.tree_cov(parent, length, 0.3), rtol=1e-12, atol=1e-13)


def momentum_covariance(mod):
    rng = np.random.default_rng(43)
    m, z0, k = 5, 3, 10
    parent, length = random_tree(rng, m)
    minv = rng.uniform(0.1, 2.0, k)
    d = rng.uniform(0.2, 2.0, m)
    A = np.stack([mod.mass_momentum(minv, d, e, z0, parent, length, 0.2, 0.8) for e in np.eye(k + parent.size)], axis=1)
    M = np.diag(1.0 / minv)
    M[z0:z0 + m, z0:z0 + m] = np.diag(d) + tree_oracle.precision_matrix(parent, length, 0.2, 0.8)
    return np.allclose(A @ A.T, M, rtol=1e-9, atol=1e-11 * np.abs(M).max())


def joint_case():
    rng = np.random.default_rng(44)
    m, nc, z0, k = 7, 3, 4, 14
    parent, length = random_tree(rng, m)
    G = rng.standard_normal((nc, nc))
    return rng, parent, length, G @ G.T + 4.0 * np.eye(nc), 0.3 * rng.standard_normal((m, nc)), \
        rng.uniform(0.1, 2.0, k), rng.uniform(0.1, 2.0, m), z0, k


def joint_solve(mod):
    rng, parent, length, A, B, minv, d, z0, k = joint_case()
    M = tree_oracle.joint_mass_matrix(minv, d, A, B, z0, parent, length, 0.3, 1.4)
    p = rng.standard_normal(k)
    got = mod.joint_mass_velocity(minv, d, A, B, p, z0, parent, length, 0.3, 1.4)
    return np.allclose(got, np.linalg.solve(M, p), rtol=1e-10, atol=1e-11)


def joint_momentum_covariance(mod):
    rng, parent, length, A, B, minv, d, z0, k = joint_case()
    M = tree_oracle.joint_mass_matrix(minv, d, A, B, z0, parent, length, 0.0, 0.9)
    Am = np.stack([mod.joint_mass_momentum(minv, d, A, B, e, z0, parent, length, 0.0, 0.9)
                   for e in np.eye(k + parent.size)], axis=1)
    return np.allclose(Am @ Am.T, M, rtol=1e-9, atol=1e-10 * np.abs(M).max())


CHECKS = [two_tip, plain_solve, brownian_covariance, momentum_covariance, joint_solve, joint_momentum_covariance]


def test_unmodified_copy_passes():
    mod = mutated("import numpy as np", "import numpy as np")
    for chk in CHECKS:
        assert chk(mod), chk.__name__


def caught(mod):
    for chk in CHECKS:
        try:
            if not chk(mod):
                return chk.__name__
        except (np.linalg.LinAlgError, FloatingPointError, ValueError):
            return chk.__name__
    return None


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mass_oracle_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    assert caught(mutated(old, new)) is not None, f"no pin catches: {name}"
