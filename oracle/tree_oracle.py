"""Oracle of the phylogenetic Brownian prior (Section 2.2, Eq. 2).

TEST INFRASTRUCTURE: used only by the tests and the bench's CPU legs.

The tips' latent values z are N(0, sigma^2 V).  V_ij is the root variance
scalar plus the length of the root path that tips i and j share (the time
from the root to their most recent common ancestor); V_ii is the root
variance plus the whole root-to-tip path (Section 2.2).  ``tree_cov`` writes V
out from that definition in NumPy; ``tree_prior`` evaluates Eq. 2 and its
derivatives by dense algebra on V (the O(M^3) route that Section 2.3.1's
dynamic programme avoids) in ``tree_oracle.c``, in long double: coalescent
trees have tip branches of ~1e-7 under a height of ~1, so V's condition number
reaches ~1e9 and FP64 dense algebra would lose the last digits that the
comparison needs.

Tree encoding: nodes 0..M-1 are the tips in the order of z, nodes M..2M-2 are
internal, parent[v] = -1 at the root, length[v] = branch length from v to its
parent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tree_oracle.c")
_SO = os.path.join(_HERE, "_build", "libtree_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str = _SRC, so: str = _SO) -> str:
    os.makedirs(os.path.dirname(so), exist_ok=True)
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                        "-std=c99", "-Wall", "-o", tmp, src, "-lm"], check=True)
        os.replace(tmp, so)
    return so


def _typed(lib):
    d, i64 = ctypes.POINTER(ctypes.c_double), ctypes.c_int64
    l64 = ctypes.POINTER(ctypes.c_int64)
    lib.tree_oracle_cov.argtypes = [i64, l64, d, ctypes.c_double, d]
    lib.tree_oracle_cov.restype = ctypes.c_int
    lib.tree_oracle_prior.argtypes = [i64, l64, d, ctypes.c_double, ctypes.c_double, d, d, d, d, d]
    lib.tree_oracle_prior.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _typed(ctypes.CDLL(build()))
    return _lib


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def load_variant(src_text: str, workdir: str):
    """Compile a modified copy of the C source (tests that plant a mistake in
    the oracle) and return its library, to pass as lib=."""
    src = os.path.join(workdir, "tree_variant.c")
    with open(src, "w") as f:
        f.write(src_text)
    return _typed(ctypes.CDLL(build(force=True, src=src, so=os.path.join(workdir, "libtree_variant.so"))))


def root_path(parent, v):
    """The nodes on the path from v up to (excluding) the root, v first."""
    path = []
    while parent[v] >= 0:
        path.append(int(v))
        v = parent[v]
    return path


def tree_cov(parent, length, root_var=0.0):
    """V (M x M, FP64) from the definition: root_var + total length of the
    branches that lie on both tips' root paths."""
    parent = np.asarray(parent, np.int64)
    length = np.asarray(length, float)
    m = (parent.size + 1) // 2
    # on[i, k] = 1 when branch k (above node k) lies on tip i's root path; the
    # shared length of tips i and j is then sum_k on[i, k] length[k] on[j, k]
    on = np.zeros((m, parent.size))
    for i in range(m):
        on[i, root_path(parent, i)] = 1.0
    return root_var + (on * length) @ on.T


def _call(parent, length, root_var, sigma2, z, want_prec=False, lib=None):
    par = np.ascontiguousarray(parent, dtype=np.int64)
    ln = np.ascontiguousarray(length, dtype=np.float64)
    m = (par.size + 1) // 2
    zz = np.ascontiguousarray(z, dtype=np.float64) if z is not None else None
    ld = np.zeros(1)
    pz, pd = np.zeros(m), np.zeros(m)
    prec = np.zeros((m, m)) if want_prec else None
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None  # noqa: E731
    rc = (lib or _load()).tree_oracle_prior(m, par.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), dp(ln), float(root_var),
                                   float(sigma2), dp(zz), dp(ld) if zz is not None else None,
                                   dp(pz) if zz is not None else None, dp(pd), dp(prec))
    if rc != 0:
        raise np.linalg.LinAlgError("V is not positive definite or the tree is malformed")
    return float(ld[0]), pz, pd, prec


def tree_prior(z, parent, length, root_var, sigma2, lib=None):
    """(log N(z; 0, sigma2 V), (sigma2 V)^-1 z, diag((sigma2 V)^-1)), dense, in long double."""
    ld, pz, pd, _ = _call(parent, length, root_var, sigma2, z, lib=lib)
    return ld, pz, pd


def precision_matrix(parent, length, root_var=0.0, sigma2=1.0):
    """(sigma2 V)^-1 (M x M), computed in long double and rounded to FP64."""
    return _call(parent, length, root_var, sigma2, None, want_prec=True)[3]


def simulate(rng, parent, length, root_var, sigma2, n_draws):
    """Draws of z by running the Brownian motion down the tree (Section 2.2): the
    root is N(0, root_var sigma2); each child is its parent plus N(0, sigma2 *
    branch length).  Returns [n_draws, M]."""
    parent = np.asarray(parent, np.int64)
    length = np.asarray(length, float)
    nn = parent.size
    m = (nn + 1) // 2
    root = int(np.flatnonzero(parent < 0)[0])
    # parents before children: order nodes by their depth in edges
    depth = np.array([len(root_path(parent, v)) for v in range(nn)])
    order = np.argsort(depth, kind="stable")
    val = np.zeros((n_draws, nn))
    val[:, root] = np.sqrt(root_var * sigma2) * rng.standard_normal(n_draws)
    for v in order:
        if v == root:
            continue
        val[:, v] = val[:, parent[v]] + np.sqrt(sigma2 * length[v]) * rng.standard_normal(n_draws)
    return val[:, :m]


# ---------------------------------------------------------------------------
# Tree-structured HMC mass matrix on the rate block (Section 2.3.2's
# preconditioner with the phylogenetic prior's full precision, Eq. 2):
#     M = diag(1 / minv) outside [z0, z0 + m),  M_z = diag(d) + (sigma2 V)^-1.
# Dense algebra from these definitions, no tree recursion.
# ---------------------------------------------------------------------------
def brownian_from_normals(parent, length, root_var, sigma2, xi_nodes):
    """The Brownian motion down the tree (Section 2.2) driven by the given node
    normals: root = sqrt(sigma2 root_var) xi[root], child = parent +
    sqrt(sigma2 length) xi[child].  Written as path sums: the value at a node
    is the root's term plus the terms of every branch on its root path.
    Returns the values at all 2M-1 nodes."""
    parent = np.asarray(parent, np.int64)
    length = np.asarray(length, float)
    xi = np.asarray(xi_nodes, float)
    root = int(np.flatnonzero(parent < 0)[0])
    base = np.sqrt(sigma2 * root_var) * xi[root]
    return np.array([base + sum(np.sqrt(sigma2 * length[e]) * xi[e] for e in root_path(parent, v))
                     for v in range(parent.size)])


def mass_velocity(d, p_z, parent, length, root_var, sigma2, refine=True):
    """(diag(d) + C^-1)^-1 p_z with C = sigma2 V, by the Woodbury identity
        (D + C^-1)^-1 = C - C D^1/2 (I + D^1/2 C D^1/2)^-1 D^1/2 C,
    which never inverts V: on coalescent trees V's condition number reaches
    ~1e9, so forming C^-1 in FP64 would lose the digits that the comparison
    needs, while I + D^1/2 C D^1/2 stays well conditioned for moderate d.
    Negative d entries count as 0.  refine: one step of iterative refinement
    with a long-double residual (below)."""
    C = sigma2 * tree_cov(parent, length, root_var)
    dd = np.maximum(np.asarray(d, float), 0.0)
    s = np.sqrt(dd)
    K = np.eye(s.size) + s[:, None] * C * s[None, :]

    def woodbury(b):
        Cb = C @ b
        return Cb - C @ (s * np.linalg.solve(K, s * Cb))

    p_z = np.asarray(p_z, float)
    v = woodbury(p_z)
    if refine:
        # one step of iterative refinement: the residual p - (D + P) v takes
        # P v from the long-double dense prior, so the Woodbury route's FP64
        # error (up to ~1e-9 of the largest entry at d ~ 100 on a 1,610-tip
        # coalescent tree) is divided by itself
        _, pv, _ = tree_prior(v, parent, length, root_var, sigma2)
        v = v + woodbury(p_z - dd * v - pv)
    return v


def mass_full_velocity(minv, d, p, z0, parent, length, root_var, sigma2):
    """M^-1 p for the whole state: minv * p outside the rate block."""
    p = np.asarray(p, float)
    v = np.asarray(minv, float) * p
    m = (np.asarray(parent).size + 1) // 2
    v[z0:z0 + m] = mass_velocity(d, p[z0:z0 + m], parent, length, root_var, sigma2)
    return v


def mass_momentum(minv, d, xi, z0, parent, length, root_var, sigma2):
    """The momentum p = A xi with A A^T = M: p_i = xi_i / sqrt(minv_i) outside
    the block; p_z = sqrt(d) xi_z + (sigma2 V)^-1 w inside, w the Brownian
    motion driven by xi[k:] (Cov w = sigma2 V, so Cov((sigma2 V)^-1 w) =
    (sigma2 V)^-1).  (sigma2 V)^-1 w comes from the long-double dense prior."""
    minv = np.asarray(minv, float)
    xi = np.asarray(xi, float)
    k = minv.size
    m = (np.asarray(parent).size + 1) // 2
    p = xi[:k] / np.sqrt(minv)
    w = brownian_from_normals(parent, length, root_var, sigma2, xi[k:])[:m]
    _, pw, _ = tree_prior(w, parent, length, root_var, sigma2)
    p[z0:z0 + m] = np.sqrt(np.maximum(np.asarray(d, float), 0.0)) * xi[z0:z0 + m] + pw
    return p


def joint_mass_matrix(minv, d, A, B, z0, parent, length, root_var, sigma2):
    """The dense joint mass: diag(1 / minv), with [[A, B^T], [B, diag(d) + P]] on
    the coordinates [0, nc) and the rate block [z0, z0 + m); P from the
    long-double prior.  For well-conditioned trees only (P is rounded to FP64)."""
    minv = np.asarray(minv, float)
    A, B = np.atleast_2d(np.asarray(A, float)), np.asarray(B, float)
    nc = A.shape[0]
    m = (np.asarray(parent).size + 1) // 2
    M = np.diag(1.0 / minv)
    M[:nc, :nc] = A
    M[z0:z0 + m, z0:z0 + m] = np.diag(np.maximum(np.asarray(d, float), 0.0)) + precision_matrix(
        parent, length, root_var, sigma2)
    M[z0:z0 + m, :nc] = B
    M[:nc, z0:z0 + m] = B.T
    return M


def joint_mass_velocity(minv, d, A, B, p, z0, parent, length, root_var, sigma2):
    """M^-1 p for the joint mass by block elimination on the rate block:
    y = M_z^-1 p_z and U = M_z^-1 B by mass_velocity (refined Woodbury, no
    inverse of V), S = A - B^T U, x_g = S^-1 (p_g - B^T y), x_z = y - U x_g;
    minv * p elsewhere."""
    A, B = np.atleast_2d(np.asarray(A, float)), np.asarray(B, float)
    nc = A.shape[0]
    m = (np.asarray(parent).size + 1) // 2
    p = np.asarray(p, float)
    x = np.asarray(minv, float) * p
    y = mass_velocity(d, p[z0:z0 + m], parent, length, root_var, sigma2)
    U = np.column_stack([mass_velocity(d, B[:, j], parent, length, root_var, sigma2) for j in range(nc)])
    S = A - B.T @ U
    xg = np.linalg.solve(S, p[:nc] - B.T @ y)
    x[:nc] = xg
    x[z0:z0 + m] = y - U @ xg
    return x


def joint_mass_momentum(minv, d, A, B, xi, z0, parent, length, root_var, sigma2):
    """p ~ N(0, M) for the joint mass from normals xi: p_z as in mass_momentum,
    then the coupled coordinates from their conditional law given p_z,
    N(B^T M_z^-1 p_z, S): p_g = U^T p_z + chol(S) xi[:nc]."""
    A, B = np.atleast_2d(np.asarray(A, float)), np.asarray(B, float)
    nc = A.shape[0]
    m = (np.asarray(parent).size + 1) // 2
    p = mass_momentum(minv, d, xi, z0, parent, length, root_var, sigma2)
    U = np.column_stack([mass_velocity(d, B[:, j], parent, length, root_var, sigma2) for j in range(nc)])
    S = A - B.T @ U
    p[:nc] = U.T @ p[z0:z0 + m] + np.linalg.cholesky(0.5 * (S + S.T)) @ np.asarray(xi, float)[:nc]
    return p
