"""FP64 NumPy oracle of the phylogenetic Brownian prior (Section 2.2, Eq. 2).

TEST INFRASTRUCTURE: used only by the tests and the bench's CPU legs.

The tips' latent values z are N(0, sigma^2 V).  V_ij is the root variance
scalar plus the length of the root path that tips i and j share (the time
from the root to their most recent common ancestor); V_ii is the root
variance plus the whole root-to-tip path (Section 2.2).  This module writes V
out entry by entry from that definition, then evaluates Eq. 2 and its
derivatives with dense linear algebra, the O(M^3) route that Section 2.3.1's
dynamic programme avoids.

Tree encoding: nodes 0..M-1 are the tips in the order of z, nodes M..2M-2 are
internal, parent[v] = -1 at the root, length[v] = branch length from v to its
parent.
"""
from __future__ import annotations

import numpy as np


def root_path(parent, v):
    """The nodes on the path from v up to (excluding) the root, v first."""
    path = []
    while parent[v] >= 0:
        path.append(int(v))
        v = parent[v]
    return path


def tree_cov(parent, length, root_var=0.0):
    """V (M x M) from the definition: root_var + total length of the branches
    that lie on both tips' root paths."""
    parent = np.asarray(parent, np.int64)
    length = np.asarray(length, float)
    m = (parent.size + 1) // 2
    # on[i, k] = 1 when branch k (above node k) lies on tip i's root path; the
    # shared length of tips i and j is then sum_k on[i, k] length[k] on[j, k]
    on = np.zeros((m, parent.size))
    for i in range(m):
        on[i, root_path(parent, i)] = 1.0
    return root_var + (on * length) @ on.T


def tree_prior(z, parent, length, root_var, sigma2):
    """(log N(z; 0, sigma2 V), (sigma2 V)^-1 z, diag((sigma2 V)^-1)) by dense algebra."""
    z = np.asarray(z, float)
    cov = sigma2 * tree_cov(parent, length, root_var)
    m = z.size
    sign, logdet = np.linalg.slogdet(cov)
    if sign <= 0:
        raise np.linalg.LinAlgError("V is not positive definite")
    prec = np.linalg.inv(cov)
    pz = prec @ z
    logdens = -0.5 * m * np.log(2 * np.pi) - 0.5 * logdet - 0.5 * float(z @ pz)
    return logdens, pz, np.diag(prec).copy()


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
