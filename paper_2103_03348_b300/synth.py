"""Seeded synthetic point patterns shaped like the paper's workloads.

This module only *draws* data: event locations, times and per-event log-rates,
plus the parameter vector at which a workload is evaluated.  It contains none
of the likelihood's arithmetic (no intensity, no integral, no derivative), so
both the CPU oracle and the CUDA path can take their inputs from it without
sharing any of the method's code.

Stand-ins for the paper's data (Section 3.2: 23,422 Ebola cases, 1,610 of them
sequenced, roughly 600 km x 600 km of West Africa over about two years; Section
3.1: "25,000 randomly generated data points").  The case table, the posterior
trees and the BEAST analysis file are not available, so every workload below is
drawn from a seeded NumPy PCG64 generator (seed = 1000 + workload index):

* ``unit_square``  N=2,000  unit square x [0,1]; Ogata thinning of the temporal
  marginal of a Hawkes process (immigrant rate 1,400, branching 0.3, decay 10);
  immigrants uniform in space, offspring displaced N(0, 0.02^2 I) from a parent
  drawn by its share of the excitation at the accepted time.  All log-rates 0.
* ``ebola_like``   N=23,422 on [0,600]^2 km x [0,730] d, 50 Gaussian hotspots
  (sigma 20 km), cluster-process offspring (Poisson(0.5) children, Exp(0.1/d)
  delays, N(0, 5^2 I) km displacements).  1,610 random events carry log-rates
  drawn N(0, V) with V the covariance of Brownian motion (sigma^2 = 1, root
  variance 0) down a random Kingman coalescent tree of 1,610 tips (Section 2.2,
  Eq. 2); the other log-rates are 0.
* ``large``        N=100,000, same generator on [0,2000]^2 km x [0,1500] d with
  556 hotspots; all log-rates i.i.d. N(0, 0.25).
* ``surrogate``    N=500,000 on [0,2000]^2 km x [0,1500] d; immigrants half
  uniform, half from 500 hotspots (sigma 20 km); offspring weight 0.6.

Every pattern is returned sorted by time (ascending), as the library requires.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Parameter order used throughout the library: (mu0, tau_x, tau_t, theta0, omega, h).
PARAM_NAMES = ("mu0", "tau_x", "tau_t", "theta0", "omega", "h")


@dataclasses.dataclass
class Workload:
    name: str
    x: np.ndarray  # float64 [N]
    y: np.ndarray  # float64 [N]
    t: np.ndarray  # float64 [N], ascending
    r: np.ndarray  # float64 [N], log-rates r_n = log theta_n
    params: np.ndarray  # float64 [6]
    sequenced: np.ndarray  # int64 indices of events whose log-rate is free
    tree_cov: np.ndarray = None  # [M, M] V of the sequenced events' tree (in `sequenced` order), or None
    tree_parent: np.ndarray = None  # [2M-1] parent of each tree node (-1 at the root); nodes 0..M-1 are the
    #                                 tips in `sequenced` order, internal nodes follow in merge order
    tree_length: np.ndarray = None  # [2M-1] length of the branch above each node (0 at the root)

    @property
    def n(self) -> int:
        return int(self.t.shape[0])


def _sorted(name, x, y, t, r, params, sequenced_mask):
    order = np.argsort(t, kind="stable")
    x, y, t, r = x[order], y[order], t[order], r[order]
    seq = np.nonzero(sequenced_mask[order])[0].astype(np.int64)
    return Workload(name, np.ascontiguousarray(x, np.float64), np.ascontiguousarray(y, np.float64),
                    np.ascontiguousarray(t, np.float64), np.ascontiguousarray(r, np.float64),
                    np.asarray(params, np.float64), seq)


def ogata_temporal(rng, n_events, nu, branching, omega, sigma_offspring):
    """Ogata thinning of a temporal Hawkes process with exponential decay.

    Intensity nu + sum_i branching*omega*exp(-omega (t - t_i)); stops after
    ``n_events`` accepted points.  The excitation state is carried as a scalar
    that decays between proposals.  Each accepted point is an immigrant with
    probability nu / (total intensity), otherwise the child of an earlier point
    drawn in proportion to that point's current excitation.  Immigrants are
    uniform on the unit square; children are displaced N(0, sigma^2 I).
    """
    t = 0.0
    excite = 0.0  # current sum_i branching*omega*exp(-omega (t - t_i))
    ts = np.empty(n_events)
    xs = np.empty(n_events)
    ys = np.empty(n_events)
    k = 0
    while k < n_events:
        bound = nu + excite  # intensity only decreases until the next event
        w = rng.exponential(1.0 / bound)
        t += w
        excite *= math.exp(-omega * w)
        u = rng.uniform()
        if u * bound > nu + excite:
            continue
        # accepted: immigrant or child?
        if rng.uniform() * (nu + excite) < nu or k == 0:
            xs[k], ys[k] = rng.uniform(), rng.uniform()
        else:
            wts = np.exp(-omega * (t - ts[:k]))
            parent = rng.choice(k, p=wts / wts.sum())
            xs[k] = xs[parent] + sigma_offspring * rng.standard_normal()
            ys[k] = ys[parent] + sigma_offspring * rng.standard_normal()
        ts[k] = t
        excite += branching * omega
        k += 1
    return xs, ys, ts


def cluster_process(rng, n_immigrants, box, t_max, centres, sigma_hot, frac_uniform,
                    branching, omega, sigma_offspring):
    """Branching (cluster) construction of a spatiotemporal Hawkes pattern.

    Immigrants: time uniform on [0, t_max]; location uniform in the box with
    probability ``frac_uniform``, else a random hotspot centre plus N(0,
    sigma_hot^2 I).  Every event has Poisson(branching) children, each delayed
    by Exp(rate omega) and displaced by N(0, sigma_offspring^2 I).
    """
    t = rng.uniform(0.0, t_max, n_immigrants)
    uni = rng.uniform(size=n_immigrants) < frac_uniform
    hot = rng.integers(0, len(centres), n_immigrants)
    x = np.where(uni, rng.uniform(0, box, n_immigrants), centres[hot, 0] + sigma_hot * rng.standard_normal(n_immigrants))
    y = np.where(uni, rng.uniform(0, box, n_immigrants), centres[hot, 1] + sigma_hot * rng.standard_normal(n_immigrants))
    xs, ys, ts = [x], [y], [t]
    px, py, pt = x, y, t
    while len(pt):
        kids = rng.poisson(branching, len(pt))
        idx = np.repeat(np.arange(len(pt)), kids)
        if len(idx) == 0:
            break
        ct = pt[idx] + rng.exponential(1.0 / omega, len(idx))
        cx = px[idx] + sigma_offspring * rng.standard_normal(len(idx))
        cy = py[idx] + sigma_offspring * rng.standard_normal(len(idx))
        xs.append(cx); ys.append(cy); ts.append(ct)
        px, py, pt = cx, cy, ct
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(ts)


def coalescent_brownian(rng, m, sigma2=1.0, root_var=0.0, return_cov=False, return_tree=False):
    """Tip values of Brownian motion down a random Kingman coalescent tree.

    Tips are contemporaneous.  While k lineages remain, the waiting time to the
    next merger is Exp(k(k-1)/2) and a uniformly random pair merges.  The root
    value is N(0, root_var*sigma2); each child is its parent plus N(0, sigma2 *
    branch length).  The tip vector is then N(0, sigma2 V) with V the tree's
    shared-path-length matrix (Section 2.2, Eq. 2).  With return_cov the tree's
    V is returned too: V_ij = root_var + (root height - height of the most
    recent common ancestor of tips i and j); the random draws are unchanged.
    """
    # Build the tree bottom-up: node heights and parent pointers.
    height = np.zeros(2 * m - 1)
    parent = np.full(2 * m - 1, -1, dtype=np.int64)
    lineages = list(range(m))
    now = 0.0
    nxt = m
    while len(lineages) > 1:
        k = len(lineages)
        now += rng.exponential(2.0 / (k * (k - 1)))
        i, j = rng.choice(k, 2, replace=False)
        a, b = lineages[i], lineages[j]
        height[nxt] = now
        parent[a] = nxt
        parent[b] = nxt
        for idx in sorted((i, j), reverse=True):
            lineages.pop(idx)
        lineages.append(nxt)
        nxt += 1
    root = lineages[0]
    value = np.zeros(2 * m - 1)
    value[root] = math.sqrt(root_var * sigma2) * rng.standard_normal()
    # internal nodes were created in increasing height: walk from the root down
    for node in range(2 * m - 2, -1, -1):
        if node == root:
            continue
        bl = height[parent[node]] - height[node]
        value[node] = value[parent[node]] + math.sqrt(sigma2 * bl) * rng.standard_normal()
    if not return_cov:
        return value[:m]
    lengths = np.zeros(2 * m - 1)
    for node in range(2 * m - 1):
        if parent[node] >= 0:
            lengths[node] = height[parent[node]] - height[node]
    # V from the tree: for every internal node, the pairs split by it share the
    # path from the root down to that node
    children = [[] for _ in range(2 * m - 1)]
    for node in range(2 * m - 1):
        if parent[node] >= 0:
            children[parent[node]].append(node)
    tips = [[k] if k < m else None for k in range(2 * m - 1)]
    cov = np.zeros((m, m))
    for node in range(m, 2 * m - 1):  # children are created before their parent
        a, b = children[node]
        shared = root_var + height[root] - height[node]
        ta, tb = np.array(tips[a]), np.array(tips[b])
        cov[np.ix_(ta, tb)] = shared
        cov[np.ix_(tb, ta)] = shared
        tips[node] = tips[a] + tips[b]
        tips[a] = tips[b] = None
    cov[np.arange(m), np.arange(m)] = root_var + height[root]
    if return_tree:
        return value[:m], cov, parent.copy(), lengths
    return value[:m], cov


def _hotspot_pattern(rng, n_target, box, t_max, n_hot, frac_uniform, branching, omega, sigma_off,
                     sigma_hot=20.0):
    centres = rng.uniform(0, box, (n_hot, 2))
    n_imm = int(math.ceil(n_target * (1.0 - branching) * 1.02))
    while True:
        x, y, t = cluster_process(rng, n_imm, box, t_max, centres, sigma_hot, frac_uniform,
                                  branching, omega, sigma_off)
        if len(t) >= n_target:
            break
        n_imm = int(n_imm * 1.05) + 1
    keep = np.argsort(t, kind="stable")[:n_target]
    return x[keep], y[keep], t[keep]


def make_unit_square(seed: int = 1000, n: int = 2000) -> Workload:
    rng = np.random.default_rng(seed)
    x, y, t = ogata_temporal(rng, n, nu=1400.0, branching=0.3, omega=10.0, sigma_offspring=0.02)
    params = (0.5, 0.1, 0.05, 0.3, 10.0, 0.02)
    return _sorted("unit_square_N2000", x, y, t, np.zeros(n), params, np.zeros(n, bool))


def make_ebola_like(seed: int = 1001, n: int = 23422, m_seq: int = 1610, box: float = 600.0,
                    t_max: float = 730.0, n_hot: int = 50) -> Workload:
    rng = np.random.default_rng(seed)
    x, y, t = _hotspot_pattern(rng, n, box, t_max, n_hot, 0.0, 0.5, 0.1, 5.0)
    r = np.zeros(n)
    seq = rng.choice(n, min(m_seq, n), replace=False)
    cov = np.zeros((0, 0))
    parent, lengths = np.zeros(0, np.int64), np.zeros(0)
    if len(seq):
        r[seq], cov, parent, lengths = coalescent_brownian(rng, len(seq), return_cov=True, return_tree=True)
    mask = np.zeros(n, bool)
    mask[seq] = True
    params = (0.5, 20.0, 30.0, 0.5, 0.1, 5.0)
    w = _sorted(f"ebola_like_N{n}", x, y, t, r, params, mask)
    # V in the order of w.sequenced (time-sorted event indices)
    tip_of = np.full(n, -1, dtype=np.int64)
    tip_of[seq] = np.arange(len(seq))
    order = np.argsort(t, kind="stable")
    tips = tip_of[order[w.sequenced]]
    w.tree_cov = np.ascontiguousarray(cov[np.ix_(tips, tips)])
    # the same tree with its tips renumbered in `sequenced` order
    m = len(seq)
    if m:
        relabel = np.arange(2 * m - 1)
        relabel[tips] = np.arange(m)  # old tip id -> new tip id
        new_parent = np.full(2 * m - 1, -1, np.int64)
        new_length = np.zeros(2 * m - 1)
        for old_id in range(2 * m - 1):
            nid = relabel[old_id]
            pa = parent[old_id]
            new_parent[nid] = relabel[pa] if pa >= 0 else -1
            new_length[nid] = lengths[old_id]
        w.tree_parent, w.tree_length = new_parent, new_length
    return w


def make_large(seed: int = 1002, n: int = 100_000) -> Workload:
    rng = np.random.default_rng(seed)
    x, y, t = _hotspot_pattern(rng, n, 2000.0, 1500.0, 556, 0.0, 0.5, 0.1, 5.0)
    r = rng.normal(0.0, 0.5, n)  # variance 0.25
    params = (0.5, 20.0, 30.0, 0.5, 0.1, 5.0)
    return _sorted(f"large_N{n}", x, y, t, r, params, np.ones(n, bool))


def make_surrogate(seed: int = 1004, n: int = 500_000) -> Workload:
    rng = np.random.default_rng(seed)
    x, y, t = _hotspot_pattern(rng, n, 2000.0, 1500.0, 500, 0.5, 0.6, 0.1, 5.0)
    params = (0.4, 20.0, 30.0, 0.6, 0.1, 5.0)
    return _sorted(f"surrogate_N{n}", x, y, t, np.zeros(n), params, np.zeros(n, bool))


def make_uniform(seed: int, n: int, box: float = 1.0, t_max: float = 1.0, r_sd: float = 0.0,
                 params=(0.5, 0.1, 0.05, 0.3, 10.0, 0.02)) -> Workload:
    """Small i.i.d. uniform pattern for unit tests (ragged sizes, edge cases)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, box, n)
    y = rng.uniform(0, box, n)
    t = rng.uniform(0, t_max, n)
    r = rng.normal(0.0, r_sd, n) if r_sd > 0 else np.zeros(n)
    return _sorted(f"uniform_N{n}", x, y, t, r, params, np.ones(n, bool))


WORKLOADS = {
    "unit_square": make_unit_square,
    "ebola_like": make_ebola_like,
    "large": make_large,
    "surrogate": make_surrogate,
}


def make(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)
