"""The O(M) tree prior kernel (Section 2.3.1's dynamic programme for Eq. 2)
against the dense oracle, and the tree-based posterior against the dense one."""
import numpy as np
import pytest

from oracle import hmc_oracle, tree_oracle
from paper_2103_03348_b300 import synth
from parity_util import FP64_TOL, scaled_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# The kernel is FP64; the dense oracle works in long double, since V's
# condition number reaches ~4e9 on the 1,610-tip coalescent tree (tip branches
# of ~5e-7 under a height of 2), where FP64 dense algebra loses ~4e-10.  The
# recursions lose a few ulps per level (a 1e-14 relative difference was
# measured on that tree); 1e-10 relative leaves room.
TREE_TOL = 1e-10


def caterpillar(m, rng):
    parent = np.full(2 * m - 1, -1)
    parent[0] = parent[1] = m
    for k in range(2, m):
        parent[k] = m + k - 1
        parent[m + k - 2] = m + k - 1
    length = rng.uniform(0.05, 1.0, 2 * m - 1)
    length[2 * m - 2] = 0.0
    return parent, length


def balanced(m, rng):
    # m a power of two: pair nodes level by level
    parent = np.full(2 * m - 1, -1)
    cur, nxt = list(range(m)), m
    while len(cur) > 1:
        new = []
        for a, b in zip(cur[0::2], cur[1::2]):
            parent[a] = parent[b] = nxt
            new.append(nxt)
            nxt += 1
        cur = new
    length = rng.uniform(0.05, 1.0, 2 * m - 1)
    length[-1] = 0.0
    return parent, length


def shuffled(parent, length, rng):
    """The same tree with its internal nodes renumbered at random."""
    m = (parent.size + 1) // 2
    perm = np.arange(parent.size)
    perm[m:] = m + rng.permutation(m - 1)
    new_parent = np.full_like(parent, -1)
    new_length = np.zeros_like(length)
    for v in range(parent.size):
        new_parent[perm[v]] = perm[parent[v]] if parent[v] >= 0 else -1
        new_length[perm[v]] = length[v]
    return new_parent, new_length


def trees():
    rng = np.random.default_rng(17)
    w = synth.make_ebola_like(n=23422, m_seq=1610)
    yield "ebola_like_1610", w.tree_parent, w.tree_length, 0.0, 1.0
    yield "caterpillar_300", *caterpillar(300, rng), 0.4, 2.0
    yield "balanced_1024", *balanced(1024, rng), 1.5, 0.3
    yield "shuffled_balanced_256", *shuffled(*balanced(256, rng), rng), 0.2, 1.0
    yield "cherry", np.array([2, 2, -1]), np.array([0.3, 0.9, 0.0]), 0.7, 1.3
    w2 = synth.make_ebola_like(seed=3, n=8000, m_seq=2500, box=300.0, t_max=300.0, n_hot=6)
    yield "coalescent_2500", w2.tree_parent, w2.tree_length, 0.05, 0.5


@pytest.mark.parametrize("case", list(trees()), ids=lambda c: c[0])
def test_tree_prior_matches_dense_oracle(case):
    from paper_2103_03348_b300 import build, tree
    build.build()
    name, parent, length, tau0, s2 = case
    m = (parent.size + 1) // 2
    z = np.random.default_rng(m).normal(0.0, 1.0, m)
    tp = tree.TreePrior(parent, length, tau0, s2)
    out = tp.evaluate(torch.tensor(z, dtype=torch.float64, device="cuda"))
    ld, pz, pd = tree_oracle.tree_prior(z, parent, length, tau0, s2)
    assert abs(out["logdens"].item() - ld) <= TREE_TOL * max(1.0, abs(ld)), name
    assert scaled_err(out["pz"].cpu().numpy(), pz) <= TREE_TOL, name
    np.testing.assert_allclose(out["pdiag"].cpu().numpy(), pd, rtol=TREE_TOL, atol=0)


def test_tree_prior_optional_outputs_and_repeatability():
    from paper_2103_03348_b300 import build, tree
    build.build()
    w = synth.make_ebola_like(seed=2, n=3000, m_seq=400, box=150.0, t_max=150.0, n_hot=4)
    tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.1, 1.0)
    z = torch.randn(400, dtype=torch.float64, device="cuda")
    a = tp.evaluate(z)
    b = tp.evaluate(z, want=("pz",))
    assert set(b) == {"pz"}
    assert torch.equal(a["pz"], b["pz"])  # one block, fixed order: bit-identical


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_tree_posterior_matches_dense_posterior(precision):
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    w = synth.make_ebola_like(seed=11, n=600, m_seq=40, box=120.0, t_max=120.0, n_hot=4)
    prec = tree_oracle.precision_matrix(w.tree_parent, w.tree_length)
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")  # noqa: E731
    seq = torch.tensor(w.sequenced, device="cuda")
    dense = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), seq, d(prec), hmc.prior_km_days(), precision)
    tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0)
    on_tree = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), seq, None, hmc.prior_km_days(), precision, tree=tp)
    q = np.concatenate([np.log(w.params), w.r[w.sequenced]])
    q[6:] += np.random.default_rng(0).normal(0, 0.3, len(q) - 6)
    qd = d(q)
    a = dense.evaluate(qd, want_hess=True)
    a = {k: v.clone() for k, v in a.items()}
    b = on_tree.evaluate(qd, want_hess=True)
    assert abs(a["logpost"].item() - b["logpost"].item()) <= 1e-12 * abs(a["logpost"].item())
    assert scaled_err(b["grad"].cpu().numpy(), a["grad"].cpu().numpy()) <= 1e-12
    assert scaled_err(b["hdiag"].cpu().numpy(), a["hdiag"].cpu().numpy()) <= 1e-12
    if precision == "fp64":
        ref = hmc_oracle.log_posterior(w.x, w.y, w.t, w.r, w.sequenced, prec, hmc.prior_km_days().as_tuple(), q)
        assert abs(b["logpost"].item() - ref[0]) <= FP64_TOL * abs(ref[0])
        assert scaled_err(b["grad"].cpu().numpy(), ref[1]) <= FP64_TOL
        assert scaled_err(b["hdiag"].cpu().numpy(), ref[2]) <= FP64_TOL
    lp = {"logpost": torch.empty((), dtype=torch.float64, device="cuda")}
    on_tree.logpost_only(qd, lp)
    assert abs(lp["logpost"].item() - b["logpost"].item()) <= 1e-12 * abs(b["logpost"].item())


def test_tree_posterior_short_chain():
    """A few HMC iterations through the tree posterior run, accept, and stay finite."""
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    w = synth.make_ebola_like(seed=11, n=600, m_seq=40, box=120.0, t_max=120.0, n_hot=4)
    d = lambda a: torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")  # noqa: E731
    tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0)
    post = hmc.Posterior(d(w.x), d(w.y), d(w.t), d(w.r), torch.tensor(w.sequenced, device="cuda"), None,
                         hmc.prior_km_days(), "fp32c", tree=tp)
    q0 = d(np.concatenate([np.log(w.params), w.r[w.sequenced]]))
    ch = hmc.sample(post, q0, n_iter=60, n_warmup=30, n_steps=10, eps0=0.05, mass_every=20, seed=1)
    assert np.all(np.isfinite(ch.draws))
    assert ch.accept.mean() > 0.3
