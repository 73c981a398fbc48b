"""The tree-structured HMC mass matrix (diag(d) + (sigma2 V)^-1 on the rate
block, applied by one tree sweep) against the dense oracle, and the sampler
with it: exact moments on a tree-correlated Gaussian, where it must mix far
better than the diagonal mass, a chain on a Hawkes posterior, graph replay and
checkpoint resume."""
import numpy as np
import pytest

from oracle import tree_oracle
from paper_2103_03348_b300 import synth
from parity_util import scaled_err
from test_gpu_tree import TREE_TOL, trees

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Z0 = 6


def dev(a):
    return torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")


def inputs(m, seed):
    rng = np.random.default_rng(seed)
    k = Z0 + m + 3
    minv = rng.uniform(0.2, 3.0, k)
    d = rng.uniform(0.0, 4.0, m)
    d[::7] = 0.0
    d[1] = -0.5  # negative curvature counts as none
    return rng, k, minv, d


@pytest.mark.parametrize("case", list(trees()), ids=lambda c: c[0])
def test_velocity_position_and_kinetic_match_oracle(case):
    from paper_2103_03348_b300 import build, tree
    build.build()
    name, parent, length, tau0, s2 = case
    m = (parent.size + 1) // 2
    rng, k, minv, d = inputs(m, m)
    p = rng.standard_normal(k)
    q0 = rng.standard_normal(k)
    tm = tree.TreeMass(tree.TreePrior(parent, length, tau0, s2), k, Z0)
    tm.d.copy_(dev(d))
    tm.factor()
    vel, q, kin, kin2 = dev(np.zeros(k)), dev(q0), dev(0.0), dev(0.0)
    tm.velocity(dev(p), dev(minv), vel=vel, q=q, eps=0.37, kinetic=kin)
    tm.velocity(dev(p), dev(minv), kinetic=kin2)
    ref = tree_oracle.mass_full_velocity(minv, d, p, Z0, parent, length, tau0, s2)
    assert scaled_err(vel.cpu().numpy(), ref) <= TREE_TOL, name
    assert abs(kin.item() - 0.5 * p @ ref) <= TREE_TOL * abs(0.5 * p @ ref), name
    assert kin.item() == kin2.item()  # same sweep, same order
    np.testing.assert_allclose(q.cpu().numpy(), q0 + 0.37 * vel.cpu().numpy(), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("case", list(trees()), ids=lambda c: c[0])
def test_momentum_matches_oracle(case):
    from paper_2103_03348_b300 import build, tree
    build.build()
    name, parent, length, tau0, s2 = case
    m = (parent.size + 1) // 2
    rng, k, minv, d = inputs(m, m + 1)
    tm = tree.TreeMass(tree.TreePrior(parent, length, tau0, s2), k, Z0)
    tm.d.copy_(dev(d))
    xi = rng.standard_normal(tm.n_normals)
    p = tm.momentum(dev(minv), dev(xi), dev(np.zeros(k)))
    ref = tree_oracle.mass_momentum(minv, d, xi, Z0, parent, length, tau0, s2)
    assert scaled_err(p.cpu().numpy(), ref) <= TREE_TOL, name


class TreeGaussPost:
    """A Gaussian target whose precision has exactly the tree mass's form:
    diag(a) outside the rate block, diag(d0) + (sigma2 V)^-1 on it; in the
    Posterior interface (tree, pd, m), with the prior part applied by the
    tree prior kernel."""

    def __init__(self, tp, a, d0):
        self.tree, self.m = tp, tp.m
        self.a, self.d0 = a, d0
        self.dim = a.numel()
        self.pd = torch.empty(self.m, dtype=torch.float64, device="cuda")
        self.calls = {"grad": 0, "hess": 0}

    def evaluate(self, q, want_hess=False, out=None):
        if out is None:
            out = {"logpost": torch.empty((), dtype=torch.float64, device=q.device),
                   "grad": torch.empty_like(q), "hdiag": torch.empty_like(q)}
        z = q[Z0:Z0 + self.m]
        pr = self.tree.evaluate(z, want=("pz", "pdiag"))
        aq = self.a * q
        aq[Z0:Z0 + self.m] = self.d0 * z + pr["pz"]
        out["logpost"].copy_(-0.5 * torch.dot(q, aq))
        out["grad"].copy_(-aq)
        if want_hess:
            self.pd.copy_(pr["pdiag"])
            h = -self.a.clone()
            h[Z0:Z0 + self.m] = -(self.d0 + pr["pdiag"])
            out["hdiag"].copy_(h)
        self.calls["hess" if want_hess else "grad"] += 1
        return out

    def status(self):
        return 0


def gauss_problem():
    from paper_2103_03348_b300 import tree
    w = synth.make_ebola_like(seed=4, n=2000, m_seq=120, box=150.0, t_max=150.0, n_hot=4)
    tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0)
    rng = np.random.default_rng(8)
    m = tp.m
    a = rng.uniform(0.5, 20.0, Z0 + m + 2)
    d0 = rng.uniform(0.0, 3.0, m)
    post = TreeGaussPost(tp, dev(a), dev(d0))
    # the exact covariance: diag(1 / a) outside, (diag(d0) + P)^-1 on the block (oracle, column by column)
    var = 1.0 / a
    var[Z0:Z0 + m] = [tree_oracle.mass_velocity(d0, e, w.tree_parent, w.tree_length, 0.0, 1.0)[j]
                      for j, e in enumerate(np.eye(m))]
    return post, var


def test_tree_mass_recovers_tree_gaussian_moments_and_beats_the_diagonal():
    from paper_2103_03348_b300 import build, hmc
    build.build()
    post, var = gauss_problem()
    q0 = dev(np.zeros(post.dim))
    kw = dict(n_iter=800, n_warmup=200, n_steps=10, eps0=0.1, mass_every=50, seed=3)
    ch = hmc.sample(post, q0, mass="tree", **kw)
    ess = hmc.ess_all(ch.draws)
    mean, v = ch.draws.mean(0), ch.draws.var(0)
    s = np.sqrt(var)
    assert 0.5 < ch.accept.mean() <= 1.0
    assert np.all(np.abs(mean) <= 5 * s / np.sqrt(ess))
    assert np.all(np.abs(v / var - 1) <= 5 * np.sqrt(2 / ess) + 0.05)
    diag = hmc.sample(post, q0, mass="diag", **kw)
    ess_diag = hmc.ess_all(diag.draws)
    rates = slice(Z0, Z0 + post.m)
    # the prior's tree correlations are preconditioned exactly: the slowest rate mixes far faster
    assert ess[rates].min() > 5 * ess_diag[rates].min()


def test_tree_mass_graph_replay_and_checkpoint_resume(tmp_path):
    from paper_2103_03348_b300 import build, hmc
    build.build()
    post, _ = gauss_problem()
    q0 = dev(np.zeros(post.dim))
    kw = dict(n_iter=30, n_warmup=30, n_steps=6, eps0=0.1, mass_every=12, seed=5, mass="tree")
    eager = hmc.sample(post, q0, use_graph=False, **kw)
    full = hmc.sample(post, q0, **kw)
    assert np.array_equal(eager.draws, full.draws) and np.array_equal(eager.accept, full.accept)
    for every in (25, 45):  # the last checkpoint falls in warm-up (25), then in sampling (45)
        ck = str(tmp_path / f"ck{every}.pt")
        hmc.sample(post, q0, checkpoint=ck, checkpoint_every=every, **kw)
        resumed = hmc.sample(post, q0, resume=ck, **kw)
        assert np.array_equal(resumed.draws, full.draws) and np.array_equal(resumed.accept, full.accept)


def test_tree_mass_chain_on_hawkes_posterior():
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    w = synth.make_ebola_like(seed=11, n=600, m_seq=40, box=120.0, t_max=120.0, n_hot=4)
    tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0)
    post = hmc.Posterior(dev(w.x), dev(w.y), dev(w.t), dev(w.r), torch.tensor(w.sequenced, device="cuda"), None,
                         hmc.prior_km_days(), "fp32c", tree=tp)
    q0 = dev(np.concatenate([np.log(w.params), w.r[w.sequenced]]))
    ch = hmc.sample(post, q0, n_iter=100, n_warmup=100, n_steps=10, eps0=0.05, mass_every=25, seed=2, mass="tree")
    assert np.all(np.isfinite(ch.logpost)) and np.all(np.isfinite(ch.draws))
    assert 0.4 < ch.accept.mean() <= 1.0
    with pytest.raises(ValueError):
        hmc.sample(post, q0, n_iter=1, n_warmup=0, mass="full")


# ---------------------------------------------------------------------------
# the joint mass: the six globals coupled to the rate block
# ---------------------------------------------------------------------------
def coupled_blocks(rng, parent, length, tau0, s2, d, strength):
    """A (6 x 6) and B (m x 6) with S = A - B^T M_z^-1 B = strength-weighted and positive definite."""
    m = (parent.size + 1) // 2
    B = rng.standard_normal((m, 6)) / np.sqrt(m)
    U = np.column_stack([tree_oracle.mass_velocity(d, B[:, j], parent, length, tau0, s2) for j in range(6)])
    G = B.T @ U
    G = 0.5 * (G + G.T)
    C = rng.standard_normal((6, 6))
    return G + strength * G + (C @ C.T) / 6 + 0.05 * np.eye(6), B


@pytest.mark.parametrize("case", [c for c in trees() if c[0] != "shuffled_balanced_256"], ids=lambda c: c[0])
def test_joint_velocity_and_momentum_match_oracle(case):
    from paper_2103_03348_b300 import build, tree
    build.build()
    name, parent, length, tau0, s2 = case
    m = (parent.size + 1) // 2
    rng, k, minv, d = inputs(m, m + 2)
    A, B = coupled_blocks(rng, parent, length, tau0, s2, d, 0.3)
    tm = tree.TreeMass(tree.TreePrior(parent, length, tau0, s2), k, Z0, nc=6)
    tm.d.copy_(dev(d))
    tm.factor()
    tm.set_coupling(A, B)
    Bc = tm.coupling_shrink * B
    p = rng.standard_normal(k)
    vel, kin = dev(np.zeros(k)), dev(0.0)
    tm.velocity(dev(p), dev(minv), vel=vel, kinetic=kin)
    ref = tree_oracle.joint_mass_velocity(minv, d, A, Bc, p, Z0, parent, length, tau0, s2)
    assert scaled_err(vel.cpu().numpy(), ref) <= TREE_TOL, name
    assert abs(kin.item() - 0.5 * p @ ref) <= TREE_TOL * abs(0.5 * p @ ref), name
    xi = rng.standard_normal(tm.n_normals)
    pg = tm.momentum(dev(minv), dev(xi), dev(np.zeros(k)))
    pref = tree_oracle.joint_mass_momentum(minv, d, A, Bc, xi, Z0, parent, length, tau0, s2)
    assert scaled_err(pg.cpu().numpy(), pref) <= TREE_TOL, name


class TreeGaussJointPost(TreeGaussPost):
    """TreeGaussPost with the globals coupled to the rates: precision
    [[Ag, Bg^T], [Bg, diag(d0) + P]] on (globals, z), diag(a) elsewhere."""

    def __init__(self, tp, a, d0, Ag, Bg):
        super().__init__(tp, a, d0)
        self.Ag, self.Bg = Ag, Bg

    def evaluate(self, q, want_hess=False, out=None):
        if out is None:
            out = {"logpost": torch.empty((), dtype=torch.float64, device=q.device),
                   "grad": torch.empty_like(q), "hdiag": torch.empty_like(q)}
        z, g = q[Z0:Z0 + self.m], q[:6]
        pr = self.tree.evaluate(z, want=("pz", "pdiag"))
        aq = self.a * q
        aq[:6] = self.Ag @ g + self.Bg.T @ z
        aq[Z0:Z0 + self.m] = self.d0 * z + pr["pz"] + self.Bg @ g
        out["logpost"].copy_(-0.5 * torch.dot(q, aq))
        out["grad"].copy_(-aq)
        if want_hess:
            self.pd.copy_(pr["pdiag"])
            h = -self.a.clone()
            h[:6] = -torch.diagonal(self.Ag)
            h[Z0:Z0 + self.m] = -(self.d0 + pr["pdiag"])
            out["hdiag"].copy_(h)
        self.calls["hess" if want_hess else "grad"] += 1
        return out


def test_joint_mass_recovers_coupled_gaussian_moments():
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    w = synth.make_ebola_like(seed=4, n=2000, m_seq=120, box=150.0, t_max=150.0, n_hot=4)
    par, ln = w.tree_parent, w.tree_length
    tp = tree.TreePrior(par, ln, 0.0, 1.0)
    rng = np.random.default_rng(9)
    m = tp.m
    a = rng.uniform(0.5, 20.0, Z0 + m + 2)
    d0 = rng.uniform(0.0, 3.0, m)
    Ag, Bg = coupled_blocks(rng, par, ln, 0.0, 1.0, d0, 0.2)
    post = TreeGaussJointPost(tp, dev(a), dev(d0), dev(Ag), dev(Bg))
    minv = 1.0 / a
    var = np.array([tree_oracle.joint_mass_velocity(minv, d0, Ag, Bg, e, Z0, par, ln, 0.0, 1.0)[j]
                    for j, e in enumerate(np.eye(post.dim))])  # diag of the target's covariance
    q0 = dev(np.zeros(post.dim))
    kw = dict(n_iter=800, n_warmup=200, n_steps=10, eps0=0.1, mass_every=50, seed=4)
    ch = hmc.sample(post, q0, mass="tree_joint", **kw)
    ess = hmc.ess_all(ch.draws)
    s = np.sqrt(var)
    assert 0.5 < ch.accept.mean() <= 1.0
    assert np.all(np.abs(ch.draws.mean(0)) <= 5 * s / np.sqrt(ess))
    assert np.all(np.abs(ch.draws.var(0) / var - 1) <= 5 * np.sqrt(2 / ess) + 0.05)
    # mixing, not only correctness: every global moves (with an exact mass and a fixed step size the
    # trajectory can land near a whole period, so ESS comparisons between masses are left to the
    # measured Hawkes chains)
    assert ess[:6].min() > 100
    block = hmc.sample(post, q0, mass="tree", **kw)  # the block mass targets the same law
    ess_b = hmc.ess_all(block.draws)
    assert np.all(np.abs(block.draws.mean(0)) <= 5 * s / np.sqrt(ess_b))


def test_joint_mass_chain_on_hawkes_posterior_and_resume(tmp_path):
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    w = synth.make_ebola_like(seed=11, n=600, m_seq=40, box=120.0, t_max=120.0, n_hot=4)
    tp = tree.TreePrior(w.tree_parent, w.tree_length, 0.0, 1.0)

    def make():
        return hmc.Posterior(dev(w.x), dev(w.y), dev(w.t), dev(w.r), torch.tensor(w.sequenced, device="cuda"), None,
                             hmc.prior_km_days(), "fp32c", tree=tp)

    q0 = dev(np.concatenate([np.log(w.params), w.r[w.sequenced]]))
    kw = dict(n_iter=60, n_warmup=60, n_steps=10, eps0=0.05, mass_every=25, seed=2, mass="tree_joint")
    full = hmc.sample(make(), q0, **kw)
    assert np.all(np.isfinite(full.logpost)) and np.all(np.isfinite(full.draws))
    assert 0.4 < full.accept.mean() <= 1.0
    ck = str(tmp_path / "ck.pt")
    hmc.sample(make(), q0, checkpoint=ck, checkpoint_every=80, **kw)
    resumed = hmc.sample(make(), q0, resume=ck, **kw)
    assert np.array_equal(resumed.draws, full.draws) and np.array_equal(resumed.accept, full.accept)
