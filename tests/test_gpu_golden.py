"""The CUDA path against the committed golden fixtures (tests/golden/, oracle
outputs stored with their inputs)."""
import json
import os

import numpy as np
import pytest

from parity_util import FP32C_GNORM_TOL, FP32C_LL_TOL, FP64_TOL, norm_rel, scaled_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def dev(a):
    return torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", ["fp64", "fp32c", "fp32c_band", "fp32c_st"])
@pytest.mark.parametrize("name", ["loglik_hand_n7.json", "loglik_uniform_n96.json"])
def test_likelihood_fixture(name, precision):
    from paper_2103_03348_b300 import build, hawkes
    build.build()
    g = load(name)
    i, e = g["inputs"], g["expected"]
    ll, grad, hd = hawkes.hess_diag(dev(i["x"]), dev(i["y"]), dev(i["t"]), dev(i["r"]), i["params"], precision)
    ll, grad, hd = ll.item(), grad.cpu().numpy(), hd.cpu().numpy()
    if precision == "fp64":
        assert abs(ll - e["loglik"]) <= FP64_TOL * abs(e["loglik"])
        assert scaled_err(grad, e["grad"]) <= FP64_TOL and scaled_err(hd, e["hdiag"]) <= FP64_TOL
    else:
        assert abs(ll - e["loglik"]) <= FP32C_LL_TOL * abs(e["loglik"])
        assert norm_rel(grad, e["grad"]) <= FP32C_GNORM_TOL
        assert norm_rel(hd, e["hdiag"]) <= 1e-4


def test_tree_fixture():
    from paper_2103_03348_b300 import build, tree
    build.build()
    i, e = load("tree_prior_m9.json")["inputs"], load("tree_prior_m9.json")["expected"]
    tp = tree.TreePrior(i["parent"], i["length"], i["root_var"], i["sigma2"])
    out = tp.evaluate(dev(i["z"]))
    assert abs(out["logdens"].item() - e["logdens"]) <= 1e-13 * abs(e["logdens"])
    np.testing.assert_allclose(out["pz"].cpu().numpy(), e["pz"], rtol=1e-12)
    np.testing.assert_allclose(out["pdiag"].cpu().numpy(), e["pdiag"], rtol=1e-12)


@pytest.mark.parametrize("prior_form", ["dense", "tree"])
def test_posterior_fixture(prior_form):
    from paper_2103_03348_b300 import build, hmc, tree
    build.build()
    g = load("posterior_n48_m9.json")
    i, e = g["inputs"], g["expected"]
    prior = hmc.Prior(tuple(i["prior_kind"]), tuple(i["prior_a"]), tuple(i["prior_b"]))
    seq = torch.tensor(i["seq"], device="cuda")
    if prior_form == "dense":
        from oracle import tree_oracle  # the dense precision is an input here, built by the definition
        prec = tree_oracle.precision_matrix(np.array(i["tree_parent"]), np.array(i["tree_length"]))
        post = hmc.Posterior(dev(i["x"]), dev(i["y"]), dev(i["t"]), dev(i["r"]), seq, dev(prec), prior, "fp64")
    else:
        tp = tree.TreePrior(i["tree_parent"], i["tree_length"], 0.0, 1.0)
        post = hmc.Posterior(dev(i["x"]), dev(i["y"]), dev(i["t"]), dev(i["r"]), seq, None, prior, "fp64", tree=tp)
    out = post.evaluate(dev(i["q"]), want_hess=True)
    assert abs(out["logpost"].item() - e["logpost"]) <= FP64_TOL * abs(e["logpost"])
    assert scaled_err(out["grad"].cpu().numpy(), e["grad"]) <= FP64_TOL
    assert scaled_err(out["hdiag"].cpu().numpy(), e["hdiag"]) <= FP64_TOL
