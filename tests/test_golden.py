"""The oracle still reproduces the committed golden fixtures (tests/golden/,
written by make_golden.py from the oracle alone), and the fixtures agree with
facts fixed by the paper's definitions."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import hmc_oracle, tree_oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["loglik_hand_n7.json", "loglik_uniform_n96.json"])
def test_oracle_reproduces_likelihood_fixture(name):
    g = load(name)
    i, e = g["inputs"], g["expected"]
    o = oracle.evaluate(np.array(i["x"]), np.array(i["y"]), np.array(i["t"]), np.array(i["r"]),
                        np.array(i["params"]), want=2)
    assert abs(o["loglik"] - e["loglik"]) <= 1e-13 * abs(e["loglik"])
    for k in ("lam", "grad", "hdiag"):
        np.testing.assert_allclose(o[k], e[k], rtol=1e-12, atol=1e-14 * np.max(np.abs(e[k])))


def test_hand_fixture_structure():
    """Events 1 and 2 share a time and a place: equal intensities, and the
    log-likelihood splits as sum log lambda - Lambda."""
    e = load("loglik_hand_n7.json")["expected"]
    assert e["lam"][1] == e["lam"][2]
    assert abs(np.sum(np.log(e["lam"])) - e["Lambda"] - e["loglik"]) <= 1e-13 * abs(e["loglik"])


def test_oracle_reproduces_tree_fixture():
    g = load("tree_prior_m9.json")
    i, e = g["inputs"], g["expected"]
    ld, pz, pd = tree_oracle.tree_prior(np.array(i["z"]), np.array(i["parent"]), np.array(i["length"]),
                                        i["root_var"], i["sigma2"])
    assert abs(ld - e["logdens"]) <= 1e-13 * abs(e["logdens"])
    np.testing.assert_allclose(pz, e["pz"], rtol=1e-12)
    np.testing.assert_allclose(pd, e["pdiag"], rtol=1e-12)
    v = np.array(e["V"])
    # by hand from the tree: tips 0 and 1 meet at node 9, whose root path is 9 -> 10 -> 14 -> 16
    assert abs(v[0, 1] - (0.25 + 0.4 + 0.3 + 0.5)) <= 1e-15
    # tips 0 and 8 meet only at the root
    assert abs(v[0, 8] - 0.25) <= 1e-15
    assert abs(v[8, 8] - (0.25 + 2.0 + 0.35)) <= 1e-15


def test_oracle_reproduces_posterior_fixture():
    g = load("posterior_n48_m9.json")
    i, e = g["inputs"], g["expected"]
    prec = tree_oracle.precision_matrix(np.array(i["tree_parent"]), np.array(i["tree_length"]))
    prior = (np.array(i["prior_kind"]), np.array(i["prior_a"]), np.array(i["prior_b"]))
    lp, gq, hq = hmc_oracle.log_posterior(np.array(i["x"]), np.array(i["y"]), np.array(i["t"]), np.array(i["r"]),
                                          np.array(i["seq"]), prec, prior, np.array(i["q"]))
    assert abs(lp - e["logpost"]) <= 1e-13 * abs(e["logpost"])
    np.testing.assert_allclose(gq, e["grad"], rtol=1e-11, atol=1e-13 * np.max(np.abs(e["grad"])))
    np.testing.assert_allclose(hq, e["hdiag"], rtol=1e-11, atol=1e-13 * np.max(np.abs(e["hdiag"])))
