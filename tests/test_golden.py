"""The FP64 oracle against cases worked by hand in exact arithmetic
(`tests/golden/hand_worked.json`; each case names the equation or algorithm
it follows and gives its derivation).  Small integer factors with unequal
entries make a transposed operand, a dropped or sign-flipped term, or a
wrong mode index change the answer."""
import ast
import json
import math
import operator
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import cpals as oc

with open(os.path.join(os.path.dirname(__file__), "golden", "hand_worked.json")) as f:
    GOLD = json.load(f)["cases"]

_OPS = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul, ast.Div: operator.truediv}


def value(x):
    """A fixture entry: a number, or an expression of integers, + - * / and
    sqrt(), evaluated with exact fractions where no square root occurs."""
    if not isinstance(x, str):
        return float(x)

    def ev(node):
        if isinstance(node, ast.Expression):
            return ev(node.body)
        if isinstance(node, ast.Constant) and isinstance(node.value, int):
            return Fraction(node.value)
        if isinstance(node, ast.BinOp) and type(node.op) in _OPS:
            a, b = ev(node.left), ev(node.right)
            if isinstance(a, float) or isinstance(b, float):
                a, b = float(a), float(b)
            return _OPS[type(node.op)](a, b)
        if isinstance(node, ast.UnaryOp) and isinstance(node.op, ast.USub):
            return -ev(node.operand)
        if isinstance(node, ast.Call) and getattr(node.func, "id", "") == "sqrt" and len(node.args) == 1:
            return math.sqrt(float(ev(node.args[0])))
        raise ValueError("unsupported expression %r" % x)

    return float(ev(ast.parse(x, mode="eval")))


def arr(x):
    return np.vectorize(value, otypes=[np.float64])(np.asarray(x, dtype=object))


def close(a, b, tol=1e-13):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (a.shape, b.shape)
    assert np.all(np.abs(a - b) <= tol * np.maximum(1.0, np.abs(b))), (a, b)


def test_leverage_scores_full_rank():
    c = GOLD["leverage_full_rank"]
    s = oc.arls_build(arr(c["U"]))
    close(s["G"], arr(c["G"]))
    close(s["Gpinv"], arr(c["G_pinv"]))
    close(s["ell"], arr(c["ell"]))
    close(s["cdf"], arr(c["cdf"]))
    close(s["C"], value(c["C"]))


def test_leverage_scores_rank_deficient():
    c = GOLD["leverage_rank_deficient"]
    s = oc.arls_build(arr(c["U"]))
    close(s["Gpinv"], arr(c["G_pinv"]))
    close(s["ell"], arr(c["ell"]))
    close(s["C"], value(c["C"]))


def test_inverse_cdf_edges_and_empty_bins():
    for case in GOLD["inverse_cdf"]["cases"]:
        ell = arr(case["ell"])
        cdf = np.cumsum(ell)
        got = oc.inverse_cdf(cdf, ell, arr(case["t"]))
        assert got.tolist() == case["i"], (case, got)


def _tensor(c):
    return np.asarray(c["idx"], dtype=np.int64), arr(c["vals"]), tuple(c["dims"]), [arr(U) for U in c["factors"]]


@pytest.mark.parametrize("n", [0, 1, 2])
def test_exact_mttkrp_every_mode(n):
    c = GOLD["mttkrp"]
    idx, vals, dims, fs = _tensor(c)
    close(oc.exact_mttkrp(idx, vals, dims, fs, n), arr(c["exact"][n]))


def test_sampled_mttkrp_selected_nonzeros_and_sketched_gram():
    c = GOLD["mttkrp"]
    idx, vals, dims, fs = _tensor(c)
    n = c["sampled_mode"]
    sidx = np.asarray(c["samp_idx"], dtype=np.int64)
    w = arr(c["w"])
    close(oc.sampled_mttkrp(idx, vals, dims, fs, n, sidx, w), arr(c["sampled"]))
    assert oc.selected_nnz(idx, dims, n, sidx) == c["selected_nnz"]
    close(oc.sketched_gram(fs, n, sidx, w), arr(c["sketched_gram"]))


def _krp_case():
    c = GOLD["krp_leverage"]
    fs = [arr(U) for U in c["factors"]]
    return c, fs, c["mode"], [U.shape[0] for U in fs]


def test_exact_krp_leverage_table():
    c, fs, n, dims = _krp_case()
    grams = [oc.gram(U) for U in fs]
    close(oc.pinv_sym(oc.hadamard_of_grams(grams, n)), arr(c["G_pinv"]))
    lev = arr(c["lev"])                       # lev[j][k], KRP key j + 3 k
    close(oc.exact_krp_leverage(fs, n), lev.T.reshape(-1))


@pytest.mark.parametrize("F", [1, 2, 3])
def test_sts_draws_follow_the_exact_leverage_law(F):
    c, fs, n, dims = _krp_case()
    grams = [oc.gram(U) for U in fs]
    trees = [oc.sts_build(U, F) for U in fs]
    J = 30000
    sidx, p, near = oc.sts_draw(trees, fs, grams, n, J, seed=11, sweep=2)
    law = arr(c["lev"]) / 2.0
    close(p, law[sidx[1], sidx[2]])
    assert np.all(law[sidx[1], sidx[2]] > 0)           # zero-mass rows never drawn
    marg = arr(c["sts_marginal_first"])
    freq = np.bincount(sidx[1], minlength=3) / J
    assert np.all(np.abs(freq - marg) < 5 * np.sqrt(marg * (1 - marg) / J))
    joint = np.zeros((3, 3))
    np.add.at(joint, (sidx[1], sidx[2]), 1.0 / J)
    assert np.all(np.abs(joint - law) < 5 * np.sqrt(law * (1 - law) / J) + 1e-12)


def test_arls_draws_follow_the_product_law():
    c, fs, n, dims = _krp_case()
    samplers = [oc.arls_build(U) for U in fs]
    sidx, p, near = oc.arls_draw(samplers, n, 20000, seed=5, sweep=0)
    close(p, np.full(p.shape, value(c["arls_p"])))
    assert np.all(sidx[n] == -1)


def test_sts_tree_nodes():
    c = GOLD["sts_tree"]
    U = arr(c["U"])
    t1 = oc.sts_build(U, 1)
    assert t1["L"] == 4
    close(t1["nodes"][4:8], arr(c["F1_nodes"]))
    close(t1["nodes"][1:4], arr(c["F1_inner"]))
    t2 = oc.sts_build(U, 2)
    assert t2["L"] == 2
    close(t2["nodes"][2:4], arr(c["F2_nodes"]))
    close(t2["nodes"][1], arr(c["F2_root"]))


def test_solve_and_renormalise():
    c = GOLD["solve_renorm"]
    Un, sigma = oc.solve_and_renorm(arr(c["Y"]), arr(c["G_pinv"]))
    close(Un, arr(c["U"]))
    close(sigma, arr(c["sigma"]))


@pytest.mark.parametrize("which", [0, 1])
def test_fit(which):
    c = GOLD["fit"]["cases"][which]
    idx, vals, dims, fs = _tensor(c)
    sigma = arr(c["sigma"])
    close(oc.fit(idx, vals, fs, sigma), value(c["fit"]))
    if "model_norm_sq" in c:
        close(oc.model_norm_sq(fs, sigma), value(c["model_norm_sq"]))
        close(oc.inner_with_model(idx, vals, fs, sigma), value(c["inner"]))


def test_sample_weights():
    c = GOLD["sample_weights"]
    close(oc.sample_weights(arr(c["p"]), c["J"]), arr(c["w"]))


def test_fixture_expressions_parse_exactly():
    assert value("2*sqrt(58)/3") == pytest.approx(2 * math.sqrt(58) / 3, rel=1e-15)
    assert value("-1/3") == -1.0 / 3.0
    with pytest.raises(ValueError):
        value("__import__('os')")
