"""STS-CP on the GPU against the FP64 oracle.

The GPU sums the tree masses in float32; a draw may therefore differ from
the oracle only where the oracle finds a decision within 1e-5 * m(root) of
its threshold (the oracle's near-tie flag at that tolerance), and at most 1%
of the draws may differ at these sizes.  Probabilities of equal draws agree
to 1e-5 relative; fits to 1e-3.
"""
import numpy as np
import pytest
import torch

from oracle import cpals as oc
from tests.gpu_common import cuda_ready, lib_or_build, make_case, create, gpu_factors, rel_frob

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ready(), reason="needs a CUDA GPU")]
TIE = 1e-5


@pytest.fixture(scope="module")
def cpd():
    return lib_or_build()


def _oracle_sts(cpd, h, fs, mode, J, seed, sweep, F):
    grams = [oc.gram(U) for U in fs]
    trees = [oc.sts_build(U, F) for U in fs]
    return oc.sts_draw(trees, fs, grams, mode, J, seed, sweep, tie_tol=TIE)


@pytest.mark.parametrize("dims,R,F,nnz", [((200, 150, 100), 8, 0, 20000),
                                           ((333, 97, 1031), 25, 0, 30000),
                                           ((120, 90, 64), 8, 1, 8000),
                                           ((120, 90, 64), 8, 3, 8000),
                                           ((50, 40, 30, 20), 6, 0, 20000)])
def test_sts_draws_match_oracle(cpd, dims, R, F, nnz):
    idx, vals, init = make_case(dims, nnz, R, seed=321)
    J = 4000
    h = create(cpd, dims, idx, vals, init, "sts", R, J, seed=17, leaf_rows=F)
    fs = gpu_factors(cpd, h)
    Fe = F or R
    for mode, sweep in [(0, 0), (len(dims) - 1, 5)]:
        gi, gp = cpd.cpd_leverage_sample(h, mode, J, sweep)
        oi, op, near = _oracle_sts(cpd, h, fs, mode, J, 17, sweep, Fe)
        gi = gi.cpu().numpy()
        mism = np.any(gi != oi, axis=0)
        assert not np.any(mism & ~near), "STS draw differs away from a near-tie"
        assert mism.mean() < 0.01
        ok = ~mism
        assert np.max(np.abs(gp.cpu().numpy()[ok] - op[ok]) / op[ok]) < 1e-5
        assert np.all(gi[mode] == -1)
    h.close()


def test_sts_sweep_stepwise_and_fit(cpd):
    dims, R, J = (200, 150, 100), 8, 2000
    idx, vals, init = make_case(dims, 20000, R, seed=1001)
    h = create(cpd, dims, idx, vals, init, "sts", R, J, seed=3001)
    for s in range(2):
        for n in range(3):
            fs = gpu_factors(cpd, h)
            oi, op, near = _oracle_sts(cpd, h, fs, n, J, 3001, s, R)
            gi, gp = cpd.cpd_leverage_sample(h, n, J, s)
            gi_np = gi.cpu().numpy()
            assert not np.any(np.any(gi_np != oi, axis=0) & ~near)
            w = 1.0 / (J * gp)
            Y, _ = cpd.cpd_sampled_mttkrp(h, n, gi, w)
            Yo = oc.sampled_mttkrp(idx, vals, dims, fs, n, gi_np, w.cpu().numpy())
            assert rel_frob(Y.cpu().numpy(), Yo) <= 1e-5
            cpd.cpd_gram_solve(h, n, Y)
    h.close()


def test_sts_end_to_end_fit(cpd):
    dims, R, J = (200, 150, 100), 8, 2000
    idx, vals, init = make_case(dims, 20000, R, seed=1001)
    h = create(cpd, dims, idx, vals, init, "sts", R, J, seed=3001)
    cpd.cpd_als_sweep(h, 5)
    f_gpu = cpd.cpd_fit(h)
    _, fits = oc.als(idx, vals, dims, [u.astype(np.float64) for u in init], "sts", 5, J=J, seed=3001)
    assert abs(f_gpu - fits[-1]) < 1e-3
    h.close()
