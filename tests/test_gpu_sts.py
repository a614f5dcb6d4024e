"""STS-CP on the GPU against the FP64 oracle.

Precision 0 (the default) keeps the tree, the running Hadamard product and
the walk's masses in double-float and the target in float64, and rescans a
leaf in double-float whenever its float32 row masses cannot decide the row.
A draw may then differ from the oracle's only where the oracle finds a
decision within 1e-12 * m(root) of its threshold (its near-tie flag); the
number of such ties is printed.  Probabilities of equal draws agree to 1e-9
relative.  Precision option 1 (float32 trees and masses) is held to the
float32 bar: ties at 1e-5 * m(root), at most 1% of the draws differing.
"""
import numpy as np
import pytest
import torch

from oracle import cpals as oc
from tests.gpu_common import cuda_ready, lib_or_build, make_case, create, gpu_factors, rel_frob

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ready(), reason="needs a CUDA GPU")]
TIE = 1e-12
TIE_FAST = 1e-5


@pytest.fixture(scope="module")
def cpd():
    return lib_or_build()


def _oracle_sts(fs, mode, J, seed, sweep, F, tie):
    grams = [oc.gram(U) for U in fs]
    trees = [oc.sts_build(U, F) for U in fs]
    return oc.sts_draw(trees, fs, grams, mode, J, seed, sweep, tie_tol=tie)


def _compare(gi, gp, oi, op, near, label):
    mism = np.any(gi != oi, axis=0)
    away = mism & ~near
    print("%s: %d draws, %d near ties, %d differing (all at ties)" % (label, gi.shape[1], int(near.sum()),
                                                                       int(mism.sum())))
    assert not np.any(away), "STS draw differs away from a near-tie: %s" % np.nonzero(away)[0][:10]
    assert int(mism.sum()) <= max(1, gi.shape[1] // 1000), "too many draws differ at ties"
    ok = ~mism
    return mism, np.max(np.abs(gp[ok] - op[ok]) / op[ok]) if ok.any() else 0.0


@pytest.mark.parametrize("dims,R,F,nnz", [((200, 150, 100), 8, 0, 20000),
                                           ((333, 97, 1031), 25, 0, 30000),
                                           ((120, 90, 64), 8, 1, 8000),
                                           ((120, 90, 64), 8, 3, 8000),
                                           ((300, 260, 170), 40, 0, 30000),
                                           ((420, 310, 260), 100, 0, 40000),
                                           ((50, 40, 30, 20), 6, 0, 20000)])
def test_sts_draws_match_oracle(cpd, dims, R, F, nnz):
    idx, vals, init = make_case(dims, nnz, R, seed=321)
    J = 4000
    h = create(cpd, dims, idx, vals, init, "sts", R, J, seed=17, leaf_rows=F)
    fs = gpu_factors(cpd, h)
    Fe = F or R
    for mode, sweep in [(0, 0), (len(dims) - 1, 5), (1, 2)]:
        gi, gp = cpd.cpd_leverage_sample(h, mode, J, sweep)
        oi, op, near = _oracle_sts(fs, mode, J, 17, sweep, Fe, TIE)
        gi = gi.cpu().numpy()
        _, perr = _compare(gi, gp.cpu().numpy(), oi, op, near, "dims %s R %d F %d mode %d" % (dims, R, Fe, mode))
        assert perr < 1e-9, perr
        assert np.all(gi[mode] == -1)
    print("leaves rescanned in double-float:", cpd.cpd_sts_rescans(h))
    h.close()


def test_sts_fast_precision_draws(cpd):
    """Precision option 1: float32 trees, masses and target."""
    dims, R, J = (200, 150, 100), 8, 4000
    idx, vals, init = make_case(dims, 20000, R, seed=321)
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method="sts", rank=R, samples=J, seed=17, fast=True)
    fs = gpu_factors(cpd, h)
    for mode, sweep in [(0, 0), (2, 5)]:
        gi, gp = cpd.cpd_leverage_sample(h, mode, J, sweep)
        oi, op, near = _oracle_sts(fs, mode, J, 17, sweep, R, TIE_FAST)
        mism, perr = _compare(gi.cpu().numpy(), gp.cpu().numpy(), oi, op, near, "fast mode %d" % mode)
        assert mism.mean() < 0.01
        assert perr < 1e-4
    assert cpd.cpd_sts_rescans(h) == 0
    h.close()


def test_sts_sweep_stepwise_and_fit(cpd):
    dims, R, J = (200, 150, 100), 8, 2000
    idx, vals, init = make_case(dims, 20000, R, seed=1001)
    h = create(cpd, dims, idx, vals, init, "sts", R, J, seed=3001)
    for s in range(2):
        for n in range(3):
            fs = gpu_factors(cpd, h)
            oi, op, near = _oracle_sts(fs, n, J, 3001, s, R, TIE)
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
    print("STS 5-round fit: GPU %.6f oracle %.6f" % (f_gpu, fits[-1]))
    assert abs(f_gpu - fits[-1]) < 1e-3
    h.close()
