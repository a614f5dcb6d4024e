"""Parity at the full size of the headline workload, in the launch
configuration the bench times: dims 100,000^3, 5e7 distinct Zipf(1.1)
nonzeros, R = 32, J = 65,536, CP-ARLS-LEV, after two captured ALS rounds.

* every one of the 65,536 draws of two mode updates equals the FP64
  oracle's inverse-CDF draw from the same factors (ties at 1e-12 C excepted),
  with probabilities to 1e-10 relative: after two rounds the factor Grams have
  condition numbers near 2e3, and the df64 pseudo-inverse is accurate to
  ~cond * 2^-48 ~ 1e-11 per factor (5.8e-12 observed);
* the downsampled MTTKRP of a full draw equals the oracle's over all 1e5 rows
  (relative Frobenius 1e-5) and selects the same nonzeros;
* the solve and renormalisation equal the oracle's for that Y;
* all 65,536 STS-CP draws of a mode update equal the oracle's walk except at
  decisions within 1e-12 m(root) of a threshold.
"""
import numpy as np
import pytest
import torch

from oracle import cpals as oc
from paper_2210_05105_gb300 import synth
from tests.gpu_common import cuda_ready, lib_or_build, rel_frob

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ready(), reason="needs a CUDA GPU")]

W = synth.WORKLOADS["zipf_1e5cube_50M"]


@pytest.fixture(scope="module")
def full():
    cpd = lib_or_build()
    dims, R, J = W["dims"], W["R"], W["J"]
    idx, vals = synth.make_tensor_torch(dims, W["nnz"], W["data_seed"], W["zipf"], W["values"], device="cuda")
    init = [torch.from_numpy(u).cuda() for u in synth.init_factors(dims, R, W["init_seed"])]
    h = cpd.cpd_create(dims, idx, vals, init, method="arls", rank=R, samples=J, seed=W["sample_seed"])
    cpd.cpd_als_sweep(h, 2)
    idx_np, vals_np = idx.cpu().numpy(), vals.cpu().numpy()
    del idx, vals, init
    torch.cuda.empty_cache()
    yield cpd, h, idx_np, vals_np
    h.close()


def _factors(cpd, h):
    return [cpd.cpd_get_factors(h, k).double().cpu().numpy() for k in range(3)]


def test_fullsize_draws_equal_oracle(full):
    cpd, h, idx, vals = full
    J = W["J"]
    fs = _factors(cpd, h)
    samplers = [oc.arls_build(U) for U in fs]
    for mode, sweep in ((0, 2), (2, 9)):
        gi, gp = cpd.cpd_leverage_sample(h, mode, J, sweep)
        oi, op, near = oc.arls_draw(samplers, mode, J, W["sample_seed"], sweep)
        gi = gi.cpu().numpy()
        mism = np.any(gi != oi, axis=0)
        print("full-size ARLS mode %d: %d draws, %d near ties, %d differing"
              % (mode, J, int(near.sum()), int(mism.sum())))
        assert not np.any(mism & ~near), "draw differs away from a tie"
        assert int(mism.sum()) <= max(1, J // 1000), "too many draws differ at ties"
        ok = ~mism
        assert np.max(np.abs(gp.cpu().numpy()[ok] - op[ok]) / op[ok]) < 1e-10


def test_fullsize_sampled_mttkrp_and_solve(full):
    cpd, h, idx, vals = full
    dims, J = W["dims"], W["J"]
    fs = _factors(cpd, h)
    mode = 1
    gi, gp = cpd.cpd_leverage_sample(h, mode, J, 4)
    w = 1.0 / (J * gp)
    Y, nsel = cpd.cpd_sampled_mttkrp(h, mode, gi, w)
    gi_np, w_np = gi.cpu().numpy(), w.cpu().numpy()
    ref = oc.sampled_mttkrp(idx, vals, dims, fs, mode, gi_np, w_np)
    Yg = Y.double().cpu().numpy()
    assert rel_frob(Yg, ref) <= 1e-5
    assert nsel == oc.selected_nnz(idx, dims, mode, gi_np)
    sigma = cpd.cpd_gram_solve(h, mode, Y).cpu().numpy()
    G = oc.hadamard_of_grams([oc.gram(U) for U in fs], mode)
    Un, sig_ref = oc.solve_and_renorm(Yg, oc.pinv_sym(G))
    assert rel_frob(cpd.cpd_get_factors(h, mode).double().cpu().numpy(), Un) <= 1e-5
    assert np.max(np.abs(sigma - sig_ref) / sig_ref) <= 1e-5


def test_fullsize_three_round_fit_matches_oracle(full):
    """Three whole ALS rounds of CP-ARLS-LEV at the full size from the same
    initial factors and uniforms: the GPU's fit and the FP64 oracle's agree
    to 1e-3 (the draws are decided on float64 scores on both sides, so the
    trajectories differ only by the float32 rounding of the factors)."""
    cpd, _, idx, vals = full
    dims, R, J = W["dims"], W["R"], W["J"]
    init = synth.init_factors(dims, R, W["init_seed"])
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=J,
                       seed=W["sample_seed"])
    cpd.cpd_als_sweep(h, 3)
    f_gpu = cpd.cpd_fit(h)
    h.close()
    _, fits = oc.als(idx, vals, dims, [u.astype(np.float64) for u in init], "arls", 3, J=J, seed=W["sample_seed"])
    print("full-size 3-round fit: GPU %.6f oracle %.6f gap %.2e" % (f_gpu, fits[-1], abs(f_gpu - fits[-1])))
    assert abs(f_gpu - fits[-1]) < 1e-3


def test_fullsize_sts_draws_match_oracle(full):
    """STS-CP at the full size, in the launch configuration of
    `bench.py --method sts` (the library's default leaf size, 8 rows here: a
    14-level tree per factor; the oracle's trees use F = R = 32, and the law
    does not depend on F): all 65,536 draws of a mode update equal the FP64
    oracle's walk on the same factors except at decisions within 1e-12 m(root)
    of a threshold (ties, counted and printed), with probabilities to 1e-9
    relative."""
    cpd, h_arls, idx, vals = full
    dims, R, J = W["dims"], W["R"], W["J"]
    fs32 = [cpd.cpd_get_factors(h_arls, k) for k in range(3)]
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(), fs32, method="sts",
                       rank=R, samples=J, seed=W["sample_seed"])
    fs = _factors(cpd, h)
    grams = [oc.gram(U) for U in fs]
    trees = [oc.sts_build(U, R) for U in fs]
    mode, sweep = 1, 3
    gi, gp = cpd.cpd_leverage_sample(h, mode, J, sweep)
    oi, op, near = oc.sts_draw(trees, fs, grams, mode, J, W["sample_seed"], sweep, tie_tol=1e-12)
    gi = gi.cpu().numpy()
    mism = np.any(gi != oi, axis=0)
    print("full-size STS: %d draws, %d near ties, %d differing, %d leaves rescanned in double-float"
          % (J, int(near.sum()), int(mism.sum()), cpd.cpd_sts_rescans(h)))
    assert not np.any(mism & ~near), "STS draw differs away from a near-tie"
    assert int(mism.sum()) <= max(1, J // 1000), "too many draws differ at ties"
    ok = ~mism
    assert np.max(np.abs(gp.cpu().numpy()[ok] - op[ok]) / op[ok]) < 1e-9
    h.close()
