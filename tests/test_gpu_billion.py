"""Parity of one mode update at the billion-scale workload (dims 8.2e6 x
1.77e5 x 8.1e6 -- the Reddit tensor's dims, Table 4 -- 1e9 distinct Zipf(1.3)
nonzeros, log(1 + Poisson(3)) values, R = 100, J = 2^17), in the launch
configuration the bench times, after one captured ALS round:

* all 131,072 CP-ARLS-LEV draws of a mode update equal the FP64 oracle's
  inverse-CDF draws from the same factors, ties excepted: a draw within
  min(1e-6, max(1e-12, 8 cond(G_k) 2^-53)) C_k of a bin boundary, cond over
  the eigenvalues the pseudo-inverse keeps (the factor Grams of this
  Zipf(1.3) tensor grow ill-conditioned, and a float64 Gram fixes G_k^+ and
  the leverage scores only to ~cond(G_k) 2^-53); probabilities agree to
  min(1e-6, 64 cond_max^2 2^-53) relative (a quadratic form in G_k^+ can
  lose cond^2);
* the downsampled MTTKRP of those draws equals the oracle's on 512 random
  output rows (their nonzeros picked out of the device COO), 1e-5 relative;
* the solve and renormalisation equal the oracle's on those rows.
The oracle cannot hold the whole tensor's per-nonzero work at this size, so
the MTTKRP and solve are compared on sampled rows."""
import numpy as np
import pytest
import torch

from oracle import cpals as oc
from paper_2210_05105_gb300 import synth
from tests.gpu_common import cuda_ready, lib_or_build, rel_frob

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ready(), reason="needs a CUDA GPU")]

W = synth.WORKLOADS["zipf_reddit_1B"]


def test_billion_scale_mode_update_matches_oracle():
    cpd = lib_or_build()
    dims, R, J = W["dims"], W["R"], W["J"]
    idx, vals, used = synth.make_tensor_device(dims, W["nnz"], W["data_seed"], W["zipf"], W["values"])
    assert idx.shape == (3, W["nnz"])
    h = cpd.cpd_create(dims, idx, vals, None, method="arls", rank=R, samples=J, seed=W["sample_seed"])
    cpd.cpd_als_sweep(h, 1)
    mode, sweep = 1, 7
    fs = [cpd.cpd_get_factors(h, k).double().cpu().numpy() for k in range(3)]
    gi, gp = cpd.cpd_leverage_sample(h, mode, J, sweep)
    samplers = [oc.arls_build(U) if k != mode else None for k, U in enumerate(fs)]
    oi, op, near = oc.arls_draw(samplers, mode, J, W["sample_seed"], sweep, tie_tol="conditioned")
    conds = [oc.gram_condition(s["G"]) for s in samplers if s is not None]
    gi_np = gi.cpu().numpy()
    mism = np.any(gi_np != oi, axis=0)
    print("billion-scale ARLS: %d draws, %d near ties, %d differing; cond(G_k) %s"
          % (J, int(near.sum()), int(mism.sum()), ["%.2e" % c for c in conds]))
    assert not np.any(mism & ~near)
    assert int(mism.sum()) <= max(1, J // 1000)   # ties stay a small minority
    ok = ~mism
    perr = np.max(np.abs(gp.cpu().numpy()[ok] - op[ok]) / op[ok])
    print("probability max rel err %.2e" % perr)
    assert perr < min(1e-6, max(1e-10, 64 * max(conds) ** 2 * 2.0 ** -53))
    assert near.sum() < J // 100                  # the window is not vacuous
    w = 1.0 / (J * gp)
    Y, nsel = cpd.cpd_sampled_mttkrp(h, mode, gi, w)
    rows = np.sort(np.random.default_rng(5).choice(dims[mode], size=512, replace=False))
    sel = torch.isin(idx[mode].long(), torch.from_numpy(rows).cuda())
    Yo = oc.sampled_mttkrp(idx[:, sel].cpu().numpy(), vals[sel].cpu().numpy(), dims, fs, mode, gi_np,
                           w.cpu().numpy())[rows]
    Yg = Y.double().cpu().numpy()
    err = rel_frob(Yg[rows], Yo)
    print("billion-scale MTTKRP on 512 rows: rel err %.2e, nnz_sel %d" % (err, nsel))
    assert err <= 1e-5
    G = oc.hadamard_of_grams([oc.gram(U) for U in fs], mode)
    Un, _ = oc.solve_and_renorm(Yg, oc.pinv_sym(G))
    cpd.cpd_gram_solve(h, mode, Y)
    Ug = cpd.cpd_get_factors(h, mode).double().cpu().numpy()
    assert rel_frob(Ug[rows], Un[rows]) <= 1e-5
    h.close()
    del idx, vals
    torch.cuda.empty_cache()
