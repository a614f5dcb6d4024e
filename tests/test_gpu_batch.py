"""Batched form and autotuner against the single-handle path."""
import numpy as np
import pytest
import torch

from tests.gpu_common import cuda_ready, lib_or_build, make_case, create, gpu_factors, rel_frob

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ready(), reason="needs a CUDA GPU")]

CASES = [((120, 90, 70), 6000, 8, 800, "arls"), ((300, 50, 40, 30), 9000, 6, 1200, "arls"),
         ((80, 200, 60), 7000, 12, 1000, "sts"), ((500, 400, 300), 20000, 16, 3000, "arls"),
         ((64, 64, 64), 3000, 4, 500, "sts")]


def _handles(cpd):
    hs = []
    for i, (dims, nnz, R, J, m) in enumerate(CASES):
        idx, vals, init = make_case(dims, nnz, R, seed=500 + i)
        hs.append(create(cpd, dims, idx, vals, init, m, R, J, seed=40 + i))
    return hs


def test_batch_graph_equals_individual_sweeps():
    """Two batched rounds equal two rounds of each handle's own graph.  The
    SpMM's float32 reductions add in a run-dependent order, so the two runs
    differ by float32 rounding; both samplers decide their draws on float64
    (CP-ARLS-LEV) or double-float (STS-CP) masses, so that rounding moves a
    draw only at a near-tie and the factors stay within 1e-3."""
    cpd = lib_or_build()
    ha = _handles(cpd)
    hb = _handles(cpd)
    b = cpd.cpd_batch_create(ha, branches=3)
    cpd.cpd_batch_sweep(b, 2)
    for h in hb:
        cpd.cpd_als_sweep(h, 2)
    for (dims, nnz, R, J, m), h1, h2 in zip(CASES, ha, hb):
        for k in range(h1.N):
            assert rel_frob(cpd.cpd_get_factors(h1, k).cpu().numpy(),
                            cpd.cpd_get_factors(h2, k).cpu().numpy()) < 1e-3, (m, k)
        assert abs(cpd.cpd_fit(h1) - cpd.cpd_fit(h2)) < 1e-4
    b.close()
    for h in ha + hb:
        h.close()


def test_autotune_picks_valid_shapes_and_keeps_results():
    cpd = lib_or_build()
    dims, nnz, R, J = (500, 400, 300), 20000, 16, 3000
    for m in ("arls", "sts"):
        idx, vals, init = make_case(dims, nnz, R, seed=77)
        h1 = create(cpd, dims, idx, vals, init, m, R, J, seed=9)
        h2 = create(cpd, dims, idx, vals, init, m, R, J, seed=9)
        bps, g, F = cpd.cpd_autotune(h1)
        assert bps in (1, 2, 4, 8) and g in (8, 16, 32)
        assert F in (R, R // 2, R // 4, R // 8)
        cpd.cpd_als_sweep(h1, 3)
        cpd.cpd_als_sweep(h2, 3)
        assert abs(cpd.cpd_fit(h1) - cpd.cpd_fit(h2)) < 1e-3
        h1.close()
        h2.close()


def test_batched_rounds_match_oracle():
    """The batched graph against the FP64 oracle: two batched ALS rounds of
    every tensor of the batch (3- and 4-mode, CP-ARLS-LEV and STS-CP) end at
    the oracle's fit from the same inputs and uniforms (within 1e-3)."""
    from oracle import cpals as oc
    cpd = lib_or_build()
    hs, inputs = [], []
    for i, (dims, nnz, R, J, m) in enumerate(CASES):
        idx, vals, init = make_case(dims, nnz, R, seed=500 + i)
        inputs.append((idx, vals, init))
        hs.append(create(cpd, dims, idx, vals, init, m, R, J, seed=40 + i))
    b = cpd.cpd_batch_create(hs, branches=3)
    cpd.cpd_batch_sweep(b, 2)
    for i, ((dims, nnz, R, J, m), h, (idx, vals, init)) in enumerate(zip(CASES, hs, inputs)):
        _, fits = oc.als(idx, vals, dims, [u.astype(np.float64) for u in init], m, 2, J=J, seed=40 + i)
        f = cpd.cpd_fit(h)
        print("batched tensor %d (%s, %s): GPU fit %.6f, oracle %.6f" % (i, m, dims, f, fits[-1]))
        assert abs(f - fits[-1]) < 1e-3
    b.close()
    for h in hs:
        h.close()
