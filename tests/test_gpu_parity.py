"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: sample indices exact except draws the oracle marks as ties
within 1e-12 of a bin boundary, at most 1 in 1000 of them (counts printed); draw probabilities 1e-12 relative (float64
on both sides); sampled and exact MTTKRP 1e-5 relative Frobenius (float32
accumulation); solve / renormalisation 1e-5; fit 1e-9 absolute for a given
model and 1e-3 between full randomized runs.
"""
import numpy as np
import pytest
import torch

from oracle import cpals as oc
from tests.gpu_common import cuda_ready, lib_or_build, make_case, create, gpu_factors, rel_frob

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ready(), reason="needs a CUDA GPU")]

SMALL = dict(dims=(200, 150, 100), nnz=20000, R=8, J=2000)


@pytest.fixture(scope="module")
def cpd():
    return lib_or_build()


def _small(cpd, method="arls", **kw):
    cfg = dict(SMALL)
    cfg.update(kw)
    idx, vals, init = make_case(cfg["dims"], cfg["nnz"], cfg["R"], seed=cfg.get("seed", 1001),
                                zipf=cfg.get("zipf", 0.0))
    h = create(cpd, cfg["dims"], idx, vals, init, method, cfg["R"], cfg["J"], seed=3001,
               leaf_rows=cfg.get("F", 0))
    return h, idx, vals, init, cfg


def test_create_normalises_and_grams(cpd):
    h, idx, vals, init, cfg = _small(cpd)
    fs = gpu_factors(cpd, h)
    for k in range(3):
        ref = oc.renormalize(init[k].astype(np.float64))
        assert rel_frob(fs[k], ref) < 1e-6
        G = cpd.cpd_get_gram(h, k).cpu().numpy()
        assert rel_frob(G, oc.gram(fs[k])) < 1e-13
    h.close()


@pytest.mark.parametrize("R,dims", [(8, (200, 150, 100)), (40, (400, 300, 250)), (100, (600, 500, 450))])
def test_arls_sampler_state_matches_oracle(cpd, R, dims):
    """Leverage scores and running sums (Algorithm 2) at R = 8 (one thread a
    row), 40 (two) and 100 (four threads sharing a row)."""
    h, idx, vals, init, cfg = _small(cpd, R=R, dims=dims)
    fs = gpu_factors(cpd, h)
    for k in range(3):
        # the Gram behind the scores: df64 kernels (register-blocked for R > 64)
        assert rel_frob(cpd.cpd_get_gram(h, k).cpu().numpy(), oc.gram(fs[k])) < 1e-13
        st = oc.arls_build(fs[k])
        ell, cdf = cpd.cpd_get_arls_state(h, k)
        assert np.max(np.abs(ell.cpu().numpy() - st["ell"]) / st["ell"].max()) < 1e-12
        assert np.max(np.abs(cdf.cpu().numpy() - st["cdf"])) < 1e-12 * st["C"]
        assert abs(st["C"] - cfg["R"]) < 1e-9           # leverage scores sum to R (Eq. 8)
    h.close()


def _tie_mismatches(gi, oi, near, label):
    """Draws whose indices differ from the oracle's: each must sit at a
    near-tie (a target within the tolerance of a bin boundary, where the two
    sides' rounding may legitimately pick either bin), and they must stay a
    small minority (at most 1 in 1000, or 1).  The counts are printed."""
    mism = np.any(gi != oi, axis=0)
    J = gi.shape[1]
    print("%s: %d draws, %d near ties, %d differing" % (label, J, int(near.sum()), int(mism.sum())))
    assert not np.any(mism & ~near), "index mismatch away from a tie"
    assert int(mism.sum()) <= max(1, J // 1000), "too many draws differ at ties"
    return mism


@pytest.mark.parametrize("mode,sweep", [(0, 0), (1, 3), (2, 7)])
def test_arls_draws_match_oracle_exactly(cpd, mode, sweep):
    h, idx, vals, init, cfg = _small(cpd, J=20000)
    fs = gpu_factors(cpd, h)
    samplers = [oc.arls_build(U) for U in fs]
    gi, gp = cpd.cpd_leverage_sample(h, mode, cfg["J"], sweep)
    oi, op, near = oc.arls_draw(samplers, mode, cfg["J"], 3001, sweep)
    gi = gi.cpu().numpy()
    mism = _tie_mismatches(gi, oi, near, "ARLS mode %d sweep %d" % (mode, sweep))
    assert np.all(gi[mode] == -1)
    ok = ~mism
    assert np.max(np.abs(gp.cpu().numpy()[ok] - op[ok]) / op[ok]) < 1e-12
    h.close()


@pytest.mark.parametrize("dims,mode", [((6007, 5003, 4001), 0), ((6007, 5003, 4001), 2),
                                       ((3001, 2003, 1009, 17, 11), 4)])
def test_arls_draws_with_staged_running_sums(cpd, dims, mode):
    """Factors long enough that the draw kernel stages only every 2nd or
    4th running sum in shared memory (ragged last stride; a 5-mode tensor
    takes the 8-mode kernel): every draw equals the oracle's inverse-CDF draw
    (ties excepted), across 40 blocks of draws."""
    R, J = 8, 20000
    idx, vals, init = make_case(dims, 30000, R, seed=41)
    h = create(cpd, dims, idx, vals, init, "arls", R, J, seed=77)
    fs = gpu_factors(cpd, h)
    samplers = [oc.arls_build(U) for U in fs]
    gi, gp = cpd.cpd_leverage_sample(h, mode, J, 5)
    oi, op, near = oc.arls_draw(samplers, mode, J, 77, 5)
    gi = gi.cpu().numpy()
    mism = _tie_mismatches(gi, oi, near, "ARLS %s mode %d" % (dims, mode))
    ok = ~mism
    assert np.max(np.abs(gp.cpu().numpy()[ok] - op[ok]) / op[ok]) < 1e-12
    h.close()


def _oracle_samples(fs, mode, J, seed, sweep):
    samplers = [oc.arls_build(U) for U in fs]
    oi, op, _ = oc.arls_draw(samplers, mode, J, seed, sweep)
    return oi, op


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_sampled_mttkrp_matches_oracle(cpd, mode):
    h, idx, vals, init, cfg = _small(cpd, J=5000)
    fs = gpu_factors(cpd, h)
    oi, op = _oracle_samples(fs, mode, cfg["J"], 11, 0)
    w = 1.0 / (cfg["J"] * op)
    Y, nsel = cpd.cpd_sampled_mttkrp(h, mode, torch.from_numpy(oi), torch.from_numpy(w))
    ref = oc.sampled_mttkrp(idx, vals, cfg["dims"], fs, mode, oi, w)
    assert rel_frob(Y.cpu().numpy(), ref) <= 1e-5
    assert nsel == oc.selected_nnz(idx, cfg["dims"], mode, oi)
    h.close()


@pytest.mark.parametrize("R,bps", [(8, 0), (16, 0), (64, 2), (128, 1), (128, 8)])
def test_sampled_mttkrp_hot_rows(cpd, R, bps):
    """Zipf rows with thousands of nonzeros: rows that the layout marks hot
    are accumulated in shared memory (and, past the slots a launch holds --
    164 hot rows against 105 slots at R = 128 with 8 blocks per SM -- through
    the global path); the result equals the oracle's for every mode, before
    and after the autotuner changes the launch shape.  R = 16, 64 and 128 run
    the kernels compiled for row strides 16, 64 and 128; R = 8 the generic one."""
    dims, nnz, J = (3000, 400, 300), 300_000, 4000
    idx, vals, init = make_case(dims, nnz, R, seed=77, zipf=1.1)
    assert np.bincount(idx[0]).max() > 2000
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=J, seed=8,
                       spmm_blocks_per_sm=bps)
    fs = gpu_factors(cpd, h)
    for tuned in (False, True):
        if tuned:
            cpd.cpd_autotune(h)
        for mode in range(3):
            oi, op = _oracle_samples(fs, mode, J, 13, 0)
            w = 1.0 / (J * op)
            Y, nsel = cpd.cpd_sampled_mttkrp(h, mode, torch.from_numpy(oi), torch.from_numpy(w))
            ref = oc.sampled_mttkrp(idx, vals, dims, fs, mode, oi, w)
            assert rel_frob(Y.cpu().numpy(), ref) <= 1e-5
            assert nsel == oc.selected_nnz(idx, dims, mode, oi)
    h.close()


@pytest.mark.parametrize("R,dims,bps", [(100, (300_000, 400, 300), 0), (128, (250_000, 40, 30), 8)])
def test_row_sorted_sampled_mttkrp_matches_oracle(cpd, R, dims, bps):
    """With R > 64, a mode whose output Y (I_0 x Rp floats, 120-128 MB)
    exceeds 96 MB takes the row-sorted SpMM: selected nonzeros counting-sorted
    by output row, each row summed in registers and stored once, or reduced
    once per 32-position chunk into stored zeros where it crosses a chunk
    boundary (the Zipf-hot rows).  The second case (1,200 KRP rows, so nearly
    every nonzero is selected; rows of up to ~1,200 nonzeros; 8 blocks per SM)
    runs the kernel compiled for Rp = 128.  Equal to the oracle within 1e-5
    for that mode and the unsorted ones, with the sorted lists holding all
    selected nonzeros and capped at 1024 (the rest through the flat-list
    SpMM afterwards)."""
    nnz, J = 400_000, 6000
    idx, vals, init = make_case(dims, nnz, R, seed=79, zipf=1.05)
    fs = None
    for cap in (0, 1000):
        h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                           [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=J, seed=8,
                           nnz_sel_capacity=cap, spmm_blocks_per_sm=bps)
        if fs is None:
            fs = gpu_factors(cpd, h)
        for mode in range(3):
            oi, op = _oracle_samples(fs, mode, J, 17, 0)
            w = 1.0 / (J * op)
            Y, nsel = cpd.cpd_sampled_mttkrp(h, mode, torch.from_numpy(oi), torch.from_numpy(w))
            ref = oc.sampled_mttkrp(idx, vals, dims, fs, mode, oi, w)
            assert rel_frob(Y.cpu().numpy(), ref) <= 1e-5, (cap, mode)
            assert nsel == oc.selected_nnz(idx, dims, mode, oi)
            if mode == 0:
                assert nsel > 1024
                # rows both inside one 32-position chunk and across chunks
                skeys = np.unique(oc.krp_key(oi, dims, 0))
                per_row = np.bincount(idx[0][np.isin(oc.krp_key(idx, dims, 0), skeys)], minlength=dims[0])
                assert np.count_nonzero(per_row > 32) > 10 and np.count_nonzero(per_row == 1) > 1000
        h.close()


def test_sampled_mttkrp_edge_cases(cpd):
    h, idx, vals, init, cfg = _small(cpd)
    fs = gpu_factors(cpd, h)
    dims = cfg["dims"]
    # J = 0: Y = 0
    Y, nsel = cpd.cpd_sampled_mttkrp(h, 0, torch.zeros((3, 0), dtype=torch.int32), torch.zeros(0, dtype=torch.float64))
    assert nsel == 0 and float(Y.abs().max()) == 0.0
    # one draw repeated, and a column with no nonzeros
    e0 = idx[:, 0]
    sidx = np.array([[-1, -1, -1, -1], [e0[1]] * 3 + [0], [e0[2]] * 3 + [0]], dtype=np.int64)
    keys = oc.krp_key(idx, dims, 0)
    empty_key = oc.krp_key(np.array([[0], [0], [0]]), dims, 0)[0]
    w = np.array([0.5, 0.25, 2.0, 1.0])
    Y, nsel = cpd.cpd_sampled_mttkrp(h, 0, torch.from_numpy(sidx), torch.from_numpy(w))
    ref = oc.sampled_mttkrp(idx, vals, dims, fs, 0, sidx, w)
    assert rel_frob(Y.cpu().numpy(), ref) <= 1e-5
    assert nsel == oc.selected_nnz(idx, dims, 0, sidx)
    assert nsel == np.count_nonzero(keys == keys[0]) + np.count_nonzero(keys == empty_key)
    h.close()


def test_exact_mttkrp_matches_oracle(cpd):
    h, idx, vals, init, cfg = _small(cpd, method="exact")
    fs = gpu_factors(cpd, h)
    for mode in range(3):
        Y = cpd.cpd_exact_mttkrp(h, mode)
        assert rel_frob(Y.cpu().numpy(), oc.exact_mttkrp(idx, vals, cfg["dims"], fs, mode)) <= 1e-5
    h.close()


def test_gram_solve_matches_oracle(cpd):
    h, idx, vals, init, cfg = _small(cpd)
    fs = gpu_factors(cpd, h)
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((cfg["dims"][1], cfg["R"])).astype(np.float32)
    sigma = cpd.cpd_gram_solve(h, 1, torch.from_numpy(Y)).cpu().numpy()
    G = oc.hadamard_of_grams([oc.gram(U) for U in fs], 1)
    U_ref, s_ref = oc.solve_and_renorm(Y.astype(np.float64), oc.pinv_sym(G))
    U_g = cpd.cpd_get_factors(h, 1).double().cpu().numpy()
    assert rel_frob(sigma, s_ref) < 1e-5
    assert rel_frob(U_g, U_ref) < 1e-5
    G1 = cpd.cpd_get_gram(h, 1).cpu().numpy()
    assert rel_frob(G1, oc.gram(U_g)) < 1e-13
    # the ARLS sampler of mode 1 was rebuilt from the new factor
    ell, _ = cpd.cpd_get_arls_state(h, 1)
    assert np.max(np.abs(ell.cpu().numpy() - oc.arls_build(U_g)["ell"])) < 1e-12 * cfg["R"]
    h.close()


def test_fit_matches_oracle(cpd):
    h, idx, vals, init, cfg = _small(cpd)
    cpd.cpd_als_sweep(h, 2)
    f = cpd.cpd_fit(h)
    fs = gpu_factors(cpd, h)
    sigma = cpd.cpd_get_sigma(h).cpu().numpy()
    assert abs(f - oc.fit(idx, vals, fs, sigma)) < 1e-9
    h.close()


def test_stepwise_sweep_matches_oracle(cpd):
    """Teacher-forced: each mode update starts from the GPU's factors."""
    h, idx, vals, init, cfg = _small(cpd)
    J = cfg["J"]
    for s in range(2):
        for n in range(3):
            fs = gpu_factors(cpd, h)
            samplers = [oc.arls_build(U) for U in fs]
            oi, op, near = oc.arls_draw(samplers, n, J, 3001, s)
            gi, gp = cpd.cpd_leverage_sample(h, n, J, s)
            gi = gi.cpu().numpy()
            _tie_mismatches(gi, oi, near, "stepwise sweep %d mode %d" % (s, n))
            w = 1.0 / (J * gp.cpu().numpy())
            Y, _ = cpd.cpd_sampled_mttkrp(h, n, torch.from_numpy(gi), torch.from_numpy(w))
            Yo = oc.sampled_mttkrp(idx, vals, cfg["dims"], fs, n, gi, w)
            assert rel_frob(Y.cpu().numpy(), Yo) <= 1e-5
            cpd.cpd_gram_solve(h, n, Y)
            Uo, _ = oc.solve_and_renorm(Y.double().cpu().numpy(),
                                        oc.pinv_sym(oc.hadamard_of_grams([oc.gram(U) for U in fs], n)))
            assert rel_frob(cpd.cpd_get_factors(h, n).double().cpu().numpy(), Uo) < 1e-5
    h.close()


def test_graph_sweep_equals_stepwise(cpd):
    """cpd_als_sweep (captured graph) performs the same updates as the
    step-wise entry points with sweep counter 0, 1, ..."""
    h1, idx, vals, init, cfg = _small(cpd)
    h2, *_ = _small(cpd)
    J = cfg["J"]
    cpd.cpd_als_sweep(h1, 2)
    for s in range(2):
        for n in range(3):
            gi, gp = cpd.cpd_leverage_sample(h2, n, J, s)
            w = 1.0 / (J * gp)
            Y, _ = cpd.cpd_sampled_mttkrp(h2, n, gi, w)
            cpd.cpd_gram_solve(h2, n, Y)
    for k in range(3):
        assert rel_frob(cpd.cpd_get_factors(h1, k).cpu().numpy(), cpd.cpd_get_factors(h2, k).cpu().numpy()) < 1e-4
    h1.close()
    h2.close()


def test_end_to_end_fit_small_uniform(cpd):
    """200x150x100, 20k uniform nonzeros, R = 8, J = 2000, 5 sweeps of
    CP-ARLS-LEV: final fit within 1e-3 of the oracle's own run."""
    h, idx, vals, init, cfg = _small(cpd)
    cpd.cpd_als_sweep(h, 5)
    f_gpu = cpd.cpd_fit(h)
    _, fits = oc.als(idx, vals, cfg["dims"], [u.astype(np.float64) for u in init], "arls", 5, J=cfg["J"], seed=3001)
    assert abs(f_gpu - fits[-1]) < 1e-3
    h.close()


def test_host_input_matches_device_input(cpd):
    cfgd = SMALL
    idx, vals, init = make_case(cfgd["dims"], cfgd["nnz"], cfgd["R"], seed=1001)
    h1 = create(cpd, cfgd["dims"], idx, vals, init, "arls", cfgd["R"], cfgd["J"], seed=3001)
    h2 = create(cpd, cfgd["dims"], idx, vals, init, "arls", cfgd["R"], cfgd["J"], seed=3001, on_host=True)
    for k in range(3):
        assert torch.equal(cpd.cpd_get_factors(h1, k), cpd.cpd_get_factors(h2, k))
    h1.close()
    h2.close()


def test_rank_deficient_gram_uses_pseudo_inverse(cpd):
    """R > I_0 makes G_0 singular: the Jacobi pseudo-inverse path must give
    the oracle's leverage scores (they sum to rank = I_0)."""
    dims = (5, 60, 40)
    idx, vals, init = make_case(dims, 3000, 8, seed=77)
    h = create(cpd, dims, idx, vals, init, "arls", 8, 500, seed=5)
    fs = gpu_factors(cpd, h)
    st = oc.arls_build(fs[0])
    ell, cdf = cpd.cpd_get_arls_state(h, 0)
    assert abs(st["C"] - 5.0) < 1e-9
    assert np.max(np.abs(ell.cpu().numpy() - st["ell"])) < 1e-9
    h.close()


def test_odd_rank_and_ragged_tiles(cpd):
    """R = 25 (not a multiple of 4: padded row stride 28) and modes that are
    not tile multiples (the solve's 64-row tiles end ragged at 97 and 1031
    rows)."""
    dims = (333, 97, 1031)
    idx, vals, init = make_case(dims, 30000, 25, seed=90)
    h = create(cpd, dims, idx, vals, init, "arls", 25, 3000, seed=9)
    fs = gpu_factors(cpd, h)
    for k in range(3):
        assert rel_frob(cpd.cpd_get_gram(h, k).cpu().numpy(), oc.gram(fs[k])) < 1e-13
    rng = np.random.default_rng(25)
    for mode in (1, 2):
        Ys = rng.standard_normal((dims[mode], 25)).astype(np.float32)
        sigma = cpd.cpd_gram_solve(h, mode, torch.from_numpy(Ys)).cpu().numpy()
        G = oc.hadamard_of_grams([oc.gram(U) for U in fs], mode)
        U_ref, s_ref = oc.solve_and_renorm(Ys.astype(np.float64), oc.pinv_sym(G))
        assert rel_frob(sigma, s_ref) < 1e-5
        assert rel_frob(cpd.cpd_get_factors(h, mode).double().cpu().numpy(), U_ref) < 1e-5
        fs[mode] = cpd.cpd_get_factors(h, mode).double().cpu().numpy()
    oi, op = _oracle_samples(fs, 2, 3000, 9, 0)
    gi, gp = cpd.cpd_leverage_sample(h, 2, 3000, 0)
    w = 1.0 / (3000 * op)
    Y, _ = cpd.cpd_sampled_mttkrp(h, 2, torch.from_numpy(oi), torch.from_numpy(w))
    assert rel_frob(Y.cpu().numpy(), oc.sampled_mttkrp(idx, vals, dims, fs, 2, oi, w)) <= 1e-5
    cpd.cpd_als_sweep(h, 1)
    fs2 = gpu_factors(cpd, h)
    f = cpd.cpd_fit(h)
    assert abs(f - oc.fit(idx, vals, fs2, cpd.cpd_get_sigma(h).cpu().numpy())) < 1e-9
    h.close()


def test_invalid_inputs_are_reported(cpd):
    dims = (10, 10, 10)
    idx, vals, init = make_case(dims, 100, 4, seed=3)
    bad = idx.copy()
    bad[1, 5] = 10                     # out of range
    with pytest.raises(cpd.CpdError) as e:
        create(cpd, dims, bad, vals, init, "arls", 4, 10, seed=1)
    assert e.value.status == 2
    dup = idx.copy()
    dup[:, 7] = dup[:, 3]              # duplicate coordinate
    with pytest.raises(cpd.CpdError) as e:
        create(cpd, dims, dup, vals, init, "arls", 4, 10, seed=1)
    assert e.value.status == 3
    h = create(cpd, dims, idx, vals, init, "arls", 4, 10, seed=1)
    sidx = np.zeros((3, 4), dtype=np.int64)
    sidx[2, 1] = 99                    # out-of-range draw: latched, reported
    with pytest.raises(cpd.CpdError) as e:
        cpd.cpd_sampled_mttkrp(h, 0, torch.from_numpy(sidx), torch.ones(4, dtype=torch.float64))
    assert e.value.status == 2
    # the handle stays usable afterwards
    Y, _ = cpd.cpd_sampled_mttkrp(h, 0, torch.zeros((3, 4), dtype=torch.int32), torch.ones(4, dtype=torch.float64))
    h.close()


def test_sketched_gram_solve_matches_oracle(cpd):
    """options.sketched_gram = 1: U_n = Y G~^+ with G~ the Gram of the draws
    (Fig. 3, bottom), step by step against the oracle."""
    dims, R, J = SMALL["dims"], SMALL["R"], SMALL["J"]
    idx, vals, init = make_case(dims, SMALL["nnz"], R, seed=1001)
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=J, seed=3001,
                       sketched_gram=True)
    for n in range(3):
        fs = gpu_factors(cpd, h)
        gi, gp = cpd.cpd_leverage_sample(h, n, J, 0)
        w = 1.0 / (J * gp)
        Y, _ = cpd.cpd_sampled_mttkrp(h, n, gi, w)
        cpd.cpd_gram_solve(h, n, Y)
        Gsk = oc.sketched_gram(fs, n, gi.cpu().numpy(), w.cpu().numpy())
        Uo, _ = oc.solve_and_renorm(Y.double().cpu().numpy(), oc.pinv_sym(Gsk))
        assert rel_frob(cpd.cpd_get_factors(h, n).double().cpu().numpy(), Uo) < 1e-5
    h.close()


def test_sketched_gram_end_to_end_fit(cpd):
    dims, R, J = SMALL["dims"], SMALL["R"], SMALL["J"]
    idx, vals, init = make_case(dims, SMALL["nnz"], R, seed=1001)
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=J, seed=3001,
                       sketched_gram=True)
    cpd.cpd_als_sweep(h, 5)
    f_gpu = cpd.cpd_fit(h)
    _, fits = oc.als(idx, vals, dims, [u.astype(np.float64) for u in init], "arls", 5, J=J, seed=3001,
                     sketched=True)
    assert abs(f_gpu - fits[-1]) < 1e-3
    h.close()


def test_fast_precision_fit_and_draws(cpd):
    """options.precision = 1 (float32 Grams, leverage scores, one Newton step
    for G^+): draws may leave the float64 law's bins only near boundaries
    (under 1% of the draws here), and the 5-round fit stays within 1e-3 of
    the oracle's."""
    dims, R, J = SMALL["dims"], SMALL["R"], SMALL["J"]
    idx, vals, init = make_case(dims, SMALL["nnz"], R, seed=1001)
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=J, seed=3001,
                       fast=True)
    fs = gpu_factors(cpd, h)
    samplers = [oc.arls_build(U) for U in fs]
    gi, _ = cpd.cpd_leverage_sample(h, 1, J, 0)
    oi, _, _ = oc.arls_draw(samplers, 1, J, 3001, 0)
    assert np.mean(np.any(gi.cpu().numpy() != oi, axis=0)) < 0.01
    cpd.cpd_als_sweep(h, 5)
    f_gpu = cpd.cpd_fit(h)
    _, fits = oc.als(idx, vals, dims, [u.astype(np.float64) for u in init], "arls", 5, J=J, seed=3001)
    assert abs(f_gpu - fits[-1]) < 1e-3
    h.close()


@pytest.mark.parametrize("R,I", [(8, 130), (32, 1000), (20, 777), (64, 5003), (100, 300)])
def test_fast_precision_gram_tensor_cores(cpd, R, I):
    """precision = 1 forms factor Grams on the tensor cores (bfloat16 x 3
    exact split, float32 accumulation; R > 64 keeps the float32 FMA loop):
    each G_k equals U_k^T U_k of the stored normalised factor to float32
    accumulation accuracy, and the columns have unit norm."""
    dims = (I, 90, 70)
    idx, vals, init = make_case(dims, 4000, R, seed=300 + R)
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=500, seed=5,
                       fast=True)
    for k in range(3):
        U = cpd.cpd_get_factors(h, k).double().cpu().numpy()
        G = cpd.cpd_get_gram(h, k).cpu().numpy()
        ref = U.T @ U
        assert np.abs(np.linalg.norm(U, axis=0) - 1.0).max() < 1e-5
        assert np.abs(G - ref).max() <= 2e-6 * np.abs(np.diag(ref)).max()
    h.close()


@pytest.mark.parametrize("method", ["arls", "sts"])
def test_zero_factor_draws_weight_zero(cpd, method):
    """A factor set to zero has no sampling distribution: draws through it
    carry probability 0 and weight 0, the downsampled MTTKRP is exactly zero
    (no NaN), and the draw stays an O(log I) search (large I, large J)."""
    dims, R, J = (200_000, 300, 250), 8, 65536
    idx, vals, init = make_case(dims, 20000, R, seed=21)
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method=method, rank=R, samples=J, seed=9)
    cpd.cpd_set_factors(h, 0, torch.zeros((dims[0], R), device="cuda"))
    for n in (1, 2):
        gi, gp = cpd.cpd_leverage_sample(h, n, J, 0)
        p = gp.cpu().numpy()
        assert not np.any(p > 0)
        gi = gi.cpu().numpy()
        for k in range(3):
            if k != n:
                assert gi[k].min() >= 0 and gi[k].max() < dims[k]
        w = torch.zeros(J, dtype=torch.float64, device="cuda")
        Y, _ = cpd.cpd_sampled_mttkrp(h, n, torch.from_numpy(gi).cuda(), w)
        assert torch.all(Y == 0)
    cpd.cpd_als_sweep(h, 1)
    for k in range(3):
        assert torch.isfinite(cpd.cpd_get_factors(h, k)).all()
    h.close()


def test_full_index_beyond_64_bits(cpd):
    """dims 5e6 x 4e6 x 1e6 (2e19 cells, more than 2^64): column keys still fit
    in 64 bits, the duplicate check takes the two-sort ordering; MTTKRPs equal
    the oracle's and a repeated coordinate is still rejected."""
    dims, R, J = (5_000_000, 4_000_000, 1_000_000), 4, 3000
    rng = np.random.default_rng(5)
    idx = np.stack([rng.integers(0, d, 20000) for d in dims]).astype(np.int32)
    vals = rng.random(20000, dtype=np.float32)
    init = [rng.standard_normal((d, R), dtype=np.float32) for d in dims]
    h = create(cpd, dims, idx, vals, init, "arls", R, J, seed=2)
    fs = gpu_factors(cpd, h)
    Y = cpd.cpd_exact_mttkrp(h, 0)
    assert rel_frob(Y.cpu().numpy(), oc.exact_mttkrp(idx, vals, dims, fs, 0)) <= 1e-5
    sidx = np.stack([idx[0, :J], idx[1, :J], np.full(J, -1)]).astype(np.int64)
    w = rng.random(J) + 0.5
    Y, nsel = cpd.cpd_sampled_mttkrp(h, 2, torch.from_numpy(sidx), torch.from_numpy(w))
    assert rel_frob(Y.cpu().numpy(), oc.sampled_mttkrp(idx, vals, dims, fs, 2, sidx, w)) <= 1e-5
    assert nsel == oc.selected_nnz(idx, dims, 2, sidx)
    h.close()
    dup = idx.copy()
    dup[:, 11] = dup[:, 4]
    with pytest.raises(cpd.CpdError) as e:
        create(cpd, dims, dup, vals, init, "arls", R, J, seed=2)
    assert e.value.status == 3


def test_duplicate_coordinates_summed_on_request(cpd):
    """duplicate_policy = 1: repeated coordinates become one nonzero holding
    the sum of their values (both in the 64-bit full-index ordering and in
    the two-sort ordering of a tensor with more than 2^64 cells)."""
    for dims in [(30, 20, 10), (5_000_000, 4_000_000, 1_000_000)]:
        rng = np.random.default_rng(8)
        base = np.stack([rng.integers(0, d, 3000) for d in dims]).astype(np.int32)
        rep = base[:, rng.integers(0, 3000, 1500)]
        idx = np.concatenate([base, rep], axis=1)
        vals = rng.random(idx.shape[1], dtype=np.float32)
        R, J = 4, 200
        init = [rng.standard_normal((d, R), dtype=np.float32) for d in dims]
        h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                           [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=J, seed=1,
                           sum_duplicates=True)
        keys = [np.asarray(x, dtype=np.int64) for x in idx]
        order = np.lexsort(keys[::-1])
        srt = idx[:, order]
        newrun = np.ones(srt.shape[1], dtype=bool)
        newrun[1:] = np.any(srt[:, 1:] != srt[:, :-1], axis=0)
        rid = np.cumsum(newrun) - 1
        uidx = srt[:, newrun]
        uvals = np.zeros(uidx.shape[1])
        np.add.at(uvals, rid, vals[order].astype(np.float64))
        fs = gpu_factors(cpd, h)
        for mode in range(3):
            Y = cpd.cpd_exact_mttkrp(h, mode)
            assert rel_frob(Y.cpu().numpy(), oc.exact_mttkrp(uidx, uvals, dims, fs, mode)) <= 1e-5
        f = cpd.cpd_fit(h)
        fo = oc.fit(uidx, uvals, fs, cpd.cpd_get_sigma(h).cpu().numpy())
        assert abs(f - fo) < 1e-9
        h.close()


def test_library_drawn_initial_factors_match_oracle_generator(cpd):
    """init_factors = NULL: the library draws U_k ~ N(0, 1) from the seed
    (Box-Muller on Philox4x64-10, key (seed, 2)); after Algorithm 1's initial
    column normalisation they equal the oracle's draws from the same
    definition (float64 there, float32 on the GPU) within 1e-6, and the
    handle then runs as if the caller had passed those factors."""
    from oracle import philox as ph
    dims, R, J, seed = (230, 170, 90), 8, 1500, 4242
    idx, vals, _ = make_case(dims, 15000, R, seed=55)
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(), None, method="arls",
                       rank=R, samples=J, seed=seed)
    init = ph.gaussian_factors(dims, R, seed)
    for k in range(3):
        got = cpd.cpd_get_factors(h, k).double().cpu().numpy()
        ref = oc.renormalize(init[k].astype(np.float64))
        assert np.max(np.abs(got - ref)) < 1e-6, k
    h2 = create(cpd, dims, idx, vals, init, "arls", R, J, seed=seed)
    cpd.cpd_als_sweep(h, 2)
    cpd.cpd_als_sweep(h2, 2)
    assert abs(cpd.cpd_fit(h) - cpd.cpd_fit(h2)) < 1e-6
    h.close()
    h2.close()


def test_non_finite_gram_reports_singular_gram(cpd):
    """A NaN that reaches a Gram leaves Eq. 4 without a pseudo-inverse: the
    eigensolver does not converge and CPD_ERR_SINGULAR_GRAM is latched and
    returned by the next synchronising call."""
    h, idx, vals, init, cfg = _small(cpd)
    Y = torch.ones((cfg["dims"][1], cfg["R"]), dtype=torch.float32, device="cuda")
    Y[3, 2] = float("nan")
    with pytest.raises(cpd.CpdError) as ei:
        cpd.cpd_gram_solve(h, 1, Y)
    assert ei.value.status == 7
    h.close()



@pytest.mark.parametrize("R", [40, 64, 99, 100, 128])
def test_tiled_solve_large_rank_matches_oracle(cpd, R):
    """Solve and renormalisation (Algorithm 1's mode update) at 32 < R <= 128 (the
    register-tiled kernel: 128-row tiles, ragged at 150 and 1031 rows, R not a
    multiple of 4 for R = 99) against the oracle's Y G^+ and column norms."""
    dims = (333, 150, 1031)
    idx, vals, init = make_case(dims, 20000, R, seed=91)
    h = create(cpd, dims, idx, vals, init, "arls", R, 1000, seed=9)
    fs = gpu_factors(cpd, h)
    rng = np.random.default_rng(R)
    for mode in (1, 2):
        Ys = rng.standard_normal((dims[mode], R)).astype(np.float32)
        sigma = cpd.cpd_gram_solve(h, mode, torch.from_numpy(Ys)).cpu().numpy()
        G = oc.hadamard_of_grams([oc.gram(U) for U in fs], mode)
        U_ref, s_ref = oc.solve_and_renorm(Ys.astype(np.float64), oc.pinv_sym(G))
        assert rel_frob(sigma, s_ref) < 1e-5, mode
        assert rel_frob(cpd.cpd_get_factors(h, mode).double().cpu().numpy(), U_ref) < 1e-5, mode
        fs[mode] = cpd.cpd_get_factors(h, mode).double().cpu().numpy()
    h.close()


@pytest.mark.parametrize("method", ["arls", "sts"])
def test_deterministic_runs_are_bitwise_equal(cpd, method):
    """options.deterministic: no floating-point atomics in the downsampled
    MTTKRP, so two runs from the same inputs give bit-identical factors, sigma
    and fit; the run stays within the method's tolerance of the oracle."""
    dims, R, J = (300, 200, 150), 16, 3000
    idx, vals, init = make_case(dims, 40000, R, seed=71, zipf=1.1)
    runs = []
    for _ in range(2):
        h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                           [torch.from_numpy(u).cuda() for u in init], method=method, rank=R, samples=J, seed=5,
                           deterministic=True)
        cpd.cpd_als_sweep(h, 3)
        runs.append(([cpd.cpd_get_factors(h, k).cpu() for k in range(3)], cpd.cpd_get_sigma(h).cpu(), cpd.cpd_fit(h)))
        h.close()
    (f1, s1, fit1), (f2, s2, fit2) = runs
    assert all(torch.equal(a, b) for a, b in zip(f1, f2))
    assert torch.equal(s1, s2) and fit1 == fit2
    _, fits = oc.als(idx, vals, dims, [u.astype(np.float64) for u in init], method, 3, J=J, seed=5)
    assert abs(fit1 - fits[-1]) < 1e-3


def test_deterministic_sampled_mttkrp_matches_oracle(cpd):
    """The deterministic path of Eq. 7 with caller draws: repeated KRP rows
    with unequal weights (their weights add), draws that miss every nonzero,
    and a hot-row (Zipf) tensor; equal to the oracle within 1e-5 and to the
    atomics path's count of selected nonzeros; repeated calls bitwise equal."""
    dims, R, J = (400, 300, 200), 12, 5000
    idx, vals, init = make_case(dims, 60000, R, seed=73, zipf=1.2)
    hd = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                        [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=J, seed=5,
                        deterministic=True)
    ha = create(cpd, dims, idx, vals, init, "arls", R, J, seed=5)
    fs = gpu_factors(cpd, hd)
    rng = np.random.default_rng(74)
    for mode in range(3):
        gi, gp = cpd.cpd_leverage_sample(ha, mode, J, 1)
        si = gi.cpu().numpy().copy()
        si[:, 100:200] = si[:, 0:100]               # repeated draws
        w = rng.uniform(0.1, 3.0, J)                # with unequal weights
        Yd, nd = cpd.cpd_sampled_mttkrp(hd, mode, torch.from_numpy(si), torch.from_numpy(w))
        Yd2, _ = cpd.cpd_sampled_mttkrp(hd, mode, torch.from_numpy(si), torch.from_numpy(w))
        Ya, na = cpd.cpd_sampled_mttkrp(ha, mode, torch.from_numpy(si), torch.from_numpy(w))
        Yo = oc.sampled_mttkrp(idx, vals, dims, fs, mode, si, w)
        assert rel_frob(Yd.cpu().numpy(), Yo) <= 1e-5, mode
        assert torch.equal(Yd, Yd2)
        assert nd == na == oc.selected_nnz(idx, dims, mode, si)
    hd.close()
    ha.close()


def test_deterministic_capacity_overflow_is_reported(cpd):
    """nnz_sel_capacity below the selected nonzeros of a call latches
    CPD_ERR_CAPACITY; the exact method has no deterministic mode."""
    dims, R, J = (100, 80, 60), 8, 2000
    idx, vals, init = make_case(dims, 20000, R, seed=75)
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=J, seed=5,
                       deterministic=True, nnz_sel_capacity=500)
    gi, gp = cpd.cpd_leverage_sample(h, 0, J, 0)
    with pytest.raises(cpd.CpdError) as ei:
        cpd.cpd_sampled_mttkrp(h, 0, gi, 1.0 / (J * gp))
    assert ei.value.status == 6
    h.close()
    with pytest.raises(cpd.CpdError) as ei:
        cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method="exact", rank=R, samples=J, seed=5,
                       deterministic=True)
    assert ei.value.status == 1


def test_tensor_core_gram_wait_runs_out_cleanly(cpd):
    """The tensor-core Gram's bounded mbarrier waits (precision option 1): with
    a short limit and no MMA issued, every wait runs out, the kernel latches
    CPD_ERR_TIMEOUT and frees its tensor memory, and the handle keeps working
    (the next Gram, with MMAs, equals the oracle's)."""
    dims, R = (600, 400, 300), 16
    idx, vals, init = make_case(dims, 20000, R, seed=31)
    h = cpd.cpd_create(dims, torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(),
                       [torch.from_numpy(u).cuda() for u in init], method="arls", rank=R, samples=500, seed=5,
                       fast=True)
    U = cpd.cpd_get_factors(h, 0).clone()
    cpd.cpd_debug_gram_wait(h, 2_000_000, suppress_mma=True)      # ~1 ms at 2 GHz
    with pytest.raises(cpd.CpdError) as ei:
        cpd.cpd_set_factors(h, 0, U)
    assert ei.value.status == 8                                    # CPD_ERR_TIMEOUT
    cpd.cpd_debug_gram_wait(h, 0, suppress_mma=False)
    for _ in range(3):                                             # TMEM was freed: allocations succeed
        cpd.cpd_set_factors(h, 0, U)
    G = cpd.cpd_get_gram(h, 0).cpu().numpy()
    ref = oc.gram(U.double().cpu().numpy())
    assert np.abs(G - ref).max() <= 2e-6 * np.abs(np.diag(ref)).max()
    h.close()
