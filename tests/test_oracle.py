"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a library
routine computing the same quantity by another route (numpy's Philox, SVD
pseudo-inverse, QR), an explicitly materialised Khatri-Rao product or
sampling matrix, a dense brute force, an invariant or a closed form.
"""
import numpy as np
import pytest

from oracle import philox as ph
from oracle import cpals as oc
from paper_2210_05105_gb300 import synth
from tests.helpers import dense_from_coo, matricize, khatri_rao_design, planted_dense


def _numpy_philox_block(ctr, key):
    """First output block of numpy's Philox for counter `ctr` (numpy
    increments its 256-bit counter before generating, so feed ctr - 1)."""
    c = np.array(ctr, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        i = 0
        while True:
            was_zero = c[i] == 0
            c[i] = c[i] - np.uint64(1)
            if not was_zero or i == 3:
                break
            i += 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=c)
    return bg.random_raw(4)


def test_philox_matches_numpy_bitgenerator():
    rng = np.random.default_rng(11)
    ctrs = [[0, 0, 0, 0], [2**64 - 1, 2**64 - 1, 3, 9], [5, 0, 2**63, 1]]
    ctrs += [list(rng.integers(0, 2**64, size=4, dtype=np.uint64)) for _ in range(40)]
    keys = [[0, 0], [2**64 - 1, 2**64 - 1]] + [list(rng.integers(0, 2**64, 2, dtype=np.uint64)) for _ in range(41)]
    for c, k in zip(ctrs, keys):
        got = ph.philox4x64([[c[0]], [c[1]], [c[2]], [c[3]]], [[k[0]], [k[1]]])[:, 0]
        assert (got == _numpy_philox_block(c, k)).all()


def test_uniform_mapping_range_and_resolution():
    w = np.array([0, 2**11 - 1, 2**11, 2**64 - 1], dtype=np.uint64)
    u = ph.uniform01(w)
    assert u[0] == 0.0 and u[1] == 0.0
    assert u[2] == 2.0 ** -53
    assert u[3] == 1.0 - 2.0 ** -53
    us = ph.draw_uniforms(3, ph.STREAM_ARLS, np.arange(200000), 1, 0, 2)
    assert us.min() >= 0.0 and us.max() < 1.0
    assert abs(us.mean() - 0.5) < 5e-3 and abs(us.var() - 1 / 12) < 2e-3


def test_gaussian_factors_follow_the_normal_law():
    """Library-side initial factors (Algorithm 1's initialisation): the Box-Muller
    transform of the Philox uniforms is N(0, 1) -- Kolmogorov-Smirnov against
    the normal CDF of scipy, first four moments, no infinities (u1 > 0) --
    and distinct factors, rows and columns get distinct counters."""
    from scipy import stats
    fs = ph.gaussian_factors((700, 300), 200, seed=5)
    z = np.concatenate([f.ravel() for f in fs]).astype(np.float64)
    assert np.all(np.isfinite(z)) and z.shape[0] == 200000
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.012 and abs(z.var() - 1.0) < 0.012
    assert abs(stats.skew(z)) < 0.03 and abs(stats.kurtosis(z)) < 0.06
    # columns are uncorrelated and the same seed reproduces the same draws
    c = np.corrcoef(fs[0][:, :20].T)
    assert np.max(np.abs(c - np.eye(20))) < 0.2
    again = ph.gaussian_factors((700, 300), 200, seed=5)
    assert all((a == b).all() for a, b in zip(fs, again))
    other = ph.gaussian_factors((700, 300), 200, seed=6)
    assert not np.array_equal(fs[0], other[0])


def test_pinv_against_svd_and_penrose_conditions():
    rng = np.random.default_rng(3)
    for R, rank in [(6, 6), (8, 5), (12, 3)]:
        B = rng.standard_normal((R, rank))
        G = B @ B.T
        P = oc.pinv_sym(G)
        assert np.allclose(P, np.linalg.pinv(G, rcond=1e-12), atol=1e-8 * np.abs(P).max())
        assert np.allclose(G @ P @ G, G, atol=1e-10 * np.abs(G).max())
        assert np.allclose(P @ G @ P, P, atol=1e-10 * np.abs(P).max())
        assert np.allclose((G @ P).T, G @ P, atol=1e-10)


def test_key_order_and_gram_hadamard_identity():
    rng = np.random.default_rng(4)
    dims = (4, 3, 5, 2)
    fs = [rng.standard_normal((d, 3)) for d in dims]
    for n in range(4):
        A = khatri_rao_design(fs, n)
        G = oc.hadamard_of_grams([oc.gram(U) for U in fs], n)
        assert np.allclose(A.T @ A, G)                       # Eq. 5
        other = [k for k in range(4) if k != n]
        grid = np.meshgrid(*[np.arange(dims[k]) for k in other], indexing="ij")
        idx = [np.zeros(grid[0].size, dtype=np.int64)] * 4
        idx = list(idx)
        for g, k in zip(grid, other):
            idx[k] = g.reshape(-1)
        keys = oc.krp_key(idx, dims, n)
        assert np.allclose(A[keys], oc.krp_rows(fs, idx, n))  # row order of Eq. 3


def test_exact_mttkrp_matches_dense_matricization():
    rng = np.random.default_rng(5)
    dims = (7, 5, 6)
    idx = synth.coo_coordinates(dims, 60, 9)
    vals = rng.standard_normal(60)
    fs = [rng.standard_normal((d, 4)) for d in dims]
    T = dense_from_coo(idx, vals, dims)
    for n in range(3):
        ref = matricize(T, n) @ khatri_rao_design(fs, n)     # Eq. 6 brute force
        assert np.allclose(oc.exact_mttkrp(idx, vals, dims, fs, n), ref)


def test_sampled_mttkrp_matches_explicit_sampling_matrix():
    rng = np.random.default_rng(6)
    dims = (6, 5, 4)
    idx = synth.coo_coordinates(dims, 50, 10)
    vals = rng.standard_normal(50)
    fs = [rng.standard_normal((d, 3)) for d in dims]
    T = dense_from_coo(idx, vals, dims)
    for n in range(3):
        J = 17
        sidx = np.stack([rng.integers(0, d, J) for d in dims])
        sidx[n] = -1
        w = rng.random(J) + 0.1
        ncols = int(np.prod([d for k, d in enumerate(dims) if k != n]))
        keys = oc.krp_key(sidx, dims, n)
        S = np.zeros((J, ncols))
        S[np.arange(J), keys] = np.sqrt(w)                   # row j: sqrt(w_j) e_key^T
        ref = matricize(T, n) @ S.T @ S @ khatri_rao_design(fs, n)   # Eq. 7
        got = oc.sampled_mttkrp(idx, vals, dims, fs, n, sidx, w)
        assert np.allclose(got, ref)


def test_selected_nnz_matches_brute_force_count():
    """nnz(mat(T, n) S^T), counted by checking every nonzero against every
    draw with plain loops (no keys): a nonzero is selected when its indices
    outside mode n equal those of some draw; repeated draws count once."""
    rng = np.random.default_rng(12)
    dims = (7, 5, 6, 3)
    idx = synth.coo_coordinates(dims, 120, 13)
    for n in range(4):
        J = 25
        sidx = np.stack([rng.integers(0, d, J) for d in dims])
        sidx[n] = -1
        sidx[:, 3] = sidx[:, 0]                              # a repeated draw
        count = 0
        for e in range(idx.shape[1]):
            for j in range(J):
                if all(idx[k, e] == sidx[k, j] for k in range(4) if k != n):
                    count += 1
                    break
        assert oc.selected_nnz(idx, dims, n, sidx) == count
    assert oc.selected_nnz(idx, dims, 0, np.zeros((4, 0), dtype=np.int64)) == 0


def test_sampled_with_every_row_once_equals_exact():
    rng = np.random.default_rng(7)
    dims = (9, 6, 5)
    idx = synth.coo_coordinates(dims, 120, 12)
    vals = rng.random(120)
    fs = [rng.standard_normal((d, 5)) for d in dims]
    for n in range(3):
        other = [k for k in range(3) if k != n]
        grid = np.meshgrid(*[np.arange(dims[k]) for k in other], indexing="ij")
        sidx = np.full((3, grid[0].size), -1, dtype=np.int64)
        for g, k in zip(grid, other):
            sidx[k] = g.reshape(-1)
        w = np.ones(sidx.shape[1])
        got = oc.sampled_mttkrp(idx, vals, dims, fs, n, sidx, w)
        assert np.allclose(got, oc.exact_mttkrp(idx, vals, dims, fs, n), rtol=1e-12, atol=1e-12)


def test_duplicate_draws_equal_summed_weight():
    rng = np.random.default_rng(8)
    dims = (8, 7, 6)
    idx = synth.coo_coordinates(dims, 150, 13)
    vals = rng.random(150)
    fs = [rng.standard_normal((d, 4)) for d in dims]
    sidx = np.stack([rng.integers(0, d, 5) for d in dims])
    sidx[0] = -1
    dup = np.concatenate([sidx, sidx[:, :2]], axis=1)
    w = np.array([0.5, 1.5, 2.0, 0.25, 1.0, 0.75, 3.0])
    merged_w = w[:5].copy()
    merged_w[:2] += w[5:]
    a = oc.sampled_mttkrp(idx, vals, dims, fs, 0, dup, w)
    b = oc.sampled_mttkrp(idx, vals, dims, fs, 0, sidx, merged_w)
    assert np.allclose(a, b)


def test_leverage_scores_sum_to_rank_and_match_qr():
    rng = np.random.default_rng(9)
    for I, R, rank in [(40, 6, 6), (30, 8, 5)]:
        U = rng.standard_normal((I, rank)) @ rng.standard_normal((rank, R))
        st = oc.arls_build(U)
        assert abs(st["ell"].sum() - rank) < 1e-9                       # Eq. 8 invariant
        Q, Rr = np.linalg.qr(U)
        keep = np.abs(np.diag(Rr)) > 1e-10 * np.abs(np.diag(Rr)).max()
        if keep.all():
            assert np.allclose(st["ell"], np.sum(Q * Q, axis=1), atol=1e-12)
        assert np.allclose(st["cdf"][-1], st["C"])


def test_exact_krp_leverage_matches_qr_of_materialised_krp():
    rng = np.random.default_rng(10)
    dims = (5, 4, 6)
    fs = [rng.standard_normal((d, 3)) for d in dims]
    for n in range(3):
        A = khatri_rao_design(fs, n)
        Q, _ = np.linalg.qr(A)
        assert np.allclose(oc.exact_krp_leverage(fs, n), np.sum(Q * Q, axis=1), atol=1e-12)


def test_inverse_cdf_edges():
    ell = np.array([0.0, 1.0, 0.0, 2.0, 0.0])
    cdf = np.cumsum(ell)
    t = np.array([0.0, 0.999, 1.0, 2.5, 3.0, 7.0])
    got = oc.inverse_cdf(cdf, ell, t)
    assert list(got) == [1, 1, 3, 3, 3, 3]          # zero-weight rows never drawn


def test_inverse_cdf_past_end_is_last_nonzero_width_bin():
    """t rounded up to the total C: the first row whose running sum reaches C.
    A positive weight absorbed by rounding (bin of zero width) is never drawn,
    past the end included; all weights zero gives row 0."""
    ell = np.array([1.0, 1e-20, 0.0])
    cdf = np.cumsum(ell)
    assert cdf[1] == cdf[0] == 1.0
    assert list(oc.inverse_cdf(cdf, ell, np.array([0.5, 1.0]))) == [0, 0]
    z = np.zeros(4)
    assert list(oc.inverse_cdf(z, z, np.array([0.0]))) == [0]


def test_zero_factor_draws_weight_zero_and_zero_update():
    """A factor of zeros (e.g. after a sampled MTTKRP that met no nonzero) has
    no leverage distribution; every KRP row through it is zero, so the exact
    MTTKRP is zero and the draws carry probability 0 and weight 0 (no NaN)."""
    rng = np.random.default_rng(3)
    dims, R, J = (6, 5, 4), 3, 50
    fs = [oc.renormalize(rng.standard_normal((d, R))) for d in dims]
    fs[0] = np.zeros_like(fs[0])
    samplers = [oc.arls_build(U) for U in fs]
    assert samplers[0]["C"] == 0.0
    idx, p, _ = oc.arls_draw(samplers, 1, J, seed=5, sweep=0)
    assert np.all(idx[0] == 0) and np.all(p == 0.0)
    w = oc.sample_weights(p, J)
    assert np.all(w == 0.0)
    coords = np.array(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")).reshape(3, -1)
    vals = rng.random(coords.shape[1])
    Y = oc.sampled_mttkrp(coords, vals, dims, fs, 1, idx, w)
    assert np.all(Y == 0.0)
    assert np.all(oc.exact_mttkrp(coords, vals, dims, fs, 1) == 0.0)
    assert np.all(oc.sample_weights(np.array([0.25, 0.0, np.nan]), 2) == np.array([2.0, 0.0, 0.0]))


def test_arls_draw_law_matches_factor_marginals():
    rng = np.random.default_rng(12)
    dims = (7, 5, 6)
    fs = [oc.renormalize(rng.standard_normal((d, 3))) for d in dims]
    samplers = [oc.arls_build(U) for U in fs]
    n, J = 1, 200000
    sidx, p, near = oc.arls_draw(samplers, n, J, seed=99, sweep=0)
    assert not near.any()
    # exact law: independent factors, P(i_k = i) = ell_k[i] / C_k (Algorithm 3)
    marg = [np.diff(np.concatenate([[0.0], s["cdf"]])) / s["C"] for s in samplers]
    assert np.allclose(p, marg[0][sidx[0]] * marg[2][sidx[2]])
    for k in (0, 2):
        freq = np.bincount(sidx[k], minlength=dims[k]) / J
        assert np.all(np.abs(freq - marg[k]) < 5 * np.sqrt(marg[k] * (1 - marg[k]) / J) + 1e-9)
    # the product law sums to one over all rows of U_{!=n}
    assert abs(np.outer(marg[0], marg[2]).sum() - 1.0) < 1e-12


def _sts_setup(dims, R, seed, F):
    rng = np.random.default_rng(seed)
    fs = [oc.renormalize(rng.standard_normal((d, R))) for d in dims]
    grams = [oc.gram(U) for U in fs]
    trees = [oc.sts_build(U, F) for U in fs]
    return fs, grams, trees


def test_sts_tree_nodes_are_block_gram_sums():
    fs, grams, trees = _sts_setup((13, 9, 7), 3, 20, F=2)
    for U, t in zip(fs, trees):
        L = t["L"]
        assert np.allclose(t["nodes"][1], U.T @ U)
        for l in range(L):
            blk = U[2 * l:2 * l + 2]
            assert np.allclose(t["nodes"][L + l], blk.T @ blk if blk.size else 0.0)


@pytest.mark.parametrize("F", [1, 2, 3])
def test_sts_walk_is_inverse_cdf_of_conditional(F):
    """At every factor the tree walk picks the inverse CDF (in row order) of
    the conditional law q_i ~ (U_k[i] (*) h)^T G_{>k} (U_k[i] (*) h)."""
    dims = (11, 6, 5)
    fs, grams, trees = _sts_setup(dims, 3, 21, F)
    n = 1
    G = oc.hadamard_of_grams(grams, n)
    Gp = oc.pinv_sym(G)
    rng = np.random.default_rng(5)
    h = rng.standard_normal((400, 3))
    u = rng.random(400)
    k = 0
    Ggt = Gp * grams[2]                       # G_{>0} = G^+ (*) G_2 for n = 1
    rows, near = oc._sts_walk(trees[k], fs[k], Ggt, h, u, 1e-9)
    x = fs[k][None, :, :] * h[:, None, :]
    q = np.einsum("jia,ab,jib->ji", x, Ggt, x)
    cq = np.cumsum(q, axis=1)
    ref = np.argmax(cq > (u * cq[:, -1])[:, None], axis=1)
    ok = (rows == ref) | near
    assert ok.all() and (~near).sum() > 350


def test_sts_draw_probability_is_exact_leverage():
    """Product of the conditionals = exact leverage of the KRP row / rank
    (QR of the materialised design matrix), and frequencies follow it."""
    dims = (6, 5, 4)
    R = 3
    fs, grams, trees = _sts_setup(dims, R, 22, F=2)
    for n in range(3):
        A = khatri_rao_design(fs, n)
        Q, _ = np.linalg.qr(A)
        lev = np.sum(Q * Q, axis=1) / R
        J = 60000
        sidx, p, near = oc.sts_draw(trees, fs, grams, n, J, seed=7, sweep=1)
        keys = oc.krp_key(sidx, dims, n)
        assert np.allclose(p, lev[keys], rtol=1e-9)
        freq = np.bincount(keys, minlength=lev.size) / J
        sd = np.sqrt(lev * (1 - lev) / J)
        assert np.all(np.abs(freq - lev) < 5 * sd + 1e-9)


def test_fit_matches_dense_residual():
    rng = np.random.default_rng(14)
    dims = (5, 4, 6)
    idx = synth.coo_coordinates(dims, 40, 3)
    vals = rng.random(40)
    fs = [rng.standard_normal((d, 3)) for d in dims]
    sigma = rng.random(3) + 0.5
    T = dense_from_coo(idx, vals, dims)
    M = np.einsum("r,ir,jr,kr->ijk", sigma, *fs)
    ref = 1 - np.linalg.norm(M - T) / np.linalg.norm(T)
    assert abs(oc.fit(idx, vals, fs, sigma) - ref) < 1e-12


def test_solve_and_renorm_properties():
    rng = np.random.default_rng(15)
    Y = rng.standard_normal((30, 4))
    B = rng.standard_normal((4, 4))
    G = B @ B.T + np.eye(4)
    U, s = oc.solve_and_renorm(Y, oc.pinv_sym(G))
    assert np.allclose(np.linalg.norm(U, axis=0), 1.0)
    assert np.allclose((U * s) @ G, Y)                     # U diag(sigma) G = Y
    Y[:, 2] = 0.0
    U, s = oc.solve_and_renorm(Y, np.eye(4))
    assert s[2] == 0.0 and np.all(U[:, 2] == 0.0)


def test_exact_als_recovers_planted_rank():
    idx, vals, _ = planted_dense((9, 8, 7), 3, 31)
    init = synth.init_factors((9, 8, 7), 3, 42)
    _, fits = oc.als(idx, vals, (9, 8, 7), init, "exact", sweeps=100)
    assert fits[-1] > 0.999


def test_randomized_als_noise_floor_scales_as_inverse_sqrt_J():
    """With the exact G^+ of Eq. 5 the sampled update is an unbiased estimate
    of the exact update (E[S^T S] = I), so on a planted exact-rank tensor the
    residual 1 - fit settles at a floor proportional to J^-1/2; STS-CP, which
    draws from the exact leverage law (beta = 1 in Theorem 2.1), sits below
    CP-ARLS-LEV at equal J."""
    dims = (9, 8, 7)
    idx, vals, _ = planted_dense(dims, 3, 31)
    init = synth.init_factors(dims, 3, 42)
    floor = {}
    for method in ("arls", "sts"):
        for J in (500, 5000):
            _, fits = oc.als(idx, vals, dims, init, method, sweeps=30, J=J, seed=5)
            floor[method, J] = 1.0 - float(np.mean(fits[-10:]))
        ratio = floor[method, 500] / floor[method, 5000]
        assert 2.0 < ratio < 5.0, (method, ratio)           # sqrt(10) = 3.16
    assert floor["sts", 500] < floor["arls", 500]
    assert floor["sts", 5000] < floor["arls", 5000]


def test_sampled_update_is_unbiased():
    """E[S^T S] = I, so the mean sampled MTTKRP over seeds -> exact MTTKRP."""
    rng = np.random.default_rng(16)
    dims = (6, 5, 4)
    idx = synth.coo_coordinates(dims, 70, 17)
    vals = rng.random(70)
    fs = [oc.renormalize(rng.standard_normal((d, 3))) for d in dims]
    samplers = [oc.arls_build(U) for U in fs]
    n, J, trials = 0, 40, 3000
    acc = np.zeros((dims[n], 3))
    acc2 = np.zeros((dims[n], 3))
    for s in range(trials):
        sidx, p, _ = oc.arls_draw(samplers, n, J, seed=1000 + s, sweep=0)
        Y = oc.sampled_mttkrp(idx, vals, dims, fs, n, sidx, oc.sample_weights(p, J))
        acc += Y
        acc2 += Y * Y
    mean = acc / trials
    sd = np.sqrt(np.maximum(acc2 / trials - mean ** 2, 0) / trials)
    exact = oc.exact_mttkrp(idx, vals, dims, fs, n)
    assert np.all(np.abs(mean - exact) <= 5 * sd + 1e-9)


def test_sketched_gram_matches_explicit_sampling_matrix():
    rng = np.random.default_rng(30)
    dims = (5, 4, 6)
    fs = [rng.standard_normal((d, 3)) for d in dims]
    for n in range(3):
        J = 23
        sidx = np.stack([rng.integers(0, d, J) for d in dims])
        sidx[n] = -1
        w = rng.random(J) + 0.2
        A = khatri_rao_design(fs, n)
        ncols = A.shape[0]
        S = np.zeros((J, ncols))
        S[np.arange(J), oc.krp_key(sidx, dims, n)] = np.sqrt(w)
        assert np.allclose(oc.sketched_gram(fs, n, sidx, w), (S @ A).T @ (S @ A))


def test_sketched_gram_als_solves_consistent_problems_exactly():
    """With the downsampled normal equations (Fig. 3, bottom) an exactly
    rank-R tensor is a consistent least-squares problem: every full-rank
    sketch recovers the exact update, so the fit reaches 1 (no J^-1/2 floor,
    unlike the unbiased exact-G^+ update)."""
    dims = (9, 8, 7)
    idx, vals, _ = planted_dense(dims, 3, 31)
    init = synth.init_factors(dims, 3, 42)
    _, fits = oc.als(idx, vals, dims, init, "arls", 60, J=200, seed=5, sketched=True)
    assert fits[-1] > 0.9999


def test_arls_tie_window_follows_gram_conditioning():
    """The conditioning-aware tie window: the leverage scores of a factor
    computed from two float64 Grams that differ by their last-bit rounding
    differ by about cond(G) 2^-53 relative, inside max(1e-12, 8 cond 2^-53),
    and the window reduces to the 1e-12 floor for a well-conditioned factor."""
    rng = np.random.default_rng(12)
    good = rng.standard_normal((4000, 6))
    assert oc.arls_tie_tolerance(oc.arls_build(good)) == 1e-12
    # columns nearly collinear: cond ~ 1e9
    base = rng.standard_normal((4000, 1))
    bad = base + 1e-4 * rng.standard_normal((4000, 6))
    st = oc.arls_build(bad)
    cond = oc.gram_condition(st["G"])
    assert cond > 1e7
    G2 = st["G"] * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=st["G"].shape))
    G2 = 0.5 * (G2 + G2.T)
    ell2 = oc.leverage_scores(bad, oc.pinv_sym(G2))
    drift = np.max(np.abs(np.cumsum(ell2) - st["cdf"])) / st["C"]
    assert drift > 1e-12                               # the fixed floor alone would not cover it
    assert drift <= oc.arls_tie_tolerance(st)
    # a singular Gram: the condition number is taken over the eigenvalues the
    # pseudo-inverse keeps, and the window stays finite (capped)
    sing = np.hstack([good[:, :3], good[:, :1]])
    st2 = oc.arls_build(sing)
    assert np.isfinite(oc.gram_condition(st2["G"]))
    assert oc.arls_tie_tolerance(st2) <= 1e-6
