"""Plain FP64 CPU oracle for randomized sparse CP-ALS (CP-ARLS-LEV and STS-CP).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct statement
of what the GPU path computes.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import it.  It shares no code with the CUDA
library and never calls it; the only things both sides see are the seeded
inputs (COO tensor, initial factors, seeds).

Paper: V. Bharadwaj, O. A. Malik, R. Murray, A. Buluc, J. Demmel,
"Distributed-Memory Randomized Algorithms for Sparse Tensor CP Decomposition",
arXiv 2210.05105.  Citations below name its sections, equations and algorithms.

Conventions
-----------
* A sparse tensor is COO: ``idx`` int array (N, nnz) of 0-based indices and
  ``vals`` (nnz,).  All arithmetic here is binary64.
* Factors U_k are (I_k, R) arrays.  Modes are 0-based.
* KRP row order (Eq. 3): U_{!=n} = U_{N-1} (.) ... (.) U_0 without U_n, so the
  index of the lowest remaining mode varies fastest.  The row ("column of
  mat(T, n)") linear key is  key = sum_{k != n} i_k * prod_{k' < k, k' != n} I_k'.

Readings of points the paper leaves open:
* Moore-Penrose pseudo-inverse (Eq. 4): symmetric eigendecomposition,
  eigenvalues <= R * 2^-52 * lambda_max are treated as zero.
* Sampling weight (Sec. 2.2 leaves the row scale of S unstated): row j of S is
  e_{row_j}^T / sqrt(J p_j), so S^T S carries weight w_j = 1 / (J p_j) on row_j;
  draws are i.i.d. with replacement (Theorem 2.1).
* Inverse-CDF draw (Algorithm 3, per factor): i = smallest index with
  CDF[i] > u * C; if rounding puts u * C at or past CDF[I-1], the first row
  whose running sum reaches C (the last row whose bin has nonzero width).
* A factor whose scores are all zero (C = 0) has no distribution; every KRP
  row through it is zero, so its draws take row 0 with probability 0 and
  weight 0.
* STS-CP (Sec. 4.1, Algorithm 5): factors are drawn in ascending mode order
  (excluding n); G_{>k} = G^+ (*) Grams of the factors drawn after k; the walk
  keeps an absolute target t = u * m(root) and goes left iff t < m(left),
  otherwise subtracts m(left) (the absolute-mass form of the r := (r-T)/(1-T),
  r := r/T rescaling).  Leaves hold F consecutive rows (F = R by default); the
  leaf count is padded to a power of two with empty leaves; a child covering no
  real row is never entered.  At a leaf the target is rescaled by
  (sum of row masses) / m(leaf) and the smallest row with cumulative mass > t
  is taken (last row of nonzero mass if none).
* Zero column norm at renormalisation (Algorithm 1's mode update): sigma_r = 0 and
  the column is left unchanged.
* Fit (Sec. 5.1): ||T - T~||^2 = ||T||^2 - 2 <T, T~> + sigma^T (*_k G_k) sigma,
  the last term exact for the dense model T~.
"""
import numpy as np

from .philox import draw_uniforms, STREAM_ARLS, STREAM_STS


# ---------------------------------------------------------------------------
# Khatri-Rao product rows and keys (Eq. 3, Fig. 3)
# ---------------------------------------------------------------------------

def krp_strides(dims, n):
    """Strides of the key of a row of U_{!=n}: lowest remaining mode fastest."""
    strides = np.zeros(len(dims), dtype=np.int64)
    acc = 1
    for k in range(len(dims)):
        if k == n:
            continue
        strides[k] = acc
        acc *= int(dims[k])
    return strides, acc


def krp_key(idx, dims, n):
    """Linear key of the KRP row selected by the indices idx[k], k != n."""
    strides, _ = krp_strides(dims, n)
    key = np.zeros(np.asarray(idx[0]).shape, dtype=np.int64)
    for k in range(len(dims)):
        if k != n:
            key = key + np.asarray(idx[k], dtype=np.int64) * strides[k]
    return key


def krp_rows(factors, idx, n):
    """Rows h = *_{k != n} U_k[i_k, :] of U_{!=n} for index arrays idx[k]."""
    R = factors[0].shape[1]
    m = np.asarray(idx[0]).shape[0]
    h = np.ones((m, R), dtype=np.float64)
    for k, U in enumerate(factors):
        if k != n:
            h *= np.asarray(U, dtype=np.float64)[np.asarray(idx[k], dtype=np.int64)]
    return h


# ---------------------------------------------------------------------------
# Grams and the pseudo-inverse (Eq. 4, Eq. 5)
# ---------------------------------------------------------------------------

def gram(U):
    """G_k = U_k^T U_k in binary64 (Eq. 5 operand)."""
    U = np.asarray(U, dtype=np.float64)
    return U.T @ U


def hadamard_of_grams(grams, n):
    """G = *_{k != n} G_k (Eq. 5)."""
    G = np.ones_like(grams[0])
    for k, Gk in enumerate(grams):
        if k != n:
            G = G * Gk
    return G


def pinv_sym(G):
    """Moore-Penrose pseudo-inverse of a symmetric PSD matrix (Eq. 4).

    Eigenvalues at or below R * 2^-52 * lambda_max are treated as zero.
    """
    G = np.asarray(G, dtype=np.float64)
    R = G.shape[0]
    lam, V = np.linalg.eigh(0.5 * (G + G.T))
    lmax = max(float(np.max(np.abs(lam))), 0.0)
    keep = lam > R * 2.0 ** -52 * lmax
    inv = np.zeros_like(lam)
    inv[keep] = 1.0 / lam[keep]
    return (V * inv) @ V.T


# ---------------------------------------------------------------------------
# MTTKRP: exact (Eq. 6) and downsampled (Eq. 7)
# ---------------------------------------------------------------------------

def exact_mttkrp(idx, vals, dims, factors, n):
    """mat(T, n) . U_{!=n}: each nonzero adds val * (KRP row) to row i_n (Eq. 6)."""
    R = factors[0].shape[1]
    h = krp_rows(factors, idx, n)
    Y = np.zeros((int(dims[n]), R), dtype=np.float64)
    np.add.at(Y, np.asarray(idx[n], dtype=np.int64), np.asarray(vals, dtype=np.float64)[:, None] * h)
    return Y


def sampled_mttkrp(idx, vals, dims, factors, n, samp_idx, w):
    """Downsampled MTTKRP mat(T, n) S^T S U_{!=n} (Eq. 7, Fig. 3 bottom).

    samp_idx: (N, J) sampled KRP rows (row n ignored); w: (J,) weights on the
    diagonal of S^T S.  S^T S is diagonal over KRP rows with entry
    D[key] = sum of w_j over draws j of that row, so every nonzero e adds
    val_e * D[key(e)] * (KRP row of e) to row i_n(e).
    """
    R = factors[0].shape[1]
    Y = np.zeros((int(dims[n]), R), dtype=np.float64)
    J = np.asarray(w).shape[0]
    if J == 0 or np.asarray(vals).shape[0] == 0:
        return Y
    skeys = krp_key(samp_idx, dims, n)
    ukeys, inv = np.unique(skeys, return_inverse=True)
    D = np.zeros(ukeys.shape[0], dtype=np.float64)
    np.add.at(D, inv, np.asarray(w, dtype=np.float64))
    ekeys = krp_key(idx, dims, n)
    pos = np.searchsorted(ukeys, ekeys)
    pos_c = np.minimum(pos, ukeys.shape[0] - 1)
    hit = ukeys[pos_c] == ekeys
    d = np.where(hit, D[pos_c], 0.0)
    sel = np.nonzero(d != 0.0)[0]
    if sel.size == 0:
        return Y
    sub_idx = [np.asarray(idx[k])[sel] for k in range(len(dims))]
    h = krp_rows(factors, sub_idx, n)
    contrib = (np.asarray(vals, dtype=np.float64)[sel] * d[sel])[:, None] * h
    np.add.at(Y, np.asarray(sub_idx[n], dtype=np.int64), contrib)
    return Y


def selected_nnz(idx, dims, n, samp_idx):
    """nnz(mat(T, n) S^T): nonzeros whose column is among the sampled rows."""
    skeys = np.unique(krp_key(samp_idx, dims, n))
    ekeys = krp_key(idx, dims, n)
    pos = np.minimum(np.searchsorted(skeys, ekeys), max(skeys.shape[0] - 1, 0))
    return int(np.count_nonzero(skeys[pos] == ekeys)) if skeys.size else 0


# ---------------------------------------------------------------------------
# CP-ARLS-LEV sampler (Appendix A, Algorithms 2 and 3; Eq. 8 per factor)
# ---------------------------------------------------------------------------

def leverage_scores(U, Gk_pinv):
    """dist_k = diag(U_k G_k^+ U_k^T) (Algorithm 2, Eq. 8 on one factor):
    row i is the dot product of row i of U_k G_k^+ with row i of U_k."""
    U = np.asarray(U, dtype=np.float64)
    return np.sum((U @ np.asarray(Gk_pinv, dtype=np.float64)) * U, axis=1)


def arls_build(U):
    """Sampler state of one factor: (G_k, G_k^+, leverage, inclusive CDF, C_k).

    Algorithm 2: G_k := U_k^T U_k, dist := diag(U_k G_k^+ U_k^T), C := ||dist||_1.
    The CDF is the running sum of the unnormalised scores in index order.
    """
    Gk = gram(U)
    Gp = pinv_sym(Gk)
    ell = leverage_scores(U, Gp)
    cdf = np.cumsum(ell)
    C = float(cdf[-1]) if cdf.size else 0.0
    return {"G": Gk, "Gpinv": Gp, "ell": ell, "cdf": cdf, "C": C}


def inverse_cdf(cdf, ell, t):
    """Smallest i with cdf[i] > t (Algorithm 3).  Past the end (t rounded up
    to the total C), the first row whose running sum reaches C, i.e. the last
    row whose bin has nonzero width.  All weights zero (C = 0): row 0."""
    i = np.searchsorted(cdf, t, side="right")
    C = cdf[-1]
    last = int(np.searchsorted(cdf, C, side="left")) if C > 0 else 0
    return np.where(i >= cdf.shape[0], last, i).astype(np.int64)


def gram_condition(Gk):
    """Condition number of the pseudo-inverse of a symmetric PSD Gram (Eq. 4):
    lambda_max over the smallest eigenvalue that pinv_sym keeps (above
    R 2^-52 lambda_max); 1 for a zero Gram."""
    G = np.asarray(Gk, dtype=np.float64)
    lam = np.linalg.eigvalsh(0.5 * (G + G.T))
    lmax = float(np.max(np.abs(lam))) if lam.size else 0.0
    kept = lam[lam > G.shape[0] * 2.0 ** -52 * lmax]
    return float(lmax / kept[0]) if kept.size else 1.0


def arls_tie_tolerance(sampler, floor=1e-12, cap=1e-6):
    """Tie window of a CP-ARLS-LEV draw on factor k, relative to C_k: a float64
    Gram is known to 2^-53 of its entries, so G_k^+ -- and every leverage
    score and running sum built on it -- is determined only to about
    cond(G_k) 2^-53 relative, whatever the arithmetic that follows.  The
    window is max(floor, 8 cond(G_k) 2^-53), capped at `cap`: past it the
    scores of a nearly singular Gram are fixed by the pseudo-inverse's cutoff,
    which both sides apply alike, and agreement is checked as such."""
    return min(cap, max(floor, 8.0 * gram_condition(sampler["G"]) * 2.0 ** -53))


def arls_draw(samplers, n, J, seed, sweep, tie_tol=1e-12):
    """Draw J rows of U_{!=n} from the product of per-factor leverage scores.

    Algorithm 3 with one processor: for each k != n, u = U(seed; j, k, n, s),
    i_k = inverse CDF of dist_k at u * C_k.  Returns (idx (N, J) with row n
    set to -1, p (J,) = prod_k ell_k[i_k] / C_k, near_tie (J,) bool marking
    draws whose target lies within tie_tol * C_k of a bin boundary).
    tie_tol is a number, or "conditioned" for arls_tie_tolerance(sampler k).
    """
    N = len(samplers)
    idx = np.full((N, J), -1, dtype=np.int64)
    p = np.ones(J, dtype=np.float64)
    near = np.zeros(J, dtype=bool)
    j = np.arange(J, dtype=np.uint64)
    for k in range(N):
        if k == n:
            continue
        s = samplers[k]
        u = draw_uniforms(seed, STREAM_ARLS, j, k, n, sweep)
        t = u * s["C"]
        ik = inverse_cdf(s["cdf"], s["ell"], t)
        idx[k] = ik
        # a factor whose scores are all zero has no distribution: its KRP
        # rows are all zero, the draw keeps row 0 and probability 0
        p = p * (s["ell"][ik] / s["C"] if s["C"] > 0 else 0.0)
        hi = s["cdf"][ik]
        lo = np.where(ik > 0, s["cdf"][np.maximum(ik - 1, 0)], 0.0)
        tol = (arls_tie_tolerance(s) if tie_tol == "conditioned" else tie_tol) * s["C"]
        near |= (np.abs(hi - t) <= tol) | ((ik > 0) & (np.abs(t - lo) <= tol))
    return idx, p, near


# ---------------------------------------------------------------------------
# STS-CP sampler (Sec. 4.1 "STS-CP", Appendix B, Algorithms 4 and 5)
# ---------------------------------------------------------------------------

def sts_build(U, F):
    """Binary tree over U_k: leaf v holds the Gram of its F-row block, each
    internal node the sum of its children's matrices (Sec. 4.1, Fig. 5).

    Heap layout: node 1 is the root, children of v are 2v and 2v+1, the L
    leaves (L a power of two >= ceil(I/F)) are nodes L..2L-1; leaf l covers
    rows [l F, min((l+1) F, I)).  Returns dict with 'nodes' (2L, R, R).
    """
    U = np.asarray(U, dtype=np.float64)
    I, R = U.shape
    nleaf = max(1, -(-I // F))
    L = 1
    while L < nleaf:
        L *= 2
    nodes = np.zeros((2 * L, R, R), dtype=np.float64)
    for l in range(nleaf):
        blk = U[l * F:min((l + 1) * F, I)]
        nodes[L + l] = blk.T @ blk
    for v in range(L - 1, 0, -1):
        nodes[v] = nodes[2 * v] + nodes[2 * v + 1]
    return {"nodes": nodes, "L": L, "F": F, "I": I}


def _node_first_row(tree, v):
    """First factor row covered by heap node v (array of node ids)."""
    L, F = tree["L"], tree["F"]
    v = np.asarray(v, dtype=np.int64).copy()
    while True:
        inner = v < L
        if not inner.any():
            break
        v = np.where(inner, 2 * v, v)
    return (v - L) * F


def _sts_walk(tree, U, Ggt, h, u, tie_tol):
    """Random walks of Algorithm 5 for a batch of draws on one factor.

    h: (m, R) running Hadamard products, u: (m,) uniforms.  Returns (rows,
    near_tie flags) for the batch.
    """
    nodes, L, F, I = tree["nodes"], tree["L"], tree["F"], tree["I"]
    m = u.shape[0]

    def mass(vs):
        # m(v) = h^T (G^v (*) G_{>k}) h, one node per draw
        return np.einsum("ja,jab,ab,jb->j", h, nodes[vs], Ggt, h)

    v = np.ones(m, dtype=np.int64)
    mroot = mass(v)
    t = u * mroot
    near = np.zeros(m, dtype=bool)
    while L > 1 and v[0] < L:
        left = 2 * v
        mL = mass(left)
        near |= np.abs(t - mL) <= tie_tol * np.abs(mroot)
        right_real = _node_first_row(tree, left + 1) < I
        go_right = (t >= mL) & right_real
        t = np.where(go_right, t - mL, t)
        v = np.where(go_right, left + 1, left)
    # leaf: row masses q_i = (U[i] (*) h)^T G_{>k} (U[i] (*) h) of its F rows
    r0 = (v - L) * F
    rows = r0[:, None] + np.arange(F)[None, :]
    valid = rows < I
    x = np.where(valid[:, :, None], U[np.minimum(rows, I - 1)], 0.0) * h[:, None, :]
    q = np.einsum("jia,ab,jib->ji", x, Ggt, x)
    mleaf = mass(v)
    qs = np.sum(q, axis=1)
    tl = np.where(mleaf > 0, t * (qs / np.where(mleaf > 0, mleaf, 1.0)), 0.0)
    cq = np.cumsum(q, axis=1)
    near |= np.any(np.abs(cq[:, :-1] - tl[:, None]) <= tie_tol * np.abs(mroot)[:, None], axis=1)
    above = cq > tl[:, None]
    has = above.any(axis=1)
    first = np.argmax(above, axis=1)
    posq = q > 0
    last_pos = np.where(posq.any(axis=1), F - 1 - np.argmax(posq[:, ::-1], axis=1), 0)
    return r0 + np.where(has, first, last_pos), near


def sts_draw(trees, factors, grams, n, J, seed, sweep, tie_tol=1e-12, batch=1024):
    """Draw J rows of U_{!=n} from the exact leverage distribution (STS-CP).

    For each draw j, for k != n in ascending order: G_{>k} = G^+ (*) Grams of
    the factors drawn after k; masses m(v) = h^T (G^v (*) G_{>k}) h; random
    walk from the root with t = u * m(root); leaf row masses
    q_i = (U_k[i] (*) h)^T G_{>k} (U_k[i] (*) h); then h := h (*) U_k[i_k].
    Returns (idx (N, J), p (J,), near_tie (J,)) where p = h^T G^+ h / <G^+, G>_F
    is the exact leverage of the drawn row over the leverage total, and
    near_tie marks draws with some decision within tie_tol * m(root) of its
    threshold (the target t = u m(root) - sum of left masses carries rounding
    on the scale of m(root), whatever the depth).  Draws are processed in batches of `batch` (they are independent).
    """
    N = len(factors)
    R = factors[0].shape[1]
    G = hadamard_of_grams(grams, n)
    Gp = pinv_sym(G)
    order = [k for k in range(N) if k != n]
    idx = np.full((N, J), -1, dtype=np.int64)
    h = np.ones((J, R), dtype=np.float64)
    near = np.zeros(J, dtype=bool)
    jj = np.arange(J, dtype=np.uint64)
    for pos, k in enumerate(order):
        Ggt = Gp.copy()
        for k2 in order[pos + 1:]:
            Ggt = Ggt * grams[k2]
        U = np.asarray(factors[k], dtype=np.float64)
        u = draw_uniforms(seed, STREAM_STS, jj, k, n, sweep)
        for b0 in range(0, J, batch):
            b1 = min(J, b0 + batch)
            rows, nt = _sts_walk(trees[k], U, Ggt, h[b0:b1], u[b0:b1], tie_tol)
            idx[k, b0:b1] = rows
            near[b0:b1] |= nt
        h = h * U[idx[k]]
    lev = np.einsum("ja,ab,jb->j", h, Gp, h)
    total = float(np.sum(Gp * G))
    return idx, lev / total, near


def exact_krp_leverage(factors, n):
    """Leverage scores of every row of the materialised U_{!=n} (tiny inputs).

    Rows are in key order; ell_row = h_row^T G^+ h_row with G = *_{k!=n} G_k.
    """
    dims = [U.shape[0] for U in factors]
    N = len(factors)
    other = [k for k in range(N) if k != n]
    grids = np.meshgrid(*[np.arange(dims[k]) for k in other], indexing="ij")
    idx = [None] * N
    for g, k in zip(grids, other):
        idx[k] = g.reshape(-1)
    idx[n] = np.zeros_like(idx[other[0]])
    keys = krp_key(idx, dims, n)
    order = np.argsort(keys)
    idx = [a[order] for a in idx]
    h = krp_rows(factors, idx, n)
    G = hadamard_of_grams([gram(U) for U in factors], n)
    return np.einsum("ja,ab,jb->j", h, pinv_sym(G), h)


# ---------------------------------------------------------------------------
# Solve and renormalise (Eq. 4, Algorithm 1's mode update)
# ---------------------------------------------------------------------------

def solve_and_renorm(Y, G_pinv):
    """U_n := Y G^+; sigma_r := ||U_n[:, r]||_2; U_n[:, r] /= sigma_r."""
    Un = np.asarray(Y, dtype=np.float64) @ G_pinv
    sigma = np.sqrt(np.sum(Un * Un, axis=0))
    safe = np.where(sigma > 0, sigma, 1.0)
    return Un / safe[None, :], sigma


def renormalize(U):
    """Algorithm 1's initial normalisation: divide each column by its 2-norm (zero columns kept)."""
    U = np.asarray(U, dtype=np.float64)
    nrm = np.sqrt(np.sum(U * U, axis=0))
    return U / np.where(nrm > 0, nrm, 1.0)[None, :]


# ---------------------------------------------------------------------------
# Fit (Sec. 5.1)
# ---------------------------------------------------------------------------

def inner_with_model(idx, vals, factors, sigma):
    """<T, T~> = sum_e val_e sum_r sigma_r prod_k U_k[i_{e,k}, r]."""
    R = factors[0].shape[1]
    m = np.ones((np.asarray(vals).shape[0], R), dtype=np.float64)
    for k, U in enumerate(factors):
        m *= np.asarray(U, dtype=np.float64)[np.asarray(idx[k], dtype=np.int64)]
    return float(np.asarray(vals, dtype=np.float64) @ (m @ np.asarray(sigma, dtype=np.float64)))


def model_norm_sq(factors, sigma):
    """||T~||_F^2 = sigma^T (*_k U_k^T U_k) sigma."""
    G = np.ones((factors[0].shape[1],) * 2)
    for U in factors:
        G = G * gram(U)
    s = np.asarray(sigma, dtype=np.float64)
    return float(s @ G @ s)


def fit(idx, vals, factors, sigma):
    """fit = 1 - ||T~ - T||_F / ||T||_F (Sec. 5.1)."""
    v = np.asarray(vals, dtype=np.float64)
    tn2 = float(v @ v)
    resid2 = tn2 - 2.0 * inner_with_model(idx, vals, factors, sigma) + model_norm_sq(factors, sigma)
    return 1.0 - np.sqrt(max(resid2, 0.0)) / np.sqrt(tn2)


# ---------------------------------------------------------------------------
# ALS driver (Algorithm 1)
# ---------------------------------------------------------------------------

def sketched_gram(factors, n, samp_idx, w):
    """Gram of the downsampled design matrix, (S U_{!=n})^T (S U_{!=n}) =
    sum_j w_j h_j h_j^T over the draws (the G~ of Fig. 3, bottom)."""
    h = krp_rows(factors, samp_idx, n)
    return h.T @ (np.asarray(w, dtype=np.float64)[:, None] * h)


def sample_weights(p, J):
    """w_j = 1 / (J p_j): diagonal of S^T S for i.i.d. draws with probability
    p_j.  A draw of probability 0 (or undefined, from an all-zero factor, whose
    KRP rows are all zero) gets weight 0."""
    p = np.asarray(p, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(p > 0, 1.0 / (J * np.where(p > 0, p, 1.0)), 0.0)


def als_mode_update(state, n, method, J, seed, sweep, leaf_rows=None, sketched=False):
    """One subproblem of Algorithm 1 (the update of mode n); updates state.

    state: dict with idx, vals, dims, factors (list of (I_k, R) float64),
    sigma, grams, and per method the sampler structures.
    Returns a dict of the intermediate quantities (samples, Y, G^+) so that
    tests can compare every step.  sketched=True solves with the Gram of the
    drawn rows (the downsampled normal equations of Fig. 3, bottom) instead of
    the Hadamard product of the factor Grams (Eq. 5).
    """
    idx, vals, dims, factors = state["idx"], state["vals"], state["dims"], state["factors"]
    grams = state["grams"]
    G = hadamard_of_grams(grams, n)
    Gp = pinv_sym(G)
    out = {"G": G, "Gpinv": Gp}
    if method == "exact":
        Y = exact_mttkrp(idx, vals, dims, factors, n)
    else:
        if method == "arls":
            sidx, p, near = arls_draw(state["samplers"], n, J, seed, sweep)
        elif method == "sts":
            sidx, p, near = sts_draw(state["trees"], factors, grams, n, J, seed, sweep)
        else:
            raise ValueError(method)
        w = sample_weights(p, J)
        Y = sampled_mttkrp(idx, vals, dims, factors, n, sidx, w)
        out.update({"samp_idx": sidx, "p": p, "w": w, "near_tie": near})
        if sketched:
            Gp = pinv_sym(sketched_gram(factors, n, sidx, w))
            out["Gpinv"] = Gp
    Un, sigma = solve_and_renorm(Y, Gp)
    out.update({"Y": Y, "U": Un, "sigma": sigma})
    factors[n] = Un
    state["sigma"] = sigma
    grams[n] = gram(Un)
    if method == "arls":
        state["samplers"][n] = arls_build(Un)
    elif method == "sts":
        F = leaf_rows or factors[0].shape[1]
        state["trees"][n] = sts_build(Un, F)
    return out


def als_init(idx, vals, dims, init_factors, method, leaf_rows=None):
    """Algorithm 1's initialisation with caller-supplied N(0,1) draws."""
    factors = [renormalize(U) for U in init_factors]
    R = factors[0].shape[1]
    state = {"idx": [np.asarray(a, dtype=np.int64) for a in idx],
             "vals": np.asarray(vals, dtype=np.float64),
             "dims": [int(d) for d in dims],
             "factors": factors,
             "sigma": np.ones(R, dtype=np.float64),
             "grams": [gram(U) for U in factors]}
    if method == "arls":
        state["samplers"] = [arls_build(U) for U in factors]
    elif method == "sts":
        F = leaf_rows or R
        state["trees"] = [sts_build(U, F) for U in factors]
    return state


def als(idx, vals, dims, init_factors, method, sweeps, J=0, seed=0, leaf_rows=None, sketched=False):
    """Run Algorithm 1 for `sweeps` rounds; returns (state, per-sweep fits)."""
    state = als_init(idx, vals, dims, init_factors, method, leaf_rows)
    fits = []
    for s in range(sweeps):
        for n in range(len(dims)):
            als_mode_update(state, n, method, J, seed, s, leaf_rows, sketched)
        fits.append(fit(state["idx"], state["vals"], state["factors"], state["sigma"]))
    return state, fits
