"""Independent constructions used to pin the oracle (dense tensors, explicit
Kronecker-built Khatri-Rao products, explicit sampling matrices)."""
import numpy as np


def dense_from_coo(idx, vals, dims):
    T = np.zeros(dims, dtype=np.float64)
    T[tuple(np.asarray(i, dtype=np.int64) for i in idx)] = vals
    return T


def matricize(T, n):
    """mat(T, n): rows i_n; columns over the other modes, lowest mode fastest."""
    return np.moveaxis(T, n, 0).reshape(T.shape[n], -1, order="F")


def khatri_rao_design(factors, n):
    """U_{!=n} = U_{N-1} (.) ... (.) U_0 (skipping n), built column by column
    with np.kron so that the lowest mode's index varies fastest (Eq. 3)."""
    R = factors[0].shape[1]
    modes = [k for k in range(len(factors)) if k != n][::-1]
    out = np.asarray(factors[modes[0]], dtype=np.float64)
    for k in modes[1:]:
        B = np.asarray(factors[k], dtype=np.float64)
        out = np.stack([np.kron(out[:, r], B[:, r]) for r in range(R)], axis=1)
    return out


def planted_dense(dims, R, seed):
    rng = np.random.default_rng(seed)
    fs = [rng.standard_normal((d, R)) for d in dims]
    T = np.zeros(dims)
    for r in range(R):
        t = fs[0][:, r]
        for f in fs[1:]:
            t = np.multiply.outer(t, f[:, r])
        T += t
    idx = np.array(np.nonzero(np.ones(dims)))
    return idx, T[tuple(idx)], T
