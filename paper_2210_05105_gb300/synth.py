"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only draws data: COO coordinates, values and the N(0,1) initial
factors.  It holds none of the CP-ALS arithmetic, so the oracle and the CUDA
library can both be fed from it without sharing any of the method's code.

Recipe (stand-ins for the FROSTT tensors of the paper's Table 4, which are not
redistributed here):
* Each mode index is pi_n(rank), rank drawn from a truncated Zipf law
  P(rank = r) proportional to (r + 1)^-s for r < I_n by inverse CDF over a
  binary64 table; pi_n is a seeded random permutation (the random index
  permutation of the paper's Sec. 4.4 load-balancing).  s = 0 gives uniform
  coordinates.
* Coordinates are made distinct by their linear key; draws continue until
  exactly nnz distinct coordinates exist, keeping the earliest-drawn ones.
* Values: uniform(0, 1), lognormal(0, 1), or log(1 + Poisson(3)) with zero
  draws redrawn (Reddit-like log counts).
All randomness comes from numpy's PCG64 with the caller's seed.
"""
import numpy as np


def _zipf_table(I, s):
    r = np.arange(1, I + 1, dtype=np.float64)
    w = r ** (-float(s)) if s else np.ones(I)
    c = np.cumsum(w)
    return c / c[-1]


def _draw_indices(rng, dims, count, s, perms, tables):
    out = np.empty((len(dims), count), dtype=np.int64)
    for k, I in enumerate(dims):
        if s == 0:
            out[k] = rng.integers(0, I, size=count)
        else:
            u = rng.random(count)
            rank = np.minimum(np.searchsorted(tables[k], u, side="right"), I - 1)
            out[k] = perms[k][rank]
    return out


def coo_coordinates(dims, nnz, seed, zipf_s=0.0):
    """Exactly nnz distinct coordinates, (N, nnz) int32, earliest draws kept."""
    dims = [int(d) for d in dims]
    total = 1
    for d in dims:
        total *= d
    if nnz > total:
        raise ValueError("nnz exceeds the number of cells")
    rng = np.random.Generator(np.random.PCG64(seed))
    perms = [rng.permutation(I) for I in dims] if zipf_s else None
    tables = [_zipf_table(I, zipf_s) for I in dims] if zipf_s else None
    mult = np.ones(len(dims), dtype=np.uint64)
    for k in range(1, len(dims)):
        mult[k] = mult[k - 1] * np.uint64(dims[k - 1])
    drawn = np.empty((len(dims), 0), dtype=np.int64)
    need = nnz
    while True:
        batch = max(1024, int(need * 1.15) + 16)
        drawn = np.concatenate([drawn, _draw_indices(rng, dims, batch, zipf_s, perms, tables)], axis=1)
        keys = np.zeros(drawn.shape[1], dtype=np.uint64)
        for k in range(len(dims)):
            keys += drawn[k].astype(np.uint64) * mult[k]
        _, first = np.unique(keys, return_index=True)
        if first.size >= nnz:
            keep = np.sort(first)[:nnz]
            return np.ascontiguousarray(drawn[:, keep], dtype=np.int32)
        need = nnz - first.size
        drawn = drawn[:, np.sort(first)]


def planted_values(idx, dims, seed):
    """Values of a planted rank-16 CP model (N(0,1) factors, seeded) at the
    coordinates idx (N, nnz), plus Gaussian noise scaled to 10% of the
    planted values' norm."""
    rng = np.random.Generator(np.random.PCG64(seed + 4241))
    A = [rng.standard_normal((int(I), PLANTED_RANK)) for I in dims]
    m = np.ones((idx.shape[1], PLANTED_RANK))
    for k in range(len(dims)):
        m *= A[k][np.asarray(idx[k], dtype=np.int64)]
    v = m.sum(axis=1)
    rms = float(np.sqrt(np.mean(v * v))) if v.size else 0.0
    v = v + rng.standard_normal(v.shape[0]) * (PLANTED_NOISE * rms)
    return v.astype(np.float32)


def coo_values(nnz, seed, kind="uniform"):
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    if kind == "uniform":
        return rng.random(nnz, dtype=np.float32)
    if kind == "lognormal":
        return rng.lognormal(0.0, 1.0, size=nnz).astype(np.float32)
    if kind == "logpoisson":
        x = rng.poisson(3.0, size=nnz)
        bad = x == 0
        while bad.any():
            x[bad] = rng.poisson(3.0, size=int(bad.sum()))
            bad = x == 0
        return np.log1p(x.astype(np.float64)).astype(np.float32)
    raise ValueError(kind)


def init_factors(dims, R, seed):
    """Unit-variance Gaussian initial factors (I_k, R) float32 (Algorithm 1's initialisation)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.standard_normal((int(I), R), dtype=np.float32) for I in dims]


def make_tensor(dims, nnz, seed, zipf_s=0.0, values="uniform"):
    idx = coo_coordinates(dims, nnz, seed, zipf_s)
    vals = planted_values(idx, dims, seed) if values == "planted16" else coo_values(nnz, seed, values)
    return idx, vals


# Named workloads (dims, nnz, Zipf exponent, value law, R, J, sweeps, seeds)
WORKLOADS = {
    "small_uniform_200x150x100": dict(dims=(200, 150, 100), nnz=20_000, zipf=0.0,
                                      values="uniform", R=8, J=2000, sweeps=5,
                                      data_seed=1001, init_seed=2001, sample_seed=3001),
    "zipf_1e5cube_5M": dict(dims=(100_000, 100_000, 100_000), nnz=5_000_000, zipf=1.1,
                            values="lognormal", R=32, J=65536, sweeps=20,
                            data_seed=1003, init_seed=2003, sample_seed=3003),
    "zipf_1e5cube_20M": dict(dims=(100_000, 100_000, 100_000), nnz=20_000_000, zipf=1.1,
                             values="lognormal", R=32, J=65536, sweeps=20,
                             data_seed=1006, init_seed=2006, sample_seed=3006),
    "zipf_1e5cube_50M": dict(dims=(100_000, 100_000, 100_000), nnz=50_000_000, zipf=1.1,
                             values="lognormal", R=32, J=65536, sweeps=20,
                             data_seed=1002, init_seed=2002, sample_seed=3002),
    # billion-scale 3-mode workload with Reddit's dims (paper Table 4): Zipf(1.3)
    # per mode, log(1 + Poisson(3)) values; drawn on the device (libzipfgen)
    "zipf_reddit_1B": dict(dims=(8_200_000, 177_000, 8_100_000), nnz=1_000_000_000, zipf=1.3,
                           values="logpoisson", R=100, J=131072, sweeps=20, generator="device",
                           data_seed=1007, init_seed=2007, sample_seed=3007),
    # the same recipe at a tenth of two dims and 2e7 nonzeros, for ncu captures
    # of the R = 100 kernels (a few GB on the device)
    "zipf_reddit_20M": dict(dims=(820_000, 177_000, 810_000), nnz=20_000_000, zipf=1.3,
                            values="logpoisson", R=100, J=131072, sweeps=20, generator="device",
                            data_seed=1008, init_seed=2008, sample_seed=3008),
    # 4-mode precision-form workload: values of a planted rank-16 CP model at
    # the drawn coordinates plus Gaussian noise of 10% of their norm (the
    # tensor's zeros are real zeros, so it is not a rank-16 tensor)
    "planted16_4mode_200M": dict(dims=(1_000_000, 500_000, 100_000, 1_000), nnz=200_000_000, zipf=1.2,
                                 values="planted16", R=64, J=65536, sweeps=20,
                                 data_seed=1005, init_seed=2005, sample_seed=3005),
}

PLANTED_RANK = 16
PLANTED_NOISE = 0.1


# Many uneven tensors decomposed together (the batched form): order 3 or 4
# alternating, nnz and dims log-uniform, R from {16, 32, 64}, J log-uniform.
BATCH_WORKLOADS = {
    "batch64_uneven": dict(T=64, nnz=(1e4, 5e6), dims=(1e3, 2e6), zipf=1.1, values="uniform",
                           ranks=(16, 32, 64), J=(4096, 65536), seed=1004, sweeps=20),
}


def batch_specs(T, nnz, dims, zipf, values, ranks, J, seed, sweeps):
    """Per-tensor workload dicts of a batched workload.  A 4-mode draw whose
    dims multiply to 2^63 or more (beyond the 64-bit linear index), or that
    would be denser than 1/8, is drawn again."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo_n, hi_n = np.log(nnz[0]), np.log(nnz[1])
    lo_d, hi_d = np.log(dims[0]), np.log(dims[1])
    out = []
    for t in range(T):
        N = 3 if t % 2 == 0 else 4
        while True:
            d = tuple(int(round(x)) for x in np.exp(rng.uniform(lo_d, hi_d, size=N)))
            z = int(round(float(np.exp(rng.uniform(lo_n, hi_n)))))
            total = 1
            for x in d:
                total *= x
            if total < 2 ** 63 and z * 8 <= total:
                break
        R = int(ranks[int(rng.integers(0, len(ranks)))])
        j = int(round(float(np.exp(rng.uniform(np.log(J[0]), np.log(J[1]))))))
        out.append(dict(dims=d, nnz=z, zipf=zipf, values=values, R=R, J=j, sweeps=sweeps,
                        data_seed=seed * 1000 + t, init_seed=seed * 1000 + 500 + t, sample_seed=seed * 1000 + 900 + t))
    return out


def _genlib():
    """The device-side generator library (libzipfgen.so, built beside libcpd)."""
    import ctypes
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libzipfgen.so")
    if not os.path.exists(path):
        raise RuntimeError("libzipfgen.so is not built (python -m paper_2210_05105_gb300.build)")
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    L.zg_generate.argtypes = [ctypes.c_int, P, P, P, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, P, P, P]
    L.zg_generate.restype = ctypes.c_int
    L.zg_values_logpoisson.argtypes = [ctypes.c_int64, ctypes.c_uint64, P, ctypes.c_int, P, P]
    L.zg_values_logpoisson.restype = ctypes.c_int
    return L


def poisson_ge1_cdf(lam=3.0, kmax=64):
    """Running sums P(X <= x | X >= 1), x = 1..kmax, of Poisson(lam) (last = 1)."""
    p = np.empty(kmax, dtype=np.float64)
    term = np.exp(-lam)
    for x in range(1, kmax + 1):
        term = term * lam / x
        p[x - 1] = term
    c = np.cumsum(p) / (1.0 - np.exp(-lam))
    c[-1] = 1.0
    return c


def make_tensor_device(dims, nnz, seed, zipf_s, values="logpoisson", device="cuda", max_draws=1 << 40):
    """Device generator for the billion-scale workload (libzipfgen): draw d
    picks i_k = perm_k[smallest r with table_k[r] > u_k(d)], u_k(d) from
    Philox4x64-10 key (seed, 7), counter (d, 0, 0, 0), word k; exactly nnz
    distinct coordinates with the earliest first draws, in first-draw order;
    values log(1 + Poisson(3)) with zeros redrawn (Philox key (seed, 8)).
    The tables are this module's truncated Zipf running sums and the
    permutations come from numpy's PCG64 with `seed`, as in coo_coordinates.
    Returns (idx (N, nnz) int32, vals (nnz,) float32, draws used)."""
    import ctypes
    import torch
    dims = [int(d) for d in dims]
    N = len(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    perms = [torch.from_numpy(rng.permutation(I).astype(np.int32)).to(device) for I in dims]
    tables = [torch.from_numpy(_zipf_table(I, zipf_s)).to(device) for I in dims]
    idx = torch.empty((N, nnz), dtype=torch.int32, device=device)
    L = _genlib()
    P = ctypes.c_void_p
    dims_a = (ctypes.c_int64 * N)(*dims)
    tab_a = (P * N)(*[t.data_ptr() for t in tables])
    perm_a = (P * N)(*[t.data_ptr() for t in perms])
    used = ctypes.c_int64(0)
    stream = P(torch.cuda.current_stream().cuda_stream)
    rc = L.zg_generate(N, ctypes.cast(dims_a, P), ctypes.cast(tab_a, P), ctypes.cast(perm_a, P), int(seed), int(nnz),
                       int(max_draws), P(idx.data_ptr()), ctypes.byref(used), stream)
    if rc != 0:
        raise RuntimeError("zg_generate failed with code %d" % rc)
    if values != "logpoisson":
        raise ValueError(values)
    cdf = torch.from_numpy(poisson_ge1_cdf(3.0)).to(device)
    vals = torch.empty(nnz, dtype=torch.float32, device=device)
    rc = L.zg_values_logpoisson(int(nnz), int(seed), P(cdf.data_ptr()), int(cdf.numel()), P(vals.data_ptr()), stream)
    if rc != 0:
        raise RuntimeError("zg_values_logpoisson failed with code %d" % rc)
    torch.cuda.synchronize()
    del perms, tables, cdf
    return idx, vals, int(used.value)


def make_tensor_torch(dims, nnz, seed, zipf_s=0.0, values="uniform", device="cuda"):
    """Device-side version of the same recipe for the large workloads (torch
    generator on `device`, seeded): returns (idx (N, nnz) int32, vals (nnz,)
    float32) torch tensors on `device`.  Exactly nnz distinct coordinates,
    earliest draws kept."""
    import torch
    dims = [int(d) for d in dims]
    N = len(dims)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    tables, perms = [], []
    for I in dims:
        if zipf_s:
            r = torch.arange(1, I + 1, dtype=torch.float64, device=device)
            c = torch.cumsum(r.pow(-float(zipf_s)), 0)
            tables.append(c / c[-1])
            perms.append(torch.randperm(I, generator=g, device=device))
    one_key = True
    total = 1
    for d in dims:
        total *= d
    if total >= 2 ** 62:
        one_key = False
    mult = []
    acc = 1
    for d in dims:
        mult.append(acc)
        acc *= d

    def draw(count):
        cols = []
        for k, I in enumerate(dims):
            if zipf_s:
                u = torch.rand(count, generator=g, device=device, dtype=torch.float64)
                rank = torch.clamp(torch.searchsorted(tables[k], u, right=True), max=I - 1)
                cols.append(perms[k][rank])
            else:
                cols.append(torch.randint(0, I, (count,), generator=g, device=device))
        return torch.stack(cols)

    drawn = torch.empty((N, 0), dtype=torch.int64, device=device)
    need = nnz
    while True:
        drawn = torch.cat([drawn, draw(max(1024, int(need * 1.15) + 16))], dim=1)
        if one_key:
            key = torch.zeros(drawn.shape[1], dtype=torch.int64, device=device)
            for k in range(N):
                key += drawn[k] * mult[k]
            _, inv = torch.unique(key, return_inverse=True)
        else:
            half = N // 2
            k1 = torch.zeros(drawn.shape[1], dtype=torch.int64, device=device)
            k2 = torch.zeros_like(k1)
            a1 = a2 = 1
            for k in range(half):
                k1 += drawn[k] * a1
                a1 *= dims[k]
            for k in range(half, N):
                k2 += drawn[k] * a2
                a2 *= dims[k]
            _, inv = torch.unique(torch.stack([k1, k2], dim=1), dim=0, return_inverse=True)
        pos = torch.arange(drawn.shape[1], device=device)
        first = torch.full((int(inv.max()) + 1,), drawn.shape[1], dtype=torch.int64, device=device)
        first.scatter_reduce_(0, inv, pos, reduce="amin")
        first, _ = torch.sort(first)
        if first.numel() >= nnz:
            idx = drawn[:, first[:nnz]].to(torch.int32).contiguous()
            break
        need = nnz - first.numel()
        drawn = drawn[:, first]
    if values == "uniform":
        vals = torch.rand(nnz, generator=g, device=device, dtype=torch.float32)
    elif values == "lognormal":
        vals = torch.randn(nnz, generator=g, device=device, dtype=torch.float32).exp()
    elif values == "planted16":
        g2 = torch.Generator(device=device)
        g2.manual_seed(int(seed) + 4241)
        A = [torch.randn(I, PLANTED_RANK, generator=g2, device=device) for I in dims]
        vals = torch.empty(nnz, dtype=torch.float32, device=device)
        step = 1 << 22
        for c0 in range(0, nnz, step):
            c1 = min(nnz, c0 + step)
            m = torch.ones(c1 - c0, PLANTED_RANK, device=device)
            for k in range(N):
                m *= A[k][idx[k, c0:c1].long()]
            vals[c0:c1] = m.sum(dim=1)
        rms = torch.sqrt(torch.mean(vals.double() ** 2)).float()
        vals += torch.randn(nnz, generator=g2, device=device) * (PLANTED_NOISE * rms)
    elif values == "logpoisson":
        x = torch.poisson(torch.full((nnz,), 3.0, device=device), generator=g)
        bad = x == 0
        while bool(bad.any()):
            x[bad] = torch.poisson(torch.full((int(bad.sum()),), 3.0, device=device), generator=g)
            bad = x == 0
        vals = torch.log1p(x).to(torch.float32)
    else:
        raise ValueError(values)
    return idx, vals
