"""Thin ctypes binding of libcpd (include/cpd.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Functions keep the C names; torch tensors provide device memory and streams.
If libcpd.so is missing, :func:`lib` raises -- there is no CPU fallback.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcpd.so")

CPD_ARLS_LEV, CPD_STS_CP, CPD_EXACT = 0, 1, 2
METHODS = {"arls": CPD_ARLS_LEV, "sts": CPD_STS_CP, "exact": CPD_EXACT}
STATUS = {0: "CPD_OK", 1: "CPD_ERR_INVALID_ARG", 2: "CPD_ERR_OUT_OF_RANGE_INDEX", 3: "CPD_ERR_DUPLICATE",
          4: "CPD_ERR_OOM", 5: "CPD_ERR_CUDA", 6: "CPD_ERR_CAPACITY", 7: "CPD_ERR_SINGULAR_GRAM",
          8: "CPD_ERR_TIMEOUT", 9: "CPD_ERR_NOT_FINITE"}
EXPORTS = ["cpd_default_options", "cpd_create", "cpd_leverage_sample", "cpd_sampled_mttkrp", "cpd_exact_mttkrp",
           "cpd_gram_solve", "cpd_als_sweep", "cpd_fit", "cpd_get_factors", "cpd_set_factors", "cpd_get_sigma",
           "cpd_get_arls_state", "cpd_get_gram", "cpd_profile", "cpd_profile_read", "cpd_sweep_kernel_count",
           "cpd_sampled_mttkrp_noalloc", "cpd_sts_rescans", "cpd_debug_gram_wait", "cpd_synchronize",
           "cpd_batch_create", "cpd_batch_sweep", "cpd_batch_synchronize", "cpd_batch_destroy", "cpd_autotune",
           "cpd_last_error", "cpd_destroy"]
PHASES = ["pinv", "draw", "probe", "scan", "spmm", "solve", "gram", "sampler", "exact", "clear"]


class cpd_options(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("rank", ctypes.c_int32), ("samples", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("leaf_rows", ctypes.c_int32), ("input_on_host", ctypes.c_int32),
                ("nnz_sel_capacity", ctypes.c_int64), ("reserved_i64", ctypes.c_int64 * 3),
                ("sketched_gram", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("spmm_blocks_per_sm", ctypes.c_int32), ("duplicate_policy", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("reserved_i32", ctypes.c_int32 * 3)]


class CpdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None
_P = ctypes.c_void_p


def lib():
    """Load libcpd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libcpd.so is not built (python -m paper_2210_05105_gb300.build)")
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, u64, st = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
    sig = {
        "cpd_default_options": ([ctypes.POINTER(cpd_options)], st),
        "cpd_create": ([i32, _P, i64, _P, _P, _P, ctypes.POINTER(cpd_options), _P, ctypes.POINTER(_P)], st),
        "cpd_leverage_sample": ([_P, i32, i64, u64, _P, _P], st),
        "cpd_sampled_mttkrp": ([_P, i32, _P, _P, i64, _P, _P], st),
        "cpd_exact_mttkrp": ([_P, i32, _P], st),
        "cpd_gram_solve": ([_P, i32, _P, _P], st),
        "cpd_als_sweep": ([_P, i32], st),
        "cpd_fit": ([_P, ctypes.POINTER(ctypes.c_double)], st),
        "cpd_get_factors": ([_P, i32, _P], st),
        "cpd_set_factors": ([_P, i32, _P], st),
        "cpd_get_sigma": ([_P, _P], st),
        "cpd_get_arls_state": ([_P, i32, _P, _P], st),
        "cpd_get_gram": ([_P, i32, _P], st),
        "cpd_profile": ([_P, i32], st),
        "cpd_profile_read": ([_P, _P, _P], st),
        "cpd_sweep_kernel_count": ([_P, _P], st),
        "cpd_synchronize": ([_P], st),
        "cpd_sts_rescans": ([_P, _P], st),
        "cpd_debug_gram_wait": ([_P, i64, i32], st),
        "cpd_batch_create": ([_P, i32, i32, _P, ctypes.POINTER(_P)], st),
        "cpd_batch_sweep": ([_P, i32], st),
        "cpd_batch_synchronize": ([_P], st),
        "cpd_batch_destroy": ([_P], None),
        "cpd_autotune": ([_P, _P], st),
        "cpd_last_error": ([_P], ctypes.c_char_p),
        "cpd_destroy": ([_P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class Handle:
    """Owner of a cpd_handle plus the tensor sizes the binding needs."""

    def __init__(self, raw, N, dims, R, J, method, device):
        self.raw = raw
        self.N, self.dims, self.R, self.J, self.method, self.device = N, dims, R, J, method, device

    def _check(self, status):
        if status != 0:
            raise CpdError(status, lib().cpd_last_error(self.raw).decode())

    def close(self):
        if self.raw:
            lib().cpd_destroy(self.raw)
            self.raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cpd_create(dims, idx, vals, init_factors, method="arls", rank=8, samples=2000, seed=0, leaf_rows=0,
               stream=None, sketched_gram=False, fast=False, spmm_blocks_per_sm=0, sum_duplicates=False,
               deterministic=False, nnz_sel_capacity=0):
    """Build a handle.  idx (N, nnz) int32, vals (nnz,) float32 and the init
    factors (list of (I_k, R) float32) must all be on the same device: all
    CUDA, or all CPU (then they are copied by the library, host input).
    init_factors=None lets the library draw the N(0, 1) initial factors from
    the seed."""
    L = lib()
    dims = [int(d) for d in dims]
    N = len(dims)
    on_host = not idx.is_cuda
    idx = idx.contiguous()
    vals = vals.contiguous()
    init = None if init_factors is None else torch.cat([u.reshape(-1) for u in init_factors]).contiguous()
    if on_host:
        idx, vals = idx.pin_memory(), vals.pin_memory()
        init = None if init is None else init.pin_memory()
    opt = cpd_options()
    L.cpd_default_options(ctypes.byref(opt))
    opt.method = METHODS[method] if isinstance(method, str) else int(method)
    opt.rank = int(rank)
    opt.samples = int(samples)
    opt.seed = int(seed)
    opt.leaf_rows = int(leaf_rows)
    opt.input_on_host = 1 if on_host else 0
    opt.sketched_gram = 1 if sketched_gram else 0
    opt.precision = 1 if fast else 0
    opt.spmm_blocks_per_sm = int(spmm_blocks_per_sm)
    opt.duplicate_policy = 1 if sum_duplicates else 0
    opt.deterministic = 1 if deterministic else 0
    opt.nnz_sel_capacity = int(nnz_sel_capacity)
    dims_arr = (ctypes.c_int64 * N)(*dims)
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    out = ctypes.c_void_p()
    st = L.cpd_create(N, ctypes.cast(dims_arr, _P), int(vals.numel()), _ptr(idx), _ptr(vals), _ptr(init),
                      ctypes.byref(opt), sp, ctypes.byref(out))
    if st != 0:
        raise CpdError(st, L.cpd_last_error(None).decode())
    dev = torch.device("cuda", torch.cuda.current_device())
    return Handle(out, N, dims, int(rank), int(samples), opt.method, dev)


def cpd_leverage_sample(h, mode, J, sweep=0):
    """-> (idx (N, J) int32 cuda, prob (J,) float64 cuda)."""
    idx = torch.empty((h.N, J), dtype=torch.int32, device=h.device)
    prob = torch.empty(J, dtype=torch.float64, device=h.device)
    h._check(lib().cpd_leverage_sample(h.raw, mode, J, sweep, _ptr(idx), _ptr(prob)))
    h._check(lib().cpd_synchronize(h.raw))
    return idx, prob


def cpd_sampled_mttkrp(h, mode, idx, w):
    """-> (Y (I_mode, R) float32 cuda, nnz_sel int)."""
    idx = idx.to(device=h.device, dtype=torch.int32).contiguous()
    w = w.to(device=h.device, dtype=torch.float64).contiguous()
    Y = torch.empty((h.dims[mode], h.R), dtype=torch.float32, device=h.device)
    nsel = torch.zeros(1, dtype=torch.int64, device=h.device)
    h._check(lib().cpd_sampled_mttkrp(h.raw, mode, _ptr(idx), _ptr(w), int(w.numel()), _ptr(Y), _ptr(nsel)))
    h._check(lib().cpd_synchronize(h.raw))
    return Y, int(nsel.item())


def cpd_exact_mttkrp(h, mode):
    Y = torch.empty((h.dims[mode], h.R), dtype=torch.float32, device=h.device)
    h._check(lib().cpd_exact_mttkrp(h.raw, mode, _ptr(Y)))
    h._check(lib().cpd_synchronize(h.raw))
    return Y


def cpd_gram_solve(h, mode, Y):
    """U_mode := Y G^+, renormalised; -> sigma (R,) float64 cuda."""
    Y = Y.to(device=h.device, dtype=torch.float32).contiguous()
    sigma = torch.empty(h.R, dtype=torch.float64, device=h.device)
    h._check(lib().cpd_gram_solve(h.raw, mode, _ptr(Y), _ptr(sigma)))
    h._check(lib().cpd_synchronize(h.raw))
    return sigma


def cpd_als_sweep(h, n_sweeps=1, sync=True):
    h._check(lib().cpd_als_sweep(h.raw, int(n_sweeps)))
    if sync:
        h._check(lib().cpd_synchronize(h.raw))


def cpd_fit(h):
    out = ctypes.c_double()
    h._check(lib().cpd_fit(h.raw, ctypes.byref(out)))
    return out.value


def cpd_get_factors(h, mode, out=None):
    U = out if out is not None else torch.empty((h.dims[mode], h.R), dtype=torch.float32, device=h.device)
    h._check(lib().cpd_get_factors(h.raw, mode, _ptr(U)))
    return U


def cpd_set_factors(h, mode, U):
    U = U.to(device=h.device, dtype=torch.float32).contiguous()
    h._check(lib().cpd_set_factors(h.raw, mode, _ptr(U)))


def cpd_get_sigma(h):
    s = torch.empty(h.R, dtype=torch.float64, device=h.device)
    h._check(lib().cpd_get_sigma(h.raw, _ptr(s)))
    return s


def cpd_get_arls_state(h, mode):
    ell = torch.empty(h.dims[mode], dtype=torch.float64, device=h.device)
    cdf = torch.empty(h.dims[mode], dtype=torch.float64, device=h.device)
    h._check(lib().cpd_get_arls_state(h.raw, mode, _ptr(ell), _ptr(cdf)))
    return ell, cdf


def cpd_get_gram(h, mode):
    G = torch.empty((h.R, h.R), dtype=torch.float64, device=h.device)
    h._check(lib().cpd_get_gram(h.raw, mode, _ptr(G)))
    return G


def cpd_profile(h, enable=True):
    h._check(lib().cpd_profile(h.raw, 1 if enable else 0))


def cpd_profile_read(h):
    """-> {phase: (milliseconds, launches)} accumulated since the last read."""
    ms = (ctypes.c_double * len(PHASES))()
    n = (ctypes.c_int64 * len(PHASES))()
    h._check(lib().cpd_profile_read(h.raw, ctypes.cast(ms, _P), ctypes.cast(n, _P)))
    return {p: (ms[i], n[i]) for i, p in enumerate(PHASES)}


def cpd_sweep_kernel_count(h):
    n = ctypes.c_int64()
    h._check(lib().cpd_sweep_kernel_count(h.raw, ctypes.cast(ctypes.byref(n), _P)))
    return n.value


class Batch:
    """One graph replaying an ALS round of several handles concurrently."""

    def __init__(self, raw, handles):
        self.raw, self.handles = raw, handles

    def close(self):
        if self.raw:
            lib().cpd_batch_destroy(self.raw)
            self.raw = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cpd_batch_create(handles, branches=8, stream=None):
    arr = (ctypes.c_void_p * len(handles))(*[h.raw for h in handles])
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream()
    out = ctypes.c_void_p()
    st = lib().cpd_batch_create(ctypes.cast(arr, _P), len(handles), int(branches),
                                ctypes.c_void_p(stream.cuda_stream if stream is not None else 0), ctypes.byref(out))
    if st != 0:
        raise CpdError(st, lib().cpd_last_error(None).decode())
    return Batch(out, list(handles))


def cpd_batch_sweep(b, n_sweeps=1, sync=True):
    st = lib().cpd_batch_sweep(b.raw, int(n_sweeps))
    if st == 0 and sync:
        st = lib().cpd_batch_synchronize(b.raw)
    if st != 0:
        raise CpdError(st, "cpd_batch_sweep")


def cpd_autotune(h):
    """-> (SpMM blocks per SM, STS lanes per draw, STS leaf rows F) chosen for this handle."""
    out = (ctypes.c_int32 * 3)()
    h._check(lib().cpd_autotune(h.raw, ctypes.cast(out, _P)))
    return out[0], out[1], out[2]


def cpd_sts_rescans(h):
    """Leaves of STS-CP draws rescanned in double-float since creation."""
    n = ctypes.c_int64()
    h._check(lib().cpd_sts_rescans(h.raw, ctypes.cast(ctypes.byref(n), _P)))
    return n.value


def cpd_debug_gram_wait(h, wait_cycles, suppress_mma=False):
    """Test hook: limit of the tensor-core Gram's bounded waits (cycles, 0 =
    default) and whether it issues its MMAs."""
    h._check(lib().cpd_debug_gram_wait(h.raw, int(wait_cycles), 1 if suppress_mma else 0))


def cpd_synchronize(h):
    h._check(lib().cpd_synchronize(h.raw))


def cpd_destroy(h):
    h.close()
