"""cpd_sampled_mttkrp_noalloc, the allocation-free downsampled MTTKRP for
callers that cannot call cudaMalloc (code running under stream capture, code
whose device memory is owned by another allocator, latency-bound callers):
called through the C ABI, its output must match the handle-based
cpd_sampled_mttkrp within the 1e-5 relative tolerance of the MTTKRP tests,
on two calls in a row (the second call sees the first call's table)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import cpals as oc
from tests.gpu_common import cuda_ready, lib_or_build, make_case, create, gpu_factors, rel_frob

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ready(), reason="needs a CUDA GPU")]


def _noalloc(cpd, dims, idx_d, vals_d, facs, R, mode, sidx, w):
    L = cpd.lib()
    f = L.cpd_sampled_mttkrp_noalloc
    P = ctypes.c_void_p
    f.argtypes = [ctypes.c_int32, P, ctypes.c_int64, P, P, P, ctypes.c_int32, ctypes.c_int32, P, P,
                  ctypes.c_int64, P, P, P]
    f.restype = ctypes.c_int
    N = len(dims)
    dims_arr = (ctypes.c_int64 * N)(*dims)
    ptrs = (ctypes.c_void_p * N)(*[u.data_ptr() for u in facs])
    Y = torch.empty((dims[mode], R), dtype=torch.float32, device="cuda")
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    sidx = sidx.to(device="cuda", dtype=torch.int32).contiguous()
    w = w.to(device="cuda", dtype=torch.float64).contiguous()
    st = f(N, ctypes.cast(dims_arr, P), int(vals_d.numel()), P(idx_d.data_ptr()), P(vals_d.data_ptr()),
           ctypes.cast(ptrs, P), R, mode, P(sidx.data_ptr()), P(w.data_ptr()), int(w.numel()), P(Y.data_ptr()),
           P(status.data_ptr()), P(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, Y, int(status.item())


def test_noalloc_matches_handle_path_twice():
    cpd = lib_or_build()
    dims, R, J = (200, 150, 100), 8, 3000
    idx, vals, init = make_case(dims, 20000, R, seed=1001)
    h = create(cpd, dims, idx, vals, init, "arls", R, J, seed=3001)
    facs = [cpd.cpd_get_factors(h, k) for k in range(3)]
    idx_d = torch.from_numpy(idx).cuda().contiguous()
    vals_d = torch.from_numpy(vals).cuda().contiguous()
    for call, (mode, sweep) in enumerate([(1, 0), (2, 4)]):
        sidx, p = cpd.cpd_leverage_sample(h, mode, J, sweep)
        w = 1.0 / (J * p)
        Y_ref, _ = cpd.cpd_sampled_mttkrp(h, mode, sidx, w)
        st, Y, status = _noalloc(cpd, dims, idx_d, vals_d, facs, R, mode, sidx, w)
        assert st == 0 and status == 0, (call, st, status)
        assert rel_frob(Y.cpu().numpy(), Y_ref.cpu().numpy()) <= 1e-5, call
    h.close()


def test_noalloc_rejects_oversized_sample_lists():
    cpd = lib_or_build()
    dims, R = (20, 10, 5), 4
    idx, vals, init = make_case(dims, 100, R, seed=5)
    facs = [torch.from_numpy(u).cuda() for u in init]
    sidx = torch.zeros((3, 65537), dtype=torch.int32)
    w = torch.ones(65537, dtype=torch.float64)
    st, _, _ = _noalloc(cpd, dims, torch.from_numpy(idx).cuda().contiguous(), torch.from_numpy(vals).cuda(), facs, R,
                        0, sidx, w)
    assert st == 6     # CPD_ERR_CAPACITY
