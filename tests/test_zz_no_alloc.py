"""cpd_sampled_mttkrp_noalloc, the allocation-free downsampled MTTKRP for
callers that cannot call cudaMalloc (code whose device memory is owned by
another allocator, latency-bound callers):
called through the C ABI, its output must match the handle-based
cpd_sampled_mttkrp and the FP64 oracle within the 1e-5 relative tolerance of
the MTTKRP tests, on two calls in a row (the second call sees the first
call's table).  Out-of-range draws and out-of-range nonzero coordinates are
skipped and reported in the status word; J = 0 gives Y = 0."""
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
        Yo = oc.sampled_mttkrp(idx, vals, dims, [f.double().cpu().numpy() for f in facs], mode,
                               sidx.cpu().numpy(), w.cpu().numpy())
        assert rel_frob(Y.cpu().numpy(), Yo) <= 1e-5, call
    h.close()


def _case():
    dims, R, J = (60, 50, 40), 6, 500
    idx, vals, init = make_case(dims, 5000, R, seed=77)
    rng = np.random.default_rng(78)
    sidx = np.stack([rng.integers(0, d, J) for d in dims]).astype(np.int32)
    w = rng.uniform(0.5, 2.0, J)
    return dims, R, idx, vals, [u.astype(np.float32) for u in init], sidx, w


def test_noalloc_out_of_range_draw_is_skipped():
    cpd = lib_or_build()
    dims, R, idx, vals, init, sidx, w = _case()
    mode = 0
    bad = sidx.copy()
    bad[1, 7] = dims[1]            # one draw past the end of mode 1
    facs = [torch.from_numpy(u).cuda() for u in init]
    st, Y, status = _noalloc(cpd, dims, torch.from_numpy(idx).cuda().contiguous(),
                             torch.from_numpy(vals).cuda().contiguous(), facs, R, mode,
                             torch.from_numpy(bad), torch.from_numpy(w))
    assert st == 0 and status == 1
    keep = np.ones(w.shape[0], dtype=bool)
    keep[7] = False
    Yo = oc.sampled_mttkrp(idx, vals, dims, [u.astype(np.float64) for u in init], mode, sidx[:, keep], w[keep])
    assert rel_frob(Y.cpu().numpy(), Yo) <= 1e-5


def test_noalloc_out_of_range_coordinate_is_skipped():
    cpd = lib_or_build()
    dims, R, idx, vals, init, sidx, w = _case()
    mode = 2
    # make every nonzero hit a drawn column, then corrupt the mode-n index of one
    idx = idx.copy()
    idx[0, :500], idx[1, :500] = sidx[0], sidx[1]
    clean = oc.sampled_mttkrp(idx[:, 1:], vals[1:], dims, [u.astype(np.float64) for u in init], mode, sidx, w)
    bad = idx.copy()
    bad[mode, 0] = dims[mode] + 5
    facs = [torch.from_numpy(u).cuda() for u in init]
    facs[mode] = torch.zeros(1, dtype=torch.float32, device="cuda")   # never read
    st, Y, status = _noalloc(cpd, dims, torch.from_numpy(np.ascontiguousarray(bad)).cuda(),
                             torch.from_numpy(vals).cuda().contiguous(), facs, R, mode,
                             torch.from_numpy(sidx), torch.from_numpy(w))
    assert st == 0 and status == 2
    assert rel_frob(Y.cpu().numpy(), clean) <= 1e-5


def test_noalloc_no_draws_gives_zero():
    cpd = lib_or_build()
    dims, R, idx, vals, init, _, _ = _case()
    facs = [torch.from_numpy(u).cuda() for u in init]
    st, Y, status = _noalloc(cpd, dims, torch.from_numpy(idx).cuda().contiguous(),
                             torch.from_numpy(vals).cuda().contiguous(), facs, R, 1,
                             torch.zeros((3, 0), dtype=torch.int32), torch.zeros(0, dtype=torch.float64))
    assert st == 0 and status == 0
    assert float(Y.abs().max()) == 0.0


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
