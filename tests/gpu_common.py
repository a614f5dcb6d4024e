"""Shared set-up of the GPU parity tests: build the library once, make
seeded inputs, and convert between the CUDA path and the oracle."""
import numpy as np
import pytest
import torch

from paper_2210_05105_gb300 import synth


def cuda_ready():
    return torch.cuda.is_available()


def lib_or_build():
    from paper_2210_05105_gb300 import build, cpd
    import os
    if not os.path.exists(cpd.LIB_PATH):
        build.build()
    return cpd


def rel_frob(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.linalg.norm(a - b)
    n = np.linalg.norm(b)
    return d / n if n > 0 else d


def make_case(dims, nnz, R, seed, zipf=0.0, values="uniform"):
    idx, vals = synth.make_tensor(dims, nnz, seed, zipf_s=zipf, values=values)
    init = synth.init_factors(dims, R, seed + 1000)
    return idx, vals, init


def create(cpd, dims, idx, vals, init, method, R, J, seed, leaf_rows=0, on_host=False):
    dev = "cpu" if on_host else "cuda"
    return cpd.cpd_create(dims, torch.from_numpy(np.ascontiguousarray(idx)).to(dev),
                          torch.from_numpy(np.ascontiguousarray(vals)).to(dev),
                          [torch.from_numpy(u).to(dev) for u in init],
                          method=method, rank=R, samples=J, seed=seed, leaf_rows=leaf_rows)


def gpu_factors(cpd, h):
    return [cpd.cpd_get_factors(h, k).double().cpu().numpy() for k in range(h.N)]
