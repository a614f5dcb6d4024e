"""The device-side input generator (libzipfgen) used for the billion-scale
workload, against a numpy statement of the same recipe on a small case: the
same Philox uniforms (key (seed, 7), counter (d, 0, 0, 0)), the same
truncated-Zipf inverse CDF and permutations, the earliest nnz distinct
coordinates in first-draw order, and log(1 + Poisson(3) | >= 1) values."""
import numpy as np
import pytest
import torch

from oracle import philox as ph
from paper_2210_05105_gb300 import synth
from tests.gpu_common import cuda_ready, lib_or_build

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ready(), reason="needs a CUDA GPU")]


def _reference(dims, nnz, seed, s):
    rng = np.random.Generator(np.random.PCG64(seed))
    perms = [rng.permutation(I) for I in dims]
    tables = [synth._zipf_table(I, s) for I in dims]
    mult = np.cumprod([1] + list(dims[:-1])).astype(np.uint64)
    M = 4096
    while True:
        d = np.arange(M, dtype=np.uint64)
        w = ph.philox4x64([d, np.zeros_like(d), np.zeros_like(d), np.zeros_like(d)],
                          [np.full(M, seed, dtype=np.uint64), np.full(M, 7, dtype=np.uint64)])
        coords = []
        for k, I in enumerate(dims):
            u = ph.uniform01(w[k])
            r = np.minimum(np.searchsorted(tables[k], u, side="right"), I - 1)
            coords.append(perms[k][r])
        key = np.zeros(M, dtype=np.uint64)
        for k in range(len(dims)):
            key += coords[k].astype(np.uint64) * mult[k]
        _, first = np.unique(key, return_index=True)
        if first.size >= nnz:
            keep = np.sort(first)[:nnz]
            idx = np.stack([c[keep] for c in coords]).astype(np.int32)
            break
        M *= 2
    e = np.arange(nnz, dtype=np.uint64)
    u = ph.uniform01(ph.philox4x64([e, np.zeros_like(e), np.zeros_like(e), np.zeros_like(e)],
                                   [np.full(nnz, seed, dtype=np.uint64), np.full(nnz, 8, dtype=np.uint64)])[0])
    cdf = synth.poisson_ge1_cdf(3.0)
    x = np.minimum(np.searchsorted(cdf, u, side="right"), cdf.size - 1) + 1
    return idx, np.log1p(x.astype(np.float64)).astype(np.float32), int(keep[-1]) + 1


@pytest.mark.parametrize("dims,nnz,s", [((300, 200, 150), 20000, 1.3), ((97, 50, 64, 30), 30000, 1.1),
                                        ((5000, 40, 7000), 100000, 1.3)])
def test_device_generator_matches_numpy_recipe(dims, nnz, s):
    lib_or_build()
    idx, vals, used = synth.make_tensor_device(dims, nnz, 123, s)
    ri, rv, rused = _reference(dims, nnz, 123, s)
    assert used == rused
    assert np.array_equal(idx.cpu().numpy(), ri)
    assert np.allclose(vals.cpu().numpy(), rv, rtol=1e-7, atol=0)
    key = np.zeros(nnz, dtype=np.uint64)
    m = 1
    for k, I in enumerate(dims):
        key += ri[k].astype(np.uint64) * np.uint64(m)
        m *= I
    assert np.unique(key).size == nnz
