// Per-mode layouts of the sparse tensor (Sec. 4.3, "Tensor Storage and Local
// MTTKRP"): for each matricization mat(T, n) the nonzeros are sorted by the
// key of their column (the KRP row of U_{!=n} they pair with), so that the
// nonzeros of one sampled column form one contiguous range.  A hash index maps
// a column key to that range, which replaces the paper's sorted-column search.
#include "common.cuh"
#include <algorithm>

namespace {

__global__ void check_indices_kernel(const int32_t* __restrict__ idx, int64_t nnz, int N,
                                     const int64_t* __restrict__ dims, const float* __restrict__ vals,
                                     int* status) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; e < nnz; e += st) {
    for (int k = 0; k < N; ++k) {
      int32_t i = idx[(int64_t)k * nnz + e];
      if (i < 0 || (int64_t)i >= dims[k]) cpd_set_status(status, CPD_ERR_OUT_OF_RANGE_INDEX);
    }
    if (!isfinite(vals[e])) cpd_set_status(status, CPD_ERR_NOT_FINITE);
  }
}

// key of nonzero e for mode n; for the first layout (n == 0) the row index is
// appended below the key (full linear index), which lets one sort both group
// the columns and expose duplicate coordinates as equal neighbours.
struct KeyArgs {
  unsigned long long stride[CPD_MAX_MODES];
  int N, n;
  unsigned long long In;
  int full;
};

__global__ void make_keys_kernel(const int32_t* __restrict__ idx, int64_t nnz, KeyArgs a,
                                 unsigned long long* __restrict__ keys, uint32_t* __restrict__ perm) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; e < nnz; e += st) {
    unsigned long long key = 0;
    for (int k = 0; k < a.N; ++k)
      if (k != a.n) key += (unsigned long long)idx[(int64_t)k * nnz + e] * a.stride[k];
    if (a.full) key = key * a.In + (unsigned long long)idx[(int64_t)a.n * nnz + e];
    keys[e] = key;
    perm[e] = (uint32_t)e;
  }
}

// Two-pass ordering for tensors whose full linear index does not fit in 64
// bits: entries first sorted by i_n (keys = i_n), then re-keyed by their
// column key in that order and sorted stably, which orders them by
// (column key, i_n) as the one-pass full index would.
__global__ void row_keys_kernel(const int32_t* __restrict__ idx_n, int64_t nnz, unsigned long long* __restrict__ keys,
                                uint32_t* __restrict__ perm) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    keys[e] = (unsigned long long)idx_n[e];
    perm[e] = (uint32_t)e;
  }
}

__global__ void rekey_kernel(const int32_t* __restrict__ idx, int64_t nnz, KeyArgs a, const uint32_t* __restrict__ perm,
                             unsigned long long* __restrict__ keys) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = perm[j];
    unsigned long long key = 0;
    for (int k = 0; k < a.N; ++k)
      if (k != a.n) key += (unsigned long long)idx[(int64_t)k * nnz + e] * a.stride[k];
    keys[j] = key;
  }
}

// Duplicates after the two-pass ordering: equal column key and equal i_n.
__global__ void duplicate_check2_kernel(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ perm,
                                        const int32_t* __restrict__ idx_n, int64_t nnz, int* status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    if (e > 0 && keys[e] == keys[e - 1] && idx_n[perm[e]] == idx_n[perm[e - 1]])
      cpd_set_status(status, CPD_ERR_DUPLICATE);
}

// Summing duplicates (duplicate_policy 1): after the mode-0 ordering, run
// heads (first entry of each distinct coordinate) ...
__global__ void run_heads_kernel(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ perm,
                                 const int32_t* __restrict__ idx0, int64_t nnz, int two_pass,
                                 uint32_t* __restrict__ head) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    bool same = e > 0 && keys[e] == keys[e - 1];
    if (same && two_pass) same = idx0[perm[e]] == idx0[perm[e - 1]];
    head[e] = same ? 0u : 1u;
  }
}

// ... and one thread per run writes the coordinate and the sum of its values
// (in sorted order, so the result is deterministic) to the run's slot.
__global__ void run_sum_kernel(const uint32_t* __restrict__ head, const uint32_t* __restrict__ rid,
                               const uint32_t* __restrict__ perm, const int32_t* __restrict__ idx,
                               const float* __restrict__ vals, int64_t nnz, int N, int64_t nu,
                               int32_t* __restrict__ idx_out, float* __restrict__ vals_out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    if (!head[e]) continue;
    const int64_t r = rid[e];
    const int64_t p = perm[e];
    for (int k = 0; k < N; ++k) idx_out[(int64_t)k * nu + r] = idx[(int64_t)k * nnz + p];
    float s = vals[p];
    for (int64_t f = e + 1; f < nnz && !head[f]; ++f) s += vals[perm[f]];
    vals_out[r] = s;
  }
}

// After sorting by full linear index, equal neighbours are duplicate coordinates.
__global__ void duplicate_check_kernel(const unsigned long long* __restrict__ keys, int64_t nnz, int* status) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; e < nnz; e += st)
    if (e > 0 && keys[e] == keys[e - 1]) cpd_set_status(status, CPD_ERR_DUPLICATE);
}

__global__ void divide_keys_kernel(unsigned long long* __restrict__ keys, int64_t nnz, unsigned long long In) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; e < nnz; e += st) keys[e] = keys[e] / In;
}

// (i_n, value) of every nonzero in input order, packed into 8 bytes, so that
// the permuting gather below makes one random access per entry, not two.
__global__ void pack_entries_kernel(const int32_t* __restrict__ idx_n, const float* __restrict__ vals, int64_t nnz,
                                    uint2* __restrict__ packed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    packed[e] = make_uint2((uint32_t)idx_n[e], __float_as_uint(vals[e]));
}

__global__ void gather_entries_kernel(const uint2* __restrict__ packed, const uint32_t* __restrict__ perm, int64_t nnz,
                                      uint2* __restrict__ ent, const unsigned long long* __restrict__ keys,
                                      uint32_t* __restrict__ flags) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; e < nnz; e += st) {
    ent[e] = packed[perm[e]];
    flags[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1u : 0u;
  }
}

// Row counts of every stride-th entry: hot rows only need to be recognised
// (their slots order them by count), and counting every entry would send
// millions of atomics to the same few Zipf-hot counters.
__global__ void count_rows_kernel(const uint2* __restrict__ ent, int64_t nnz, int64_t stride,
                                  uint32_t* __restrict__ counts) {
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * stride; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x * stride)
    atomicAdd(&counts[ent[e].x], 1u);
}

// rows with at least `min_count` nonzeros -> (count, row) pairs, any order
__global__ void hot_candidates_kernel(const uint32_t* __restrict__ counts, int64_t I, uint32_t min_count,
                                      unsigned long long* __restrict__ keys, uint32_t* __restrict__ rows,
                                      uint32_t* __restrict__ ncand) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = counts[i];
    if (c >= min_count) {
      const uint32_t at = atomicAdd(ncand, 1u);
      keys[at] = c;
      rows[at] = (uint32_t)i;
    }
  }
}

// after an ascending sort of the candidates: slot s = the s-th largest count
__global__ void hot_assign_kernel(const uint32_t* __restrict__ rows_sorted, uint32_t ncand, int H,
                                  int32_t* __restrict__ hot_rows, uint32_t* __restrict__ code) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < H; s += gridDim.x * blockDim.x) {
    const uint32_t r = rows_sorted[ncand - 1 - (uint32_t)s];
    hot_rows[s] = (int32_t)r;
    code[r] = CPD_HOT_BIT | (uint32_t)s;
  }
}

__global__ void hot_mark_kernel(uint2* __restrict__ ent, int64_t nnz, const uint32_t* __restrict__ code) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = code[ent[e].x];
    if (c & CPD_HOT_BIT) ent[e].x = c;
  }
}

__global__ void fiber_begin_kernel(const uint32_t* __restrict__ flags_in, const uint32_t* __restrict__ fid,
                                   int64_t nnz, uint32_t* __restrict__ fbeg) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; e < nnz; e += st)
    if (flags_in[e]) fbeg[fid[e]] = (uint32_t)e;
}

__global__ void table_insert_kernel(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ fbeg,
                                    int64_t nf, uint32_t nnz, FiberSlot* __restrict__ table,
                                    unsigned long long mask, int* status) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; f < nf; f += st) {
    uint32_t b = fbeg[f];
    uint32_t e = (f + 1 < nf) ? fbeg[f + 1] : nnz;
    unsigned long long key = keys[b];
    unsigned long long s = cpd_mix64(key) & mask;
    bool placed = false;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
      unsigned long long old = atomicCAS(&table[s].key, CPD_EMPTY64, key);
      if (old == CPD_EMPTY64) {
        table[s].beg = b;
        table[s].len = e - b;
        placed = true;
        break;
      }
      s = (s + 1) & mask;
    }
    if (!placed) cpd_set_status(status, CPD_ERR_CAPACITY);
  }
}

int bits_for(unsigned long long maxval) {
  int b = 0;
  while (b < 64 && (maxval >> b) != 0ull) ++b;
  return b;
}

// The layout build's stream-ordered temporaries (32 bytes a nonzero): freed
// in order on the success path (before its final synchronisation, so the pool
// can return the memory), and by the destructor on every error return
// (duplicate coordinates, an allocation that fails).
struct StreamTemps {
  cudaStream_t st;
  void* p[7];
  explicit StreamTemps(cudaStream_t s) : st(s) {
    for (void*& q : p) q = nullptr;
  }
  template <typename T> cudaError_t alloc(T** q, size_t bytes, int slot) {
    const cudaError_t e = cudaMallocAsync((void**)q, bytes, st);
    if (e == cudaSuccess) p[slot] = (void*)*q;
    return e;
  }
  cudaError_t release(int slot) {
    void* q = p[slot];
    p[slot] = nullptr;
    return q ? cudaFreeAsync(q, st) : cudaSuccess;
  }
  cudaError_t release_all() {
    cudaError_t first = cudaSuccess;
    for (int k = 0; k < 7; ++k) {
      const cudaError_t e = release(k);
      if (first == cudaSuccess) first = e;
    }
    return first;
  }
  ~StreamTemps() {
    for (void* q : p)
      if (q && cudaFreeAsync(q, st) != cudaSuccess) (void)cudaGetLastError();
  }
};

}  // namespace

cpd_status cpd_build_layouts(cpd_ctx* h) {
  int64_t nnz = h->nnz;
  const int N = h->N;
  cudaStream_t st = h->stream;
  const int grid = h->num_sms * 8, thr = 256;

  StreamTemps tmp(st);
  int64_t* d_dims = nullptr;
  CPD_CUDA(h, tmp.alloc(&d_dims, sizeof(int64_t) * CPD_MAX_MODES, 6));
  CPD_CUDA(h, cudaMemcpyAsync(d_dims, h->dims, sizeof(int64_t) * N, cudaMemcpyHostToDevice, st));
  if (nnz > 0) {
    check_indices_kernel<<<grid, thr, 0, st>>>(h->idx, nnz, N, d_dims, h->vals, h->status);
    CPD_LAUNCH(h, "check_indices");
  }
  int hs = 0;
  CPD_CUDA(h, cudaMemcpyAsync(&hs, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPD_CUDA(h, cudaStreamSynchronize(st));
  CPD_CUDA(h, tmp.release(6));
  if (hs != 0) {
    return cpd_fail(h, (cpd_status)hs, hs == CPD_ERR_OUT_OF_RANGE_INDEX ? "coordinate out of range"
                                                                      : "non-finite tensor value");
  }

  unsigned long long *keys = nullptr, *keys_tmp = nullptr;
  uint32_t *perm = nullptr, *perm_tmp = nullptr, *flags = nullptr, *fid = nullptr;
  size_t m = (size_t)std::max<int64_t>(nnz, 1);
  CPD_CUDA(h, tmp.alloc(&keys, m * 8, 0));
  CPD_CUDA(h, tmp.alloc(&keys_tmp, m * 8, 1));
  CPD_CUDA(h, tmp.alloc(&perm, m * 4, 2));
  CPD_CUDA(h, tmp.alloc(&perm_tmp, m * 4, 3));
  CPD_CUDA(h, tmp.alloc(&flags, m * 4, 4));
  CPD_CUDA(h, tmp.alloc(&fid, m * 4, 5));

  // duplicate_policy 1: order by coordinate once, sum repeated coordinates
  // into a compacted COO, then build every layout from it
  if (h->opt.duplicate_policy == 1 && nnz > 1) {
    KeyArgs a;
    unsigned long long acc = 1;
    for (int k = 0; k < CPD_MAX_MODES; ++k) a.stride[k] = 0;
    for (int k = 1; k < N; ++k) { a.stride[k] = acc; acc *= (unsigned long long)h->dims[k]; }
    const bool two_pass = (long double)acc * (long double)h->dims[0] >= 18446744073709551615.0L;
    a.N = N; a.n = 0; a.In = (unsigned long long)h->dims[0]; a.full = !two_pass;
    cpd_status s;
    if (two_pass) {
      row_keys_kernel<<<grid, thr, 0, st>>>(h->idx, nnz, keys, perm);
      if ((s = cpd_radix_sort_u64(h, keys, perm, nnz, bits_for(a.In - 1ull), keys_tmp, perm_tmp)) != CPD_OK) return s;
      rekey_kernel<<<grid, thr, 0, st>>>(h->idx, nnz, a, perm, keys);
      if ((s = cpd_radix_sort_u64(h, keys, perm, nnz, bits_for(acc - 1ull), keys_tmp, perm_tmp)) != CPD_OK) return s;
    } else {
      make_keys_kernel<<<grid, thr, 0, st>>>(h->idx, nnz, a, keys, perm);
      if ((s = cpd_radix_sort_u64(h, keys, perm, nnz, bits_for(acc * a.In - 1ull), keys_tmp, perm_tmp)) != CPD_OK)
        return s;
    }
    run_heads_kernel<<<grid, thr, 0, st>>>(keys, perm, h->idx, nnz, two_pass ? 1 : 0, flags);
    CPD_LAUNCH(h, "run heads");
    uint32_t* d_total = (uint32_t*)keys_tmp;
    if ((s = cpd_scan_u32(h, flags, fid, nnz, d_total)) != CPD_OK) return s;
    uint32_t nu = 0;
    CPD_CUDA(h, cudaMemcpyAsync(&nu, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CPD_CUDA(h, cudaStreamSynchronize(st));
    if ((int64_t)nu < nnz) {
      int32_t* idx2 = nullptr;
      float* vals2 = nullptr;
      if ((s = cpd_alloc(h, &idx2, (size_t)N * nu)) != CPD_OK) return s;
      if ((s = cpd_alloc(h, &vals2, (size_t)nu)) != CPD_OK) return s;
      run_sum_kernel<<<grid, thr, 0, st>>>(flags, fid, perm, h->idx, h->vals, nnz, N, nu, idx2, vals2);
      CPD_LAUNCH(h, "run sums");
      CPD_CUDA(h, cudaStreamSynchronize(st));
      cpd_free(h, h->idx);
      cpd_free(h, h->vals);
      h->idx = idx2;
      h->vals = vals2;
      h->nnz = nu;
      nnz = nu;
    }
  }

  for (int n = 0; n < N; ++n) {
    ModeLayout& L = h->mode[n];
    KeyArgs a;
    unsigned long long acc = 1;
    for (int k = 0; k < CPD_MAX_MODES; ++k) a.stride[k] = 0;
    for (int k = 0; k < N; ++k) {
      if (k == n) continue;
      a.stride[k] = acc;
      L.stride[k] = acc;
      acc *= (unsigned long long)h->dims[k];
    }
    // mode 0 carries the duplicate check: one sort by the full linear index
    // when it fits in 64 bits, else two stable sorts (i_0, then column key)
    const bool two_pass = (n == 0) && (long double)acc * (long double)h->dims[n] >= 18446744073709551615.0L;
    a.N = N; a.n = n; a.In = (unsigned long long)h->dims[n]; a.full = (n == 0) && !two_pass;
    unsigned long long maxkey = acc - 1ull;            // largest column key
    if (a.full) maxkey = acc * a.In - 1ull;            // full linear index
    cpd_status s = cpd_alloc(h, &L.ent, m);
    if (s != CPD_OK) return s;
    if (nnz == 0) {
      L.n_fibers = 0;
      L.mask = 15;
      if ((s = cpd_alloc(h, &L.table, 16)) != CPD_OK) return s;
      CPD_CUDA(h, cudaMemsetAsync(L.table, 0xff, 16 * sizeof(FiberSlot), st));
      continue;
    }
    if (two_pass) {
      row_keys_kernel<<<grid, thr, 0, st>>>(h->idx + (int64_t)n * nnz, nnz, keys, perm);
      CPD_LAUNCH(h, "row keys");
      if ((s = cpd_radix_sort_u64(h, keys, perm, nnz, bits_for(a.In - 1ull), keys_tmp, perm_tmp)) != CPD_OK) return s;
      rekey_kernel<<<grid, thr, 0, st>>>(h->idx, nnz, a, perm, keys);
      CPD_LAUNCH(h, "rekey");
      if ((s = cpd_radix_sort_u64(h, keys, perm, nnz, bits_for(maxkey), keys_tmp, perm_tmp)) != CPD_OK) return s;
      duplicate_check2_kernel<<<grid, thr, 0, st>>>(keys, perm, h->idx + (int64_t)n * nnz, nnz, h->status);
      CPD_LAUNCH(h, "duplicate check");
    } else {
      make_keys_kernel<<<grid, thr, 0, st>>>(h->idx, nnz, a, keys, perm);
      CPD_LAUNCH(h, "make_keys");
      if ((s = cpd_radix_sort_u64(h, keys, perm, nnz, bits_for(maxkey), keys_tmp, perm_tmp)) != CPD_OK) return s;
      if (n == 0) {
        duplicate_check_kernel<<<grid, thr, 0, st>>>(keys, nnz, h->status);
        divide_keys_kernel<<<grid, thr, 0, st>>>(keys, nnz, a.In);
        CPD_LAUNCH(h, "duplicate check");
      }
    }
    uint2* packed = reinterpret_cast<uint2*>(keys_tmp);   // sort scratch, free until the scan below
    pack_entries_kernel<<<grid, thr, 0, st>>>(h->idx + (int64_t)n * nnz, h->vals, nnz, packed);
    gather_entries_kernel<<<grid, thr, 0, st>>>(packed, perm, nnz, L.ent, keys, flags);
    CPD_LAUNCH(h, "gather_entries");
    uint32_t* d_total = (uint32_t*)keys_tmp;   // scratch word
    if ((s = cpd_scan_u32(h, flags, fid, nnz, d_total)) != CPD_OK) return s;
    uint32_t nf = 0;
    CPD_CUDA(h, cudaMemcpyAsync(&nf, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CPD_CUDA(h, cudaMemcpyAsync(&hs, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CPD_CUDA(h, cudaStreamSynchronize(st));
    if (hs == CPD_ERR_DUPLICATE) return cpd_fail(h, CPD_ERR_DUPLICATE, "duplicate coordinates in the COO input");
    L.n_fibers = nf;
    uint32_t* fbeg = perm_tmp;   // reuse: the sort is done
    fiber_begin_kernel<<<grid, thr, 0, st>>>(flags, fid, nnz, fbeg);
    CPD_LAUNCH(h, "fiber_begin");
    unsigned long long cap = 16;
    while (cap < 2ull * (unsigned long long)nf) cap <<= 1;
    L.mask = cap - 1;
    if ((s = cpd_alloc(h, &L.table, cap)) != CPD_OK) return s;
    CPD_CUDA(h, cudaMemsetAsync(L.table, 0xff, cap * sizeof(FiberSlot), st));
    table_insert_kernel<<<grid, thr, 0, st>>>(keys, fbeg, nf, (uint32_t)nnz, L.table, L.mask, h->status);
    CPD_LAUNCH(h, "table_insert");

    // hot rows of mode n: count, keep rows with >= CPD_HOT_MIN_COUNT
    // nonzeros, sort by count, give the hottest hot_cap of them slots
    if (h->hot_cap > 0) {
      const int64_t In = h->dims[n];
      uint32_t* counts = nullptr;
      if ((s = cpd_alloc(h, &counts, (size_t)In)) != CPD_OK) return s;
      L.row_code = counts;
      CPD_CUDA(h, cudaMemsetAsync(counts, 0, (size_t)In * 4, st));
      CPD_CUDA(h, cudaMemsetAsync(flags, 0, sizeof(uint32_t), st));    // candidate counter
      const int64_t stride = std::max<int64_t>(1, nnz / (int64_t(1) << 22));   // about 4M counted entries
      count_rows_kernel<<<grid, thr, 0, st>>>(L.ent, nnz, stride, counts);
      const uint32_t min_count = (uint32_t)std::max<int64_t>(1, CPD_HOT_MIN_COUNT / stride);
      const unsigned rgrid = (unsigned)std::min<int64_t>(cpd_ceil_div(In, thr), (int64_t)h->num_sms * 8);
      hot_candidates_kernel<<<rgrid, thr, 0, st>>>(counts, In, min_count, keys, perm, flags);
      CPD_LAUNCH(h, "hot candidates");
      uint32_t ncand = 0;
      CPD_CUDA(h, cudaMemcpyAsync(&ncand, flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
      CPD_CUDA(h, cudaStreamSynchronize(st));
      if (ncand > 0) {
        if ((s = cpd_radix_sort_u64(h, keys, perm, ncand, 32, keys_tmp, perm_tmp)) != CPD_OK) return s;
        const int H = (int)std::min<int64_t>(ncand, h->hot_cap);
        if ((s = cpd_alloc(h, &L.hot_rows, (size_t)H)) != CPD_OK) return s;
        hot_assign_kernel<<<cpd_ceil_div(H, 256), 256, 0, st>>>(perm, ncand, H, L.hot_rows, counts);
        hot_mark_kernel<<<grid, thr, 0, st>>>(L.ent, nnz, counts);
        CPD_LAUNCH(h, "hot rows");
        L.n_hot = H;
      }
    }
  }
  CPD_CUDA(h, tmp.release_all());
  CPD_CUDA(h, cudaMemcpyAsync(&hs, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CPD_CUDA(h, cudaStreamSynchronize(st));
  if (hs != 0) return cpd_fail(h, (cpd_status)hs, "layout build failed on the device");
  return CPD_OK;
}
