// Seeded synthetic COO tensors on the device (input generator; none of the
// CP-ALS arithmetic lives here).  Built as its own library, libzipfgen.so,
// separate from libcpd.so.
//
// Recipe (the device form of the generator used for the small workloads):
// draw d = 0, 1, 2, ... picks, for each mode k < N <= 4, the uniform
// u_k = top 53 bits of word k of Philox4x64-10 with key (seed, 7) and counter
// (d, 0, 0, 0), times 2^-53; rank_k = the smallest r with table_k[r] > u_k
// (table_k the running sums of the truncated Zipf law, clamped to I_k - 1)
// and i_k = perm_k[rank_k].  The first draw of a coordinate keeps it; exactly
// nnz distinct coordinates are returned, those with the earliest first draws,
// in the order of their first draws.  Values: log(1 + x) with x drawn from
// Poisson(lambda) conditioned on x >= 1 (Poisson redrawn at zero), by inverse
// CDF of the uniform of Philox4x64-10 key (seed, 8), counter (position, 0, 0, 0).
//
// Dedup: an open-addressing set of 64-bit linear keys in device memory; each
// cell keeps the smallest draw index that hit it (atomicMin), so the result
// does not depend on the order in which threads insert.
#include <cuda_runtime.h>
#include <stdint.h>
#include <algorithm>
#include <vector>

namespace {

constexpr unsigned long long EMPTY = 0xffffffffffffffffull;

__device__ __forceinline__ void philox(unsigned long long c[4], unsigned long long k0, unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    const unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const unsigned long long x0 = hi1 ^ c[1] ^ k0, x2 = hi0 ^ c[3] ^ k1;
    c[0] = x0; c[1] = lo1; c[2] = x2; c[3] = lo0;
  }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

struct GenArgs {
  const double* table[4];
  const int32_t* perm[4];
  int64_t dims[4];
  unsigned long long mult[4];
  int N;
  unsigned long long seed;
};

__global__ void insert_kernel(GenArgs a, unsigned long long d0, unsigned long long count,
                              unsigned long long* __restrict__ keys, unsigned long long* __restrict__ first,
                              unsigned long long mask, unsigned long long* __restrict__ distinct, int* __restrict__ full) {
  for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < count;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long d = d0 + t;
    unsigned long long c[4] = {d, 0ull, 0ull, 0ull};
    philox(c, a.seed, 7ull);
    unsigned long long key = 0;
    for (int k = 0; k < a.N; ++k) {
      const double u = (double)(c[k] >> 11) * 0x1.0p-53;
      const double* tb = a.table[k];
      int64_t lo = 0, hi = a.dims[k];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (tb[mid] > u) hi = mid; else lo = mid + 1;
      }
      if (lo > a.dims[k] - 1) lo = a.dims[k] - 1;
      key += (unsigned long long)a.perm[k][lo] * a.mult[k];
    }
    unsigned long long s = mix64(key) & mask;
    bool placed = false;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
      const unsigned long long old = atomicCAS(keys + s, EMPTY, key);
      if (old == EMPTY || old == key) {
        if (old == EMPTY) atomicAdd(distinct, 1ull);
        atomicMin(first + s, d);
        placed = true;
        break;
      }
      s = (s + 1) & mask;
    }
    if (!placed) atomicExch(full, 1);
  }
}

// bit (first - d0) for every cell first drawn in [d0, d1)
__global__ void mark_window_kernel(const unsigned long long* __restrict__ keys, const unsigned long long* __restrict__ first,
                                   unsigned long long cap, unsigned long long d0, unsigned long long d1,
                                   unsigned long long* __restrict__ bits) {
  for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap;
       s += (unsigned long long)gridDim.x * blockDim.x) {
    if (keys[s] == EMPTY) continue;
    const unsigned long long f = first[s];
    if (f >= d0 && f < d1) atomicOr(bits + ((f - d0) >> 6), 1ull << ((f - d0) & 63));
  }
}

// bit d for every kept cell (first draw d < T)
__global__ void mark_kept_kernel(const unsigned long long* __restrict__ keys, const unsigned long long* __restrict__ first,
                                 unsigned long long cap, unsigned long long T, unsigned long long* __restrict__ bits) {
  for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap;
       s += (unsigned long long)gridDim.x * blockDim.x) {
    if (keys[s] == EMPTY) continue;
    const unsigned long long f = first[s];
    if (f < T) atomicOr(bits + (f >> 6), 1ull << (f & 63));
  }
}

constexpr int SCAN_B = 1024;

// popcount of each word, summed per block of SCAN_B words
__global__ void block_count_kernel(const unsigned long long* __restrict__ bits, int64_t nw,
                                   unsigned long long* __restrict__ bsum) {
  __shared__ unsigned long long red[32];
  const int64_t w = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  unsigned long long c = w < nw ? (unsigned long long)__popcll(bits[w]) : 0ull;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int i = 0; i < SCAN_B / 32; ++i) t += red[i];
    bsum[blockIdx.x] = t;
  }
}

// exclusive prefix of set bits before each word (block offsets from the host scan)
__global__ void word_prefix_kernel(const unsigned long long* __restrict__ bits, int64_t nw,
                                   const unsigned long long* __restrict__ boff, unsigned long long* __restrict__ wpre) {
  __shared__ unsigned long long ws[32];
  const int64_t w = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned long long c = w < nw ? (unsigned long long)__popcll(bits[w]) : 0ull;
  unsigned long long x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  unsigned long long base = boff[blockIdx.x];
  for (int i = 0; i < wid; ++i) base += ws[i];
  if (w < nw) wpre[w] = base + x - c;
}

__global__ void emit_kernel(const unsigned long long* __restrict__ keys, const unsigned long long* __restrict__ first,
                            unsigned long long cap, unsigned long long T, const unsigned long long* __restrict__ bits,
                            const unsigned long long* __restrict__ wpre, GenArgs a, int64_t nnz,
                            int32_t* __restrict__ idx_out) {
  for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < cap;
       s += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long key = keys[s];
    if (key == EMPTY) continue;
    const unsigned long long f = first[s];
    if (f >= T) continue;
    const unsigned long long below = bits[f >> 6] & ((1ull << (f & 63)) - 1ull);
    const unsigned long long pos = wpre[f >> 6] + (unsigned long long)__popcll(below);
    if (pos >= (unsigned long long)nnz) continue;
    unsigned long long rem = key;
    for (int k = a.N - 1; k >= 0; --k) {
      const unsigned long long ik = rem / a.mult[k];
      rem -= ik * a.mult[k];
      idx_out[(int64_t)k * nnz + (int64_t)pos] = (int32_t)ik;
    }
  }
}

__global__ void values_kernel(int64_t nnz, unsigned long long seed, const double* __restrict__ cdf, int ncdf,
                              float* __restrict__ vals) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long c[4] = {(unsigned long long)e, 0ull, 0ull, 0ull};
    philox(c, seed, 8ull);
    const double u = (double)(c[0] >> 11) * 0x1.0p-53;
    int x = 0;
    while (x < ncdf - 1 && !(cdf[x] > u)) ++x;     // smallest x with cdf[x] > u
    vals[e] = (float)log1p((double)(x + 1));
  }
}

}  // namespace

extern "C" {

// Returns 0 on success; 1 bad arguments; 2 CUDA error; 3 the draw budget ran
// out before nnz distinct coordinates were found.  *draws_used (host) = T,
// the number of draws whose first hits were kept.
int zg_generate(int N, const int64_t* dims, const double* const* tables, const int32_t* const* perms,
                uint64_t seed, int64_t nnz, int64_t max_draws, int32_t* idx_out, int64_t* draws_used,
                void* stream) {
  if (N < 1 || N > 4 || nnz < 1 || !dims || !tables || !perms || !idx_out) return 1;
  cudaStream_t st = (cudaStream_t)stream;
  GenArgs a;
  a.N = N;
  a.seed = seed;
  unsigned long long acc = 1;
  long double prod = 1.0L;
  for (int k = 0; k < 4; ++k) { a.table[k] = nullptr; a.perm[k] = nullptr; a.dims[k] = 1; a.mult[k] = 0; }
  for (int k = 0; k < N; ++k) {
    if (dims[k] < 1 || dims[k] > 0x7fffffffll) return 1;
    a.table[k] = tables[k];
    a.perm[k] = perms[k];
    a.dims[k] = dims[k];
    a.mult[k] = acc;
    acc *= (unsigned long long)dims[k];
    prod *= (long double)dims[k];
  }
  if (prod >= 18446744073709551615.0L || (long double)nnz > prod) return 1;
  unsigned long long cap = 1024;
  while ((long double)cap < 1.6L * (long double)nnz) cap <<= 1;
  const unsigned long long mask = cap - 1;
  unsigned long long *keys = nullptr, *first = nullptr, *distinct = nullptr;
  int* full = nullptr;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMalloc(&keys, cap * 8) != cudaSuccess || cudaMalloc(&first, cap * 8) != cudaSuccess ||
      cudaMalloc(&distinct, 8) != cudaSuccess || cudaMalloc(&full, 4) != cudaSuccess) {
    cudaFree(keys); cudaFree(first); cudaFree(distinct); cudaFree(full);
    cudaGetLastError();
    return 2;
  }
  int rc = 0;
  cudaMemsetAsync(keys, 0xff, cap * 8, st);
  cudaMemsetAsync(first, 0xff, cap * 8, st);
  cudaMemsetAsync(distinct, 0, 8, st);
  cudaMemsetAsync(full, 0, 4, st);
  const unsigned long long chunk = std::max<unsigned long long>(1ull << 16, (unsigned long long)nnz / 8);
  unsigned long long d0 = 0, have = 0, before = 0;
  const unsigned grid = (unsigned)sms * 16;
  while (true) {
    if ((long long)d0 >= max_draws) { rc = 3; break; }
    insert_kernel<<<grid, 256, 0, st>>>(a, d0, chunk, keys, first, mask, distinct, full);
    int hfull = 0;
    cudaMemcpyAsync(&have, distinct, 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&hfull, full, 4, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = 2; break; }
    if (hfull) { rc = 2; break; }
    if (have >= (unsigned long long)nnz) break;
    before = have;
    d0 += chunk;
  }
  unsigned long long T = 0;
  unsigned long long *bits = nullptr, *bsum = nullptr, *wpre = nullptr;
  if (rc == 0) {
    // threshold inside the last chunk: the (nnz - before)-th new cell by first draw
    const unsigned long long need = (unsigned long long)nnz - before;
    const unsigned long long nwc = (chunk + 63) / 64;
    std::vector<unsigned long long> hb(nwc);
    if (cudaMalloc(&bits, nwc * 8) != cudaSuccess) rc = 2;
    if (rc == 0) {
      cudaMemsetAsync(bits, 0, nwc * 8, st);
      mark_window_kernel<<<grid, 256, 0, st>>>(keys, first, cap, d0, d0 + chunk, bits);
      cudaMemcpyAsync(hb.data(), bits, nwc * 8, cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) rc = 2;
      cudaFree(bits);
      bits = nullptr;
    }
    if (rc == 0) {
      unsigned long long seen = 0;
      for (unsigned long long w = 0; w < nwc && T == 0; ++w) {
        const unsigned long long c = (unsigned long long)__builtin_popcountll(hb[w]);
        if (seen + c >= need) {
          unsigned long long x = hb[w];
          for (int b = 0; b < 64; ++b) {
            if ((x >> b) & 1ull) {
              if (++seen == need) { T = d0 + w * 64 + (unsigned long long)b + 1ull; break; }
            }
          }
        } else {
          seen += c;
        }
      }
      if (T == 0) rc = 2;
    }
  }
  if (rc == 0) {
    const int64_t nw = (int64_t)((T + 63) / 64);
    const int64_t nb = (nw + SCAN_B - 1) / SCAN_B;
    if (cudaMalloc(&bits, (size_t)nw * 8) != cudaSuccess || cudaMalloc(&bsum, (size_t)nb * 8) != cudaSuccess ||
        cudaMalloc(&wpre, (size_t)nw * 8) != cudaSuccess) {
      rc = 2;
    } else {
      cudaMemsetAsync(bits, 0, (size_t)nw * 8, st);
      mark_kept_kernel<<<grid, 256, 0, st>>>(keys, first, cap, T, bits);
      block_count_kernel<<<(unsigned)nb, SCAN_B, 0, st>>>(bits, nw, bsum);
      std::vector<unsigned long long> hs((size_t)nb);
      cudaMemcpyAsync(hs.data(), bsum, (size_t)nb * 8, cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) rc = 2;
      if (rc == 0) {
        unsigned long long run = 0;
        for (auto& v : hs) { const unsigned long long c = v; v = run; run += c; }
        if (run != (unsigned long long)nnz) rc = 2;
        cudaMemcpyAsync(bsum, hs.data(), (size_t)nb * 8, cudaMemcpyHostToDevice, st);
        word_prefix_kernel<<<(unsigned)nb, SCAN_B, 0, st>>>(bits, nw, bsum, wpre);
        emit_kernel<<<grid, 256, 0, st>>>(keys, first, cap, T, bits, wpre, a, nnz, idx_out);
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = 2;
      }
    }
  }
  if (cudaGetLastError() != cudaSuccess && rc == 0) rc = 2;
  cudaFree(bits); cudaFree(bsum); cudaFree(wpre);
  cudaFree(keys); cudaFree(first); cudaFree(distinct); cudaFree(full);
  if (draws_used) *draws_used = (int64_t)T;
  return rc;
}

// vals[e] = log(1 + x_e), x_e ~ Poisson conditioned on x >= 1, by inverse CDF
// over cdf[0..ncdf) (device, cdf[x - 1] = P(X <= x | X >= 1), last entry 1).
int zg_values_logpoisson(int64_t nnz, uint64_t seed, const double* cdf, int ncdf, float* vals, void* stream) {
  if (nnz < 0 || !cdf || ncdf < 1 || (nnz > 0 && !vals)) return 1;
  if (nnz == 0) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  values_kernel<<<(unsigned)sms * 16, 256, 0, (cudaStream_t)stream>>>(nnz, seed, cdf, ncdf, vals);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
