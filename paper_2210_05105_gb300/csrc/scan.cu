// Device-wide exclusive scan of uint32 and a stable LSD radix sort of
// (uint64 key, uint32 payload) pairs.  Used to build the per-mode layouts
// (sort nonzeros by KRP-row key, number the fibers) and the flat work list of
// the sampled MTTKRP.
#include "common.cuh"
#include <algorithm>

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of one value per thread; returns the block total.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* excl_out, uint32_t* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(CPD_FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < THREADS / 32 ? smem[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(CPD_FULL, s, o);
      if (lane >= o) s += y;
    }
    if (lane < THREADS / 32) smem[lane] = s;
  }
  __syncthreads();
  uint32_t warp_base = warp ? smem[warp - 1] : 0;
  uint32_t total = smem[THREADS / 32 - 1];
  *excl_out = warp_base + x - v;
  __syncthreads();
  return total;
}

__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ bsum) {
  __shared__ uint32_t sm[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t e = base + i;
    if (e < n) s += in[e];
  }
  uint32_t ex;
  uint32_t tot = block_exclusive_scan<SCAN_THREADS>(s, &ex, sm);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One block of 1024 threads: exclusive scan of nb block sums in place.
__global__ void scan_single_kernel(uint32_t* bsum, int64_t nb, uint32_t* total) {
  __shared__ uint32_t sm[32];
  int64_t per = (nb + 1023) / 1024;
  int64_t b0 = (int64_t)threadIdx.x * per;
  uint32_t s = 0;
  for (int64_t i = 0; i < per; ++i) {
    int64_t e = b0 + i;
    if (e < nb) s += bsum[e];
  }
  uint32_t ex;
  uint32_t tot = block_exclusive_scan<1024>(s, &ex, sm);
  uint32_t run = ex;
  for (int64_t i = 0; i < per; ++i) {
    int64_t e = b0 + i;
    if (e < nb) { uint32_t v = bsum[e]; bsum[e] = run; run += v; }
  }
  if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void scan_down_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                                 const uint32_t* __restrict__ bsum) {
  __shared__ uint32_t sm[32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t e = base + i;
    v[i] = e < n ? in[e] : 0;
    s += v[i];
  }
  uint32_t ex;
  block_exclusive_scan<SCAN_THREADS>(s, &ex, sm);
  uint32_t run = ex + bsum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t e = base + i;
    if (e < n) { out[e] = run; run += v[i]; }
  }
}

// ---- radix sort -----------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;   // 4096 keys per block
constexpr int RS_WARPS = RS_THREADS / 32;

// n_dev (device, may be NULL): the element count when it is only known on the
// device (a captured sweep); n is then the capacity the grid was sized for.
__global__ void radix_hist_kernel(const unsigned long long* __restrict__ keys, int64_t n, int shift,
                                  uint32_t* __restrict__ counts, int64_t nblk, const uint32_t* __restrict__ n_dev) {
  __shared__ uint32_t hist[256];
  if (n_dev) n = min(n, (int64_t)*n_dev);
  hist[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int64_t e = base + (int64_t)r * RS_THREADS + threadIdx.x;
    if (e < n) atomicAdd(&hist[(keys[e] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nblk + blockIdx.x] = hist[threadIdx.x];
}

// Stable scatter: element order inside a tile is (round, thread); ranks among
// equal digits come from warp match masks, then a prefix over warps.  The
// tile is first reordered by digit in shared memory (its digit counts are the
// differences of consecutive global offsets), then written out in that order,
// so that each digit's run of the tile goes to consecutive addresses instead
// of one scattered 8-byte write per key.
constexpr size_t RS_SMEM = (size_t)RS_TILE * (sizeof(unsigned long long) + sizeof(uint32_t));
__global__ void __launch_bounds__(RS_THREADS) radix_scatter_kernel(
    const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ vin, unsigned long long* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ offs, int64_t nblk,
    const uint32_t* __restrict__ n_dev) {
  extern __shared__ unsigned long long sk[];                       // RS_TILE keys, by digit
  uint32_t* sv = reinterpret_cast<uint32_t*>(sk + RS_TILE);         // RS_TILE payloads
  __shared__ uint32_t gbase[256], lbase[256], base[256];
  __shared__ uint32_t wc[RS_WARPS][256];
  if (n_dev) n = min(n, (int64_t)*n_dev);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t tile = (int64_t)blockIdx.x * RS_TILE;
  // this tile's count of digit t: offsets are scanned in (digit, block) order
  const int64_t oi = (int64_t)t * nblk + blockIdx.x;
  const uint32_t g0 = offs[oi];
  const uint32_t g1 = oi + 1 < 256 * nblk ? offs[oi + 1] : (uint32_t)n;
  gbase[t] = g0;
  lbase[t] = g1 - g0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) wc[w][t] = 0;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {          // inclusive scan of the counts
    const uint32_t v = t >= o ? lbase[t - o] : 0u;
    __syncthreads();
    lbase[t] += v;
    __syncthreads();
  }
  lbase[t] -= g1 - g0;                          // exclusive: the digit's first slot in the tile
  base[t] = lbase[t];
  __syncthreads();
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int64_t e = tile + (int64_t)r * RS_THREADS + t;
    bool valid = e < n;
    unsigned long long k = valid ? kin[e] : 0ull;
    uint32_t v = valid ? vin[e] : 0u;
    uint32_t d = valid ? (uint32_t)((k >> shift) & 255u) : 256u;
    uint32_t peers = __match_any_sync(CPD_FULL, d);
    uint32_t rank = __popc(peers & lt_mask);
    int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wc[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = base[t];
#pragma unroll
      for (int w = 0; w < RS_WARPS; ++w) { uint32_t c = wc[w][t]; wc[w][t] = run; run += c; }
      base[t] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = wc[warp][d] + rank;   // slot in the tile
      sk[pos] = k;
      sv[pos] = v;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) wc[w][t] = 0;
    __syncthreads();
  }
  const int64_t tn = n - tile < RS_TILE ? n - tile : RS_TILE;
  for (int i = t; i < (int)tn; i += RS_THREADS) {
    const unsigned long long k = sk[i];
    const uint32_t d = (uint32_t)((k >> shift) & 255u);
    const uint32_t pos = gbase[d] + ((uint32_t)i - lbase[d]);
    kout[pos] = k;
    vout[pos] = sv[i];
  }
}

}  // namespace

// Exclusive scan of n uint32 values (in may equal out); *total (device, may be
// NULL) receives the sum.  Sums must fit in 32 bits.
cpd_status cpd_scan_u32(cpd_ctx* h, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total) {
  if (n <= 0) {
    if (total) CPD_CUDA(h, cudaMemsetAsync(total, 0, sizeof(uint32_t), h->stream));
    return CPD_OK;
  }
  int64_t nb = cpd_ceil_div(n, SCAN_TILE);
  uint32_t* bsum = nullptr;
  CPD_CUDA(h, cudaMallocAsync((void**)&bsum, nb * sizeof(uint32_t), h->stream));
  scan_reduce_kernel<<<(unsigned)nb, SCAN_THREADS, 0, h->stream>>>(in, n, bsum);
  scan_single_kernel<<<1, 1024, 0, h->stream>>>(bsum, nb, total);
  scan_down_kernel<<<(unsigned)nb, SCAN_THREADS, 0, h->stream>>>(in, out, n, bsum);
  CPD_LAUNCH(h, "scan kernels");
  CPD_CUDA(h, cudaFreeAsync(bsum, h->stream));
  return CPD_OK;
}

// The same scan with caller scratch bsum of ceil(n / 2048) words (no
// allocation, so it can be captured in a graph).
int64_t cpd_scan_u32_scratch(int64_t n) { return cpd_ceil_div(std::max<int64_t>(n, 1), SCAN_TILE); }
cpd_status cpd_scan_u32_buf(cpd_ctx* h, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                            uint32_t* bsum, cudaStream_t st) {
  if (n <= 0) {
    if (total) CPD_CUDA(h, cudaMemsetAsync(total, 0, sizeof(uint32_t), st));
    return CPD_OK;
  }
  const int64_t nb = cpd_ceil_div(n, SCAN_TILE);
  scan_reduce_kernel<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, bsum);
  scan_single_kernel<<<1, 1024, 0, st>>>(bsum, nb, total);
  scan_down_kernel<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, bsum);
  CPD_LAUNCH(h, "scan kernels");
  return CPD_OK;
}

// Stable LSD radix sort of (keys, vals) on the low `bits` bits of the keys.
// The scatter's shared-memory limit (its 48 KB tile beside its static
// arrays); called at set-up, outside any stream capture.
cpd_status cpd_radix_init(cpd_ctx* h) { return cpd_smem_attr(h, (const void*)radix_scatter_kernel, 64 * 1024); }

// The sorted result ends in keys/vals; keys_tmp/vals_tmp are scratch of n.
cpd_status cpd_radix_sort_u64(cpd_ctx* h, unsigned long long* keys, uint32_t* vals, int64_t n, int bits,
                              unsigned long long* keys_tmp, uint32_t* vals_tmp) {
  if (n <= 1 || bits <= 0) return CPD_OK;
  {
    const cpd_status si = cpd_radix_init(h);
    if (si != CPD_OK) return si;
  }
  int64_t nblk = cpd_ceil_div(n, RS_TILE);
  uint32_t* counts = nullptr;
  CPD_CUDA(h, cudaMallocAsync((void**)&counts, (size_t)nblk * 256 * sizeof(uint32_t), h->stream));
  unsigned long long *ka = keys, *kb = keys_tmp;
  uint32_t *va = vals, *vb = vals_tmp;
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    int shift = 8 * p;
    radix_hist_kernel<<<(unsigned)nblk, RS_THREADS, 0, h->stream>>>(ka, n, shift, counts, nblk, nullptr);
    CPD_LAUNCH(h, "radix_hist");
    cpd_status s = cpd_scan_u32(h, counts, counts, nblk * 256, nullptr);
    if (s != CPD_OK) return s;
    radix_scatter_kernel<<<(unsigned)nblk, RS_THREADS, RS_SMEM, h->stream>>>(ka, va, kb, vb, n, shift, counts, nblk,
                                                                             nullptr);
    CPD_LAUNCH(h, "radix_scatter");
    unsigned long long* tk = ka; ka = kb; kb = tk;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  if (ka != keys) {
    CPD_CUDA(h, cudaMemcpyAsync(keys, ka, n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, h->stream));
    CPD_CUDA(h, cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, h->stream));
  }
  CPD_CUDA(h, cudaFreeAsync(counts, h->stream));
  return CPD_OK;
}

// The same sort for a count known only on the device (*n_dev <= cap): grids
// are sized for cap, blocks past the count exit at once, and the result is
// left in whichever buffer pair the last pass wrote (*out_k, *out_v), so no
// copy of cap elements is needed.  counts: 256 * ceil(cap / 4096) words.
cpd_status cpd_radix_sort_u64_dev(cpd_ctx* h, unsigned long long* keys, uint32_t* vals, int64_t cap,
                                  const uint32_t* n_dev, int bits, unsigned long long* keys_tmp, uint32_t* vals_tmp,
                                  uint32_t* counts, unsigned long long** out_k, uint32_t** out_v) {
  unsigned long long *ka = keys, *kb = keys_tmp;
  uint32_t *va = vals, *vb = vals_tmp;
  if (cap > 1 && bits > 0) {
    const int64_t nblk = cpd_ceil_div(cap, RS_TILE);
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
      const int shift = 8 * p;
      radix_hist_kernel<<<(unsigned)nblk, RS_THREADS, 0, h->stream>>>(ka, cap, shift, counts, nblk, n_dev);
      CPD_LAUNCH(h, "radix_hist");
      cpd_status s = cpd_scan_u32(h, counts, counts, nblk * 256, nullptr);
      if (s != CPD_OK) return s;
      radix_scatter_kernel<<<(unsigned)nblk, RS_THREADS, RS_SMEM, h->stream>>>(ka, va, kb, vb, cap, shift, counts,
                                                                               nblk, n_dev);
      CPD_LAUNCH(h, "radix_scatter");
      unsigned long long* tk = ka; ka = kb; kb = tk;
      uint32_t* tv = va; va = vb; vb = tv;
    }
  }
  *out_k = ka;
  *out_v = va;
  return CPD_OK;
}

