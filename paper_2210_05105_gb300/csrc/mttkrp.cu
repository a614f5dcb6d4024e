// Downsampled MTTKRP  Y = mat(T, n) S^T S U_{!=n}  (Eq. 7, Fig. 2 bottom) and
// the exact MTTKRP of Eq. 6.
//
// Sampled path, three launches after clearing Y and the per-call tables:
//  1. probe  (one warp per draw): KRP-row key of the draw, hash lookup of its
//     nonzero range in the mode layout, merge with earlier draws of the same
//     column (their weights add: S^T S is diagonal over KRP rows), and for
//     the first draw of a column the KRP row h = *_{k != n} U_k[i_k, :];
//  2. scan   (one block): offsets of each distinct column's nonzeros in the
//     flat list of selected nonzeros, total nnz(mat(T, n) S^T);
//  3. spmm   (persistent grid): warps take 32 consecutive selected nonzeros
//     (load balanced regardless of column lengths) and add
//     w_col * val * h_col into row i_n of Y.
#include "common.cuh"
#include <algorithm>
#include <cstring>

namespace {

struct MArgs {
  const float* U[CPD_MAX_MODES];
  int64_t dims[CPD_MAX_MODES];
  unsigned long long stride[CPD_MAX_MODES];
  int N, n, R, Rp;
  const FiberSlot* table;
  unsigned long long mask;
  const uint2* ent;
  uint32_t* dd_tag;
  double* dd_w;
  uint32_t dmask;
  uint32_t* uq_slot;
  uint32_t* uq_len;
  uint32_t* uq_off;
  float* H;
  uint32_t* counters;
  int* status;
  uint32_t uq_cap;
};

__device__ __forceinline__ bool fiber_lookup(const FiberSlot* __restrict__ table, unsigned long long mask,
                                             unsigned long long key, uint32_t& beg, uint32_t& len) {
  unsigned long long s = cpd_mix64(key) & mask;
  for (unsigned long long probe = 0; probe <= mask; ++probe) {
    const ulonglong2 raw = *reinterpret_cast<const ulonglong2*>(table + s);
    if (raw.x == key) {
      beg = (uint32_t)(raw.y & 0xffffffffull);
      len = (uint32_t)(raw.y >> 32);
      return true;
    }
    if (raw.x == CPD_EMPTY64) return false;
    s = (s + 1) & mask;
  }
  return false;
}

__global__ void probe_kernel(MArgs a, const int32_t* __restrict__ idx, const double* __restrict__ w, int64_t J) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool mine = lane < a.N && lane != a.n;
  for (int64_t j = warp; j < J; j += nwarps) {
    int32_t ik = mine ? idx[(int64_t)lane * J + j] : 0;
    bool bad = mine && (ik < 0 || (int64_t)ik >= a.dims[lane]);
    if (__any_sync(CPD_FULL, bad)) {
      if (lane == 0) cpd_set_status(a.status, CPD_ERR_OUT_OF_RANGE_INDEX);
      continue;
    }
    unsigned long long key = mine ? (unsigned long long)ik * a.stride[lane] : 0ull;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) key += __shfl_xor_sync(CPD_FULL, key, o);   // lanes 0..7 hold the modes
    key = __shfl_sync(CPD_FULL, key, 0);
    uint32_t beg = 0, len = 0, u = 0;
    int won = 0, found = 0;
    if (lane == 0) {
      found = fiber_lookup(a.table, a.mask, key, beg, len);
      if (found) {
        uint32_t s = (uint32_t)cpd_mix64((unsigned long long)beg) & a.dmask;
        for (uint32_t probe = 0; probe <= a.dmask; ++probe) {
          uint32_t old = atomicCAS(&a.dd_tag[s], CPD_EMPTY32, beg);
          if (old == CPD_EMPTY32) { won = 1; break; }
          if (old == beg) break;
          s = (s + 1) & a.dmask;
        }
        atomicAdd(&a.dd_w[s], w[j]);
        if (won) {
          u = atomicAdd(&a.counters[0], 1u);
          if (u < a.uq_cap) { a.uq_slot[u] = s; a.uq_len[u] = len; }
          else { cpd_set_status(a.status, CPD_ERR_CAPACITY); won = 0; }
        }
      }
    }
    won = __shfl_sync(CPD_FULL, won, 0);
    if (!won) continue;
    u = __shfl_sync(CPD_FULL, u, 0);
    for (int r = lane; r < a.Rp; r += 32) {
      float v = r < a.R ? 1.0f : 0.0f;
      for (int k = 0; k < a.N; ++k) {
        int32_t ikk = __shfl_sync(CPD_FULL, ik, k);
        if (k != a.n && r < a.R) v *= a.U[k][(int64_t)ikk * a.Rp + r];
      }
      a.H[(int64_t)u * a.Rp + r] = v;
    }
  }
}

// One block: exclusive offsets of the distinct columns' nonzero counts.
__global__ void __launch_bounds__(1024) scan_kernel(MArgs a, int64_t* __restrict__ out_nnz_sel) {
  __shared__ uint32_t wsum[32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const uint32_t nu = min(a.counters[0], a.uq_cap);
  const uint32_t per = (nu + 1023) / 1024;
  const uint32_t b0 = t * per;
  uint32_t s = 0;
  for (uint32_t q = 0; q < per; ++q)
    if (b0 + q < nu) s += a.uq_len[b0 + q];
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(CPD_FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t v = wsum[lane];
    uint32_t z = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(CPD_FULL, z, o);
      if (lane >= o) z += y;
    }
    wsum[lane] = z - v;
  }
  __syncthreads();
  uint32_t run = wsum[wid] + x - s;
  for (uint32_t q = 0; q < per; ++q)
    if (b0 + q < nu) { uint32_t v = a.uq_len[b0 + q]; a.uq_off[b0 + q] = run; run += v; }
  if (t == 1023) {
    a.uq_off[nu] = run;
    a.counters[1] = run;
    if (out_nnz_sel) *out_nnz_sel = (int64_t)run;
  }
}

__global__ void __launch_bounds__(256) spmm_kernel(MArgs a, float* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t nu = min(a.counters[0], a.uq_cap);
  const uint32_t total = a.counters[1];
  const int64_t nchunks = ((int64_t)total + 31) / 32;
  const int C = a.Rp / 4;                 // float4 chunks per row
  const int E = C >= 32 ? 1 : 32 / C;     // nonzeros per warp instruction
  const int sub = C >= 32 ? 0 : lane / C; // which of the E nonzeros this lane serves
  const int q = C >= 32 ? lane : lane % C;
  for (int64_t c = warp; c < nchunks; c += nwarps) {
    const int64_t p = c * 32 + lane;
    // The 32 positions of the chunk meet at most 32 consecutive segments:
    // one search finds the first, the window of their offsets goes to the
    // lanes, and each lane locates its own segment in the window by shuffles.
    uint32_t seg0 = 0;
    if (lane == 0) {
      uint32_t lo = 0, hi = nu - 1;        // last segment with offset <= c * 32
      const uint32_t p0 = (uint32_t)(c * 32);
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (a.uq_off[mid] <= p0) lo = mid; else hi = mid - 1;
      }
      seg0 = lo;
    }
    seg0 = __shfl_sync(CPD_FULL, seg0, 0);
    const uint32_t wseg = seg0 + lane;
    const uint32_t woff = wseg < nu ? a.uq_off[wseg] : 0xffffffffu;
    uint32_t loc = 0;                      // last window slot with offset <= p
#pragma unroll
    for (int b = 16; b > 0; b >>= 1) {
      const uint32_t o = __shfl_sync(CPD_FULL, woff, (int)(loc + b));
      if (o <= (uint32_t)p) loc += b;
    }
    const uint32_t segoff = __shfl_sync(CPD_FULL, woff, (int)loc);
    uint32_t row = 0, useg = 0;
    float scale = 0.0f;
    if (p < total) {
      useg = seg0 + loc;
      const uint32_t slot = a.uq_slot[useg];
      const uint32_t e = a.dd_tag[slot] + ((uint32_t)p - segoff);
      const uint2 en = a.ent[e];
      row = en.x;
      scale = (float)(a.dd_w[slot] * (double)__uint_as_float(en.y));
    }
    const int cnt = (int)((int64_t)total - c * 32 < 32 ? (int64_t)total - c * 32 : 32);
    // C lanes cover one row of Rp floats with 16-byte vector reductions, so
    // one warp instruction updates E = 32 / C selected nonzeros at once.
    for (int j0 = 0; j0 < cnt; j0 += E) {
      const int jj = j0 + sub;
      const int src = jj < 32 ? jj : 31;
      const uint32_t rj = __shfl_sync(CPD_FULL, row, src);
      const float sj = __shfl_sync(CPD_FULL, scale, src);
      const uint32_t uj = __shfl_sync(CPD_FULL, useg, src);
      if (sub < E && jj < cnt) {
        for (int qq = q; qq < C; qq += 32) {
          const float4 hv = reinterpret_cast<const float4*>(a.H + (int64_t)uj * a.Rp)[qq];
          float* yp = Y + (int64_t)rj * a.Rp + 4 * qq;
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(yp), "f"(sj * hv.x), "f"(sj * hv.y),
                       "f"(sj * hv.z), "f"(sj * hv.w)
                       : "memory");
        }
      }
    }
  }
}

// Exact MTTKRP over the input-order COO: a warp takes 32 nonzeros.
__global__ void exact_kernel(MArgs a, const int32_t* __restrict__ idx, const float* __restrict__ vals, int64_t nnz,
                             float* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c0 = warp * 32; c0 < nnz; c0 += nwarps * 32) {
    const int64_t e = c0 + lane;
    int32_t ii[CPD_MAX_MODES];
#pragma unroll
    for (int k = 0; k < CPD_MAX_MODES; ++k) ii[k] = (k < a.N && e < nnz) ? idx[(int64_t)k * nnz + e] : 0;
    const float v = e < nnz ? vals[e] : 0.0f;
    const int cnt = (int)(nnz - c0 < 32 ? nnz - c0 : 32);
    for (int j = 0; j < cnt; ++j) {
      const float vj = __shfl_sync(CPD_FULL, v, j);
      int32_t ij[CPD_MAX_MODES];
#pragma unroll
      for (int k = 0; k < CPD_MAX_MODES; ++k) ij[k] = __shfl_sync(CPD_FULL, ii[k], j);
      for (int r = lane; r < a.R; r += 32) {
        float m = vj;
        for (int k = 0; k < a.N; ++k)
          if (k != a.n) m *= a.U[k][(int64_t)ij[k] * a.Rp + r];
        atomicAdd(Y + (int64_t)ij[a.n] * a.Rp + r, m);
      }
    }
  }
}

MArgs make_args(cpd_ctx* h, int mode) {
  MArgs a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k < h->N; ++k) {
    a.U[k] = h->U[k];
    a.dims[k] = h->dims[k];
    a.stride[k] = h->mode[mode].stride[k];
  }
  a.N = h->N; a.n = mode; a.R = h->R; a.Rp = h->Rp;
  a.table = h->mode[mode].table;
  a.mask = h->mode[mode].mask;
  a.ent = h->mode[mode].ent;
  a.dd_tag = h->dd_tag; a.dd_w = h->dd_w; a.dmask = h->dedup_mask;
  a.uq_slot = h->uq_slot; a.uq_len = h->uq_len; a.uq_off = h->uq_off;
  a.H = h->H; a.counters = h->counters; a.status = h->status;
  a.uq_cap = (uint32_t)h->Jcap;
  return a;
}

}  // namespace

// Y (I_mode x Rp, internal stride) := mat(T, mode) S^T S U_{!=mode}.
cpd_status cpd_sampled_mttkrp_launch(cpd_ctx* h, int mode, const int32_t* idx, const double* w, const double* p,
                                     int64_t J, float* Y, int64_t* out_nnz_sel) {
  (void)p;
  cudaStream_t st = h->stream;
  {
    PhaseTimer pt(h, CPD_PHASE_CLEAR);
    CPD_CUDA(h, cudaMemsetAsync(Y, 0, (size_t)h->dims[mode] * h->Rp * sizeof(float), st));
    CPD_CUDA(h, cudaMemsetAsync(h->dd_tag, 0xff, ((size_t)h->dedup_mask + 1) * sizeof(uint32_t), st));
    CPD_CUDA(h, cudaMemsetAsync(h->dd_w, 0, ((size_t)h->dedup_mask + 1) * sizeof(double), st));
    CPD_CUDA(h, cudaMemsetAsync(h->counters, 0, 4 * sizeof(uint32_t), st));
  }
  MArgs a = make_args(h, mode);
  if (J > 0) {
    PhaseTimer pt(h, CPD_PHASE_PROBE);
    int grid = (int)std::min<int64_t>(cpd_ceil_div(J * 32, 256), (int64_t)h->num_sms * 16);
    probe_kernel<<<grid, 256, 0, st>>>(a, idx, w, J);
    CPD_LAUNCH(h, "probe");
  }
  {
    PhaseTimer pt(h, CPD_PHASE_SCAN);
    scan_kernel<<<1, 1024, 0, st>>>(a, out_nnz_sel);
    CPD_LAUNCH(h, "scan");
  }
  {
    PhaseTimer pt(h, CPD_PHASE_SPMM);
    spmm_kernel<<<h->num_sms * 8, 256, 0, st>>>(a, Y);
    CPD_LAUNCH(h, "spmm");
  }
  return CPD_OK;
}

cpd_status cpd_exact_mttkrp_launch(cpd_ctx* h, int mode, float* Y) {
  cudaStream_t st = h->stream;
  PhaseTimer pt(h, CPD_PHASE_EXACT);
  CPD_CUDA(h, cudaMemsetAsync(Y, 0, (size_t)h->dims[mode] * h->Rp * sizeof(float), st));
  if (h->nnz == 0) return CPD_OK;
  MArgs a = make_args(h, mode);
  exact_kernel<<<h->num_sms * 8, 256, 0, st>>>(a, h->idx, h->vals, h->nnz, Y);
  CPD_LAUNCH(h, "exact_mttkrp");
  return CPD_OK;
}
