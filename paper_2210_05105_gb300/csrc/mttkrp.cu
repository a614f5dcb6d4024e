// Downsampled MTTKRP  Y = mat(T, n) S^T S U_{!=n}  (Eq. 7, Fig. 3 bottom) and
// the exact MTTKRP of Eq. 6.
//
// Sampled path, two launches after clearing Y and the per-call tables:
//  1. probe  (one lane per draw): KRP-row key of the draw, hash lookup of its
//     nonzero range in the mode layout, merge with earlier draws of the same
//     column (their weights add: S^T S is diagonal over KRP rows); the first
//     draw of a column reserves its place in the flat list of selected
//     nonzeros and writes the KRP row h = *_{k != n} U_k[i_k, :];
//  2. spmm   (persistent grid): warps take 32 consecutive selected nonzeros
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
  float* dd_w;
  uint32_t dmask;
  uint32_t* uq_slot;
  uint32_t* chunk_seg;
  uint32_t* uq_off;
  uint32_t* uq_beg;
  float* H;
  uint32_t* counters;
  int* status;
  uint32_t uq_cap;
  const int32_t* hot_rows;   // row of each hot slot (entries carry CPD_HOT_BIT | slot)
  int n_hot;                 // hot slots accumulated in shared memory by this launch
  const uint32_t* row_code;  // per row of mode n: CPD_HOT_BIT | slot for hot rows (exact MTTKRP)
  uint32_t* dslot;           // deterministic mode: each draw's dedup slot (no weight atomics), else null
  uint32_t* uq_len;          // deterministic mode: nonzeros of each distinct column, else null
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

// One lane per draw: KRP-row key, hash lookup of the column's nonzero range,
// merge with earlier draws of the same column (weights add: S^T S is
// diagonal over KRP rows).  The first draw of a column takes, with one 64-bit
// atomic, both its index u among the distinct columns and the offset of its
// nonzeros in the flat list of selected nonzeros (so no separate scan).  The
// warp then writes the KRP row h_u = *_{k != n} U_k[i_k, :] of each such
// column and marks the 32-nonzero chunks that start inside its range.
__global__ void probe_kernel(MArgs a, const int32_t* __restrict__ idx, const double* __restrict__ w, int64_t J) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(a.counters);
  for (int64_t j0 = warp * 32; j0 < J; j0 += nwarps * 32) {
    const int64_t j = j0 + lane;
    const bool valid = j < J;
    int32_t ik[CPD_MAX_MODES];
    unsigned long long key = 0;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < CPD_MAX_MODES; ++k) {
      ik[k] = 0;
      if (k < a.N && k != a.n && valid) {
        ik[k] = idx[(int64_t)k * J + j];
        if (ik[k] < 0 || (int64_t)ik[k] >= a.dims[k]) bad = true;
        key += (unsigned long long)(bad ? 0 : ik[k]) * a.stride[k];
      }
    }
    if (bad) cpd_set_status(a.status, CPD_ERR_OUT_OF_RANGE_INDEX);
    uint32_t beg = 0, len = 0, u = 0, off = 0;
    bool won = false;
    uint32_t myslot = CPD_EMPTY32;
    if (valid && !bad && fiber_lookup(a.table, a.mask, key, beg, len)) {
      uint32_t sl = (uint32_t)cpd_mix64((unsigned long long)beg) & a.dmask;
      for (uint32_t probe = 0; probe <= a.dmask; ++probe) {
        const uint32_t old = atomicCAS(&a.dd_tag[sl], CPD_EMPTY32, beg);
        if (old == CPD_EMPTY32) { won = true; break; }
        if (old == beg) break;
        sl = (sl + 1) & a.dmask;
      }
      if (!a.dslot) atomicAdd(&a.dd_w[sl], (float)w[j]);   // deterministic mode: summed in draw order later
      myslot = sl;
      if (won) u = sl;                      // the slot, until the index is known
    }
    if (a.dslot && valid) a.dslot[j] = myslot;
    // One 64-bit atomic per warp reserves the warp's winners' indices and
    // nonzero ranges at once; lanes place themselves by a prefix sum.
    const unsigned wm = __ballot_sync(CPD_FULL, won);
    if (wm) {
      const uint32_t mylen = won ? len : 0u;
      uint32_t incl = mylen;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(CPD_FULL, incl, o);
        if (lane >= o) incl += t;
      }
      const uint32_t tot = __shfl_sync(CPD_FULL, incl, 31);
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(ctr, ((unsigned long long)__popc(wm) << 32) | (unsigned long long)tot);
      base = __shfl_sync(CPD_FULL, base, 0);
      if (won) {
        const uint32_t sl = u;
        u = (uint32_t)(base >> 32) + (uint32_t)__popc(wm & ((1u << lane) - 1u));
        off = (uint32_t)(base & 0xffffffffull) + incl - mylen;
        if (u < a.uq_cap) {
          a.uq_slot[u] = sl; a.uq_off[u] = off; a.uq_beg[u] = beg;
          if (a.uq_len) a.uq_len[u] = len;
        }
        else { cpd_set_status(a.status, CPD_ERR_CAPACITY); won = false; }
      }
    }
    if (won) {
      // the winning lane writes its column's KRP row (16-byte vectors; rows
      // are independent, so the lanes' gathers overlap) ...
      float4* hrow = reinterpret_cast<float4*>(a.H + (int64_t)u * a.Rp);
      for (int v0 = 0; v0 < a.Rp / 4; v0 += 8) {       // 8 vectors in flight per factor
        float4 x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = make_float4(1.f, 1.f, 1.f, 1.f);
#pragma unroll
        for (int k = 0; k < CPD_MAX_MODES; ++k) {
          if (k < a.N && k != a.n) {
            const float4* f = reinterpret_cast<const float4*>(a.U[k] + (int64_t)ik[k] * a.Rp) + v0;
            float4 fv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) fv[q] = (v0 + q < a.Rp / 4) ? __ldg(f + q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 8; ++q) { x[q].x *= fv[q].x; x[q].y *= fv[q].y; x[q].z *= fv[q].z; x[q].w *= fv[q].w; }
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (v0 + q < a.Rp / 4) hrow[v0 + q] = x[q];
      }
      // ... and marks the chunks c whose first position 32 c lies in its range
      const uint32_t c1 = (off + 31) >> 5, c2 = (off + len - 1) >> 5;
      for (uint32_t c = c1; c <= c2; ++c) a.chunk_seg[c] = u;
    }
  }
}

// One step of a lane group: selected position jj of the chunk (row code r,
// weight sj, distinct column uj, all shuffled from lane jj) adds sj * h_uj
// into its output row.  The lane group's KRP row hv stays in registers while
// the drawn column does not change.
__device__ __forceinline__ void spmm_step(const MArgs& a, int Rp, int C, int q, int Hs, float* __restrict__ hot_acc,
                                          float* __restrict__ Y, uint32_t r, float sj, uint32_t uj, uint32_t& cu,
                                          float4& hv) {
  if (uj != cu) {
    hv = reinterpret_cast<const float4*>(a.H)[(int64_t)uj * C + q];
    cu = uj;
  }
  if (r & CPD_HOT_BIT) {
    const uint32_t slot = r & ~CPD_HOT_BIT;
    if ((int)slot < Hs) {
      // column 4 q + c of the slot's row lives at c C + q: the C lanes of a
      // group add into consecutive words (distinct banks)
      float* acc = hot_acc + (size_t)slot * (Rp + 1) + q;
      atomicAdd(acc, sj * hv.x);
      atomicAdd(acc + C, sj * hv.y);
      atomicAdd(acc + 2 * C, sj * hv.z);
      atomicAdd(acc + 3 * C, sj * hv.w);
      if (q == 0) reinterpret_cast<unsigned int*>(hot_acc + (size_t)Hs * (Rp + 1))[slot] = 1u;
      return;
    }
    r = (uint32_t)a.hot_rows[slot];
  }
  float* yp = Y + (int64_t)r * Rp + 4 * q;
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(yp), "f"(sj * hv.x), "f"(sj * hv.y),
               "f"(sj * hv.z), "f"(sj * hv.w)
               : "memory");
}

// Position p of the flat list of selected nonzeros (chunk c = p / 32 of a
// warp, one position per lane) -> its row code, weight x value and distinct
// column.  The 32 positions of a chunk meet at most 32 consecutive segments
// starting at the one the probe recorded for the chunk; the window of their
// offsets goes to the lanes, and each lane finds its own segment in the
// window by shuffles.  All 32 lanes take part; positions >= total get
// scale 0.
__device__ __forceinline__ void locate_selected(const MArgs& a, uint32_t nu, uint32_t total, int64_t c, int lane,
                                                uint32_t& row, float& scale, uint32_t& useg) {
  const int64_t p = c * 32 + lane;
  const uint32_t seg0 = a.chunk_seg[c];
  const uint32_t wseg = seg0 + lane;
  const uint32_t woff = wseg < nu ? a.uq_off[wseg] : 0xffffffffu;
  uint32_t loc = 0;                      // last window slot with offset <= p
#pragma unroll
  for (int b = 16; b > 0; b >>= 1) {
    const uint32_t o = __shfl_sync(CPD_FULL, woff, (int)(loc + b));
    if (o <= (uint32_t)p) loc += b;
  }
  const uint32_t segoff = __shfl_sync(CPD_FULL, woff, (int)loc);
  row = 0; useg = 0; scale = 0.0f;
  if (p < total) {
    useg = seg0 + loc;
    // the entry's address does not wait for the dedup slot: the column's
    // first entry was recorded by the probe
    const uint32_t slot = a.uq_slot[useg];
    const uint32_t e = a.uq_beg[useg] + ((uint32_t)p - segoff);
    const uint2 en = a.ent[e];
    row = en.x;
    scale = a.dd_w[slot] * __uint_as_float(en.y);
  }
}

// The cnt (<= 32) nonzeros held one per lane (row code, scale, column) of a
// warp.  C lanes cover one row of Rp floats (C <= 32 since R <= 128) with
// 16-byte vector reductions, so one warp instruction updates E = 32 / C
// selected nonzeros at once.  Consecutive nonzeros of a lane group often
// belong to the same drawn column, so its KRP row is kept in registers and
// loaded again only when the column changes.
template <int RPT>
__device__ __forceinline__ void spmm_warp(const MArgs& a, int Rp, int C, int E, int sub, int q, int Hs,
                                          float* __restrict__ hot_acc, float* __restrict__ Y, uint32_t row,
                                          float scale, uint32_t useg, int cnt) {
  uint32_t cu = 0xffffffffu;
  float4 hv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (RPT && (E * C == 32 || E == 1) && cnt == 32) {
    // a full chunk and a lane-group shape that fills the warp (or one group
    // of C < 32 lanes, the others idle): every step is valid (four steps
    // unrolled at Rp >= 32, two at Rp = 16: more would spill at 32 registers)
#pragma unroll (RPT >= 32 ? 4 : 2)
    for (int j0 = 0; j0 < 32; j0 += E) {
      const int jj = E == 1 ? j0 : j0 + sub;
      const uint32_t r = __shfl_sync(CPD_FULL, row, jj);
      const float sj = __shfl_sync(CPD_FULL, scale, jj);
      const uint32_t uj = __shfl_sync(CPD_FULL, useg, jj);
      if (E * C == 32 || sub < E) spmm_step(a, Rp, C, q, Hs, hot_acc, Y, r, sj, uj, cu, hv);
    }
  } else {
    for (int j0 = 0; j0 < cnt; j0 += E) {
      const int jj = j0 + sub;
      const int src = jj < 32 ? jj : 31;
      const uint32_t r = __shfl_sync(CPD_FULL, row, src);
      const float sj = __shfl_sync(CPD_FULL, scale, src);
      const uint32_t uj = __shfl_sync(CPD_FULL, useg, src);
      if (!(sub < E && jj < cnt)) continue;
      spmm_step(a, Rp, C, q, Hs, hot_acc, Y, r, sj, uj, cu, hv);
    }
  }
}

// Row-sorted SpMM, for outputs Y larger than L2 (R > 64).  There the vector
// reductions of the flat-list SpMM miss L2 and read-modify-write DRAM
// sectors; most cold rows take only a few selected nonzeros, so even the
// zeros of a cleared Y come back from DRAM.  Instead the selected nonzeros
// of the cold rows are counting-sorted by output row (count, scan, scatter of
// one full 32-byte record each, so no DRAM sector is read back), and a flat
// pass over the sorted list (warps take 32 consecutive positions, load
// balanced) sums each run of one row in registers: a row whose nonzeros all
// lie in one 32-position chunk is stored once, a row crossing a chunk
// boundary gets one vector reduction per chunk into zeros that a streaming
// pass stored beforehand (with the rows that have no sorted nonzeros), so Y
// is written, not read, except for those rows.  The rows this launch keeps in
// shared memory (the hot rows) stay out of the sort: the flat-list SpMM takes
// them afterwards in column order (their KRP rows reused across a column's
// run), together with every position past the sorted list's capacity.
struct RowSort {
  uint32_t* cnt;        // I: per-row counts (pass 0), counted down by pass 1
  const uint32_t* off;  // I + 1: row offsets (off[I] = sorted positions)
  uint4* rec;           // 2 cap: 32-byte records {row, scale bits, column, 0; 0, 0, 0, 0}, sorted
  uint32_t cap;         // multiple of 32
  int64_t I;
};

// PASS 0 counts the selected nonzeros of each cold row; PASS 1 places them
// at off[row] + (count, decremented).  A warp a chunk of 32 positions
// (positions < min(total, cap)); entries of rows with a shared-memory slot of
// this launch (slot < Hs) are skipped.
template <int PASS>
__global__ void __launch_bounds__(256) rowsort_kernel(MArgs a, int Hs, RowSort rs) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long pk = *reinterpret_cast<const unsigned long long*>(a.counters);
  const uint32_t nu = min((uint32_t)(pk >> 32), a.uq_cap);
  const uint32_t lim = min((uint32_t)(pk & 0xffffffffull), rs.cap);
  const int64_t nchunks = ((int64_t)lim + 31) / 32;
  for (int64_t c = warp; c < nchunks; c += nwarps) {
    uint32_t code, useg;
    float scale;
    locate_selected(a, nu, lim, c, lane, code, scale, useg);
    if (c * 32 + lane >= (int64_t)lim) continue;
    uint32_t row = code;
    if (code & CPD_HOT_BIT) {
      const uint32_t slot = code & ~CPD_HOT_BIT;
      if ((int)slot < Hs) continue;
      row = (uint32_t)a.hot_rows[slot];
    }
    if (PASS == 0) {
      atomicAdd(&rs.cnt[row], 1u);
    } else {
      const uint32_t at = rs.off[row] + atomicSub(&rs.cnt[row], 1u) - 1u;
      uint4* r = rs.rec + 2 * (size_t)at;
      r[0] = make_uint4(row, __float_as_uint(scale), useg, 0u);
      r[1] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

// Zeros for every row without sorted nonzeros and every row whose nonzeros
// cross a 32-position chunk boundary (those take vector reductions); C lanes
// a row.
__global__ void __launch_bounds__(1024, 2) rowsort_zero_kernel(float* __restrict__ Y, int Rp, RowSort rs) {
  const int lane = threadIdx.x & 31;
  const int C = Rp / 4;
  const int E = C >= 32 ? 1 : 32 / C;
  const int sub = C >= 32 ? 0 : lane / C;
  const int q = C >= 32 ? lane : lane % C;
  if (sub >= E) return;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t ngroups = (((int64_t)gridDim.x * blockDim.x) >> 5) * E;
  for (int64_t r = warp * E + sub; r < rs.I; r += ngroups) {
    const uint32_t b = rs.off[r], e = rs.off[r + 1];
    if (b == e || (b >> 5) != ((e - 1) >> 5))
      reinterpret_cast<float4*>(Y + r * Rp)[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

// The sorted positions, 32 a warp (Rp > 64: one lane group of C <= 32 lanes
// a warp).  RS_BATCH positions at a time have their KRP rows loaded before
// they are summed; a run of one row ends in a store (row inside the chunk) or a
// vector reduction (row crossing the chunk's first or last position).
constexpr int RS_BATCH = 4;
template <int RPT>
__global__ void __launch_bounds__(512, 2) rowsort_flat_kernel(MArgs a, float* __restrict__ Y, RowSort rs) {
  const int Rp = RPT ? RPT : a.Rp;
  const int C = Rp / 4;
  const int lane = threadIdx.x & 31;
  const int q = lane;                       // lanes >= C take part in the shuffles only
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t lim = rs.off[rs.I];
  const int64_t nchunks = ((int64_t)lim + 31) / 32;
  const float4* H4 = reinterpret_cast<const float4*>(a.H);
  for (int64_t c = warp; c < nchunks; c += nwarps) {
    const int64_t p = c * 32 + lane;
    const bool in = p < (int64_t)lim;
    const uint4 rc = in ? rs.rec[2 * p] : make_uint4(0xffffffffu, 0u, 0u, 0u);
    const uint32_t row = rc.x;
    const float sc = __uint_as_float(rc.y);
    const uint32_t col = rc.z;
    const uint32_t prev = c > 0 ? rs.rec[2 * (c * 32 - 1)].x : 0xffffffffu;
    const uint32_t next = c * 32 + 32 < (int64_t)lim ? rs.rec[2 * (c * 32 + 32)].x : 0xffffffffu;
    const int cnt = (int)((int64_t)lim - c * 32 < 32 ? (int64_t)lim - c * 32 : 32);
    uint32_t cur = __shfl_sync(CPD_FULL, row, 0);
    bool first = true;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    auto flush = [&](bool span) {
      if (q < C) {
        float* yp = Y + (int64_t)cur * Rp + 4 * q;
        if (span)
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(yp), "f"(acc.x), "f"(acc.y),
                       "f"(acc.z), "f"(acc.w)
                       : "memory");
        else
          *reinterpret_cast<float4*>(yp) = acc;
      }
    };
    for (int j0 = 0; j0 < cnt; j0 += RS_BATCH) {
      uint32_t rj[RS_BATCH];
      float sj[RS_BATCH];
      float4 hv[RS_BATCH];
#pragma unroll
      for (int u = 0; u < RS_BATCH; ++u) {
        const int jj = min(j0 + u, 31);
        rj[u] = __shfl_sync(CPD_FULL, row, jj);
        sj[u] = __shfl_sync(CPD_FULL, sc, jj);
        const uint32_t cj = __shfl_sync(CPD_FULL, col, jj);
        hv[u] = (j0 + u < cnt && q < C) ? H4[(int64_t)cj * C + q] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      }
#pragma unroll
      for (int u = 0; u < RS_BATCH; ++u) {
        if (j0 + u < cnt) {
          if (rj[u] != cur) {
            flush(first && cur == prev);
            first = false;
            cur = rj[u];
            acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          }
          acc.x = fmaf(sj[u], hv[u].x, acc.x); acc.y = fmaf(sj[u], hv[u].y, acc.y);
          acc.z = fmaf(sj[u], hv[u].z, acc.z); acc.w = fmaf(sj[u], hv[u].w, acc.w);
        }
      }
    }
    flush((first && cur == prev) || cur == next);
  }
}

// RPT: the row stride Rp as a compile-time constant (lane-group shape and
// address arithmetic fold), or 0 for a.Rp at run time.  hot_below: the
// positions below 32 c_begin were row-sorted except the shared-memory rows'.
template <int RPT>
__global__ void __launch_bounds__(1024, 2) spmm_kernel(MArgs a, float* __restrict__ Y, int64_t* __restrict__ out_nnz_sel,
                                                       int64_t c_begin, int hot_below) {
  // hot rows: one float row (stride Rp + 1, so rows start in different banks;
  // column 4 q + c at c Rp / 4 + q) per slot, and a touched flag per slot;
  // flushed to Y once per block
  extern __shared__ float hot_acc[];
  const int Rp = RPT ? RPT : a.Rp;
  const int S = Rp + 1;
  const int Hs = a.n_hot;
  unsigned int* touched = reinterpret_cast<unsigned int*>(hot_acc + (size_t)Hs * S);
  for (int i = threadIdx.x; i < Hs * S; i += blockDim.x) hot_acc[i] = 0.0f;
  for (int i = threadIdx.x; i < Hs; i += blockDim.x) touched[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long pk = *reinterpret_cast<const unsigned long long*>(a.counters);
  const uint32_t nu = min((uint32_t)(pk >> 32), a.uq_cap);
  const uint32_t total = (uint32_t)(pk & 0xffffffffull);
  if (out_nnz_sel && blockIdx.x == 0 && threadIdx.x == 0) *out_nnz_sel = (int64_t)total;
  const int64_t nchunks = ((int64_t)total + 31) / 32;
  const int C = Rp / 4;                   // float4 chunks per row
  const int E = C >= 32 ? 1 : 32 / C;     // nonzeros per warp instruction
  const int sub = C >= 32 ? 0 : lane / C; // which of the E nonzeros this lane serves
  const int q = C >= 32 ? lane : lane % C;
  // Below 32 c_begin (the row-sorted list's positions) only the entries of
  // this launch's shared-memory rows are taken, moved to the front of the
  // chunk in order by a ballot; from 32 c_begin on, every entry.
  for (int64_t c = (hot_below ? 0 : c_begin) + warp; c < nchunks; c += nwarps) {
    uint32_t row, useg;
    float scale;
    locate_selected(a, nu, total, c, lane, row, scale, useg);
    int cnt = (int)((int64_t)total - c * 32 < 32 ? (int64_t)total - c * 32 : 32);
    if (hot_below && c < c_begin) {
      const bool keep = lane < cnt && (row & CPD_HOT_BIT) && (int)(row & ~CPD_HOT_BIT) < Hs;
      const unsigned km = __ballot_sync(CPD_FULL, keep);
      cnt = __popc(km);
      if (cnt == 0) continue;
      const int src = lane < cnt ? (int)__fns(km, 0, lane + 1) : 0;
      row = __shfl_sync(CPD_FULL, row, src);
      scale = __shfl_sync(CPD_FULL, scale, src);
      useg = __shfl_sync(CPD_FULL, useg, src);
    }
    spmm_warp<RPT>(a, Rp, C, E, sub, q, Hs, hot_acc, Y, row, scale, useg, cnt);
  }
  // flush the block's hot rows that it touched
  __syncthreads();
  for (int i = threadIdx.x; i < Hs * C; i += blockDim.x) {
    const int slot = i / C, qq = i - slot * C;
    if (!touched[slot]) continue;
    const float* acc = hot_acc + (size_t)slot * S + qq;
    float* yp = Y + (int64_t)a.hot_rows[slot] * Rp + 4 * qq;
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(yp), "f"(acc[0]), "f"(acc[C]),
                 "f"(acc[2 * C]), "f"(acc[3 * C])
                 : "memory");
  }
}

// One launch instead of four memsets: Y = 0, dedup tags = empty, dedup
// weights = 0, packed counters = 0.
__global__ void clear_kernel(float4* __restrict__ Y, int64_t ny4, uint4* __restrict__ tag, float4* __restrict__ dw,
                             int64_t nd4, uint32_t* __restrict__ counters) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = t0; i < ny4; i += st) Y[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int64_t i = t0; i < nd4; i += st) {
    tag[i] = make_uint4(CPD_EMPTY32, CPD_EMPTY32, CPD_EMPTY32, CPD_EMPTY32);
    dw[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  if (t0 < 4) counters[t0] = 0u;
}

// Exact MTTKRP (Eq. 6) over the input-order COO: a warp takes 32 nonzeros;
// as in the sampled SpMM, C = Rp / 4 lanes cover one row with 16-byte
// vectors (E = 32 / C nonzeros per warp instruction), the KRP row of a
// nonzero is formed from its factor rows on the fly, and hot output rows
// accumulate in shared memory before one flush per block.
template <int NM>   // NM >= N: index registers per lane
__global__ void __launch_bounds__(512, 2) exact_kernel(MArgs a, const int32_t* __restrict__ idx,
                                                        const float* __restrict__ vals, int64_t nnz,
                                                        float* __restrict__ Y) {
  extern __shared__ float hot_acc[];
  const int S = a.Rp + 1;
  const int Hs = a.n_hot;
  unsigned int* touched = reinterpret_cast<unsigned int*>(hot_acc + (size_t)Hs * S);
  for (int i = threadIdx.x; i < Hs * S; i += blockDim.x) hot_acc[i] = 0.0f;
  for (int i = threadIdx.x; i < Hs; i += blockDim.x) touched[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int C = a.Rp / 4;
  const int E = C >= 32 ? 1 : 32 / C;
  const int sub = C >= 32 ? 0 : lane / C;
  const int q = C >= 32 ? lane : lane % C;
  for (int64_t c0 = warp * 32; c0 < nnz; c0 += nwarps * 32) {
    const int64_t e = c0 + lane;
    int32_t ii[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) ii[k] = (k < a.N && e < nnz) ? idx[(int64_t)k * nnz + e] : 0;
    const float v = e < nnz ? vals[e] : 0.0f;
    const int cnt = (int)(nnz - c0 < 32 ? nnz - c0 : 32);
    for (int j0 = 0; j0 < cnt; j0 += E) {
      const int jj = j0 + sub;
      const int src = jj < 32 ? jj : 31;
      int32_t ij[NM];
#pragma unroll
      for (int k = 0; k < NM; ++k) ij[k] = __shfl_sync(CPD_FULL, ii[k], src);
      const float vj = __shfl_sync(CPD_FULL, v, src);
      if (!(sub < E && jj < cnt)) continue;
      float4 hv = make_float4(vj, vj, vj, vj);
      for (int k = 0; k < a.N; ++k) {
        if (k == a.n) continue;
        const float4 u = reinterpret_cast<const float4*>(a.U[k] + (int64_t)ij[k] * a.Rp)[q];
        hv.x *= u.x; hv.y *= u.y; hv.z *= u.z; hv.w *= u.w;
      }
      const uint32_t row = (uint32_t)ij[a.n];
      const uint32_t code = a.row_code ? a.row_code[row] : 0u;
      if ((code & CPD_HOT_BIT) && (int)(code & ~CPD_HOT_BIT) < Hs) {
        const uint32_t slot = code & ~CPD_HOT_BIT;
        float* acc = hot_acc + (size_t)slot * S + q;   // column 4 q + c at c C + q
        atomicAdd(acc, hv.x);
        atomicAdd(acc + C, hv.y);
        atomicAdd(acc + 2 * C, hv.z);
        atomicAdd(acc + 3 * C, hv.w);
        if (q == 0) touched[slot] = 1u;
      } else {
        float* yp = Y + (int64_t)row * a.Rp + 4 * q;
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(yp), "f"(hv.x), "f"(hv.y), "f"(hv.z),
                     "f"(hv.w)
                     : "memory");
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < Hs * C; i += blockDim.x) {
    const int slot = i / C, qq = i - slot * C;
    if (!touched[slot]) continue;
    const float* acc = hot_acc + (size_t)slot * S + qq;
    float* yp = Y + (int64_t)a.hot_rows[slot] * a.Rp + 4 * qq;
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(yp), "f"(acc[0]), "f"(acc[C]),
                 "f"(acc[2 * C]), "f"(acc[3 * C])
                 : "memory");
  }
}

// Rows of the downsampled design matrix S U_{!=n}: sqrt(w_j) h_j, one warp
// per draw (their Gram is the sketched Gram of Fig. 3, bottom).
__global__ void sketch_rows_kernel(MArgs a, const int32_t* __restrict__ idx, const double* __restrict__ w, int64_t J,
                                   float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp; j < J; j += nwarps) {
    const bool mine = lane < a.N && lane != a.n;
    int32_t ik = mine ? idx[(int64_t)lane * J + j] : 0;
    const bool bad = mine && (ik < 0 || (int64_t)ik >= a.dims[lane]);
    const bool any_bad = __any_sync(CPD_FULL, bad);
    const float sw = (float)sqrt(fmax(w[j], 0.0));
    for (int r = lane; r < a.Rp; r += 32) {
      float v = (r < a.R && !any_bad) ? sw : 0.0f;
      for (int k = 0; k < a.N; ++k) {
        const int32_t ikk = __shfl_sync(CPD_FULL, ik, k);
        if (k != a.n && r < a.R && !any_bad) v *= a.U[k][(int64_t)ikk * a.Rp + r];
      }
      out[j * a.Rp + r] = v;
    }
  }
}

}  // namespace

// SpMM launch shape for `bps` blocks per SM: 1024 threads per block up to two
// blocks, then 2048 / bps; the shared memory of an SM is split evenly among
// its blocks and holds as many hot rows (Rp + 1 floats and a flag) as fit.
int cpd_spmm_threads(int bps) { return bps <= 2 ? 1024 : 2048 / bps; }
int cpd_spmm_hot_slots(int Rp, int bps) {
  const size_t budget = (size_t)(220 * 1024) / (size_t)std::max(bps, 1);
  return (int)(budget / ((size_t)(Rp + 1) * 4 + 4));
}
// dynamic shared memory of the sampled SpMM: the hot rows and their flags
static size_t spmm_smem(int threads, int n_hot, int Rp) {
  (void)threads;
  return (size_t)n_hot * ((size_t)(Rp + 1) * 4 + 4);
}
cpd_status cpd_spmm_init(cpd_ctx* h) {
  const size_t shm = spmm_smem(cpd_spmm_threads(1), cpd_spmm_hot_slots(h->Rp, 1), h->Rp);
  for (const void* f : {(const void*)spmm_kernel<0>, (const void*)spmm_kernel<16>, (const void*)spmm_kernel<32>,
                        (const void*)spmm_kernel<64>, (const void*)spmm_kernel<100>,
                        (const void*)spmm_kernel<128>}) {
    const cpd_status s = cpd_smem_attr(h, f, shm);
    if (s != CPD_OK) return s;
  }
  const cpd_status s4 = cpd_smem_attr(h, (const void*)exact_kernel<4>, shm);
  return s4 != CPD_OK ? s4 : cpd_smem_attr(h, (const void*)exact_kernel<CPD_MAX_MODES>, shm);
}

// Row-sorted SpMM for every mode whose output Y (I_n x Rp floats, Rp > 64)
// exceeds 96 MB, three quarters of L2: per-row counts and offsets for the
// largest such mode, and sorted lists of min(nnz, nnz_sel_capacity or 2^27)
// selected nonzeros shared by the modes; selected nonzeros past them take the
// flat-list path.
cpd_status cpd_rowsort_alloc(cpd_ctx* h) {
  if (h->opt.deterministic || h->nnz == 0 || h->Rp <= 64) return CPD_OK;
  int64_t imax = 0;
  for (int k = 0; k < h->N; ++k) {
    h->mode[k].row_sorted = h->dims[k] * (int64_t)h->Rp * 4 > ((int64_t)96 << 20);
    if (h->mode[k].row_sorted) imax = std::max(imax, h->dims[k]);
  }
  if (imax == 0) return CPD_OK;
  int64_t cap = h->opt.nnz_sel_capacity > 0 ? h->opt.nnz_sel_capacity : ((int64_t)1 << 27);
  cap = std::min<int64_t>(cap, h->nnz);
  cap = std::min<int64_t>(cpd_ceil_div(cap, 32) * 32, (int64_t)0xffffffe0ll);
  cpd_status s;
  if ((s = cpd_alloc(h, &h->rs_cnt, (size_t)imax + 1)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->rs_off, (size_t)imax + 1)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->rs_bsum, (size_t)cpd_scan_u32_scratch(imax))) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->rs_rec, (size_t)2 * cap)) != CPD_OK) return s;
  h->rs_cap = cap;
  return CPD_OK;
}

namespace {

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
  a.uq_slot = h->uq_slot; a.chunk_seg = h->chunk_seg; a.uq_off = h->uq_off; a.uq_beg = h->uq_beg;
  a.H = h->H; a.counters = h->counters; a.status = h->status;
  a.uq_cap = (uint32_t)h->Jcap;
  return a;
}

}  // namespace

// Y (I_mode x Rp, internal stride) := mat(T, mode) S^T S U_{!=mode}.
// Y = 0 (rows of `mode`), dedup tables empty, counters 0, on stream st.
cpd_status cpd_clear_launch(cpd_ctx* h, int mode, float* Y, cudaStream_t st) {
  // (row-sorted modes: the SpMM stores every row of Y itself)
  const bool sorted = h->rs_cap > 0 && h->mode[mode].row_sorted;
  const int64_t ny4 = sorted ? 0 : h->dims[mode] * (int64_t)h->Rp / 4;      // Rp is a multiple of 4
  const int64_t nd4 = ((int64_t)h->dedup_mask + 1) / 4;          // 2J slots, a power of two >= 4
  clear_kernel<<<h->num_sms * 4, 256, 0, st>>>(reinterpret_cast<float4*>(Y), ny4,
                                                reinterpret_cast<uint4*>(h->dd_tag),
                                                reinterpret_cast<float4*>(h->dd_w), nd4, h->counters);
  CPD_LAUNCH(h, "clear");
  return CPD_OK;
}

cpd_status cpd_sampled_mttkrp_launch(cpd_ctx* h, int mode, const int32_t* idx, const double* w, const double* p,
                                     int64_t J, float* Y, int64_t* out_nnz_sel, cudaEvent_t cleared) {
  (void)p;
  cudaStream_t st = h->stream;
  if (cleared) {
    CPD_CUDA(h, cudaStreamWaitEvent(st, cleared, 0));     // cleared on the forked branch
  } else {
    PhaseTimer pt(h, CPD_PHASE_CLEAR);
    const cpd_status s = cpd_clear_launch(h, mode, Y, st);
    if (s != CPD_OK) return s;
  }
  MArgs a = make_args(h, mode);
  if (h->opt.deterministic) { a.dslot = h->dslot; a.uq_len = h->uq_len; }
  if (J > 0) {
    PhaseTimer pt(h, CPD_PHASE_PROBE);
    int grid = (int)std::min<int64_t>(cpd_ceil_div(J, 256), (int64_t)h->num_sms * 16);
    probe_kernel<<<grid, 256, 0, st>>>(a, idx, w, J);
    CPD_LAUNCH(h, "probe");
  }
  if (h->opt.deterministic) {
    PhaseTimer pt(h, CPD_PHASE_SPMM);
    const cpd_status sd = cpd_det_mttkrp(h, mode, w, J, Y, out_nnz_sel);
    if (sd != CPD_OK) return sd;
  } else {
    PhaseTimer pt(h, CPD_PHASE_SPMM);
    const int bps = h->tune_spmm_bps;
    a.n_hot = std::min(h->mode[mode].n_hot, cpd_spmm_hot_slots(h->Rp, bps));
    a.hot_rows = h->mode[mode].hot_rows;
    const size_t shm = spmm_smem(cpd_spmm_threads(bps), a.n_hot, h->Rp);
    const dim3 grid(h->num_sms * bps), block(cpd_spmm_threads(bps));
    RowSort rs;
    memset(&rs, 0, sizeof(rs));
    const bool sorted = h->rs_cap > 0 && h->mode[mode].row_sorted;
    int64_t c_begin = 0;
    if (sorted) {
      const int64_t I = h->dims[mode];
      rs.cnt = h->rs_cnt; rs.off = h->rs_off; rs.rec = h->rs_rec;
      rs.cap = (uint32_t)h->rs_cap; rs.I = I;
      CPD_CUDA(h, cudaMemsetAsync(h->rs_cnt, 0, (size_t)I * sizeof(uint32_t), st));
      const int g = h->num_sms * 8;
      rowsort_kernel<0><<<g, 256, 0, st>>>(a, a.n_hot, rs);
      CPD_LAUNCH(h, "spmm row count");
      const cpd_status ss = cpd_scan_u32_buf(h, h->rs_cnt, h->rs_off, I, h->rs_off + I, h->rs_bsum, st);
      if (ss != CPD_OK) return ss;
      rowsort_kernel<1><<<g, 256, 0, st>>>(a, a.n_hot, rs);
      CPD_LAUNCH(h, "spmm row scatter");
      rowsort_zero_kernel<<<h->num_sms * 2, 1024, 0, st>>>(Y, h->Rp, rs);
      CPD_LAUNCH(h, "spmm row zeros");
      if (h->Rp == 128)
        rowsort_flat_kernel<128><<<h->num_sms * 2, 512, 0, st>>>(a, Y, rs);
      else if (h->Rp == 100)
        rowsort_flat_kernel<100><<<h->num_sms * 2, 512, 0, st>>>(a, Y, rs);
      else
        rowsort_flat_kernel<0><<<h->num_sms * 2, 512, 0, st>>>(a, Y, rs);
      CPD_LAUNCH(h, "spmm rows");
      c_begin = (int64_t)h->rs_cap / 32;    // then the positions past the sorted lists
    }
    const int hb = sorted ? 1 : 0;
    switch (h->Rp) {
      case 16: spmm_kernel<16><<<grid, block, shm, st>>>(a, Y, out_nnz_sel, c_begin, hb); break;
      case 32: spmm_kernel<32><<<grid, block, shm, st>>>(a, Y, out_nnz_sel, c_begin, hb); break;
      case 64: spmm_kernel<64><<<grid, block, shm, st>>>(a, Y, out_nnz_sel, c_begin, hb); break;
      case 100: spmm_kernel<100><<<grid, block, shm, st>>>(a, Y, out_nnz_sel, c_begin, hb); break;
      case 128: spmm_kernel<128><<<grid, block, shm, st>>>(a, Y, out_nnz_sel, c_begin, hb); break;
      default: spmm_kernel<0><<<grid, block, shm, st>>>(a, Y, out_nnz_sel, c_begin, hb); break;
    }
    CPD_LAUNCH(h, "spmm");
  }
  if (h->opt.sketched_gram) return cpd_sketch_gram(h, mode, idx, w, J);
  return CPD_OK;
}

// Sketched Gram sum_j w_j h_j h_j^T of a draw list into h->Gsk (uses h->H as
// scratch, after the SpMM has consumed it).
cpd_status cpd_sketch_gram(cpd_ctx* h, int mode, const int32_t* idx, const double* w, int64_t J) {
  MArgs a = make_args(h, mode);
  if (J > 0) {
    int grid = (int)std::min<int64_t>(cpd_ceil_div(J * 32, 256), (int64_t)h->num_sms * 16);
    sketch_rows_kernel<<<grid, 256, 0, h->stream>>>(a, idx, w, J, h->H);
    CPD_LAUNCH(h, "sketch_rows");
  }
  return cpd_gram(h, h->H, J, h->Gsk);
}

cpd_status cpd_exact_mttkrp_launch(cpd_ctx* h, int mode, float* Y) {
  cudaStream_t st = h->stream;
  PhaseTimer pt(h, CPD_PHASE_EXACT);
  CPD_CUDA(h, cudaMemsetAsync(Y, 0, (size_t)h->dims[mode] * h->Rp * sizeof(float), st));
  if (h->nnz == 0) return CPD_OK;
  MArgs a = make_args(h, mode);
  const int bps = 2;   // two 512-thread blocks per SM (64 registers a thread)
  a.n_hot = h->mode[mode].row_code ? std::min(h->mode[mode].n_hot, cpd_spmm_hot_slots(h->Rp, bps)) : 0;
  a.hot_rows = h->mode[mode].hot_rows;
  a.row_code = h->mode[mode].row_code;
  const size_t shm = (size_t)a.n_hot * ((size_t)(h->Rp + 1) * 4 + 4);
  if (h->N <= 4)
    exact_kernel<4><<<h->num_sms * bps, 512, shm, st>>>(a, h->idx, h->vals, h->nnz, Y);
  else
    exact_kernel<CPD_MAX_MODES><<<h->num_sms * bps, 512, shm, st>>>(a, h->idx, h->vals, h->nnz, Y);
  CPD_LAUNCH(h, "exact_mttkrp");
  return CPD_OK;
}
