// Deterministic downsampled MTTKRP Y = mat(T, n) S^T S U_{!=n} (Eq. 7) for
// options.deterministic = 1: the same sum as mttkrp.cu's, with every
// floating-point addition in an order fixed by the inputs, so that repeated
// runs agree bit for bit.
//
//  1. The probe (mttkrp.cu) records each draw's dedup slot instead of adding
//     its weight with an atomic; the draws are sorted stably by slot and each
//     slot's weight is summed in draw order (float64, then rounded).
//  2. The distinct sampled columns are put in canonical order (sorted by the
//     position of their first nonzero in the mode layout) and their nonzeros
//     listed in that order; the list is sorted stably by output row, so each
//     row's contributions sit together in layout order.
//  3. A warp takes 256 consecutive sorted positions and sums each row's run
//     sequentially; runs inside the chunk are stored to Y directly, runs that
//     cross a chunk boundary leave partial sums that one pass adds in chunk
//     order.
// Element counts that only the device knows (distinct columns, selected
// nonzeros) are read by the kernels, so the whole sequence can be captured in
// the sweep's CUDA graph.
#include "common.cuh"
#include <algorithm>

namespace {

constexpr int DET_CHUNK = 256;
constexpr int DET_WARPS = 8;

int bits_of(unsigned long long v) {
  int b = 0;
  while (b < 64 && (v >> b) != 0ull) ++b;
  return b;
}

__global__ void weight_keys_kernel(const uint32_t* __restrict__ dslot, int64_t J, uint32_t dcap,
                                   unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < J; j += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = dslot[j];
    keys[j] = s == CPD_EMPTY32 ? (unsigned long long)dcap : (unsigned long long)s;
    vals[j] = (uint32_t)j;
  }
}

// first position of each slot's run sums that slot's weights in draw order
__global__ void weight_sum_kernel(const unsigned long long* __restrict__ keys, const uint32_t* __restrict__ vals,
                                  int64_t J, uint32_t dcap, const double* __restrict__ w, float* __restrict__ dd_w) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < J; p += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[p];
    if (k >= dcap || (p > 0 && keys[p - 1] == k)) continue;
    double s = 0.0;
    for (int64_t q = p; q < J && keys[q] == k; ++q) s += w[vals[q]];
    dd_w[k] = (float)s;
  }
}

// distinct columns keyed by the layout position of their first nonzero
__global__ void col_keys_kernel(const uint32_t* __restrict__ counters, const uint32_t* __restrict__ uq_beg, int64_t cap,
                                unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals,
                                uint32_t* __restrict__ words) {
  const unsigned long long pk = *reinterpret_cast<const unsigned long long*>(counters);
  const uint32_t nu = (uint32_t)min((unsigned long long)(pk >> 32), (unsigned long long)cap);
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < cap; u += (int64_t)gridDim.x * blockDim.x) {
    keys[u] = (uint32_t)u < nu ? (unsigned long long)uq_beg[u] : 0xffffffffull;
    vals[u] = (uint32_t)u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) words[2] = nu;
}

__global__ void col_len_kernel(const uint32_t* __restrict__ cols, const uint32_t* __restrict__ uq_len,
                               const uint32_t* __restrict__ words, int64_t cap, uint32_t* __restrict__ len) {
  const uint32_t nu = words[2];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < cap; r += (int64_t)gridDim.x * blockDim.x)
    len[r] = (uint32_t)r < nu ? uq_len[cols[r]] : 0u;
}

// the kept count: min(scan total, capacity); CPD_ERR_CAPACITY if cut
__global__ void sel_count_kernel(uint32_t* __restrict__ words, int64_t sel_cap, int* __restrict__ status) {
  const uint32_t total = words[1];
  words[0] = (int64_t)total > sel_cap ? (uint32_t)sel_cap : total;
  if ((int64_t)total > sel_cap) cpd_set_status(status, CPD_ERR_CAPACITY);
}

// canonical list: a warp per distinct column in canonical order writes its
// nonzeros' output rows (the sort keys), positions, layout entries, column
__global__ void materialize_kernel(const uint32_t* __restrict__ cols, const uint32_t* __restrict__ off,
                                   const uint32_t* __restrict__ uq_beg, const uint32_t* __restrict__ uq_len,
                                   const uint32_t* __restrict__ words, const uint2* __restrict__ ent,
                                   const int32_t* __restrict__ hot_rows, int64_t sel_cap,
                                   unsigned long long* __restrict__ rkeys, uint32_t* __restrict__ rvals,
                                   uint32_t* __restrict__ sel_e, uint32_t* __restrict__ sel_u) {
  const uint32_t nu = words[2];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < (int64_t)nu; r += nwarps) {
    const uint32_t u = cols[r];
    const uint32_t beg = uq_beg[u], len = uq_len[u], o = off[r];
    for (uint32_t i = lane; i < len; i += 32) {
      const int64_t q = (int64_t)o + i;
      if (q >= sel_cap) break;
      const uint32_t e = beg + i;
      uint32_t code = ent[e].x;
      if (code & CPD_HOT_BIT) code = (uint32_t)hot_rows[code & ~CPD_HOT_BIT];
      rkeys[q] = code;
      rvals[q] = (uint32_t)q;
      sel_e[q] = e;
      sel_u[q] = u;
    }
  }
}

// Per chunk of DET_CHUNK sorted positions: each row's run summed in order.
// flags: bit 0 the first run continues from the previous chunk, bit 1 the
// last run continues into the next, bit 2 the chunk holds one run.
template <int NPL>
__global__ void __launch_bounds__(DET_WARPS * 32) reduce_kernel(
    const unsigned long long* __restrict__ rkeys, const uint32_t* __restrict__ rvals, const uint32_t* __restrict__ words,
    const uint32_t* __restrict__ sel_e, const uint32_t* __restrict__ sel_u, const uint2* __restrict__ ent,
    const uint32_t* __restrict__ uq_slot, const float* __restrict__ dd_w, const float* __restrict__ H, int Rp,
    float* __restrict__ Y, float* __restrict__ part, uint32_t* __restrict__ flags) {
  __shared__ float s_sc[DET_WARPS][DET_CHUNK];
  __shared__ uint32_t s_u[DET_WARPS][DET_CHUNK];
  __shared__ uint32_t s_row[DET_WARPS][DET_CHUNK];
  const uint32_t n = words[0];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = (int64_t)blockIdx.x * DET_WARPS + wid;
  const int64_t nwarps = (int64_t)gridDim.x * DET_WARPS;
  const int64_t nch = ((int64_t)n + DET_CHUNK - 1) / DET_CHUNK;
  float* sc = s_sc[wid];
  uint32_t* su = s_u[wid];
  uint32_t* srow = s_row[wid];
  for (int64_t c = warp; c < nch; c += nwarps) {
    const int64_t base = c * DET_CHUNK;
    const int cnt = (int)min((int64_t)DET_CHUNK, (int64_t)n - base);
    for (int t = lane; t < cnt; t += 32) {
      const uint32_t q = rvals[base + t];
      const uint32_t u = sel_u[q];
      const uint2 en = ent[sel_e[q]];
      sc[t] = dd_w[uq_slot[u]] * __uint_as_float(en.y);
      su[t] = u;
      srow[t] = (uint32_t)rkeys[base + t];
    }
    __syncwarp();
    const bool cin = base > 0 && (uint32_t)rkeys[base - 1] == srow[0];
    const bool cout = base + cnt < (int64_t)n && (uint32_t)rkeys[base + cnt] == srow[cnt - 1];
    float acc[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) acc[i] = 0.0f;
    uint32_t cur = srow[0];
    bool first_run = true;
    float* pc = part + (size_t)c * 2 * Rp;
    for (int t = 0; t < cnt; ++t) {
      const uint32_t r = srow[t];
      if (r != cur) {
        float* dst = (first_run && cin) ? pc : Y + (int64_t)cur * Rp;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
          const int comp = lane + 32 * i;
          if (comp < Rp) dst[comp] = acc[i];
          acc[i] = 0.0f;
        }
        first_run = false;
        cur = r;
      }
      const float s = sc[t];
      const float* hr = H + (int64_t)su[t] * Rp;
#pragma unroll
      for (int i = 0; i < NPL; ++i) {
        const int comp = lane + 32 * i;
        if (comp < Rp) acc[i] = fmaf(s, hr[comp], acc[i]);
      }
    }
    const bool single = first_run;
    float* dst;
    if (single) dst = (cin || cout) ? pc : Y + (int64_t)cur * Rp;
    else dst = cout ? pc + Rp : Y + (int64_t)cur * Rp;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
      const int comp = lane + 32 * i;
      if (comp < Rp) dst[comp] = acc[i];
    }
    if (lane == 0) flags[c] = (cin ? 1u : 0u) | (cout ? 2u : 0u) | (single ? 4u : 0u);
    __syncwarp();
  }
}

// A run crossing chunk boundaries: the chunk holding its first position adds
// its partial and the following chunks' first-run partials in chunk order.
__global__ void combine_kernel(const unsigned long long* __restrict__ rkeys, const uint32_t* __restrict__ words,
                               const float* __restrict__ part, const uint32_t* __restrict__ flags, int Rp,
                               float* __restrict__ Y) {
  const uint32_t n = words[0];
  const int64_t nch = ((int64_t)n + DET_CHUNK - 1) / DET_CHUNK;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < nch; c += nwarps) {
    const uint32_t f = flags[c];
    if (!(f & 2u) || ((f & 4u) && (f & 1u))) continue;      // not the first chunk of a split run
    const int64_t last = min((c + 1) * DET_CHUNK, (int64_t)n) - 1;
    const uint32_t row = (uint32_t)rkeys[last];
    for (int comp = lane; comp < Rp; comp += 32) {
      float s = part[(size_t)c * 2 * Rp + ((f & 4u) ? 0 : Rp) + comp];
      for (int64_t c2 = c + 1; c2 < nch; ++c2) {
        s += part[(size_t)c2 * 2 * Rp + comp];
        const uint32_t f2 = flags[c2];
        if (!((f2 & 4u) && (f2 & 2u))) break;
      }
      Y[(int64_t)row * Rp + comp] = s;
    }
  }
}

}  // namespace

cpd_status cpd_det_alloc(cpd_ctx* h) {
  cpd_status s;
  if ((s = cpd_radix_init(h)) != CPD_OK) return s;
  h->sel_cap = h->opt.nnz_sel_capacity > 0 ? std::min<int64_t>(h->opt.nnz_sel_capacity, std::max<int64_t>(h->nnz, 1))
                                          : std::max<int64_t>(h->nnz, 1);
  const int64_t kc = std::max<int64_t>(h->Jcap, h->sel_cap);
  const int64_t nch = cpd_ceil_div(h->sel_cap, DET_CHUNK);
  if ((s = cpd_alloc(h, &h->dslot, (size_t)h->Jcap)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->uq_len, (size_t)h->Jcap)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->dkeys, (size_t)kc)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->dkeys2, (size_t)kc)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->dvals, (size_t)kc)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->dvals2, (size_t)kc)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->dcounts, (size_t)256 * cpd_ceil_div(kc, 4096))) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->dlen, (size_t)h->Jcap + 1)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->dwords, 4)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->sel_e, (size_t)h->sel_cap)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->sel_u, (size_t)h->sel_cap)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->dpart, (size_t)nch * 2 * h->Rp)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->dflags, (size_t)nch)) != CPD_OK) return s;
  return CPD_OK;
}

// After the probe (which filled dslot, uq_len, the distinct-column lists and
// H): weights, canonical list, row sort, reduction into Y (already zero).
cpd_status cpd_det_mttkrp(cpd_ctx* h, int mode, const double* w, int64_t J, float* Y, int64_t* out_nnz_sel) {
  cudaStream_t st = h->stream;
  const int g = h->num_sms * 4;
  unsigned long long* ok;
  uint32_t* ov;
  cpd_status s;
  if (J > 0) {
    const uint32_t dcap = h->dedup_mask + 1;
    weight_keys_kernel<<<g, 256, 0, st>>>(h->dslot, J, dcap, h->dkeys, h->dvals);
    CPD_LAUNCH(h, "det weight keys");
    if ((s = cpd_radix_sort_u64_dev(h, h->dkeys, h->dvals, J, nullptr, bits_of(dcap), h->dkeys2, h->dvals2, h->dcounts,
                                    &ok, &ov)) != CPD_OK)
      return s;
    weight_sum_kernel<<<g, 256, 0, st>>>(ok, ov, J, dcap, w, h->dd_w);
    CPD_LAUNCH(h, "det weight sums");
  }
  // canonical column order and offsets
  const int64_t cap = h->Jcap;
  col_keys_kernel<<<g, 256, 0, st>>>(h->counters, h->uq_beg, cap, h->dkeys, h->dvals, h->dwords);
  CPD_LAUNCH(h, "det column keys");
  if ((s = cpd_radix_sort_u64_dev(h, h->dkeys, h->dvals, cap, nullptr, 32, h->dkeys2, h->dvals2, h->dcounts, &ok,
                                  &ov)) != CPD_OK)
    return s;
  uint32_t* cols = ov;
  // the column list must survive the next sort, which reuses dvals/dvals2:
  // keep it in uq_off (the atomics path's offsets, unused here)
  CPD_CUDA(h, cudaMemcpyAsync(h->uq_off, cols, (size_t)cap * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  cols = h->uq_off;
  col_len_kernel<<<g, 256, 0, st>>>(cols, h->uq_len, h->dwords, cap, h->dlen);
  CPD_LAUNCH(h, "det column lengths");
  if ((s = cpd_scan_u32(h, h->dlen, h->dlen, cap, h->dwords + 1)) != CPD_OK) return s;
  sel_count_kernel<<<1, 1, 0, st>>>(h->dwords, h->sel_cap, h->status);
  materialize_kernel<<<g, 256, 0, st>>>(cols, h->dlen, h->uq_beg, h->uq_len, h->dwords, h->mode[mode].ent,
                                        h->mode[mode].hot_rows, h->sel_cap, h->dkeys, h->dvals, h->sel_e, h->sel_u);
  CPD_LAUNCH(h, "det materialize");
  // stable sort by output row: each row's entries stay in layout order
  if ((s = cpd_radix_sort_u64_dev(h, h->dkeys, h->dvals, h->sel_cap, h->dwords, bits_of((unsigned long long)h->dims[mode]),
                                  h->dkeys2, h->dvals2, h->dcounts, &ok, &ov)) != CPD_OK)
    return s;
  const int blocks = h->num_sms * 4;
  const int Rp = h->Rp;
  if (Rp <= 32)
    reduce_kernel<1><<<blocks, DET_WARPS * 32, 0, st>>>(ok, ov, h->dwords, h->sel_e, h->sel_u, h->mode[mode].ent,
                                                       h->uq_slot, h->dd_w, h->H, Rp, Y, h->dpart, h->dflags);
  else if (Rp <= 64)
    reduce_kernel<2><<<blocks, DET_WARPS * 32, 0, st>>>(ok, ov, h->dwords, h->sel_e, h->sel_u, h->mode[mode].ent,
                                                       h->uq_slot, h->dd_w, h->H, Rp, Y, h->dpart, h->dflags);
  else
    reduce_kernel<4><<<blocks, DET_WARPS * 32, 0, st>>>(ok, ov, h->dwords, h->sel_e, h->sel_u, h->mode[mode].ent,
                                                       h->uq_slot, h->dd_w, h->H, Rp, Y, h->dpart, h->dflags);
  CPD_LAUNCH(h, "det reduce");
  combine_kernel<<<blocks, 256, 0, st>>>(ok, h->dwords, h->dpart, h->dflags, Rp, Y);
  CPD_LAUNCH(h, "det combine");
  if (out_nnz_sel) {
    // the selected-nonzero count the probe reserved (low word of the packed counter)
    CPD_CUDA(h, cudaMemsetAsync(out_nnz_sel, 0, sizeof(int64_t), st));
    CPD_CUDA(h, cudaMemcpyAsync(out_nnz_sel, h->counters, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
  }
  return CPD_OK;
}
