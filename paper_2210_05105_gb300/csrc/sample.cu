// Leverage-score samplers of the Khatri-Rao product U_{!=n}.
//
// CP-ARLS-LEV (Appendix A, Algorithms 2-3): per factor k the scores
// ell_k[i] = U_k[i] G_k^+ U_k[i]^T and their running sums (the inverse-CDF
// table); a draw picks i_k independently per factor k != n.  Scores and
// running sums are float64 so the inverse CDF takes the same decisions as a
// float64 statement of Algorithm 3 up to ties at the last bits.
//
// STS-CP (Sec. 4.1, Appendix B, Algorithms 4-5) lives in sts.cu.
#include "common.cuh"
#include <algorithm>
#include <cstring>

namespace {

constexpr int LEV_THREADS = 256;
#ifndef CPD_LEV_UNROLL
#define CPD_LEV_UNROLL 4
#endif
// pairs of terms per iteration of the inner loop: 4 spends fewer issue slots
// on loop and address arithmetic (20.6 ms against 23.3 ms with 1, for the
// leverage scores and CDF of 8.2e6 rows at R = 100)
constexpr int LEV_UNROLL = CPD_LEV_UNROLL;

// ell_i = u_i^T X u_i with X = G_k^+ (Algorithm 2) as
// sum_a u_a v_a, v_a = sum_{b>=a} c_ab X_ab u_b (c = 1 on the diagonal, 2 off
// it).  One row per thread; the block's 256 rows sit column-major in shared
// memory (conflict-free), the coefficients split into float32 hi + lo (all
// threads read the same entry: broadcast).  Each v_a and the outer sum are
// Dot2 compensated dot products (exact leading products, TwoSum) in df64 on
// the float32 pipes, i.e. to ~2^-48 relative instead of float64 FMAs at 1/64
// rate.  Also writes the sum of each block's scores.  (The tile's row stride
// 257 keeps the transposing stores free of bank conflicts.)
// SPLIT threads share a row: thread part h takes rows a = h, h + SPLIT, ...
// of the triangle, and part 0 merges the partial double-floats in part order
// (deterministic).  With ROWS = 2 a thread carries rows t and t + 128 of the
// block's 256, so each coefficient load and the loop control serve two rows
// (blockDim = SPLIT * LEV_THREADS / ROWS).  Large R gives each row R(R+1)/2
// terms while the transposed tile limits a block per SM, so the split
// supplies the warps that hide the df64 chains' latency.
// The coefficients of the quadratic form once per launch: pair p of the
// row-major upper triangle (a <= b) holds c_ab X_ab as float32 hi + lo.
__global__ void lev_coef_kernel(const double* __restrict__ X, int R, float2* __restrict__ xs) {
  const int npairs = R * (R + 1) / 2;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
    int a = 0, rem = p;
    while (rem >= R - a) { rem -= R - a; ++a; }
    const int b = a + rem;
    const double x = (a == b ? 1.0 : 2.0) * X[a * R + b];
    const float hi = (float)x;
    xs[p] = make_float2(hi, (float)(x - (double)hi));
  }
}

template <int SPLIT, int ROWS>
__global__ void __launch_bounds__(LEV_THREADS / ROWS * SPLIT) lev_kernel(const float* __restrict__ U, int64_t I,
                                                                         int R, int Rp, const float2* __restrict__ xg,
                                                                         double* __restrict__ ell,
                                                                         double* __restrict__ blk, int fast) {
  constexpr int RT = LEV_THREADS / ROWS;           // row slots per part
  constexpr int NT = RT * SPLIT;
  extern __shared__ float4 lsm4[];
  const int npairs = R * (R + 1) / 2;
  float2* Xs = reinterpret_cast<float2*>(lsm4);                 // npairs (hi, lo), row-major upper triangle
  float* us = reinterpret_cast<float*>(Xs + npairs);            // Rp x 257: column c of row t at c * 257 + t
  __shared__ double red[LEV_THREADS / 32];
  __shared__ float2 partial[SPLIT > 1 ? SPLIT - 1 : 1][LEV_THREADS];
  const int tid = threadIdx.x;
  const int t = tid % RT, h = tid / RT;
  for (int p = tid; p < npairs; p += NT) Xs[p] = xg[p];
  const int64_t r0 = (int64_t)blockIdx.x * LEV_THREADS;
  {
    // coalesced rows -> transposed tile: thread tid takes column tid % 128
    // (Rp <= 128) of rows tid / 128, + NT / 128, ...
    const int c = tid & 127;
    if (c < Rp)
      for (int rr = tid >> 7; rr < LEV_THREADS; rr += NT >> 7)
        us[c * (LEV_THREADS + 1) + rr] = (r0 + rr < I) ? U[(r0 + rr) * Rp + c] : 0.0f;
  }
  __syncthreads();
  // rows t + q RT of the block, q < ROWS
  float lh[ROWS], ll[ROWS];
#pragma unroll
  for (int q = 0; q < ROWS; ++q) { lh[q] = 0.0f; ll[q] = 0.0f; }
  if (fast) {                          // float32 (precision option 1)
    for (int a = h; a < R; a += SPLIT) {
      int p = a * R - a * (a - 1) / 2;
      float ua[ROWS];
#pragma unroll
      for (int q = 0; q < ROWS; ++q) ua[q] = us[a * (LEV_THREADS + 1) + t + q * RT];
      for (int b = a; b < R; ++b, ++p) {
        const float x = Xs[p].x;
#pragma unroll
        for (int q = 0; q < ROWS; ++q) lh[q] = fmaf(ua[q] * us[b * (LEV_THREADS + 1) + t + q * RT], x, lh[q]);
      }
    }
  } else {
    // Horner-like split of the quadratic form: for each a the inner sum
    // v_a = sum_{b >= a} X'_ab u_b is a compensated dot product (the Dot2
    // step of Ogita, Rump and Oishi: exact leading product, TwoSum into
    // vh, all rounding errors and the X'_ab low parts gathered in vl), then
    // l += u_a v_a by the same step.  Per term 11 float32 operations instead
    // of 14 for accumulating each exact product u_a u_b X'_ab into l.  Even
    // and odd b run as two independent chains, merged per a.
    for (int a = h; a < R; a += SPLIT) {
      int p = a * R - a * (a - 1) / 2;
      float vh[ROWS], vl[ROWS], vh2[ROWS], vl2[ROWS];
#pragma unroll
      for (int q = 0; q < ROWS; ++q) { vh[q] = 0.0f; vl[q] = 0.0f; vh2[q] = 0.0f; vl2[q] = 0.0f; }
      int b = a;
#pragma unroll LEV_UNROLL
      for (; b + 1 < R; b += 2, p += 2) {
        const float2 x0 = Xs[p], x1 = Xs[p + 1];
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
          const float ub0 = us[b * (LEV_THREADS + 1) + t + q * RT], ub1 = us[(b + 1) * (LEV_THREADS + 1) + t + q * RT];
          df_dot_step_f(vh[q], vl[q], x0.x, x0.y, ub0);
          df_dot_step_f(vh2[q], vl2[q], x1.x, x1.y, ub1);
        }
      }
      if (b < R) {
        const float2 x = Xs[p];
#pragma unroll
        for (int q = 0; q < ROWS; ++q) df_dot_step_f(vh[q], vl[q], x.x, x.y, us[b * (LEV_THREADS + 1) + t + q * RT]);
      }
#pragma unroll
      for (int q = 0; q < ROWS; ++q) {
        df_merge(vh[q], vl[q], vh2[q], vl2[q]);
        df_renorm(vh[q], vl[q]);
        df_dot_step_f(lh[q], ll[q], vh[q], vl[q], us[a * (LEV_THREADS + 1) + t + q * RT]);
      }
    }
  }
  if (SPLIT > 1) {
    if (h > 0)
#pragma unroll
      for (int q = 0; q < ROWS; ++q) partial[h - 1][t + q * RT] = make_float2(lh[q], ll[q]);
    __syncthreads();
    if (h == 0)
      for (int g = 0; g < SPLIT - 1; ++g)
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
          const float2 o = partial[g][t + q * RT];
          if (fast) lh[q] += o.x; else df_merge(lh[q], ll[q], o.x, o.y);
        }
  }
  if (h > 0) return;
  double lsum = 0.0;
#pragma unroll
  for (int q = 0; q < ROWS; ++q) {
    const int64_t i = r0 + t + q * RT;
    if (i < I) {
      const double l = df_value(lh[q], ll[q]);
      ell[i] = l;
      lsum += l;
    }
  }
  // block sum in a fixed order (the RT threads of part 0)
  double sw = warp_sum(lsum);
  if ((t & 31) == 0) red[t >> 5] = sw;
  asm volatile("bar.sync 1, %0;" ::"n"(RT));
  if (t == 0) {
    double b = 0.0;
    for (int w = 0; w < RT / 32; ++w) b += red[w];
    blk[blockIdx.x] = b;
  }
}

// blk[b] := sum of the block sums before b (exclusive scan in place, one
// block of 1024 threads): thread t adds its run of consecutive block sums in
// order, the run totals are scanned across the block, and each thread writes
// its run's prefixes.  A fixed order, so the result is deterministic.
__global__ void __launch_bounds__(1024) blk_scan_kernel(double* __restrict__ blk, int64_t nb) {
  __shared__ double part[1024];
  const int t = threadIdx.x;
  const int64_t per = (nb + 1023) / 1024;
  const int64_t b0 = (int64_t)t * per, b1 = b0 + per < nb ? b0 + per : nb;
  double s = 0.0;
  for (int64_t b = b0; b < b1; ++b) s += blk[b];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {         // inclusive scan of the run totals
    const double v = t >= o ? part[t - o] : 0.0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  double run = t > 0 ? part[t - 1] : 0.0;
  for (int64_t b = b0; b < b1; ++b) {
    const double v = blk[b];
    blk[b] = run;
    run += v;
  }
}

// cdf[i] = (sum of the scores of all earlier blocks, from blk_scan_kernel) +
// inclusive scan of the block's scores.
__global__ void __launch_bounds__(LEV_THREADS) cdf_kernel(const double* __restrict__ ell, int64_t I,
                                                          const double* __restrict__ blk, double* __restrict__ cdf) {
  __shared__ double wsum[LEV_THREADS / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t i = (int64_t)blockIdx.x * LEV_THREADS + t;
  double v = i < I ? ell[i] : 0.0;
  double x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double y = __shfl_up_sync(CPD_FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  double base = blk[blockIdx.x];
  for (int q = 0; q < w; ++q) base += wsum[q];
  if (i < I) cdf[i] = base + x;
}

struct DrawArgs {
  const double* cdf[CPD_MAX_MODES];
  const double* ell[CPD_MAX_MODES];
  int64_t dims[CPD_MAX_MODES];
  int N, n;
  unsigned long long seed;
  int64_t sstride;            // every sstride-th running sum is staged in shared memory
  int soff[CPD_MAX_MODES];    // factor k's samples: soff[k] .. soff[k] + scnt[k] - 1
  int scnt[CPD_MAX_MODES];    // ceil(I_k / sstride) (0 for the mode being updated)
};
constexpr int DRAW_THREADS = 512;
constexpr size_t DRAW_SMEM = 46 * 1024;   // staged samples of the running sums (no opt-in needed)

// Algorithm 3 with one processor: per factor k != n, i_k = smallest i with
// cdf_k[i] > u * C_k (past the end: the row where the running sum reaches C_k).
// A factor with C_k = 0 (all scores zero) draws row 0 with probability 0.
// The block first stages every sstride-th running sum of each factor in
// shared memory; a draw's binary search runs there first (m = first staged
// sample above t), which brackets i_k to the sstride rows after sample m - 1,
// and only that bracket is searched in global memory.  For non-decreasing
// running sums the result is the full search's.
template <int NM>   // NM >= N
__global__ void __launch_bounds__(DRAW_THREADS) arls_draw_kernel(DrawArgs a, int64_t J,
                                                                 const unsigned long long* __restrict__ d_sweep,
                                                                 unsigned long long h_sweep,
                                                                 int32_t* __restrict__ out_idx,
                                                                 double* __restrict__ out_p, double* __restrict__ out_w) {
  extern __shared__ long long samp[];
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    if (k >= a.N || a.scnt[k] == 0) continue;
    const long long* cb = reinterpret_cast<const long long*>(a.cdf[k]);
    for (int m = threadIdx.x; m < a.scnt[k]; m += blockDim.x) samp[a.soff[k] + m] = cb[(int64_t)m * a.sstride];
  }
  __syncthreads();
  const unsigned long long s = d_sweep ? *d_sweep : h_sweep;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < J; j += (int64_t)gridDim.x * blockDim.x) {
    // the factors' binary searches advance together (their loads overlap)
    int64_t lo[NM], hi[NM];
    long long tb[NM];
    double t[NM], C[NM];
    bool zero = false;
    int steps = 0;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      lo[k] = 0; hi[k] = 0; tb[k] = 0; t[k] = 0.0; C[k] = 0.0;
      if (k >= a.N) continue;
      if (k == a.n) { out_idx[(int64_t)k * J + j] = -1; continue; }
      const int64_t I = a.dims[k];
      C[k] = a.cdf[k][I - 1];
      if (!(C[k] > 0.0) || !isfinite(C[k])) {     // all scores zero: no distribution, weight 0
        zero = true;
        continue;
      }
      t[k] = cpd_uniform(a.seed, CPD_STREAM_ARLS, (unsigned long long)j, (unsigned long long)k,
                         (unsigned long long)a.n, s) * C[k];
      tb[k] = __double_as_longlong(t[k]);       // non-negative: bit order = value order
      // staged samples: m = first sample above t, so rows <= (m - 1) sstride
      // have running sums <= t and row m sstride (if it exists) one above t
      const long long* sk = samp + a.soff[k];
      int ml = 0, mh = a.scnt[k];
      while (ml < mh) {
        const int mid = (ml + mh) >> 1;
        if (sk[mid] > tb[k]) mh = mid; else ml = mid + 1;
      }
      lo[k] = ml == 0 ? 0 : (int64_t)(ml - 1) * a.sstride + 1;
      hi[k] = ml < a.scnt[k] ? (int64_t)ml * a.sstride : I;
      if (lo[k] > hi[k]) lo[k] = hi[k];
      int d = 0;
      while ((int64_t(1) << d) <= hi[k] - lo[k]) ++d;
      steps = d > steps ? d : steps;
    }
    for (int it = 0; it < steps; ++it) {
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        if (lo[k] < hi[k]) {
          const int64_t mid = (lo[k] + hi[k]) >> 1;
          if (reinterpret_cast<const long long*>(a.cdf[k])[mid] > tb[k]) hi[k] = mid; else lo[k] = mid + 1;
        }
      }
    }
    double p = zero ? 0.0 : 1.0;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      if (k >= a.N || k == a.n) continue;
      const int64_t I = a.dims[k];
      if (!(C[k] > 0.0) || !isfinite(C[k])) { out_idx[(int64_t)k * J + j] = 0; continue; }
      int64_t i = lo[k];
      if (i >= I) i = cpd_inverse_cdf(a.cdf[k], I, t[k]);   // t rounded up to C: rare
      out_idx[(int64_t)k * J + j] = (int32_t)i;
      if (!zero) p *= a.ell[k][i] / C[k];
    }
    if (out_p) out_p[j] = p;
    if (out_w) out_w[j] = cpd_weight(J, p);
  }
}

size_t lev_smem(int R) {
  const int npairs = R * (R + 1) / 2;
  return (size_t)npairs * 8 + (size_t)(LEV_THREADS + 1) * cpd_pad4(R) * 4;
}

// R > 64: 16 threads share a row and each carries 4 rows (1024-thread
// blocks): 18.1 ms against 18.5 (8 x 2) and 20.6 (8 x 4) for the leverage
// scores and CDF of 8.2e6 rows at R = 100
#ifndef CPD_LEV_WSPLIT
#define CPD_LEV_WSPLIT 16        // threads a row for R > 64
#endif
#ifndef CPD_LEV_WROWS
#define CPD_LEV_WROWS 4          // rows a thread for R > 64
#endif
int lev_split(int R) { return R > 64 ? 8 : R > 32 ? 4 : 1; }

cpd_status quadform_cdf(cpd_ctx* h, const float* U, int64_t I, const double* X, double* q, double* blk,
                        double* cdf) {
  lev_coef_kernel<<<(h->R * (h->R + 1) / 2 + 255) / 256, 256, 0, h->stream>>>(X, h->R, h->lev_xs);
  CPD_LAUNCH(h, "lev coefficients");
  const float2* xg = h->lev_xs;
  const int64_t nb = cpd_ceil_div(I, LEV_THREADS);
  const int sp = lev_split(h->R);
  if (sp == 8)          // R > 64
    lev_kernel<CPD_LEV_WSPLIT, CPD_LEV_WROWS><<<(unsigned)nb, LEV_THREADS / CPD_LEV_WROWS * CPD_LEV_WSPLIT,
                                               lev_smem(h->R), h->stream>>>(U, I, h->R, h->Rp, xg, q, blk,
                                                                            h->opt.precision);
  else if (sp == 4)     // 32 < R <= 64
    lev_kernel<4, 2><<<(unsigned)nb, LEV_THREADS / 2 * 4, lev_smem(h->R), h->stream>>>(U, I, h->R, h->Rp, xg, q, blk,
                                                                                      h->opt.precision);
  else
    lev_kernel<1, 1><<<(unsigned)nb, LEV_THREADS, lev_smem(h->R), h->stream>>>(U, I, h->R, h->Rp, xg, q, blk,
                                                                              h->opt.precision);
  CPD_LAUNCH(h, "lev");
  blk_scan_kernel<<<1, 1024, 0, h->stream>>>(blk, nb);
  CPD_LAUNCH(h, "lev block scan");
  cdf_kernel<<<(unsigned)nb, LEV_THREADS, 0, h->stream>>>(q, I, blk, cdf);
  CPD_LAUNCH(h, "cdf");
  return CPD_OK;
}

cpd_status launch_lev(cpd_ctx* h, int k) {
  PhaseTimer pt(h, CPD_PHASE_SAMPLER);
  return quadform_cdf(h, h->U[k], h->dims[k], h->Gkpinv[k], h->ell[k], h->blk[k], h->cdf[k]);
}

}  // namespace

// q[i] = U[i] X U[i]^T for symmetric X (df64), in blk the sums of the
// 256-row blocks before each block, and the inclusive
// float64 running sums cdf (used by CP-ARLS-LEV and by the first STS factor).
cpd_status cpd_quadform_cdf(cpd_ctx* h, const float* U, int64_t I, const double* X, double* q, double* blk,
                            double* cdf) {
  return quadform_cdf(h, U, I, X, q, blk, cdf);
}

// Kernels with more than 48 KB of dynamic shared memory need an opt-in (set
// once, outside any stream capture).
cpd_status cpd_sample_init(cpd_ctx* h) {
  {
    const cpd_status sa = cpd_alloc(h, &h->lev_xs, (size_t)h->R * (h->R + 1) / 2);
    if (sa != CPD_OK) return sa;
  }
  for (const void* f : {(const void*)lev_kernel<1, 1>, (const void*)lev_kernel<4, 2>,
                        (const void*)lev_kernel<CPD_LEV_WSPLIT, CPD_LEV_WROWS>}) {
    const cpd_status st_ = cpd_smem_attr(h, f, lev_smem(h->R));
    if (st_ != CPD_OK) return st_;
  }
  return CPD_OK;
}

cpd_status cpd_sts_refresh(cpd_ctx* h, int mode);
cpd_status cpd_sts_draw(cpd_ctx* h, int mode, int64_t J, const unsigned long long* d_sweep,
                        unsigned long long sweep, int32_t* out_idx, double* out_p, double* out_w);

// Algorithm 2 (CP-ARLS-LEV build) or Algorithm 4 (STS-CP build) for factor
// `mode`, from its current U and Gram.
cpd_status cpd_refresh_sampler(cpd_ctx* h, int k) {
  if (h->opt.method == CPD_STS_CP) return cpd_sts_refresh(h, k);
  if (h->opt.method != CPD_ARLS_LEV) return CPD_OK;
  cpd_status s = cpd_pinv_into(h, h->G[k], h->Gkpinv[k]);
  if (s != CPD_OK) return s;
  return launch_lev(h, k);
}

cpd_status cpd_draw(cpd_ctx* h, int mode, int64_t J, const unsigned long long* d_sweep, unsigned long long sweep,
                    int32_t* out_idx, double* out_p, double* out_w) {
  if (h->opt.method == CPD_STS_CP) return cpd_sts_draw(h, mode, J, d_sweep, sweep, out_idx, out_p, out_w);
  DrawArgs a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k < h->N; ++k) { a.cdf[k] = h->cdf[k]; a.ell[k] = h->ell[k]; a.dims[k] = h->dims[k]; }
  a.N = h->N; a.n = mode; a.seed = h->opt.seed;
  if (J <= 0) return CPD_OK;
  PhaseTimer pt(h, CPD_PHASE_DRAW);
  // the smallest power-of-two stride whose samples of all factors fit
  int64_t st = 1;
  for (;;) {
    int64_t tot = 0;
    for (int k = 0; k < h->N; ++k)
      if (k != mode) tot += cpd_ceil_div(h->dims[k], st);
    if (tot * (int64_t)sizeof(long long) <= (int64_t)DRAW_SMEM) break;
    st *= 2;
  }
  a.sstride = st;
  int off = 0;
  for (int k = 0; k < h->N; ++k) {
    a.soff[k] = off;
    a.scnt[k] = k == mode ? 0 : (int)cpd_ceil_div(h->dims[k], st);
    off += a.scnt[k];
  }
  const size_t shm = (size_t)off * sizeof(long long);
  // at most two blocks per SM: the samples are staged once per block
  int grid = (int)std::min<int64_t>(cpd_ceil_div(J, DRAW_THREADS), (int64_t)h->num_sms * 2);
  if (h->N <= 4)
    arls_draw_kernel<4><<<grid, DRAW_THREADS, shm, h->stream>>>(a, J, d_sweep, sweep, out_idx, out_p, out_w);
  else
    arls_draw_kernel<CPD_MAX_MODES><<<grid, DRAW_THREADS, shm, h->stream>>>(a, J, d_sweep, sweep, out_idx, out_p,
                                                                            out_w);
  CPD_LAUNCH(h, "arls_draw");
  return CPD_OK;
}
