// Dense kernels of the ALS update: Grams (Eq. 5 operands), Hadamard product
// of Grams and its Moore-Penrose pseudo-inverse (Eq. 4-5), the solve
// U_n = Y G^+ with column renormalisation (Algorithm 1's mode update), and the
// fit of Sec. 5.1.
//
// Precision: factor storage and the solve GEMM are float32; Grams, the R x R
// algebra and the fit accumulate in float64 (the sampler's inverse CDF is
// decided on float64 leverage scores, so the Grams feeding them are float64).
#include "common.cuh"
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>

namespace {

constexpr int TR = 64;          // rows per tile
constexpr int TRP = TR + 4;     // padded column stride of the Gram tile (floats)
constexpr int DTHREADS = 256;

// ---- column sums of squares (float64 partials per block) ----------------
// Thread (g, c) of a block accumulates column c over rows g, g+groups, ...
__device__ __forceinline__ void store_col_partials(double acc, int R, int groups, double* __restrict__ out_blk) {
  __shared__ double red[DTHREADS];
  const int t = threadIdx.x;
  red[t] = acc;
  __syncthreads();
  if (t < R) {
    double s = 0.0;
    for (int g = 0; g < groups; ++g) s += red[g * R + t];
    out_blk[t] = s;
  }
  __syncthreads();
}

__global__ void colsq_kernel(const float* __restrict__ U, int64_t I, int R, int Rp, double* __restrict__ part) {
  const int groups = DTHREADS / R;
  const int t = threadIdx.x, c = t % R, g = t / R;
  double acc = 0.0;
  if (g < groups) {
    for (int64_t i = (int64_t)blockIdx.x * groups + g; i < I; i += (int64_t)gridDim.x * groups) {
      float v = U[i * Rp + c];
      acc += (double)(v * v);
    }
  }
  store_col_partials(g < groups ? acc : 0.0, R, groups, part + (int64_t)blockIdx.x * R);
}

// sigma_r = sqrt(sum of partials): one block per column, fixed order.
__global__ void sigma_kernel(const double* __restrict__ part, int nblk, int R, double* __restrict__ sigma) {
  __shared__ double red[32];
  const int r = blockIdx.x, t = threadIdx.x;
  double s = 0.0;
  for (int b = t; b < nblk; b += blockDim.x) s += part[(int64_t)b * R + r];
  s = warp_sum(s);
  if ((t & 31) == 0) red[t >> 5] = s;
  __syncthreads();
  if (t == 0) {
    double z = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) z += red[w];
    sigma[r] = sqrt(z);
  }
}

// U_out = U_in / sigma (columns with sigma = 0 kept), padded columns zeroed,
// and float64 Gram partials of the stored float32 values.  Per 64-row tile a
// thread accumulates its Gram entries as df64 sums of exact float32 products
// (error ~ 64 * 2^-48 of the sum of |terms|), then adds them into float64.
template <int MAXP>
__global__ void __launch_bounds__(DTHREADS) normalize_gram_kernel(
    const float* __restrict__ Uin, float* __restrict__ Uout, int64_t I, int R, int Rp,
    const double* __restrict__ sigma, int do_scale, double* __restrict__ gpart, int fast) {
  extern __shared__ float4 tile4[];
  float* tile = reinterpret_cast<float*>(tile4);        // R columns x TRP float32
  __shared__ float inv[CPD_MAX_RANK];
  __shared__ unsigned char pa[8320], pb[8320];
  const int t = threadIdx.x;
  const int npairs = R * (R + 1) / 2;
  for (int r = t; r < R; r += DTHREADS) {
    double s = do_scale ? sigma[r] : 0.0;
    inv[r] = (s > 0.0) ? (float)(1.0 / s) : 1.0f;
  }
  // pair table of the upper triangle, row-major
  for (int p = t; p < npairs; p += DTHREADS) {
    int a = 0, rem = p;
    while (rem >= R - a) { rem -= R - a; ++a; }
    pa[p] = (unsigned char)a;
    pb[p] = (unsigned char)(a + rem);
  }
  __syncthreads();
  // df64 accumulators (4 chains per entry for ILP) live across all tiles of
  // the block: a block holds ~I / gridDim rows, so the df64 error stays near
  // (rows per block) * 2^-48 of the sum of |terms|; float64 only at the end.
  // (with many entries per thread, R > 72, the entries themselves give the
  // instruction-level parallelism: one chain each, rows outer, entries inner)
  constexpr int CH = MAXP > 9 ? 1 : 4;
  float ah[MAXP][CH], al[MAXP][CH];
#pragma unroll
  for (int m = 0; m < MAXP; ++m)
#pragma unroll
    for (int c = 0; c < CH; ++c) { ah[m][c] = 0.0f; al[m][c] = 0.0f; }
  const int64_t ntiles = cpd_ceil_div(I, TR);
  for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const int64_t r0 = tl * TR;
    // tile column-major with a padded column stride TRP: column c of rows
    // rr..rr+3 is one 16-byte read, and the eight lanes of a phase that read
    // consecutive columns hit distinct banks
    for (int e = t; e < TR * Rp; e += DTHREADS) {
      int rr = e / Rp, c = e % Rp;
      int64_t i = r0 + rr;
      if (i < I) {
        float v = 0.0f;
        if (c < R) v = Uin[i * Rp + c] * inv[c];
        Uout[i * Rp + c] = v;
        if (c < R) tile[c * TRP + rr] = v;
      } else if (c < R) {
        tile[c * TRP + rr] = 0.0f;
      }
    }
    __syncthreads();
    if constexpr (CH == 1) {
      for (int q = 0; q < TR / 4; ++q) {
#pragma unroll
        for (int m = 0; m < MAXP; ++m) {
          const int p = t + m * DTHREADS;
          if (p < npairs) {
            const float4 x = reinterpret_cast<const float4*>(tile + pa[p] * TRP)[q];
            const float4 y = reinterpret_cast<const float4*>(tile + pb[p] * TRP)[q];
            if (fast) {
              ah[m][0] = fmaf(x.x, y.x, ah[m][0]);
              ah[m][0] = fmaf(x.y, y.y, ah[m][0]);
              ah[m][0] = fmaf(x.z, y.z, ah[m][0]);
              ah[m][0] = fmaf(x.w, y.w, ah[m][0]);
            } else {
              df_fma(ah[m][0], al[m][0], x.x, y.x);
              df_fma(ah[m][0], al[m][0], x.y, y.y);
              df_fma(ah[m][0], al[m][0], x.z, y.z);
              df_fma(ah[m][0], al[m][0], x.w, y.w);
            }
          }
        }
      }
    } else {
#pragma unroll
    for (int m = 0; m < MAXP; ++m) {
      int p = t + m * DTHREADS;
      if (p < npairs) {
        const float4* ca = reinterpret_cast<const float4*>(tile + pa[p] * TRP);
        const float4* cb = reinterpret_cast<const float4*>(tile + pb[p] * TRP);
        if (fast) {                      // float32 accumulation (precision option 1)
#pragma unroll 4
          for (int q = 0; q < TR / 4; ++q) {
            const float4 x = ca[q], y = cb[q];
            ah[m][0] = fmaf(x.x, y.x, ah[m][0]);
            ah[m][1] = fmaf(x.y, y.y, ah[m][1]);
            ah[m][2] = fmaf(x.z, y.z, ah[m][2]);
            ah[m][3] = fmaf(x.w, y.w, ah[m][3]);
          }
        } else {
#pragma unroll 4
          for (int q = 0; q < TR / 4; ++q) {
            const float4 x = ca[q], y = cb[q];
            df_fma(ah[m][0], al[m][0], x.x, y.x);
            df_fma(ah[m][CH > 1 ? 1 : 0], al[m][CH > 1 ? 1 : 0], x.y, y.y);
            df_fma(ah[m][CH > 2 ? 2 : 0], al[m][CH > 2 ? 2 : 0], x.z, y.z);
            df_fma(ah[m][CH > 3 ? 3 : 0], al[m][CH > 3 ? 3 : 0], x.w, y.w);
          }
        }
      }
    }
    }
    __syncthreads();
  }
  double* out = gpart + (int64_t)blockIdx.x * npairs;
#pragma unroll
  for (int m = 0; m < MAXP; ++m) {
    int p = t + m * DTHREADS;
    if (p < npairs) {
      if constexpr (CH == 4) {
        df_merge(ah[m][0], al[m][0], ah[m][CH - 3], al[m][CH - 3]);
        df_merge(ah[m][CH - 2], al[m][CH - 2], ah[m][CH - 1], al[m][CH - 1]);
        df_merge(ah[m][0], al[m][0], ah[m][CH - 2], al[m][CH - 2]);
      }
      out[p] = df_value(ah[m][0], al[m][0]);
    }
  }
}

// Register-blocked Gram for R > 64 (precision 0): thread (rg, bi) owns the
// 4 x 4 block bi of the Gram's upper block triangle (columns 4 a0 .. + 3 by
// 4 b0 .. + 3) for the rows of row group rg.  Per row it reads two float4 of
// the row-major tile and adds 16 exact float32 products into 16 independent
// double-float chains; every GB_FLUSH tiles of GB_TR rows the chains are
// added into float64 accumulators, so each df64 chain spans at most 1,024 / nrg
// rows (error ~ that many 2^-48 of the sum of |terms|; the float64 adds run at
// 1/64 of the float32 rate, so they are kept rare).  Tiles of 128 rows halve
// the share of the tile loads' latency left uncovered between barriers.  Each
// (block, row group) writes its own float64 partial Gram (gram_reduce_kernel
// sums them in a fixed order).
#ifndef CPD_GB_MINB
#define CPD_GB_MINB 2            // resident blocks per SM the register budget is sized for
#endif
#ifndef CPD_GB_TR
#define CPD_GB_TR 128
#endif
#ifndef CPD_GB_MAXT
#define CPD_GB_MAXT 416
#endif
constexpr int GB_TR = CPD_GB_TR;
constexpr int GB_FLUSH = 1024 / GB_TR;
constexpr int GB_MAXT = CPD_GB_MAXT;   // threads: one row group of nblk <= 406 blocks (R <= 112), 16 chains each
__global__ void __launch_bounds__(GB_MAXT, CPD_GB_MINB) gram_blk_kernel(
    const float* __restrict__ Uin, float* __restrict__ Uout, int64_t I, int R, int Rp,
    const double* __restrict__ sigma, int do_scale, double* __restrict__ gpart, int nrg) {
  extern __shared__ float4 gbs4[];
  // the float64 flush accumulators live in shared memory (16 per thread, at
  // [j * blockDim + t] for entry j: conflict-free), the tile after them
  double* acc64 = reinterpret_cast<double*>(gbs4);
  float* tile = reinterpret_cast<float*>(acc64 + 16 * blockDim.x);   // TR x Rp, row-major
  __shared__ __align__(16) float inv[CPD_MAX_RANK];                 // read as float4
  __shared__ unsigned char ba[CPD_MAX_RANK / 4 * (CPD_MAX_RANK / 4 + 1) / 2];
  __shared__ unsigned char bb[CPD_MAX_RANK / 4 * (CPD_MAX_RANK / 4 + 1) / 2];
  const int t = threadIdx.x;
  const int nb4 = Rp / 4;
  const int nblk = nb4 * (nb4 + 1) / 2;
  for (int r = t; r < Rp; r += blockDim.x) {     // 0 for the padding columns
    double sv = do_scale && r < R ? sigma[r] : 0.0;
    inv[r] = r >= R ? 0.0f : (sv > 0.0) ? (float)(1.0 / sv) : 1.0f;
  }
  for (int e = t; e < nblk; e += blockDim.x) {
    int a = 0, rem = e;
    while (rem >= nb4 - a) { rem -= nb4 - a; ++a; }
    ba[e] = (unsigned char)a;
    bb[e] = (unsigned char)(a + rem);
  }
  __syncthreads();
  // tile loads as 16-byte vectors: thread t takes vector t % nb4 of rows
  // t / nb4, + lstep, ... (threads past lstep * nb4 load nothing)
  const int lc4 = t % nb4, lstep = (int)blockDim.x / nb4;
  const int lr0 = t / nb4 < lstep ? t / nb4 : GB_TR;
  const float4 lsc = *reinterpret_cast<const float4*>(inv + 4 * lc4);
  const int bi = t % nblk, rg = t / nblk;
  const bool active = rg < nrg;
  const int a0 = 4 * ba[bi], b0 = 4 * bb[bi];
  float ah[4][4], al[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { ah[i][j] = 0.0f; al[i][j] = 0.0f; acc64[(4 * i + j) * blockDim.x + t] = 0.0; }
  const int64_t ntiles = cpd_ceil_div(I, GB_TR);
  int nt = 0;
  for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const int64_t r0 = tl * GB_TR;
    __syncthreads();                             // previous tile consumed
    for (int rr = lr0; rr < GB_TR; rr += lstep) {
      const int64_t i = r0 + rr;
      float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (i < I) {
        const float4 u = reinterpret_cast<const float4*>(Uin + i * Rp)[lc4];
        v = make_float4(u.x * lsc.x, u.y * lsc.y, u.z * lsc.z, u.w * lsc.w);
        reinterpret_cast<float4*>(Uout + i * Rp)[lc4] = v;
      }
      reinterpret_cast<float4*>(tile + rr * Rp)[lc4] = v;
    }
    __syncthreads();
    if (active) {
#pragma unroll 1
      for (int rr = rg; rr < GB_TR; rr += nrg) {
        const float4 x = *reinterpret_cast<const float4*>(tile + rr * Rp + a0);
        const float4 y = *reinterpret_cast<const float4*>(tile + rr * Rp + b0);
        const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) df_fma(ah[i][j], al[i][j], xv[i], yv[j]);
      }
      if (++nt == GB_FLUSH) {
        nt = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc64[(4 * i + j) * blockDim.x + t] += df_value(ah[i][j], al[i][j]);
            ah[i][j] = 0.0f;
            al[i][j] = 0.0f;
          }
      }
    }
  }
  if (!active) return;
  double* out = gpart + ((int64_t)blockIdx.x * nrg + rg) * (R * (R + 1) / 2);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = a0 + i, b = b0 + j;
      if (a <= b && b < R)
        out[a * R - a * (a - 1) / 2 + (b - a)] = acc64[(4 * i + j) * blockDim.x + t] + df_value(ah[i][j], al[i][j]);
    }
}

// G = sum of block partials, one warp per Gram entry: lane l sums the
// partials l, l+32, ... in order, then a fixed butterfly (deterministic).
__global__ void gram_reduce_kernel(const double* __restrict__ gpart, int nblk, int R, double* __restrict__ G) {
  const int npairs = R * (R + 1) / 2;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < npairs; p += nw) {
    int a = 0, rem = p;
    while (rem >= R - a) { rem -= R - a; ++a; }
    const int b = a + rem;
    double s = 0.0;
    for (int k = lane; k < nblk; k += 32) s += gpart[(int64_t)k * npairs + p];
    s = warp_sum(s);
    if (lane == 0) {
      G[a * R + b] = s;
      G[b * R + a] = s;
    }
  }
}

// ---- pseudo-inverse of a symmetric PSD R x R matrix ----------------------
struct PinvJob {
  const double* in[CPD_MAX_MODES];  // Hadamard factors
  int nin;
  double* out_had;                  // may be null
  double* out_pinv;
  float* out_split;                 // may be null: out_pinv as float32 hi (R x R) then lo (R x R)
  double* scratch;                  // 2 R x R float64 (global)
  int* status;                      // latched CPD_ERR_SINGULAR_GRAM if the eigensolver fails
};
struct PinvJobs { PinvJob job[2]; };

__device__ double block_sum_d(double v, double* red) {
  const int t = threadIdx.x;
  v = warp_sum(v);
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (t < 32) {
    s = (t < (int)(blockDim.x >> 5)) ? red[t] : 0.0;
    s = warp_sum(s);
  }
  if (t == 0) red[32] = s;
  __syncthreads();
  double r = red[32];
  __syncthreads();
  return r;
}

constexpr int PINV_FAST_R = 64;
constexpr int PINV_FAST_R2 = 104; // the fast path up to here: 12 entries a thread of 1024, 5 R^2 floats of shared memory
constexpr int PINV_THREADS = 1024;
constexpr int PINV_PER_T = 4;   // entries per thread of the fast path (R * R / 4 threads, at least one warp)

// Unevaluated float32 pairs (hi, lo) with |lo| <= ulp(hi) / 2 (df64).
struct dd {
  float h, l;
};
__device__ __forceinline__ dd dd_norm(float h, float l) {     // fast two-sum, |h| >= |l|
  const float s = __fadd_rn(h, l);
  return {s, __fsub_rn(l, __fsub_rn(s, h))};
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return dd_norm(p, e);
}
__device__ __forceinline__ dd dd_sub(dd a, dd b) {
  float s, e;
  df_two_sum(a.h, -b.h, s, e);
  return dd_norm(s, __fadd_rn(e, __fsub_rn(a.l, b.l)));
}
// 1 / a: approximate float32 reciprocal r, then r + r (1 - a r) in df64
// (~2^-46 relative: the refinement squares the start's error)
__device__ __forceinline__ dd dd_recip(dd a) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(a.h));
  const dd res = dd_sub(dd{1.0f, 0.0f}, dd_mul(a, dd{r, 0.0f}));
  const dd c = dd_mul(dd{r, 0.0f}, res);
  float s, e;
  df_two_sum(r, c.h, s, e);
  return dd_norm(s, __fadd_rn(e, c.l));
}

// Fast path for R <= 104 on the float32 pipes: Gauss-Jordan elimination in
// df64 (G split exactly into float32 hi + lo; each thread keeps its own
// entries in registers, the owners of row and column k publish them, one
// barrier per step) gives X ~ G^{-1} to ~cond(G) 2^-44; Newton-Schulz steps
// X <- X + X (I - G X) with G X in df64 then bring X to ~2^-48 relative.  A
// step taken from residual W = I - G X leaves residual W^2 (plus the df64
// floor ~ cond(G) 2^-48), so the iteration stops after the step whose
// incoming max |W| is below 1e-7: X is then within ~1e-14 of G^{-1}
// (relative), the accuracy class of a float64 factorisation.  Returns false
// (nothing written) when a pivot is at most 1e-9 * max diag (the same test
// as the float64 elimination, so the eigen-decomposition decides) or max |W|
// does not reach 1e-7 within the allowed steps.
template <int PT>   // entries per thread: R * R <= PT * blockDim
__device__ bool pinv_fast(const PinvJob& jb, int R, float* sm, int max_newton) {
  __shared__ float2 rowk[2][PINV_FAST_R2], colk[2][PINV_FAST_R2];
  __shared__ float red[32];
  const int t = threadIdx.x, nt = blockDim.x;
  const int RR = R * R;
  float* Gh = sm;
  float* Gl = Gh + RR;
  float* Xh = Gl + RR;
  float* Xl = Xh + RR;
  float* W = Xl + RR;
  for (int e = t; e < RR; e += nt) {
    double v = 1.0;
    for (int k = 0; k < jb.nin; ++k) v *= jb.in[k][e];
    if (jb.out_had) jb.out_had[e] = v;
    const float hi = (float)v;
    Gh[e] = hi;
    Gl[e] = (float)(v - (double)hi);
  }
  int eij[PT];   // (row << 16) | column of each entry, -1 past R * R
  dd w[PT];
#pragma unroll
  for (int m = 0; m < PT; ++m) {
    const int e = t + m * nt;
    eij[m] = e < RR ? ((e / R) << 16) | (e % R) : -1;
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < PT; ++m) {
    const int e = t + m * nt;
    w[m] = eij[m] >= 0 ? dd{Gh[e], Gl[e]} : dd{0.0f, 0.0f};
  }
  float maxd = 0.0f;
  for (int a = 0; a < R; ++a) maxd = fmaxf(maxd, fabsf(Gh[a * R + a]));
  for (int k = 0; k < R; ++k) {
    const int b = k & 1;
#pragma unroll
    for (int m = 0; m < PT; ++m) {
      if (eij[m] < 0) continue;
      const int i = eij[m] >> 16, j = eij[m] & 0xffff;
      if (i == k) rowk[b][j] = make_float2(w[m].h, w[m].l);
      if (j == k) colk[b][i] = make_float2(w[m].h, w[m].l);
    }
    __syncthreads();
    const dd piv{rowk[b][k].x, rowk[b][k].y};
    if (!(piv.h > 1e-9f * maxd) || !isfinite(piv.h)) return false;    // uniform
    const dd inv = dd_recip(piv);
#pragma unroll
    for (int m = 0; m < PT; ++m) {
      if (eij[m] < 0) continue;
      const int i = eij[m] >> 16, j = eij[m] & 0xffff;
      const dd rj{rowk[b][j].x, rowk[b][j].y}, ci{colk[b][i].x, colk[b][i].y};
      // branch-free step: the pivot column is treated as the identity column
      // (r_k := 1, w := 0 there), so every entry runs the same instructions
      const bool jk = (j == k);
      const dd r1{jk ? 1.0f : rj.h, jk ? 0.0f : rj.l};
      const dd wb{jk ? 0.0f : w[m].h, jk ? 0.0f : w[m].l};
      const dd sv = dd_mul(r1, inv);
      const dd gv = dd_sub(wb, dd_mul(ci, sv));
      w[m] = (i == k) ? sv : gv;
    }
  }
#pragma unroll
  for (int m = 0; m < PT; ++m)
    if (eij[m] >= 0) { Xh[t + m * nt] = w[m].h; Xl[t + m * nt] = w[m].l; }
  __syncthreads();
  bool ok = false;
  for (int it = 0; it < max_newton && !ok; ++it) {
    // W = I - G X with G X in df64
    float emax = 0.0f;
    for (int e = t; e < RR; e += nt) {
      const int i = e / R, j = e % R;
      float ah = 0.0f, al = 0.0f;
      for (int k = 0; k < R; ++k) {
        const float gh = Gh[i * R + k], gl = Gl[i * R + k], xh = Xh[k * R + j], xl = Xl[k * R + j];
        df_fma(ah, al, gh, xh);
        al = __fmaf_rn(gh, xl, __fmaf_rn(gl, xh, al));
      }
      const float ev = __fsub_rn(__fsub_rn(i == j ? 1.0f : 0.0f, ah), al);
      W[e] = ev;
      emax = fmaxf(emax, fabsf(ev));
    }
    emax = fmaxf(emax, __shfl_xor_sync(CPD_FULL, emax, 16));
    emax = fmaxf(emax, __shfl_xor_sync(CPD_FULL, emax, 8));
    emax = fmaxf(emax, __shfl_xor_sync(CPD_FULL, emax, 4));
    emax = fmaxf(emax, __shfl_xor_sync(CPD_FULL, emax, 2));
    emax = fmaxf(emax, __shfl_xor_sync(CPD_FULL, emax, 1));
    if ((t & 31) == 0) red[t >> 5] = emax;
    __syncthreads();
    float em = 0.0f;
    for (int q = 0; q < nt / 32; ++q) em = fmaxf(em, red[q]);
    if (!isfinite(em)) return false;
    // X <- X + X W (the correction is small: float32 suffices)
    float corr[PT];
#pragma unroll
    for (int m = 0; m < PT; ++m) {
      const int e = t + m * nt;
      float c = 0.0f;
      if (e < RR) {
        const int i = e / R, j = e % R;
        for (int k = 0; k < R; ++k) c = fmaf(Xh[i * R + k], W[k * R + j], c);
      }
      corr[m] = c;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < PT; ++m) {
      const int e = t + m * nt;
      if (e < RR) {
        float sh, se;
        df_two_sum(Xh[e], corr[m], sh, se);
        Xl[e] = __fadd_rn(Xl[e], se);
        Xh[e] = sh;
      }
    }
    __syncthreads();
    ok = em < 1e-7f || max_newton == 1;
  }
  if (!ok) return false;
  for (int e = t; e < RR; e += nt) {
    const int i = e / R, j = e % R;
    const double p = 0.5 * (df_value(Xh[e], Xl[e]) + df_value(Xh[j * R + i], Xl[j * R + i]));
    jb.out_pinv[e] = p;
    if (jb.out_split) {               // the solve's float32 copy, and its float32 remainder
      const float hi = (float)p;
      jb.out_split[e] = hi;
      jb.out_split[RR + e] = (float)(p - (double)hi);
    }
  }
  return true;
}

// Inverse of a symmetric positive definite G by Gauss-Jordan elimination
// without pivoting (the pivots are the Cholesky / LDL^T pivots) when every
// pivot exceeds 1e-9 * max diag; otherwise a parallel (round-robin) cyclic
// Jacobi eigendecomposition with eigenvalues <= R 2^-52 lambda_max dropped.
// One block; each elimination step copies row and column k aside, then every
// thread updates its entries (two barriers per step, no serial thread).
// Returns whether the float32 split of the result was written too (the fast
// path writes it with the result).
__device__ __forceinline__ bool pinv_body(const PinvJob& jb, int R, int fast) {
  extern __shared__ double A[];                     // R x R
  __shared__ double red[40];
  __shared__ int sp[64], sq[64];
  __shared__ double sc[64], ss[64];
  __shared__ double rowk[CPD_MAX_RANK], colk[CPD_MAX_RANK];
  const int t = threadIdx.x, nt = blockDim.x;
  const int RR = R * R;
  if (R <= PINV_FAST_R && pinv_fast<PINV_PER_T>(jb, R, reinterpret_cast<float*>(A), fast ? 1 : 6)) return true;
  if (R > PINV_FAST_R && R <= PINV_FAST_R2 && (int)blockDim.x * 12 >= R * R &&
      pinv_fast<12>(jb, R, reinterpret_cast<float*>(A), fast ? 1 : 6))
    return true;
  for (int e = t; e < RR; e += nt) {
    double v = 1.0;
    for (int k = 0; k < jb.nin; ++k) v *= jb.in[k][e];
    A[e] = v;
    if (jb.out_had) jb.out_had[e] = v;
  }
  __syncthreads();
  double maxdiag = 0.0;
  for (int a = 0; a < R; ++a) maxdiag = fmax(maxdiag, fabs(A[a * R + a]));
  bool singular = false;
  for (int k = 0; k < R; ++k) {
    if (t < R) { rowk[t] = A[k * R + t]; colk[t] = A[t * R + k]; }
    __syncthreads();
    const double piv = rowk[k];
    if (!(piv > 1e-9 * maxdiag) || !isfinite(piv)) { singular = true; break; }   // uniform
    const double inv = 1.0 / piv;
    for (int e = t; e < RR; e += nt) {
      const int i = e / R, j = e % R;
      double v;
      if (i == k) v = (j == k) ? inv : rowk[j] * inv;
      else if (j == k) v = -colk[i] * inv;
      else v = A[e] - colk[i] * (rowk[j] * inv);
      A[e] = v;
    }
    __syncthreads();
  }
  double* V = jb.scratch + RR;        // R x R
  if (!singular) {
    for (int e = t; e < RR; e += nt) {
      const int i = e / R, j = e % R;
      jb.out_pinv[e] = 0.5 * (A[e] + A[j * R + i]);
    }
    return false;
  }
  // -- Jacobi fallback: reload A, V = I
  __syncthreads();
  for (int e = t; e < RR; e += nt) {
    double v = 1.0;
    for (int k = 0; k < jb.nin; ++k) v *= jb.in[k][e];
    A[e] = v;
    V[e] = (e / R == e % R) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int Re = R + (R & 1);
  const int npair = Re / 2;
  const double eps = 2.220446049250313e-16;
  bool converged = false;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int e = t; e < RR; e += nt) {
      double v = A[e];
      if (e / R == e % R) dg += v * v; else off += v * v;
    }
    off = block_sum_d(off, red);
    dg = block_sum_d(dg, red);
    if (off <= ((double)R * eps) * ((double)R * eps) * dg) { converged = true; break; }   // uniform
    for (int rnd = 0; rnd < Re - 1; ++rnd) {
      if (t < npair) {
        int i = t;
        int a = (i == 0) ? 0 : ((i - 1 + rnd) % (Re - 1)) + 1;
        int k2 = Re - 1 - i;
        int b = ((k2 - 1 + rnd) % (Re - 1)) + 1;
        int p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, s = 0.0;
        if (q < R) {
          double apq = A[p * R + q];
          if (fabs(apq) > 1e-300 && fabs(apq) > eps * sqrt(fabs(A[p * R + p] * A[q * R + q]))) {
            double tau = (A[q * R + q] - A[p * R + p]) / (2.0 * apq);
            double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
        } else {
          q = -1;
        }
        sp[i] = p; sq[i] = q; sc[i] = c; ss[i] = s;
      }
      __syncthreads();
      for (int e = t; e < npair * R; e += nt) {       // rows: A <- J^T A
        int i = e / R, j = e % R;
        int p = sp[i], q = sq[i];
        if (q >= 0) {
          double c = sc[i], s = ss[i];
          double ap = A[p * R + j], aq = A[q * R + j];
          A[p * R + j] = c * ap - s * aq;
          A[q * R + j] = s * ap + c * aq;
        }
      }
      __syncthreads();
      for (int e = t; e < npair * R; e += nt) {       // columns: A <- A J, V <- V J
        int i = e / R, j = e % R;
        int p = sp[i], q = sq[i];
        if (q >= 0) {
          double c = sc[i], s = ss[i];
          double ap = A[j * R + p], aq = A[j * R + q];
          A[j * R + p] = c * ap - s * aq;
          A[j * R + q] = s * ap + c * aq;
          double vp = V[j * R + p], vq = V[j * R + q];
          V[j * R + p] = c * vp - s * vq;
          V[j * R + q] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
  }
  // 60 cyclic sweeps converge quadratically for any finite symmetric
  // matrix; not converging means non-finite entries (a NaN or Inf reached
  // the Grams): no pseudo-inverse exists
  if (!converged && t == 0 && jb.status) cpd_set_status(jb.status, CPD_ERR_SINGULAR_GRAM);
  double lmax = 0.0;
  for (int a = 0; a < R; ++a) lmax = fmax(lmax, fabs(A[a * R + a]));
  const double cut = (double)R * 0x1.0p-52 * lmax;
  for (int e = t; e < RR; e += nt) {
    int a = e / R, b = e % R;
    double s = 0.0;
    for (int m = 0; m < R; ++m) {
      double lam = A[m * R + m];
      if (lam > cut) s += V[a * R + m] * (V[b * R + m] / lam);
    }
    jb.out_pinv[e] = s;
  }
  return false;
}

// Every path of pinv_body leaves the block together, so the float32 split of
// the result (the solve's operand), when the fast path did not write it, can
// follow one barrier later.
__global__ void __launch_bounds__(PINV_THREADS) pinv_kernel(PinvJobs jobs, int R, int fast) {
  const PinvJob& jb = jobs.job[blockIdx.x];
  const bool split_done = pinv_body(jb, R, fast);
  if (jb.out_split && !split_done) {
    __syncthreads();
    for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
      const double p = jb.out_pinv[e];
      const float hi = (float)p;
      jb.out_split[e] = hi;
      jb.out_split[R * R + e] = (float)(p - (double)hi);
    }
  }
}

// ---- solve: Uw = Y P, P = G^+ rounded to float32 ---------------------------
// Four threads per row, each owning a quarter of the RB (>= Rp) columns;
// the row of Y in registers, P in shared memory read as 16-byte vectors (one
// load feeds four FMAs per thread).  o = fma(y_a, P[a][c], o), a = 0..R-1: the
// float32 accumulation bounds the error, so G^+'s float32 remainder is not
// carried.  Column sums of squares:
// shuffles over the 8 rows a warp holds, then per-warp shared partials and a
// fixed-order sum per block.
template <int RB>
__global__ void __launch_bounds__(DTHREADS) solve_kernel(
    const float* __restrict__ Y, const float* __restrict__ P2, float* __restrict__ Uw, int64_t I, int R,
    int Rp, double* __restrict__ colpart) {
  constexpr int CPT = RB / 4;          // columns per thread
  extern __shared__ float4 sm4[];
  float* Phi = reinterpret_cast<float*>(sm4);   // R x RB, zero past R
  __shared__ double wsq[DTHREADS / 32][CPD_MAX_RANK];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int q = t & 3, rl = t >> 2;
  for (int e = t; e < R * RB; e += DTHREADS) {     // G^+ rounded to float32 (by pinv_kernel)
    const int a = e / RB, c = e % RB;
    Phi[e] = c < R ? P2[a * R + c] : 0.0f;
  }
  for (int c = lane; c < CPD_MAX_RANK; c += 32) wsq[wid][c] = 0.0;
  __syncthreads();
  const int c0 = q * CPT;
  float csq[CPT];
#pragma unroll
  for (int cc = 0; cc < CPT; ++cc) csq[cc] = 0.0f;
  for (int64_t r0 = (int64_t)blockIdx.x * (DTHREADS / 4); r0 < I; r0 += (int64_t)gridDim.x * (DTHREADS / 4)) {
    const int64_t i = r0 + rl;
    const bool live = i < I;
    float y[RB];
    const float4* yrow = reinterpret_cast<const float4*>(Y + (live ? i : 0) * Rp);
#pragma unroll
    for (int v = 0; v < RB / 4; ++v) {
      const float4 x = (live && 4 * v < Rp) ? yrow[v] : make_float4(0.f, 0.f, 0.f, 0.f);
      y[4 * v] = x.x; y[4 * v + 1] = x.y; y[4 * v + 2] = x.z; y[4 * v + 3] = x.w;
    }
    float out[CPT];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) out[cc] = 0.0f;
#pragma unroll
    for (int a = 0; a < RB; ++a) {
      if (a < R) {
        const float ya = y[a];
        const float4* ph = reinterpret_cast<const float4*>(Phi + a * RB + c0);
#pragma unroll
        for (int v = 0; v < CPT / 4; ++v) {
          const float4 h4 = ph[v];
          out[4 * v] = fmaf(ya, h4.x, out[4 * v]);
          out[4 * v + 1] = fmaf(ya, h4.y, out[4 * v + 1]);
          out[4 * v + 2] = fmaf(ya, h4.z, out[4 * v + 2]);
          out[4 * v + 3] = fmaf(ya, h4.w, out[4 * v + 3]);
        }
      }
    }
    if (live) {
      float4* urow = reinterpret_cast<float4*>(Uw + i * Rp + c0);
#pragma unroll
      for (int v = 0; v < CPT / 4; ++v)
        if (c0 + 4 * v < Rp) urow[v] = make_float4(out[4 * v], out[4 * v + 1], out[4 * v + 2], out[4 * v + 3]);
    }
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc)
      if (live) csq[cc] = fmaf(out[cc], out[cc], csq[cc]);
  }
  // (float32 suffices: a thread holds a few rows; float64 only per block)
#pragma unroll
  for (int cc = 0; cc < CPT; ++cc) {
    float sq = csq[cc];
    sq += __shfl_xor_sync(CPD_FULL, sq, 4);
    sq += __shfl_xor_sync(CPD_FULL, sq, 8);
    sq += __shfl_xor_sync(CPD_FULL, sq, 16);
    if (lane < 4 && c0 + cc < R) wsq[wid][c0 + cc] = (double)sq;
  }
  __syncthreads();
  for (int c = t; c < R; c += DTHREADS) {
    double s = 0.0;
    for (int w = 0; w < DTHREADS / 32; ++w) s += wsq[w][c];
    colpart[(int64_t)blockIdx.x * R + c] = s;
  }
}

// ---- solve for R <= 32: one output column per lane ------------------------
// Lane c of every warp owns output column c and holds column c of P (G^+ in
// float32) in registers.  The block stages SOLVE_TR rows of Y in shared memory
// (the next tile is loaded into registers while the current one is used);
// warp w takes rows w, w + 8, ... of the tile, two at a time, reading each
// row as 16-byte broadcasts.  Every output sums its terms in the same order
// as solve_kernel: o = fma(y_a, P[a][c], o), a = 0..R-1.
constexpr int SOLVE_TR = 64;
__global__ void __launch_bounds__(DTHREADS, 2) solve_lane_kernel(
    const float* __restrict__ Y, const float* __restrict__ P2, float* __restrict__ Uw, int64_t I, int R, int Rp,
    double* __restrict__ colpart) {
  constexpr int RB = 32;
  __shared__ float4 ys4[SOLVE_TR * RB / 4];       // tile row r at r * RB / 4; columns >= Rp stay zero
  __shared__ float wsq[DTHREADS / 32][32];
  const int t = threadIdx.x, c = t & 31, wid = t >> 5;
  float ph[RB];
#pragma unroll
  for (int a = 0; a < RB; ++a) ph[a] = (a < R && c < R) ? P2[a * R + c] : 0.0f;
  const int C4 = Rp / 4;                          // float4 per row of Y (Rp <= 32)
  const int nv = SOLVE_TR * C4;                   // float4 per tile (<= 512 = 2 per thread)
  for (int e = t; e < SOLVE_TR * RB / 4; e += DTHREADS) ys4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4* Y4 = reinterpret_cast<const float4*>(Y);
  float4 pre[2];
  auto load_tile = [&](int64_t r0) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = t + k * DTHREADS;
      pre[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < nv) {
        const int row = e / C4, c4 = e - row * C4;
        if (r0 + row < I) pre[k] = Y4[(r0 + row) * C4 + c4];
      }
    }
  };
  float csq = 0.0f;
  int64_t r0 = (int64_t)blockIdx.x * SOLVE_TR;
  if (r0 < I) load_tile(r0);
  for (; r0 < I; r0 += (int64_t)gridDim.x * SOLVE_TR) {
    __syncthreads();                              // the previous tile has been used
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = t + k * DTHREADS;
      if (e < nv) {
        const int row = e / C4, c4 = e - row * C4;
        ys4[row * (RB / 4) + c4] = pre[k];
      }
    }
    __syncthreads();
    const int64_t rn = r0 + (int64_t)gridDim.x * SOLVE_TR;
    if (rn < I) load_tile(rn);
    for (int rr = wid; rr < SOLVE_TR; rr += 16) {   // rows rr and rr + 8 of the tile
      const float4* y0 = ys4 + rr * (RB / 4);
      const float4* y1 = ys4 + (rr + 8) * (RB / 4);
      float o0 = 0.0f, o1 = 0.0f;
#pragma unroll
      for (int v = 0; v < RB / 4; ++v) {
        const float4 a0 = y0[v], a1 = y1[v];
        o0 = fmaf(a0.x, ph[4 * v], o0);
        o1 = fmaf(a1.x, ph[4 * v], o1);
        o0 = fmaf(a0.y, ph[4 * v + 1], o0);
        o1 = fmaf(a1.y, ph[4 * v + 1], o1);
        o0 = fmaf(a0.z, ph[4 * v + 2], o0);
        o1 = fmaf(a1.z, ph[4 * v + 2], o1);
        o0 = fmaf(a0.w, ph[4 * v + 3], o0);
        o1 = fmaf(a1.w, ph[4 * v + 3], o1);
      }
      const int64_t i0 = r0 + rr, i1 = r0 + rr + 8;
      if (i0 < I) {
        if (c < Rp) Uw[i0 * Rp + c] = o0;
        csq = fmaf(o0, o0, csq);
      }
      if (i1 < I) {
        if (c < Rp) Uw[i1 * Rp + c] = o1;
        csq = fmaf(o1, o1, csq);
      }
    }
  }
  // (float32 suffices: a lane holds a few rows; float64 only per block)
  wsq[wid][c] = csq;
  __syncthreads();
  for (int cc = t; cc < R; cc += DTHREADS) {
    double s = 0.0;
    for (int w = 0; w < DTHREADS / 32; ++w) s += (double)wsq[w][cc];
    colpart[(int64_t)blockIdx.x * R + cc] = s;
  }
}

// ---- solve for 32 < R <= 128: register-tiled Y P ------------------------------
// A block of TXN TY threads (TY x TXN) computes tiles of 8 TY rows x NB
// columns (NB = 64, 112 or 128 >= Rp; TXN = 16, 14, 16): thread (ty, tx) owns
// rows 8 ty .. 8 ty + 7 and columns TC tx .. TC tx + TC - 1 (TC = NB / TXN),
// 8 TC accumulators in registers.  (NB = 112 saves the eighth of the FMAs that
// NB = 128 spends on zero columns at R = 100.)  P = G^+ rounded to float32 (R x NB, zero past R) stays in shared
// memory for the whole grid-stride loop; each tile of Y is staged transposed
// (Rp x tile rows, consecutive lanes loading consecutive rows, so the
// transposing stores do not conflict).  Per k the thread reads 8 values of Y
// and TC of P as 16-byte vectors and issues 8 TC FMAs: o = fma(y_a, P[a][c],
// o), a = 0..R-1.  The float32 accumulation bounds the error (about 2^-24
// sum_a |y_a P_ac| per output); carrying G^+'s float32 remainder as a second
// FMA per term did not reduce it measurably, so it is left out here.
template <int NB, int TY, int TXN>
__global__ void __launch_bounds__(TXN * TY, 2) solve_tile_kernel(
    const float* __restrict__ Y, const float* __restrict__ P2, float* __restrict__ Uw, int64_t I, int R, int Rp,
    double* __restrict__ colpart) {
  constexpr int TC = NB / TXN;
  static_assert(TC % 4 == 0, "16-byte vectors of P");
  constexpr int TM = 8 * TY, YS = TM + 4, NT = TXN * TY;
  extern __shared__ float4 sm4[];
  float* Ph = reinterpret_cast<float*>(sm4);     // R x NB
  float* Ys = Ph + R * NB;                       // Rp x YS (transposed tile; rows >= R hold Y's zero padding)
  __shared__ float wsq[TY][NB];
  const int t = threadIdx.x, tx = t % TXN, ty = t / TXN;
  for (int e = t; e < R * NB; e += NT) {
    const int a = e / NB, c = e % NB;
    Ph[e] = c < R ? P2[a * R + c] : 0.0f;
  }
  float csq[TC];
#pragma unroll
  for (int j = 0; j < TC; ++j) csq[j] = 0.0f;
  const int C4 = Rp / 4;
  const float4* Y4 = reinterpret_cast<const float4*>(Y);
  for (int64_t r0 = (int64_t)blockIdx.x * TM; r0 < I; r0 += (int64_t)gridDim.x * TM) {
    __syncthreads();                             // previous tile consumed (and G^+ staged)
    // lanes take consecutive rows of one float4 column of the tile
    for (int e = t; e < TM * C4; e += NT) {
      const int row = e % TM, c4 = e / TM;
      const float4 v = (r0 + row < I) ? Y4[(r0 + row) * C4 + c4] : make_float4(0.f, 0.f, 0.f, 0.f);
      Ys[(4 * c4 + 0) * YS + row] = v.x;
      Ys[(4 * c4 + 1) * YS + row] = v.y;
      Ys[(4 * c4 + 2) * YS + row] = v.z;
      Ys[(4 * c4 + 3) * YS + row] = v.w;
    }
    __syncthreads();
    float acc[8][TC];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < TC; ++j) acc[i][j] = 0.0f;
#pragma unroll 2
    for (int a = 0; a < R; ++a) {
      const float4 y0 = *reinterpret_cast<const float4*>(Ys + a * YS + 8 * ty);
      const float4 y1 = *reinterpret_cast<const float4*>(Ys + a * YS + 8 * ty + 4);
      const float yv[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
      float ph[TC];
#pragma unroll
      for (int v = 0; v < TC / 4; ++v) {
        const float4 h4 = *reinterpret_cast<const float4*>(Ph + a * NB + TC * tx + 4 * v);
        ph[4 * v] = h4.x; ph[4 * v + 1] = h4.y; ph[4 * v + 2] = h4.z; ph[4 * v + 3] = h4.w;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TC; ++j) acc[i][j] = fmaf(yv[i], ph[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t row = r0 + 8 * ty + i;
      if (row < I) {
#pragma unroll
        for (int v = 0; v < TC / 4; ++v) {
          const int c = TC * tx + 4 * v;
          if (c < Rp)
            *reinterpret_cast<float4*>(Uw + row * Rp + c) =
                make_float4(acc[i][4 * v], acc[i][4 * v + 1], acc[i][4 * v + 2], acc[i][4 * v + 3]);
        }
#pragma unroll
        for (int j = 0; j < TC; ++j) csq[j] = fmaf(acc[i][j], acc[i][j], csq[j]);
      }
    }
  }
  // column sums of squares: per (ty, column) in shared memory, then a fixed-
  // order sum over ty in float64 per block
#pragma unroll
  for (int j = 0; j < TC; ++j) wsq[ty][TC * tx + j] = csq[j];
  __syncthreads();
  for (int c = t; c < R; c += NT) {
    double s = 0.0;
    for (int y = 0; y < TY; ++y) s += (double)wsq[y][c];
    colpart[(int64_t)blockIdx.x * R + c] = s;
  }
}

static size_t solve_tile_smem(int R, int NB, int TY) {
  return ((size_t)R * NB + (size_t)cpd_pad4(R) * (8 * TY + 4)) * sizeof(float);
}
// 256-row tiles of 512 threads were measured slower than 128-row tiles of
// 256 threads at R = 100 (22.6 against 20.0 ms a round for the factors of an
// 8.2e6 x 1.77e5 x 8.1e6 tensor), so TY = 16 is used throughout
static int solve_tile_ty(int R, int NB) { (void)R; (void)NB; return 16; }

static int solve_rb(int R) { return R <= 16 ? 16 : R <= 32 ? 32 : R <= 64 ? 64 : 128; }

// ---- fit ------------------------------------------------------------------
struct FitArgs {
  const float* U[CPD_MAX_MODES];
  int N, R, Rp;
};

// <T, T~> partial per block: a warp takes 32 nonzeros, lane r owns rank
// component r (and r + 32, ...).
__global__ void fit_inner_kernel(const int32_t* __restrict__ idx, const float* __restrict__ vals, int64_t nnz,
                                 FitArgs a, const double* __restrict__ sigma, double* __restrict__ part) {
  __shared__ double red[40];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float sg[CPD_MAX_RANK / 32];
#pragma unroll
  for (int q = 0; q < CPD_MAX_RANK / 32; ++q) {
    int r = lane + 32 * q;
    sg[q] = r < a.R ? (float)sigma[r] : 0.0f;
  }
  double acc = 0.0;
  for (int64_t c0 = warp * 32; c0 < nnz; c0 += nwarps * 32) {
    int64_t e = c0 + lane;
    float v = e < nnz ? vals[e] : 0.0f;
    int32_t ii[CPD_MAX_MODES];
#pragma unroll
    for (int k = 0; k < CPD_MAX_MODES; ++k) ii[k] = (k < a.N && e < nnz) ? idx[(int64_t)k * nnz + e] : 0;
    int cnt = (int)(nnz - c0 < 32 ? nnz - c0 : 32);
    float part32 = 0.0f;
    // (unrolled so that the factor-row gathers of several nonzeros are in
    // flight at once; the additions keep their order)
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
      const float vj = __shfl_sync(CPD_FULL, v, j);
      int32_t ij[CPD_MAX_MODES];
#pragma unroll
      for (int k = 0; k < CPD_MAX_MODES; ++k) ij[k] = __shfl_sync(CPD_FULL, ii[k], j);
#pragma unroll
      for (int q = 0; q < CPD_MAX_RANK / 32; ++q) {
        int r = lane + 32 * q;
        if (32 * q < a.R) {
          float m = sg[q];
#pragma unroll
          for (int k = 0; k < CPD_MAX_MODES; ++k)
            if (k < a.N) m *= (r < a.R) ? a.U[k][(int64_t)ij[k] * a.Rp + r] : 0.0f;
          part32 = fmaf(vj, m, part32);
        }
      }
    }
    acc += (double)part32;
  }
  double s = block_sum_d(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// <T, T~> over the fibers of mode m (the mode with the fewest rows, whose
// factor L2 keeps): T~ = sum_r sigma_r *_k U_k[:, r], so a fiber with
// indices (i_k)_{k != m} adds sum_r h_r z_r, h_r = sigma_r *_{k != m}
// U_k[i_k, r] formed once per fiber and z_r = sum_e v_e U_m[i_e, r] over its
// nonzeros.  Each nonzero thus gathers one row of U_m instead of N factor
// rows.  A warp scans 32 slots of mode m's fiber table at a time and takes
// the occupied ones one by one (C = Rp / 4 lanes, 16-byte vectors); z is
// summed in float32 over runs of 32 nonzeros and in float64 across runs, and
// each lane adds its fibers' terms in float64.
struct FitFiberArgs {
  const float* U[CPD_MAX_MODES];
  int64_t dims[CPD_MAX_MODES];
  const FiberSlot* table;
  unsigned long long cap;
  const uint2* ent;
  const int32_t* hot_rows;
  int N, m, R, Rp;
};
__global__ void __launch_bounds__(256) fit_fiber_kernel(FitFiberArgs a, const double* __restrict__ sigma,
                                                        double* __restrict__ part) {
  __shared__ double red[40];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int C = a.Rp / 4;
  const bool act = lane < C;
  const int q = act ? lane : 0;
  float sgv[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) sgv[c] = (act && 4 * q + c < a.R) ? (float)sigma[4 * q + c] : 0.0f;
  const float4 sg = make_float4(sgv[0], sgv[1], sgv[2], sgv[3]);
  const float4* Um = reinterpret_cast<const float4*>(a.U[a.m]);
  double tot = 0.0;
  for (int64_t s0 = warp * 32; s0 < (int64_t)a.cap; s0 += nwarps * 32) {
    FiberSlot fs;
    fs.key = CPD_EMPTY64; fs.beg = 0; fs.len = 0;
    if (s0 + lane < (int64_t)a.cap) fs = a.table[s0 + lane];
    unsigned occ = __ballot_sync(CPD_FULL, fs.key != CPD_EMPTY64);
    while (occ) {
      const int j = __ffs(occ) - 1;
      occ &= occ - 1u;
      unsigned long long key = __shfl_sync(CPD_FULL, fs.key, j);
      const uint32_t beg = __shfl_sync(CPD_FULL, fs.beg, j), len = __shfl_sync(CPD_FULL, fs.len, j);
      // h = sigma * (rows of the other factors); key = sum_k i_k stride_k
      // in mixed radix over the modes k != m in increasing order
      float4 hv = sg;
      const int klast = a.m == a.N - 1 ? a.N - 2 : a.N - 1;     // its index is what remains of the key
#pragma unroll
      for (int k = 0; k < CPD_MAX_MODES; ++k) {
        if (k >= a.N || k == a.m) continue;
        int64_t ik;
        if (k == klast) {
          ik = (int64_t)key;
        } else {
          const unsigned long long qk = key / (unsigned long long)a.dims[k];
          ik = (int64_t)(key - qk * (unsigned long long)a.dims[k]);
          key = qk;
        }
        const float4 u = reinterpret_cast<const float4*>(a.U[k] + ik * a.Rp)[q];
        hv.x *= u.x; hv.y *= u.y; hv.z *= u.z; hv.w *= u.w;
      }
      double zx = 0.0, zy = 0.0, zz = 0.0, zw = 0.0;
      for (uint32_t e0 = 0; e0 < len; e0 += 32) {
        const uint32_t n = len - e0 < 32u ? len - e0 : 32u;
        const uint2 en = lane < (int)n ? a.ent[beg + e0 + lane] : make_uint2(0u, 0u);
        uint32_t row = en.x;
        if (row & CPD_HOT_BIT) row = (uint32_t)a.hot_rows[row & ~CPD_HOT_BIT];
        const float v = __uint_as_float(en.y);
        float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 4
        for (uint32_t t = 0; t < n; ++t) {
          const uint32_t rt = __shfl_sync(CPD_FULL, row, (int)t);
          const float vt = __shfl_sync(CPD_FULL, v, (int)t);
          const float4 u = Um[(int64_t)rt * C + q];
          z.x = fmaf(vt, u.x, z.x); z.y = fmaf(vt, u.y, z.y); z.z = fmaf(vt, u.z, z.z); z.w = fmaf(vt, u.w, z.w);
        }
        zx += z.x; zy += z.y; zz += z.z; zw += z.w;
      }
      if (act) tot += (double)hv.x * zx + (double)hv.y * zy + (double)hv.z * zz + (double)hv.w * zw;
    }
  }
  double s = block_sum_d(tot, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void fit_final_kernel(const double* __restrict__ part, int nblk, FitArgs a, const double* G0,
                                 const double* G1, const double* G2, const double* G3, const double* G4,
                                 const double* G5, const double* G6, const double* G7,
                                 const double* __restrict__ sigma, double* __restrict__ out) {
  __shared__ double red[40];
  const double* Gs[8] = {G0, G1, G2, G3, G4, G5, G6, G7};
  const int t = threadIdx.x;
  double ip = 0.0;
  for (int b = t; b < nblk; b += blockDim.x) ip += part[b];
  ip = block_sum_d(ip, red);
  double mn = 0.0;
  for (int e = t; e < a.R * a.R; e += blockDim.x) {
    double v = sigma[e / a.R] * sigma[e % a.R];
    for (int k = 0; k < a.N; ++k) v *= Gs[k][e];
    mn += v;
  }
  mn = block_sum_d(mn, red);
  if (t == 0) { out[0] = ip; out[1] = mn; }
}

}  // namespace

// ---- launchers --------------------------------------------------------------

static cpd_status gram_from(cpd_ctx* h, const float* Uin, float* Uout, int64_t I, const double* sigma, int do_scale,
                            double* G) {
  const int R = h->R;
  PhaseTimer pt(h, CPD_PHASE_GRAM);
  if (cpd_gram_tc_supported(h) && I > 0) {      // tensor cores (fast precision option)
    int nblk = 0;
    cpd_status s = cpd_gram_tc_launch(h, Uin, Uout, I, sigma, do_scale, &nblk);
    if (s != CPD_OK) return s;
    gram_reduce_kernel<<<std::max(1, (R * (R + 1) / 2 + 7) / 8), 256, 0, h->stream>>>(h->Gpart, nblk, R, G);
    CPD_LAUNCH(h, "gram_reduce");
    return CPD_OK;
  }
  size_t shm = (size_t)TRP * R * sizeof(float);
  const int npairs = R * (R + 1) / 2;
  if (R > 64 && !h->opt.precision && (h->Rp / 4) * (h->Rp / 4 + 1) / 2 <= GB_MAXT) {
    // register-blocked kernel: (4x4 blocks of the upper block triangle) x row
    // groups per CTA, one CTA per SM, one partial per (CTA, row group)
    const int nb4 = h->Rp / 4, nblk = nb4 * (nb4 + 1) / 2;
    const int nrg = 1;
    if (nblk > GB_MAXT) return cpd_fail(h, CPD_ERR_INVALID_ARG, "Gram block triangle exceeds the kernel's block size");
    const int grid = std::max(1, std::min(CPD_GB_MINB * h->num_sms, h->gram_blocks / nrg));
    const size_t gshm = (size_t)16 * nblk * nrg * sizeof(double) + (size_t)GB_TR * h->Rp * sizeof(float);
    gram_blk_kernel<<<grid, nblk * nrg, gshm, h->stream>>>(Uin, Uout, I, R, h->Rp, sigma, do_scale, h->Gpart, nrg);
    CPD_LAUNCH(h, "gram_blk");
    gram_reduce_kernel<<<std::max(1, (npairs + 7) / 8), 256, 0, h->stream>>>(h->Gpart, grid * nrg, R, G);
    CPD_LAUNCH(h, "gram_reduce");
    return CPD_OK;
  }
  // Gram entries per thread: ceil(npairs / 256) rounded up to 1, 3, 9 or 33
  if (npairs <= DTHREADS)
    normalize_gram_kernel<1><<<h->gram_blocks, DTHREADS, shm, h->stream>>>(Uin, Uout, I, R, h->Rp, sigma, do_scale,
                                                                           h->Gpart, h->opt.precision);
  else if (npairs <= 3 * DTHREADS)
    normalize_gram_kernel<3><<<h->gram_blocks, DTHREADS, shm, h->stream>>>(Uin, Uout, I, R, h->Rp, sigma, do_scale,
                                                                           h->Gpart, h->opt.precision);
  else if (npairs <= 9 * DTHREADS)
    normalize_gram_kernel<9><<<h->gram_blocks, DTHREADS, shm, h->stream>>>(Uin, Uout, I, R, h->Rp, sigma, do_scale,
                                                                           h->Gpart, h->opt.precision);
  else
    normalize_gram_kernel<33><<<h->gram_blocks, DTHREADS, shm, h->stream>>>(Uin, Uout, I, R, h->Rp, sigma, do_scale,
                                                                            h->Gpart, h->opt.precision);
  CPD_LAUNCH(h, "normalize_gram");
  gram_reduce_kernel<<<std::max(1, (R * (R + 1) / 2 + 7) / 8), 256, 0, h->stream>>>(h->Gpart, h->gram_blocks, R, G);
  CPD_LAUNCH(h, "gram_reduce");
  return CPD_OK;
}

cpd_status cpd_gram(cpd_ctx* h, const float* U, int64_t I, double* G) {
  return gram_from(h, U, (float*)U, I, nullptr, 0, G);
}

// Algorithm 1's initialisation: normalise the columns of the initial factors.
cpd_status cpd_renormalize_inputs(cpd_ctx* h) {
  const int R = h->R;
  for (int k = 0; k < h->N; ++k) {
    colsq_kernel<<<h->gram_blocks, DTHREADS, 0, h->stream>>>(h->U[k], h->dims[k], R, h->Rp, h->colsq);
    sigma_kernel<<<R, 256, 0, h->stream>>>(h->colsq, h->gram_blocks, R, h->sigma);
    CPD_LAUNCH(h, "colsq/sigma");
    cpd_status s = gram_from(h, h->U[k], h->U[k], h->dims[k], h->sigma, 1, h->G[k]);
    if (s != CPD_OK) return s;
  }
  return CPD_OK;
}

static size_t pinv_smem(int R) {
  size_t slow = (size_t)R * R * sizeof(double);
  size_t fast = R <= PINV_FAST_R2 ? (size_t)5 * R * R * sizeof(float) : 0;
  return std::max(slow, fast);
}

static cpd_status launch_pinv(cpd_ctx* h, const PinvJobs& jobs, int njobs) {
  PhaseTimer pt(h, CPD_PHASE_PINV);
  const int R = h->R;
  size_t shm = pinv_smem(R);
  // the fast path's work per entry is fixed, so fewer threads with four
  // entries each issue fewer redundant per-step instructions
  const int threads = R <= PINV_FAST_R ? std::max(32, (R * R / PINV_PER_T + 31) / 32 * 32) : PINV_THREADS;
  pinv_kernel<<<njobs, threads, shm, h->stream>>>(jobs, R, h->opt.precision);
  CPD_LAUNCH(h, "pinv");
  return CPD_OK;
}

// G = *_{k != mode} G_k into Gout and its pseudo-inverse into Pout.
cpd_status cpd_hadamard_pinv(cpd_ctx* h, int mode, double* Gout, double* Pout, double* scratch) {
  PinvJobs jobs;
  memset(&jobs, 0, sizeof(jobs));
  PinvJob& j = jobs.job[0];
  for (int k = 0; k < h->N; ++k)
    if (k != mode) j.in[j.nin++] = h->G[k];
  j.out_had = Gout;
  j.out_pinv = Pout;
  j.out_split = Pout == h->Gnpinv ? h->Gnpinv_split : nullptr;
  j.scratch = scratch ? scratch : h->Gpart;   // 2 R^2 doubles
  j.status = h->status;
  return launch_pinv(h, jobs, 1);
}

cpd_status cpd_pinv_into(cpd_ctx* h, const double* G, double* P) {
  PinvJobs jobs;
  memset(&jobs, 0, sizeof(jobs));
  jobs.job[0].in[0] = G;
  jobs.job[0].nin = 1;
  jobs.job[0].out_pinv = P;
  jobs.job[0].out_split = P == h->Gnpinv ? h->Gnpinv_split : nullptr;
  jobs.job[0].scratch = h->Gpart;
  jobs.job[0].status = h->status;
  return launch_pinv(h, jobs, 1);
}

// U_mode = Y G^+ (G^+ already in h->Gnpinv), sigma, renormalise, Gram.
cpd_status cpd_solve_renorm(cpd_ctx* h, int mode, const float* Y, double* out_sigma) {
  const int R = h->R;
  const int64_t I = h->dims[mode];
  {
    PhaseTimer pt(h, CPD_PHASE_SOLVE);
    const int rb = solve_rb(R);
    size_t shm = (size_t)(R * rb) * sizeof(float);
    int nblk = h->gram_blocks;                  // column partials summed by sigma_kernel
    if (rb == 32) {
      // two resident blocks per SM (its launch bounds cap it at 128 registers a thread)
      nblk = (int)std::min<int64_t>(std::min(nblk, h->num_sms * 2), std::max<int64_t>(cpd_ceil_div(I, SOLVE_TR), 1));
      solve_lane_kernel<<<nblk, DTHREADS, 0, h->stream>>>(Y, h->Gnpinv_split, h->Uwork, I, R, h->Rp, h->colsq);
    } else if (rb == 16)
      solve_kernel<16><<<h->gram_blocks, DTHREADS, shm, h->stream>>>(Y, h->Gnpinv_split, h->Uwork, I, R, h->Rp, h->colsq);
    else {
      // as many blocks as are resident together (two per SM up to R ~ 100,
      // where the tile and G^+ take 104 KB of shared memory a block)
      const int nb = rb == 64 ? 64 : (R <= 112 ? 112 : 128), ty = solve_tile_ty(R, nb);
      const int threads = nb == 112 ? 14 * ty : 16 * ty;
      const void* fn = nb == 64 ? (const void*)solve_tile_kernel<64, 16, 16>
                                : nb == 112 ? (const void*)solve_tile_kernel<112, 16, 14>
                                            : (const void*)solve_tile_kernel<128, 16, 16>;
      const size_t sh = solve_tile_smem(R, nb, ty);
      int occ = 1;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, sh) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
      }
      nblk = (int)std::min<int64_t>(std::min<int64_t>((int64_t)occ * h->num_sms, h->gram_blocks),
                                    std::max<int64_t>(cpd_ceil_div(I, 8 * ty), 1));
      if (nb == 64)
        solve_tile_kernel<64, 16, 16><<<nblk, threads, sh, h->stream>>>(Y, h->Gnpinv_split, h->Uwork, I, R, h->Rp,
                                                                        h->colsq);
      else if (nb == 112)
        solve_tile_kernel<112, 16, 14><<<nblk, threads, sh, h->stream>>>(Y, h->Gnpinv_split, h->Uwork, I, R, h->Rp,
                                                                         h->colsq);
      else
        solve_tile_kernel<128, 16, 16><<<nblk, threads, sh, h->stream>>>(Y, h->Gnpinv_split, h->Uwork, I, R, h->Rp,
                                                                         h->colsq);
    }
    CPD_LAUNCH(h, "solve");
    sigma_kernel<<<R, 256, 0, h->stream>>>(h->colsq, nblk, R, h->sigma);
    CPD_LAUNCH(h, "sigma");
  }
  if (out_sigma && out_sigma != h->sigma)
    CPD_CUDA(h, cudaMemcpyAsync(out_sigma, h->sigma, R * sizeof(double), cudaMemcpyDefault, h->stream));
  return gram_from(h, h->Uwork, h->U[mode], I, h->sigma, 1, h->G[mode]);
}

// d_out[0] = <T, T~>, d_out[1] = ||T~||^2.
cpd_status cpd_fit_launch(cpd_ctx* h, double* d_out) {
  FitArgs a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k < h->N; ++k) a.U[k] = h->U[k];
  a.N = h->N; a.R = h->R; a.Rp = h->Rp;
  int nblk = h->gram_blocks;
  if (h->nnz > 0 && h->opt.deterministic) {
    // input order: the fiber table's slot order depends on its insertion
    // race, so the fiber walk's sum would not repeat bit for bit
    fit_inner_kernel<<<nblk, 256, 0, h->stream>>>(h->idx, h->vals, h->nnz, a, h->sigma, h->colsq);
  } else if (h->nnz > 0) {
    // the fibers of the mode with the fewest rows
    int m = 0;
    for (int k = 1; k < h->N; ++k)
      if (h->dims[k] < h->dims[m]) m = k;
    FitFiberArgs f;
    memset(&f, 0, sizeof(f));
    for (int k = 0; k < h->N; ++k) { f.U[k] = h->U[k]; f.dims[k] = h->dims[k]; }
    f.table = h->mode[m].table;
    f.cap = h->mode[m].mask + 1;
    f.ent = h->mode[m].ent;
    f.hot_rows = h->mode[m].hot_rows;
    f.N = h->N; f.m = m; f.R = h->R; f.Rp = h->Rp;
    fit_fiber_kernel<<<nblk, 256, 0, h->stream>>>(f, h->sigma, h->colsq);
  } else {
    CPD_CUDA(h, cudaMemsetAsync(h->colsq, 0, nblk * sizeof(double), h->stream));
  }
  const double* G[8];
  for (int k = 0; k < 8; ++k) G[k] = h->G[k < h->N ? k : 0];
  fit_final_kernel<<<1, 256, 0, h->stream>>>(h->colsq, nblk, a, G[0], G[1], G[2], G[3], G[4], G[5], G[6], G[7],
                                             h->sigma, d_out);
  CPD_LAUNCH(h, "fit");
  return CPD_OK;
}

// Kernels with more than 48 KB of dynamic shared memory need an opt-in.
cpd_status cpd_dense_init(cpd_ctx* h) {
  const int R = h->R;
  size_t s1 = (size_t)TRP * R * sizeof(float);
  size_t s2 = pinv_smem(R);
  size_t s3 = (size_t)(R * solve_rb(R)) * sizeof(float);
  const std::pair<const void*, size_t> attrs[] = {
      {(const void*)normalize_gram_kernel<1>, s1}, {(const void*)normalize_gram_kernel<3>, s1},
      {(const void*)normalize_gram_kernel<9>, s1}, {(const void*)normalize_gram_kernel<33>, s1},
      {(const void*)pinv_kernel, s2},              {(const void*)solve_kernel<16>, s3},
      {(const void*)solve_kernel<32>, s3},
      {(const void*)gram_blk_kernel, (size_t)16 * GB_MAXT * sizeof(double) + (size_t)GB_TR * CPD_MAX_RANK * sizeof(float)},
      {(const void*)solve_tile_kernel<64, 16, 16>, solve_tile_smem(std::min(R, 64), 64, 16)},
      {(const void*)solve_tile_kernel<112, 16, 14>, solve_tile_smem(std::min(R, 112), 112, 16)},
      {(const void*)solve_tile_kernel<128, 16, 16>, solve_tile_smem(R, 128, 16)}};
  for (const auto& a : attrs) {
    const cpd_status st = cpd_smem_attr(h, a.first, a.second);
    if (st != CPD_OK) return st;
  }
  return CPD_OK;
}
