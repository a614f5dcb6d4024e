// STS-CP: draws from the exact leverage-score distribution of U_{!=n}
// (Sec. 4.1 "STS-CP", Appendix B, Algorithms 4-5).
//
// Build (Algorithm 4 with one processor): per factor k a complete binary tree
// in heap order; leaf l holds the Gram of rows [l F, (l+1) F) of U_k, every
// internal node the sum of its children.  Matrices are stored as their upper
// triangle (a <= b, row-major), float32.  Leaf count L is a power of two; the
// leaves past the last row stay zero.
//
// Draw (Algorithm 5 with one processor): one warp per draw j.  For the factors
// k != n in ascending order, with h the Hadamard product of the rows already
// drawn (all ones at first) and G_{>k} = G^+ (*) Grams of the factors drawn
// after k:
//   m(v) = h^T (G^v (*) G_{>k}) h = sum_p c_p G^v_p M_p,  M_p = G_{>k,ab} h_a h_b
// (c_p = 2 off the diagonal); the walk keeps the absolute target
// t = u m(root), goes left iff t < m(left) and otherwise subtracts
// m(left); at the leaf the row masses q_i = (U_k[i] (*) h)^T G_{>k} (U_k[i] (*) h)
// are scanned (target rescaled by sum q / m(leaf)).  The draw probability is
// the exact leverage of the drawn row over the leverage total,
// p = h^T G^+ h / <G^+, G>_F.
//
// Precision.  A decision at depth d must resolve the target to a small
// fraction of m(v) ~ 2^-d m(root), and the target t = u m(root) - sum m(left)
// carries the rounding of every mass subtracted on the way, on the scale of
// m(root).  To take the decisions of a float64 statement of Algorithm 5
// (all but those within ~1e-13 m(root) of a threshold), precision option 0
// keeps the node Grams, the running Hadamard product h, the matrices
// M = G_{>k} (*) h h^T and the masses as double-floats (hi + lo float32
// pairs; exact TwoProduct, TwoSum accumulation) and the target in float64.
// The leaf's row masses are first computed in float32 with a bound on their
// error; only when a row boundary lies within that bound of the target is
// the leaf rescanned in double-float (rare: ~1e-4 of the draws).
// Precision option 1 keeps float32 trees, masses and target.
#include "common.cuh"
#include <algorithm>
#include <cstring>

namespace {

constexpr int STS_NW = 4;   // warps per block

__device__ __forceinline__ void pair_of(int p, int R, int& a, int& b) {
  int aa = 0, rem = p;
  while (rem >= R - aa) { rem -= R - aa; ++aa; }
  a = aa;
  b = aa + rem;
}

// Leaf Grams (float32 trees, precision 1): one block per leaf, the leaf's
// rows staged in shared memory.
__global__ void sts_leaf_kernel(const float* __restrict__ U, int64_t I, int R, int Rp, int F, int64_t L,
                                int64_t nleaf, float* __restrict__ tree) {
  extern __shared__ float rows[];      // F x R
  const int npairs = R * (R + 1) / 2;
  const int nstride = (npairs + 3) & ~3;
  for (int64_t l = blockIdx.x; l < nleaf; l += gridDim.x) {
    const int64_t r0 = l * F;
    const int nr = (int)(I - r0 < F ? I - r0 : F);
    __syncthreads();
    for (int e = threadIdx.x; e < F * R; e += blockDim.x) {
      int i = e / R, c = e % R;
      rows[e] = i < nr ? U[(r0 + i) * Rp + c] : 0.0f;
    }
    __syncthreads();
    float* out = tree + (L + l) * nstride;
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
      int a, b;
      pair_of(p, R, a, b);
      float s = 0.0f;
      for (int i = 0; i < nr; ++i) s = fmaf(rows[i * R + a], rows[i * R + b], s);
      out[p] = s;
    }
  }
}

// One level of the upward sums: nodes [lo, 2 lo), nstride floats per node
// (the packed upper triangle padded to a multiple of 4; the padding is 0).
__global__ void sts_up_kernel(float* __restrict__ tree, int64_t lo, int nstride) {
  const int64_t total = lo * nstride / 4;
  float4* t4 = reinterpret_cast<float4*>(tree);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = lo + e / (nstride / 4);
    const int64_t q = e % (nstride / 4);
    const float4 x = t4[(2 * v) * (nstride / 4) + q], y = t4[(2 * v + 1) * (nstride / 4) + q];
    t4[v * (nstride / 4) + q] = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
  }
}

// The upper levels [1, 2 lo) in one block, level by level (they are small;
// one launch instead of log2(lo) + 1).
__global__ void sts_up_top_kernel(float* __restrict__ tree, int64_t lo, int nstride) {
  float4* t4 = reinterpret_cast<float4*>(tree);
  const int q4 = nstride / 4;
  for (int64_t l = lo; l >= 1; l >>= 1) {
    for (int64_t e = threadIdx.x; e < l * q4; e += blockDim.x) {
      const int64_t v = l + e / q4, q = e % q4;
      const float4 x = t4[(2 * v) * q4 + q], y = t4[(2 * v + 1) * q4 + q];
      t4[v * q4 + q] = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
    }
    __syncthreads();
  }
}

// Double-float trees (precision 0): node v = hi[npad] then lo[npad].
// Leaf Grams with exact products and TwoSum accumulation over the leaf's rows.
__global__ void sts_leaf_df_kernel(const float* __restrict__ U, int64_t I, int R, int Rp, int F, int64_t L,
                                   int64_t nleaf, int npad, float* __restrict__ tree) {
  extern __shared__ float rows[];      // F x R
  const int npairs = R * (R + 1) / 2;
  for (int64_t l = blockIdx.x; l < nleaf; l += gridDim.x) {
    const int64_t r0 = l * F;
    const int nr = (int)(I - r0 < F ? I - r0 : F);
    __syncthreads();
    for (int e = threadIdx.x; e < F * R; e += blockDim.x) {
      int i = e / R, c = e % R;
      rows[e] = i < nr ? U[(r0 + i) * Rp + c] : 0.0f;
    }
    __syncthreads();
    float* out = tree + (L + l) * (2 * (int64_t)npad);
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
      int a, b;
      pair_of(p, R, a, b);
      float sh = 0.0f, sl = 0.0f;
      for (int i = 0; i < nr; ++i) df_fma(sh, sl, rows[i * R + a], rows[i * R + b]);
      df_renorm(sh, sl);
      out[p] = sh;
      out[npad + p] = sl;
    }
  }
}

__device__ __forceinline__ void df_add4(float4& xh, float4& xl, const float4 yh, const float4 yl) {
  float s, e;
  df_two_sum(xh.x, yh.x, s, e); xh.x = s; xl.x = __fadd_rn(__fadd_rn(xl.x, yl.x), e); df_renorm(xh.x, xl.x);
  df_two_sum(xh.y, yh.y, s, e); xh.y = s; xl.y = __fadd_rn(__fadd_rn(xl.y, yl.y), e); df_renorm(xh.y, xl.y);
  df_two_sum(xh.z, yh.z, s, e); xh.z = s; xl.z = __fadd_rn(__fadd_rn(xl.z, yl.z), e); df_renorm(xh.z, xl.z);
  df_two_sum(xh.w, yh.w, s, e); xh.w = s; xl.w = __fadd_rn(__fadd_rn(xl.w, yl.w), e); df_renorm(xh.w, xl.w);
}

// One level of double-float upward sums: nodes [lo, 2 lo).
__global__ void sts_up_df_kernel(float* __restrict__ tree, int64_t lo, int npad) {
  const int q4 = npad / 4;
  const int64_t total = lo * q4;
  float4* t4 = reinterpret_cast<float4*>(tree);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = lo + e / q4, q = e % q4;
    float4 xh = t4[(2 * v) * 2 * q4 + q], xl = t4[(2 * v) * 2 * q4 + q4 + q];
    const float4 yh = t4[(2 * v + 1) * 2 * q4 + q], yl = t4[(2 * v + 1) * 2 * q4 + q4 + q];
    df_add4(xh, xl, yh, yl);
    t4[v * 2 * q4 + q] = xh;
    t4[v * 2 * q4 + q4 + q] = xl;
  }
}

__global__ void sts_up_top_df_kernel(float* __restrict__ tree, int64_t lo, int npad) {
  float4* t4 = reinterpret_cast<float4*>(tree);
  const int q4 = npad / 4;
  for (int64_t l = lo; l >= 1; l >>= 1) {
    for (int64_t e = threadIdx.x; e < l * q4; e += blockDim.x) {
      const int64_t v = l + e / q4, q = e % q4;
      float4 xh = t4[(2 * v) * 2 * q4 + q], xl = t4[(2 * v) * 2 * q4 + q4 + q];
      const float4 yh = t4[(2 * v + 1) * 2 * q4 + q], yl = t4[(2 * v + 1) * 2 * q4 + q4 + q];
      df_add4(xh, xl, yh, yl);
      t4[v * 2 * q4 + q] = xh;
      t4[v * 2 * q4 + q4 + q] = xl;
    }
    __syncthreads();
  }
}

struct GgtArgs {
  const double* G[CPD_MAX_MODES];
  double* out[CPD_MAX_MODES];
  int N, n, R;
};

// G_{>k} = G^+ (*) (*)_{k' > k, k' != n} G_{k'} for every k != n, and the
// leverage total Z = <G^+, G>_F.
__global__ void sts_ggt_kernel(GgtArgs a, const double* __restrict__ Gp, const double* __restrict__ Gh,
                               double* __restrict__ Z) {
  __shared__ double red[32];
  const int RR = a.R * a.R;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) {
    for (int k = 0; k < a.N; ++k) {
      if (k == a.n) continue;
      double v = Gp[e];
      for (int k2 = k + 1; k2 < a.N; ++k2)
        if (k2 != a.n) v *= a.G[k2][e];
      a.out[k][e] = v;
    }
  }
  double s = 0.0;
  for (int e = threadIdx.x; e < RR; e += blockDim.x) s += Gp[e] * Gh[e];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double z = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) z += red[w];
    *Z = z;
  }
}

struct StsArgs {
  const float* tree;
  const float* U;
  const double* Ggt;
  const double* Z;
  float* Hs;
  int32_t* out_idx;
  double* out_p;
  double* out_w;
  const unsigned long long* d_sweep;
  unsigned long long h_sweep, seed;
  int64_t I, L, J;
  int R, Rp, F, D, npairs, k, n, N, first, last;
};

// Group-wide sum over the G lanes of a lane group (G a power of two <= 32).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(CPD_FULL, v, o);
  return v;
}

// A warp walks 32 / G draws at once, G lanes per draw: the tree is complete,
// so every group descends the same number of levels and only the loaded
// nodes differ, which gives the latency-bound descent 32 / G independent
// memory streams per warp.
template <int RB, int G>
__global__ void __launch_bounds__(STS_NW * 32) sts_draw_kernel(StsArgs a) {
  constexpr int DPW = 32 / G;                                      // draws per warp
  extern __shared__ float4 sm4[];
  float* Gs = reinterpret_cast<float*>(sm4);                      // R x R
  const int R = a.R, Rp = a.Rp, npairs = a.npairs;
  const int npad = (npairs + 3) & ~3;
  unsigned char* pa = reinterpret_cast<unsigned char*>(Gs + R * R);
  unsigned char* pb = pa + npad;
  // per-group scratch from the first 16-byte boundary after the pair tables
  float* wbase = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sm4) +
                                          (((size_t)R * R * 4 + 2 * (size_t)npad + 15) & ~(size_t)15));
  const int per_group = npad + Rp + ((a.F + 3) & ~3);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane % G;
  float* M = wbase + (wid * DPW + grp) * per_group;
  float* hs = M + npad;
  float* qb = hs + Rp;

  for (int e = threadIdx.x; e < R * R; e += blockDim.x) Gs[e] = (float)a.Ggt[e];
  for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
    int x, y;
    pair_of(p, R, x, y);
    pa[p] = (unsigned char)x;
    pb[p] = (unsigned char)y;
  }
  __syncthreads();
  const unsigned long long s = a.d_sweep ? *a.d_sweep : a.h_sweep;
  const double Z = *a.Z;
  const int64_t warp = (int64_t)blockIdx.x * STS_NW + wid;
  const int64_t nwarps = (int64_t)gridDim.x * STS_NW;

  // m(v) = sum_p G^v_p M_p over the node's padded packed triangle, 16-byte
  // vectors, two accumulators
  const float4* M4 = reinterpret_cast<const float4*>(M);
  auto mass = [&](int64_t v) -> float {
    const float4* g4 = reinterpret_cast<const float4*>(a.tree + v * npad);
    float acc0 = 0.0f, acc1 = 0.0f;
    for (int q = gl; q < npad / 4; q += G) {
      const float4 gv = g4[q], mv = M4[q];
      acc0 = fmaf(gv.x, mv.x, acc0);
      acc1 = fmaf(gv.y, mv.y, acc1);
      acc0 = fmaf(gv.z, mv.z, acc0);
      acc1 = fmaf(gv.w, mv.w, acc1);
    }
    return group_sum<G>(acc0 + acc1);
  };

  for (int64_t jb = warp * DPW; jb < a.J; jb += nwarps * DPW) {
    const int64_t j = jb + grp;
    const bool live = j < a.J;
    const int64_t jj = live ? j : a.J - 1;           // dead groups shadow a live draw, write nothing
    for (int r = gl; r < Rp; r += G) hs[r] = a.Hs[jj * Rp + r];
    __syncwarp();
    for (int p = gl; p < npad; p += G) {
      if (p < npairs) {
        const int x = pa[p], y = pb[p];
        M[p] = (x == y ? 1.0f : 2.0f) * Gs[x * R + y] * hs[x] * hs[y];
      } else {
        M[p] = 0.0f;
      }
    }
    __syncwarp();
    const double u = cpd_uniform(a.seed, CPD_STREAM_STS, (unsigned long long)jj, (unsigned long long)a.k,
                                 (unsigned long long)a.n, s);
    // float32 target: the masses themselves are float32 sums, so a float64
    // target would not make the decisions more exact (and FP64 is slow here)
    float t = (float)u * mass(1);
    int64_t v = 1;
    for (int depth = 0; depth < a.D; ++depth) {
      const int64_t left = 2 * v;
      const float mL = mass(left);
      const int64_t rfirst = (((left + 1) << (a.D - depth - 1)) - a.L) * a.F;
      if (t >= mL && rfirst < a.I) { t -= mL; v = left + 1; }
      else v = left;
    }
    const int64_t r0 = (v - a.L) * a.F;
    const int nr = (int)(a.I - r0 < a.F ? a.I - r0 : a.F);
    const float mleaf = mass(v);
    // row masses of the leaf, rows gl, gl + G, ... of the group
    float qpart = 0.0f;
    for (int i = gl; i < a.F; i += G) {
      float q = 0.0f;
      if (i < nr) {
        const float* urow = a.U + (r0 + i) * Rp;
        float x[RB];
#pragma unroll
        for (int c = 0; c < RB; ++c) x[c] = (c < R) ? urow[c] * hs[c] : 0.0f;
        // outer index at run time (x_c recomputed, same bits) keeps the
        // unrolled body at RB FMAs
#pragma unroll 2
        for (int c = 0; c < R; ++c) {
          float y = 0.0f;
#pragma unroll
          for (int b = 0; b < RB; ++b)
            if (b < R) y = fmaf(Gs[c * R + b], x[b], y);
          q = fmaf(urow[c] * hs[c], y, q);
        }
        qb[i] = q;
      }
      qpart += q;
    }
    __syncwarp();
    const float qs = group_sum<G>(qpart);
    const float tl = mleaf > 0.0f ? t * (qs / mleaf) : 0.0f;
    int found = -1;
    float carry = 0.0f;
    const unsigned gmask = (G == 32) ? CPD_FULL : (((1u << G) - 1u) << (grp * G));
    for (int c0 = 0; c0 < a.F; c0 += G) {
      const int i = c0 + gl;
      const float qd = (i < nr) ? qb[i] : 0.0f;
      float cum = qd;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        const float y = __shfl_up_sync(CPD_FULL, cum, o, G);
        if (gl >= o) cum += y;
      }
      cum += carry;
      const unsigned hit = __ballot_sync(CPD_FULL, i < nr && cum > tl) & gmask;
      if (found < 0 && hit) found = c0 + (__ffs(hit) - 1) - grp * G;
      carry = __shfl_sync(CPD_FULL, cum, G - 1, G);
    }
    // If rounding put the target past the end, take the last row of nonzero
    // mass.  Computed by every lane: `found` differs between the lane groups
    // of a warp, and warp votes must not sit under group-dependent branches.
    int fallback = 0;
    for (int c0 = 0; c0 < a.F; c0 += G) {
      const int i = c0 + gl;
      const unsigned pos = __ballot_sync(CPD_FULL, i < nr && qb[i] > 0.0f) & gmask;
      if (pos) fallback = c0 + (31 - __clz(pos)) - grp * G;
    }
    if (found < 0) found = fallback;
    const int64_t ik = r0 + found;
    if (gl == 0 && live) a.out_idx[(int64_t)a.k * a.J + j] = (int32_t)ik;
    __syncwarp();
    for (int r = gl; r < Rp; r += G) {
      const float hn = (r < R) ? hs[r] * a.U[ik * Rp + r] : 0.0f;
      hs[r] = hn;
      if (!a.last && live) a.Hs[j * Rp + r] = hn;
    }
    __syncwarp();
    if (a.last) {
      // G_{>k} of the last factor is G^+: leverage of the drawn KRP row
      float acc = 0.0f;
      for (int p = gl; p < npairs; p += G) {
        const int x = pa[p], y = pb[p];
        acc = fmaf((x == y ? 1.0f : 2.0f) * Gs[x * R + y], hs[x] * hs[y], acc);
      }
      acc = group_sum<G>(acc);
      if (gl == 0 && live) {
        const double prob = (double)acc / Z;
        if (a.out_p) a.out_p[j] = prob;
        if (a.out_w) a.out_w[j] = cpd_weight(a.J, prob);
      }
    }
    __syncwarp();
  }
}

struct StsDfArgs {
  const float* tree;       // double-float nodes, stride 2 npad
  const float* U;
  const double* Ggt;       // R x R, G_{>k}
  const double* Z;
  float* Hs;               // J x 2Rp: h as hi (Rp) then lo (Rp)
  int32_t* out_idx;
  double* out_p;
  double* out_w;
  int* fallbacks;
  const unsigned long long* d_sweep;
  unsigned long long h_sweep, seed;
  int64_t I, L, J;
  int R, Rp, F, D, npairs, k, n, last;
};

// Bytes of shared memory of the double-float walk: the coefficients
// c_p G_{>k,ab} as hi, lo and the pair tables, then per draw in flight M
// (hi, lo), h (hi, lo), the leaf's float32 row masses and a float64 buffer.
size_t sts_df_smem(int R, int F, int G, int nw) {
  const int npad = ((R * (R + 1) / 2) + 3) & ~3;
  const int Rp = cpd_pad4(R), Fp = (F + 3) & ~3;
  const size_t head = (((size_t)npad * 8 + 2 * (size_t)npad + 15) & ~(size_t)15) + 16;
  const size_t per_group = (size_t)(2 * npad + 2 * Rp + Fp + 2 * Fp) * 4;
  return head + (size_t)nw * (32 / G) * per_group;
}

// Algorithm 5 for factor k (not the first drawn) in double-float.  A warp
// walks 32 / G draws, G lanes each.  Node masses are Dot2 sums of the node's
// double-float Gram against M = c (*) G_{>k} (*) h h^T; the target is float64.
// At the leaf the row masses q_i = x_i^T G_{>k} x_i, x_i = U_k[i] (*) h, are
// computed in float32 (upper triangle: R(R+1)/2 + R FMAs a row) together
// with ||x_i||^2; with ga the largest absolute row sum of G_{>k}, the float32
// error of a running sum of q is below c1 * ga * (running sum of ||x||^2)
// + c2 * |running sum of q| (c1 ~ (2R + 8) 2^-24 from the two chained dot
// products and the rounding of their inputs, c2 ~ (F/G + 8) 2^-24 from the
// scan).  If every row boundary of every draw of the warp is farther than
// that from the target, the float32 choice is the exact one; otherwise the
// warp rescans its leaves in double-float.
template <int RB, int G>
__global__ void __launch_bounds__(STS_NW * 32) sts_walk_df_kernel(StsDfArgs a) {
  constexpr int DPW = 32 / G;
  extern __shared__ float4 sm4[];
  const int R = a.R, Rp = a.Rp, npairs = a.npairs, F = a.F;
  const int npad = (npairs + 3) & ~3;
  const int Fp = (F + 3) & ~3;
  float* Gh = reinterpret_cast<float*>(sm4);
  float* Gl = Gh + npad;
  unsigned char* pa = reinterpret_cast<unsigned char*>(Gl + npad);
  unsigned char* pb = pa + npad;
  float* misc = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sm4) +
                                         (((size_t)npad * 8 + 2 * (size_t)npad + 15) & ~(size_t)15));
  float* wbase = misc + 4;
  const int per_group = 2 * npad + 2 * Rp + Fp + 2 * Fp;
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane % G;
  float* Mh = wbase + (wid * DPW + grp) * per_group;
  float* Ml = Mh + npad;
  float* hh = Ml + npad;
  float* hl = hh + Rp;
  float* qb = hl + Rp;
  double* qd = reinterpret_cast<double*>(qb + Fp);
  float* eb = reinterpret_cast<float*>(qd);          // ||x||^2 during the float32 pass

  if (threadIdx.x == 0) misc[0] = 0.0f;
  for (int p = threadIdx.x; p < npad; p += blockDim.x) {
    if (p < npairs) {
      int x, y;
      pair_of(p, R, x, y);
      const double g = (x == y ? 1.0 : 2.0) * a.Ggt[x * R + y];
      const float gh = (float)g;
      Gh[p] = gh;
      Gl[p] = (float)(g - (double)gh);
      pa[p] = (unsigned char)x;
      pb[p] = (unsigned char)y;
    } else {
      Gh[p] = 0.0f; Gl[p] = 0.0f; pa[p] = 0; pb[p] = 0;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    double rs = 0.0;
    for (int b = 0; b < R; ++b) rs += fabs(a.Ggt[c * R + b]);
    atomicMax(reinterpret_cast<int*>(misc), __float_as_int((float)rs * 1.0001f));   // non-negative: int order
  }
  __syncthreads();
  const float c1 = (float)(2 * R + 8) * 0x1.02p-24f * misc[0];
  const float c2 = (float)((F + G - 1) / G + 8) * 0x1.02p-24f;
  const unsigned long long s = a.d_sweep ? *a.d_sweep : a.h_sweep;
  const int64_t warp = (int64_t)blockIdx.x * nw + wid;
  const int64_t nwarps = (int64_t)gridDim.x * nw;
  const unsigned gmask = (G == 32) ? CPD_FULL : (((1u << G) - 1u) << (grp * G));

  // m(v) in double-float, summed over the group; every lane of the group
  // gets the same bits (the butterfly's merges are symmetric)
  auto mass = [&](int64_t v) -> double {
    const float4* th4 = reinterpret_cast<const float4*>(a.tree + v * 2 * (int64_t)npad);
    const float4* tl4 = th4 + npad / 4;
    const float4* mh4 = reinterpret_cast<const float4*>(Mh);
    const float4* ml4 = reinterpret_cast<const float4*>(Ml);
    float s0h = 0.0f, s0l = 0.0f, s1h = 0.0f, s1l = 0.0f;
    const int nq = npad / 4;
    int q = gl;
    // four vectors of the node per lane in flight: the walk is bound by the
    // latency of these L2 loads, not by the double-float arithmetic
    for (; q + 3 * G < nq; q += 4 * G) {
      float4 th[4], tl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { th[u] = th4[q + u * G]; tl[u] = tl4[q + u * G]; }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 mh = mh4[q + u * G], ml = ml4[q + u * G];
        df_dot_step(s0h, s0l, th[u].x, tl[u].x, mh.x, ml.x);
        df_dot_step(s1h, s1l, th[u].y, tl[u].y, mh.y, ml.y);
        df_dot_step(s0h, s0l, th[u].z, tl[u].z, mh.z, ml.z);
        df_dot_step(s1h, s1l, th[u].w, tl[u].w, mh.w, ml.w);
      }
    }
    for (; q < nq; q += G) {
      const float4 th = th4[q], tl = tl4[q], mh = mh4[q], ml = ml4[q];
      df_dot_step(s0h, s0l, th.x, tl.x, mh.x, ml.x);
      df_dot_step(s1h, s1l, th.y, tl.y, mh.y, ml.y);
      df_dot_step(s0h, s0l, th.z, tl.z, mh.z, ml.z);
      df_dot_step(s1h, s1l, th.w, tl.w, mh.w, ml.w);
    }
    df_merge(s0h, s0l, s1h, s1l);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(CPD_FULL, s0h, o), ol = __shfl_xor_sync(CPD_FULL, s0l, o);
      df_merge(s0h, s0l, oh, ol);
    }
    return df_value(s0h, s0l);
  };

  for (int64_t jb = warp * DPW; jb < a.J; jb += nwarps * DPW) {
    const int64_t j = jb + grp;
    const bool live = j < a.J;
    const int64_t jj = live ? j : a.J - 1;           // dead groups shadow a live draw, write nothing
    for (int r = gl; r < Rp; r += G) {
      hh[r] = a.Hs[jj * 2 * Rp + r];
      hl[r] = a.Hs[jj * 2 * Rp + Rp + r];
    }
    __syncwarp();
    for (int p = gl; p < npad; p += G) {
      float mh = 0.0f, ml = 0.0f;
      if (p < npairs) {
        const int x = pa[p], y = pb[p];
        float ph, pl;
        df_mul(hh[x], hl[x], hh[y], hl[y], ph, pl);
        df_mul(Gh[p], Gl[p], ph, pl, mh, ml);
      }
      Mh[p] = mh;
      Ml[p] = ml;
    }
    __syncwarp();
    const double u = cpd_uniform(a.seed, CPD_STREAM_STS, (unsigned long long)jj, (unsigned long long)a.k,
                                 (unsigned long long)a.n, s);
    double t = u * mass(1);
    int64_t v = 1;
    for (int depth = 0; depth < a.D; ++depth) {
      const int64_t left = 2 * v;
      const double mL = mass(left);
      const int64_t rfirst = (((left + 1) << (a.D - depth - 1)) - a.L) * a.F;
      if (t >= mL && rfirst < a.I) { t -= mL; v = left + 1; }
      else v = left;
    }
    const int64_t r0 = (v - a.L) * a.F;
    const int nr = (int)(a.I - r0 < a.F ? a.I - r0 : a.F);
    // float32 row masses and ||x||^2 of the leaf
    for (int i = gl; i < F; i += G) {
      float q = 0.0f, e2 = 0.0f;
      if (i < nr) {
        const float* urow = a.U + (r0 + i) * Rp;
        float x[RB];
#pragma unroll
        for (int c = 0; c < RB; ++c) x[c] = (c < R) ? urow[c] * hh[c] : 0.0f;
        if constexpr (RB <= 64) {
          int pc = 0;                                 // start of packed row c
#pragma unroll
          for (int c = 0; c < RB; ++c) {
            if (c < R) {
              float y = 0.0f;
#pragma unroll
              for (int b = c; b < RB; ++b)
                if (b < R) y = fmaf(Gh[pc + b - c], x[b], y);
              q = fmaf(x[c], y, q);
              e2 = fmaf(x[c], x[c], e2);
              pc += R - c;
            }
          }
        } else {
          // large R: outer index at run time (x_c recomputed, same bits),
          // the packed row read where b >= c
          int pc = 0;
#pragma unroll 1
          for (int c = 0; c < R; ++c) {
            float y = 0.0f;
#pragma unroll
            for (int b = 0; b < RB; ++b)
              if (b < R && b >= c) y = fmaf(Gh[pc + b - c], x[b], y);
            const float xc = urow[c] * hh[c];
            q = fmaf(xc, y, q);
            e2 = fmaf(xc, xc, e2);
            pc += R - c;
          }
        }
      }
      if (i < F) { qb[i] = q; eb[i] = e2; }
    }
    __syncwarp();
    const float tf = (float)t;
    int found = -1;
    bool unsure = false;
    float carry = 0.0f, carrye = 0.0f;
    for (int c0 = 0; c0 < F; c0 += G) {
      const int i = c0 + gl;
      float cum = (i < nr) ? qb[i] : 0.0f, cume = (i < nr) ? eb[i] : 0.0f;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        const float y = __shfl_up_sync(CPD_FULL, cum, o, G);
        const float ye = __shfl_up_sync(CPD_FULL, cume, o, G);
        if (gl >= o) { cum += y; cume += ye; }
      }
      cum += carry;
      cume += carrye;
      if (i < nr) {
        const float tol = c1 * cume + c2 * fabsf(cum) + 0x1p-23f * fabsf(tf);
        if (!(fabsf(cum - tf) > tol)) unsure = true;
      }
      const unsigned hit = __ballot_sync(CPD_FULL, i < nr && cum > tf) & gmask;
      if (found < 0 && hit) found = c0 + (__ffs(hit) - 1) - grp * G;
      carry = __shfl_sync(CPD_FULL, cum, G - 1, G);
      carrye = __shfl_sync(CPD_FULL, cume, G - 1, G);
    }
    int fallback = 0;
    for (int c0 = 0; c0 < F; c0 += G) {
      const int i = c0 + gl;
      const unsigned pos = __ballot_sync(CPD_FULL, i < nr && qb[i] > 0.0f) & gmask;
      if (pos) fallback = c0 + (31 - __clz(pos)) - grp * G;
    }
    if (found < 0) found = fallback;
    if (__any_sync(CPD_FULL, unsure)) {
      // rescan the leaves of the whole warp in double-float (for a draw whose
      // float32 choice was certain this gives the same row)
      __syncwarp();
      for (int i = gl; i < F; i += G) {
        double qv = 0.0;
        if (i < nr) {
          const float* urow = a.U + (r0 + i) * Rp;
          float sh = 0.0f, sl = 0.0f;
          for (int p = 0; p < npairs; ++p) {
            const int x = pa[p], y = pb[p];
            float xh, xl, yh, yl, ph, pl;
            df_mul_f(hh[x], hl[x], urow[x], xh, xl);
            df_mul_f(hh[y], hl[y], urow[y], yh, yl);
            df_mul(xh, xl, yh, yl, ph, pl);
            df_dot_step(sh, sl, Gh[p], Gl[p], ph, pl);
          }
          qv = df_value(sh, sl);
        }
        qd[i] = qv;
      }
      __syncwarp();
      double cumd = 0.0;
      int f = -1, lastpos = 0;
      for (int i = 0; i < nr; ++i) {
        cumd += qd[i];
        if (f < 0 && cumd > t) f = i;
        if (qd[i] > 0.0) lastpos = i;
      }
      found = f >= 0 ? f : lastpos;
      if (gl == 0 && live && a.fallbacks) atomicAdd(a.fallbacks, 1);
    }
    const int64_t ik = r0 + found;
    if (gl == 0 && live) a.out_idx[(int64_t)a.k * a.J + j] = (int32_t)ik;
    __syncwarp();
    for (int r = gl; r < Rp; r += G) {
      float nh = 0.0f, nl = 0.0f;
      if (r < R) df_mul_f(hh[r], hl[r], a.U[ik * Rp + r], nh, nl);
      hh[r] = nh;
      hl[r] = nl;
      if (!a.last && live) {
        a.Hs[j * 2 * Rp + r] = nh;
        a.Hs[j * 2 * Rp + Rp + r] = nl;
      }
    }
    __syncwarp();
    if (a.last) {
      // G_{>k} of the last factor is G^+: leverage of the drawn KRP row
      float sh = 0.0f, sl = 0.0f;
      for (int p = gl; p < npairs; p += G) {
        const int x = pa[p], y = pb[p];
        float ph, pl;
        df_mul(hh[x], hl[x], hh[y], hl[y], ph, pl);
        df_dot_step(sh, sl, Gh[p], Gl[p], ph, pl);
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(CPD_FULL, sh, o), ol = __shfl_xor_sync(CPD_FULL, sl, o);
        df_merge(sh, sl, oh, ol);
      }
      if (gl == 0 && live) {
        const double prob = df_value(sh, sl) / *a.Z;
        if (a.out_p) a.out_p[j] = prob;
        if (a.out_w) a.out_w[j] = cpd_weight(a.J, prob);
      }
    }
    __syncwarp();
  }
}

// The first factor drawn has h = 1, so its conditional row masses
// q_i = U_k[i] G_{>k} U_k[i]^T are the same for every draw and the tree's node
// masses are partial sums of them: the walk is an inverse CDF over q
// (computed once, in df64, by cpd_quadform_cdf).  One thread per draw.
__global__ void sts_first_kernel(const double* __restrict__ cdf, const double* __restrict__ q, int64_t I,
                                 const float* __restrict__ U, int Rp, float* __restrict__ Hs,
                                 int32_t* __restrict__ out_idx, double* __restrict__ out_p, double* __restrict__ out_w,
                                 const double* __restrict__ Zp, int last, int k, int n, int64_t J,
                                 unsigned long long seed, const unsigned long long* __restrict__ d_sweep,
                                 unsigned long long h_sweep, int df) {
  const unsigned long long s = d_sweep ? *d_sweep : h_sweep;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < J; j += (int64_t)gridDim.x * blockDim.x) {
    const double C = cdf[I - 1];
    const bool degenerate = !(C > 0.0) || !isfinite(C);    // all row masses zero
    const double t = cpd_uniform(seed, CPD_STREAM_STS, (unsigned long long)j, (unsigned long long)k,
                                 (unsigned long long)n, s) * C;
    const int64_t lo = degenerate ? 0 : cpd_inverse_cdf(cdf, I, t);
    out_idx[(int64_t)k * J + j] = (int32_t)lo;
    out_idx[(int64_t)n * J + j] = -1;
    if (last) {
      const double prob = degenerate ? 0.0 : q[lo] / *Zp;
      if (out_p) out_p[j] = prob;
      if (out_w) out_w[j] = cpd_weight(J, prob);
    } else {
      const float4* src = reinterpret_cast<const float4*>(U + lo * Rp);
      float4* dst = reinterpret_cast<float4*>(Hs + j * Rp * (df ? 2 : 1));
      for (int v = 0; v < Rp / 4; ++v) dst[v] = src[v];
      if (df)                                   // lo part of the double-float h
        for (int v = 0; v < Rp / 4; ++v) dst[Rp / 4 + v] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
}

// shared memory of the float32 walk with G lanes per draw
size_t sts_smem(int R, int F, int G) {
  const int npairs = R * (R + 1) / 2;
  const int npad = (npairs + 3) & ~3;
  const int Rp = cpd_pad4(R);
  const int per_group = npad + Rp + ((F + 3) & ~3);
  return (((size_t)R * R * 4 + 2 * (size_t)npad + 15) & ~(size_t)15) + (size_t)STS_NW * (32 / G) * per_group * 4;
}

constexpr size_t STS_SMEM_MAX = 227 * 1024;

// warps per block of the double-float walk: the most (<= 4) that fit
int sts_df_warps(int R, int F, int G) {
  for (int nw = STS_NW; nw >= 1; nw >>= 1)
    if (sts_df_smem(R, F, G, nw) <= STS_SMEM_MAX) return nw;
  return 0;
}

template <int RB, int G>
cpd_status launch_draw_g(cpd_ctx* h, const StsArgs& a) {
  const size_t shm = sts_smem(h->R, h->F, G);
  const int64_t blocks = std::min<int64_t>(cpd_ceil_div(a.J, STS_NW * (32 / G)), (int64_t)h->num_sms * 16);
  sts_draw_kernel<RB, G><<<(unsigned)blocks, STS_NW * 32, shm, h->stream>>>(a);
  CPD_LAUNCH(h, "sts_draw");
  return CPD_OK;
}

template <int RB, int G>
cpd_status launch_walk_df_g(cpd_ctx* h, const StsDfArgs& a) {
  const int nw = sts_df_warps(h->R, h->F, G);
  if (nw == 0) return cpd_fail(h, CPD_ERR_INVALID_ARG, "STS-CP walk does not fit in shared memory");
  const size_t shm = sts_df_smem(h->R, h->F, G, nw);
  const int64_t blocks = std::min<int64_t>(cpd_ceil_div(a.J, nw * (32 / G)), (int64_t)h->num_sms * 16);
  sts_walk_df_kernel<RB, G><<<(unsigned)blocks, nw * 32, shm, h->stream>>>(a);
  CPD_LAUNCH(h, "sts_walk_df");
  return CPD_OK;
}

template <int RB>
cpd_status launch_draw(cpd_ctx* h, const StsArgs& a) {
  if (h->tune_sts_g == 8) return launch_draw_g<RB, 8>(h, a);
  if (h->tune_sts_g == 32) return launch_draw_g<RB, 32>(h, a);
  return launch_draw_g<RB, 16>(h, a);
}

template <int RB>
cpd_status launch_walk_df(cpd_ctx* h, const StsDfArgs& a) {
  if (h->tune_sts_g == 8) return launch_walk_df_g<RB, 8>(h, a);
  if (h->tune_sts_g == 32) return launch_walk_df_g<RB, 32>(h, a);
  return launch_walk_df_g<RB, 16>(h, a);
}

template <int RB>
cpd_status set_draw_smem(cpd_ctx* h) {
  if (h->tree_df) {
    for (int g : {8, 16, 32}) {
      const int nw = sts_df_warps(h->R, h->F, g);
      if (nw == 0) continue;
      const void* f = g == 8 ? (const void*)sts_walk_df_kernel<RB, 8>
                             : g == 16 ? (const void*)sts_walk_df_kernel<RB, 16> : (const void*)sts_walk_df_kernel<RB, 32>;
      const cpd_status st_ = cpd_smem_attr(h, f, sts_df_smem(h->R, h->F, g, nw));
      if (st_ != CPD_OK) return st_;
    }
    return CPD_OK;
  }
  if (sts_smem(h->R, h->F, 8) <= STS_SMEM_MAX)
    { const cpd_status st_ = cpd_smem_attr(h, (const void*)sts_draw_kernel<RB, 8>, sts_smem(h->R, h->F, 8)); if (st_ != CPD_OK) return st_; }
  if (sts_smem(h->R, h->F, 16) <= STS_SMEM_MAX)
    { const cpd_status st_ = cpd_smem_attr(h, (const void*)sts_draw_kernel<RB, 16>, sts_smem(h->R, h->F, 16)); if (st_ != CPD_OK) return st_; }
  if (sts_smem(h->R, h->F, 32) <= STS_SMEM_MAX)
    { const cpd_status st_ = cpd_smem_attr(h, (const void*)sts_draw_kernel<RB, 32>, sts_smem(h->R, h->F, 32)); if (st_ != CPD_OK) return st_; }
  return CPD_OK;
}

}  // namespace

// Whether the walk with G lanes per draw fits in shared memory.
bool cpd_sts_group_fits(cpd_ctx* h, int G) {
  if (h->tree_df) return sts_df_warps(h->R, h->F, G) > 0;
  return sts_smem(h->R, h->F, G) <= STS_SMEM_MAX;
}

// Bytes of the trees of all factors for leaf size F.
size_t cpd_sts_tree_bytes(const cpd_ctx* h, int F) {
  const size_t npairs = (size_t)(((h->R * (h->R + 1) / 2) + 3) & ~3);   // padded node stride
  size_t total = 0;
  for (int k = 0; k < h->N; ++k) {
    const int64_t nleaf = cpd_ceil_div(h->dims[k], F);
    int64_t L = 1;
    while (L < nleaf) L <<= 1;
    total += (size_t)(2 * L) * npairs * sizeof(float) * (h->tree_df ? 2 : 1);
  }
  return total;
}

bool cpd_sts_leaf_rows_valid(const cpd_ctx* h, int F) {
  if (F < 1 || F > 1024 || (int64_t)F * h->R > 16384) return false;
  if (h->tree_df) return sts_df_warps(h->R, F, 32) > 0;
  return sts_smem(h->R, F, 32) <= STS_SMEM_MAX;
}

// (Re)allocate the trees for leaf size h->F (the old ones are freed) and set
// the launch limits that depend on F.
static cpd_status sts_trees(cpd_ctx* h) {
  const int R = h->R;
  const int npad = ((R * (R + 1) / 2) + 3) & ~3;   // packed triangle padded to 4
  h->tree_stride = npad * (h->tree_df ? 2 : 1);
  if (!cpd_sts_leaf_rows_valid(h, h->F))
    return cpd_fail(h, CPD_ERR_INVALID_ARG, "STS-CP leaf_rows must satisfy 1 <= F <= 1024, F * R <= 16384 "
                                            "and the walk's shared memory must fit");
  if (!cpd_sts_group_fits(h, h->tune_sts_g)) h->tune_sts_g = cpd_sts_group_fits(h, 16) ? 16 : 32;
  cpd_status s;
  for (int k = 0; k < h->N; ++k) {
    if (h->tree[k]) { cpd_free(h, h->tree[k]); h->tree[k] = nullptr; }
    const int64_t nleaf = cpd_ceil_div(h->dims[k], h->F);
    int64_t L = 1;
    while (L < nleaf) L <<= 1;
    h->L[k] = L;
    if ((s = cpd_alloc(h, &h->tree[k], (size_t)(2 * L) * h->tree_stride)) != CPD_OK) return s;
    CPD_CUDA(h, cudaMemsetAsync(h->tree[k], 0, (size_t)(2 * L) * h->tree_stride * sizeof(float), h->stream));
  }
  if ((s = set_draw_smem<32>(h)) != CPD_OK) return s;
  if ((s = set_draw_smem<64>(h)) != CPD_OK) return s;
  if ((s = set_draw_smem<128>(h)) != CPD_OK) return s;
  return cpd_smem_attr(h, h->tree_df ? (const void*)sts_leaf_df_kernel : (const void*)sts_leaf_kernel,
                       (size_t)h->F * R * 4);
}

cpd_status cpd_sts_alloc(cpd_ctx* h) {
  const int R = h->R;
  h->tune_sts_g = 16;
  h->tree_df = h->opt.precision == 0;
  if (h->opt.leaf_rows <= 0) {
    // default leaf size: the smallest of 8, 16, 32 (below R) whose trees fit
    // in 8 GB, else R.  Small leaves shorten each walk's leaf scan (R = 100,
    // 2e7 nonzeros: 2.18 sweeps/s at F = 100, 3.03 at 50, 4.11 at 25, 4.47
    // at 10), while the trees grow as I / F nodes of R(R+1)/2 entries.
    h->F = R;
    for (int F : {8, 16, 32})
      if (F < R && cpd_sts_leaf_rows_valid(h, F) && cpd_sts_tree_bytes(h, F) <= ((size_t)8 << 30)) {
        h->F = F;
        break;
      }
  }
  cpd_status s;
  if ((s = sts_trees(h)) != CPD_OK) return s;
  for (int k = 0; k < h->N; ++k)
    if ((s = cpd_alloc(h, &h->sts_ggt[k], (size_t)R * R)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->sts_Z, 1)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->sts_h, (size_t)std::max<int64_t>(h->opt.samples, 1) * h->Rp * (h->tree_df ? 2 : 1))) !=
      CPD_OK)
    return s;
  if ((s = cpd_alloc(h, &h->sts_q, (size_t)h->Imax)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->sts_cdf, (size_t)h->Imax)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->sts_blk, (size_t)cpd_ceil_div(h->Imax, 256))) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->sts_fallbacks, 1)) != CPD_OK) return s;
  CPD_CUDA(h, cudaMemsetAsync(h->sts_fallbacks, 0, sizeof(int), h->stream));
  return CPD_OK;
}

cpd_status cpd_sts_refresh(cpd_ctx* h, int k);

// New leaf size: trees rebuilt from the current factors.
cpd_status cpd_sts_set_leaf_rows(cpd_ctx* h, int F) {
  h->F = F;
  cpd_status s = sts_trees(h);
  for (int k = 0; k < h->N && s == CPD_OK; ++k) s = cpd_sts_refresh(h, k);
  return s;
}

// Algorithm 4 with one processor: leaf Grams, then the levels upward.
cpd_status cpd_sts_refresh(cpd_ctx* h, int k) {
  PhaseTimer pt(h, CPD_PHASE_SAMPLER);
  const int R = h->R, npad = ((R * (R + 1) / 2) + 3) & ~3;
  const int64_t I = h->dims[k], L = h->L[k];
  const int64_t nleaf = cpd_ceil_div(I, h->F);
  const int grid = (int)std::min<int64_t>(nleaf, (int64_t)h->num_sms * 8);
  if (h->tree_df)
    sts_leaf_df_kernel<<<grid, 256, (size_t)h->F * R * 4, h->stream>>>(h->U[k], I, R, h->Rp, h->F, L, nleaf, npad,
                                                                       h->tree[k]);
  else
    sts_leaf_kernel<<<grid, 256, (size_t)h->F * R * 4, h->stream>>>(h->U[k], I, R, h->Rp, h->F, L, nleaf, h->tree[k]);
  CPD_LAUNCH(h, "sts_leaf");
  int64_t lo = L / 2;
  for (; lo > 64; lo /= 2) {
    const int64_t total = lo * npad / 4;
    const int g = (int)std::min<int64_t>(cpd_ceil_div(total, 256), (int64_t)h->num_sms * 8);
    if (h->tree_df) sts_up_df_kernel<<<g, 256, 0, h->stream>>>(h->tree[k], lo, npad);
    else sts_up_kernel<<<g, 256, 0, h->stream>>>(h->tree[k], lo, npad);
    CPD_LAUNCH(h, "sts_up");
  }
  if (lo >= 1) {
    if (h->tree_df) sts_up_top_df_kernel<<<1, 1024, 0, h->stream>>>(h->tree[k], lo, npad);
    else sts_up_top_kernel<<<1, 1024, 0, h->stream>>>(h->tree[k], lo, npad);
    CPD_LAUNCH(h, "sts_up_top");
  }
  return CPD_OK;
}

// Requires h->Gn / h->Gnpinv of `mode` (cpd_hadamard_pinv) on the stream.
cpd_status cpd_sts_draw(cpd_ctx* h, int mode, int64_t J, const unsigned long long* d_sweep, unsigned long long sweep,
                        int32_t* out_idx, double* out_p, double* out_w) {
  if (J <= 0) return CPD_OK;
  PhaseTimer pt(h, CPD_PHASE_DRAW);
  GgtArgs g;
  memset(&g, 0, sizeof(g));
  for (int k = 0; k < h->N; ++k) { g.G[k] = h->G[k]; g.out[k] = h->sts_ggt[k]; }
  g.N = h->N; g.n = mode; g.R = h->R;
  sts_ggt_kernel<<<1, 256, 0, h->stream>>>(g, h->Gnpinv, h->Gn, h->sts_Z);
  CPD_LAUNCH(h, "sts_ggt");
  int firstk = -1, lastk = -1;
  for (int k = 0; k < h->N; ++k)
    if (k != mode) { if (firstk < 0) firstk = k; lastk = k; }
  for (int k = 0; k < h->N; ++k) {
    if (k == mode) continue;
    if (k == firstk) {
      cpd_status s = cpd_quadform_cdf(h, h->U[k], h->dims[k], h->sts_ggt[k], h->sts_q, h->sts_blk, h->sts_cdf);
      if (s != CPD_OK) return s;
      const int grid = (int)std::min<int64_t>(cpd_ceil_div(J, 256), (int64_t)h->num_sms * 8);
      sts_first_kernel<<<grid, 256, 0, h->stream>>>(h->sts_cdf, h->sts_q, h->dims[k], h->U[k], h->Rp, h->sts_h,
                                                    out_idx, out_p, out_w, h->sts_Z, k == lastk, k, mode, J,
                                                    h->opt.seed, d_sweep, sweep, h->tree_df ? 1 : 0);
      CPD_LAUNCH(h, "sts_first");
      continue;
    }
    int D = 0;
    while ((1ll << D) < h->L[k]) ++D;
    cpd_status s;
    if (h->tree_df) {
      StsDfArgs a;
      memset(&a, 0, sizeof(a));
      a.tree = h->tree[k]; a.U = h->U[k]; a.Ggt = h->sts_ggt[k]; a.Z = h->sts_Z; a.Hs = h->sts_h;
      a.out_idx = out_idx; a.out_p = out_p; a.out_w = out_w; a.fallbacks = h->sts_fallbacks;
      a.d_sweep = d_sweep; a.h_sweep = sweep; a.seed = h->opt.seed;
      a.I = h->dims[k]; a.L = h->L[k]; a.J = J;
      a.R = h->R; a.Rp = h->Rp; a.F = h->F; a.npairs = h->R * (h->R + 1) / 2;
      a.D = D; a.k = k; a.n = mode; a.last = (k == lastk);
      if (h->R <= 32) s = launch_walk_df<32>(h, a);
      else if (h->R <= 64) s = launch_walk_df<64>(h, a);
      else s = launch_walk_df<128>(h, a);
    } else {
      StsArgs a;
      memset(&a, 0, sizeof(a));
      a.tree = h->tree[k]; a.U = h->U[k]; a.Ggt = h->sts_ggt[k]; a.Z = h->sts_Z; a.Hs = h->sts_h;
      a.out_idx = out_idx; a.out_p = out_p; a.out_w = out_w;
      a.d_sweep = d_sweep; a.h_sweep = sweep; a.seed = h->opt.seed;
      a.I = h->dims[k]; a.L = h->L[k]; a.J = J;
      a.R = h->R; a.Rp = h->Rp; a.F = h->F; a.npairs = h->R * (h->R + 1) / 2;
      a.D = D; a.k = k; a.n = mode; a.N = h->N; a.first = (k == firstk); a.last = (k == lastk);
      if (h->R <= 32) s = launch_draw<32>(h, a);
      else if (h->R <= 64) s = launch_draw<64>(h, a);
      else s = launch_draw<128>(h, a);
    }
    if (s != CPD_OK) return s;
  }
  return CPD_OK;
}

// Leaves rescanned in double-float since creation (precision 0); 0 otherwise.
cpd_status cpd_sts_fallback_count(cpd_ctx* h, int64_t* out) {
  *out = 0;
  if (!h->sts_fallbacks) return CPD_OK;
  int v = 0;
  CPD_CUDA(h, cudaMemcpyAsync(&v, h->sts_fallbacks, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CPD_CUDA(h, cudaStreamSynchronize(h->stream));
  *out = v;
  return CPD_OK;
}
