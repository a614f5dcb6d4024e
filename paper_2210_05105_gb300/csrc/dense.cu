// Dense kernels of the ALS update: Grams (Eq. 5 operands), Hadamard product
// of Grams and its Moore-Penrose pseudo-inverse (Eq. 4-5), the solve
// U_n = Y G^+ with column renormalisation (Algorithm 1 lines 6-8), and the
// fit of Sec. 5.1.
//
// Precision: factor storage and the solve GEMM are float32; Grams, the R x R
// algebra and the fit accumulate in float64 (the sampler's inverse CDF is
// decided on float64 leverage scores, so the Grams feeding them are float64).
#include "common.cuh"
#include <algorithm>
#include <cmath>
#include <cstring>

namespace {

constexpr int TR = 64;          // rows per tile
constexpr int DTHREADS = 256;
constexpr int MAXP = 33;        // ceil(128 * 129 / 2 / 256) Gram pairs per thread

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

// sigma_r = sqrt(sum of partials), fixed order.
__global__ void sigma_kernel(const double* __restrict__ part, int nblk, int R, double* __restrict__ sigma) {
  int r = threadIdx.x;
  if (r < R) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * R + r];
    sigma[r] = sqrt(s);
  }
}

// U_out = U_in / sigma (columns with sigma = 0 kept), padded columns zeroed,
// and float64 Gram partials of the stored float32 values.  Per 64-row tile a
// thread accumulates its Gram entries as df64 sums of exact float32 products
// (error ~ 64 * 2^-48 of the sum of |terms|), then adds them into float64.
__global__ void __launch_bounds__(DTHREADS) normalize_gram_kernel(
    const float* __restrict__ Uin, float* __restrict__ Uout, int64_t I, int R, int Rp,
    const double* __restrict__ sigma, int do_scale, double* __restrict__ gpart) {
  extern __shared__ float tile[];                      // TR x R float32
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
  double acc[MAXP];
#pragma unroll
  for (int m = 0; m < MAXP; ++m) acc[m] = 0.0;
  const int64_t ntiles = cpd_ceil_div(I, TR);
  for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const int64_t r0 = tl * TR;
    for (int e = t; e < TR * Rp; e += DTHREADS) {
      int rr = e / Rp, c = e % Rp;
      int64_t i = r0 + rr;
      if (i < I) {
        float v = 0.0f;
        if (c < R) v = Uin[i * Rp + c] * inv[c];
        Uout[i * Rp + c] = v;
        if (c < R) tile[rr * R + c] = v;
      } else if (c < R) {
        tile[rr * R + c] = 0.0f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < MAXP; ++m) {
      int p = t + m * DTHREADS;
      if (p < npairs) {
        const int a = pa[p], b = pb[p];
        float hi = 0.0f, lo = 0.0f;
#pragma unroll 8
        for (int rr = 0; rr < TR; ++rr) df_fma(hi, lo, tile[rr * R + a], tile[rr * R + b]);
        acc[m] += df_value(hi, lo);
      }
    }
    __syncthreads();
  }
  double* out = gpart + (int64_t)blockIdx.x * npairs;
#pragma unroll
  for (int m = 0; m < MAXP; ++m) {
    int p = t + m * DTHREADS;
    if (p < npairs) out[p] = acc[m];
  }
}

// G = sum of block partials in fixed order; full symmetric R x R.
__global__ void gram_reduce_kernel(const double* __restrict__ gpart, int nblk, int R, double* __restrict__ G) {
  const int npairs = R * (R + 1) / 2;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
    int a = 0, rem = p;
    while (rem >= R - a) { rem -= R - a; ++a; }
    int b = a + rem;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += gpart[(int64_t)k * npairs + p];
    G[a * R + b] = s;
    G[b * R + a] = s;
  }
}

// ---- pseudo-inverse of a symmetric PSD R x R matrix ----------------------
struct PinvJob {
  const double* in[CPD_MAX_MODES];  // Hadamard factors
  int nin;
  double* out_had;                  // may be null
  double* out_pinv;
  double* out_factor;               // may be null: B with G^+ = B^T B
  int* out_tri;                     // may be null: 1 if B is lower triangular
  double* scratch;                  // 2 R x R float64 (global)
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

// Cholesky G = L L^T and G^{-1} = L^{-T} L^{-1} when every pivot exceeds
// 1e-9 * max diag; otherwise a parallel (round-robin) cyclic Jacobi
// eigendecomposition with eigenvalues <= R 2^-52 lambda_max dropped.
__global__ void __launch_bounds__(DTHREADS) pinv_kernel(PinvJobs jobs, int R) {
  extern __shared__ double A[];                     // R x R
  __shared__ double red[40];
  __shared__ int flag;
  __shared__ int sp[64], sq[64];
  __shared__ double sc[64], ss[64];
  const PinvJob& jb = jobs.job[blockIdx.x];
  const int t = threadIdx.x, nt = blockDim.x;
  const int RR = R * R;
  for (int e = t; e < RR; e += nt) {
    double v = 1.0;
    for (int k = 0; k < jb.nin; ++k) v *= jb.in[k][e];
    A[e] = v;
    if (jb.out_had) jb.out_had[e] = v;
  }
  if (t == 0) flag = 0;
  __syncthreads();
  double maxdiag = 0.0;
  for (int a = 0; a < R; ++a) maxdiag = fmax(maxdiag, fabs(A[a * R + a]));
  // -- Cholesky, lower triangle in place
  for (int k = 0; k < R; ++k) {
    if (t == 0) {
      double d = A[k * R + k];
      if (!(d > 1e-9 * maxdiag) || !isfinite(d)) flag = 1;
      else A[k * R + k] = sqrt(d);
    }
    __syncthreads();
    if (flag) break;
    const double lkk = A[k * R + k];
    for (int i = k + 1 + t; i < R; i += nt) A[i * R + k] /= lkk;
    __syncthreads();
    const int m = R - k - 1;
    for (int e = t; e < m * m; e += nt) {
      int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) A[i * R + j] -= A[i * R + k] * A[j * R + k];
    }
    __syncthreads();
  }
  double* W = jb.scratch;             // R x R
  double* V = jb.scratch + RR;        // R x R
  if (!flag) {
    // W = L^{-1}, one column per thread
    for (int j = t; j < R; j += nt) {
      for (int i = 0; i < j; ++i) W[i * R + j] = 0.0;
      W[j * R + j] = 1.0 / A[j * R + j];
      for (int i = j + 1; i < R; ++i) {
        double s = 0.0;
        for (int m = j; m < i; ++m) s = fma(A[i * R + m], W[m * R + j], s);
        W[i * R + j] = -s / A[i * R + i];
      }
    }
    __syncthreads();
    for (int e = t; e < RR; e += nt) {
      int a = e / R, b = e % R;
      int m0 = a > b ? a : b;
      double s = 0.0;
      for (int m = m0; m < R; ++m) s = fma(W[m * R + a], W[m * R + b], s);
      jb.out_pinv[e] = s;
      if (jb.out_factor) jb.out_factor[e] = W[e];
    }
    if (t == 0 && jb.out_tri) *jb.out_tri = 1;
    return;
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
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int e = t; e < RR; e += nt) {
      double v = A[e];
      if (e / R == e % R) dg += v * v; else off += v * v;
    }
    off = block_sum_d(off, red);
    dg = block_sum_d(dg, red);
    if (off <= ((double)R * eps) * ((double)R * eps) * dg) break;
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
    if (jb.out_factor) {   // row m of B: sqrt(1 / lambda_m) v_m^T
      double lam = A[a * R + a];
      jb.out_factor[e] = (lam > cut) ? V[b * R + a] / sqrt(lam) : 0.0;
    }
  }
  if (t == 0 && jb.out_tri) *jb.out_tri = 0;
}

// ---- solve: Uw = Y (P_hi + P_lo), float32 with the float64 G^+ split ----
__global__ void __launch_bounds__(DTHREADS) solve_kernel(
    const float* __restrict__ Y, const double* __restrict__ P, float* __restrict__ Uw, int64_t I, int R,
    int Rp, double* __restrict__ colpart) {
  extern __shared__ float sm[];
  float* Phi = sm;                 // R x R
  float* Plo = sm + R * R;         // R x R
  float* Yt = sm + 2 * R * R;      // TR x R
  const int t = threadIdx.x;
  for (int e = t; e < R * R; e += DTHREADS) {
    double p = P[e];
    float hi = (float)p;
    Phi[e] = hi;
    Plo[e] = (float)(p - (double)hi);
  }
  const int groups = DTHREADS / R;
  const int c = t % R, g = t / R;
  double acc = 0.0;
  const int64_t ntiles = cpd_ceil_div(I, TR);
  __syncthreads();
  for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const int64_t r0 = tl * TR;
    for (int e = t; e < TR * R; e += DTHREADS) {
      int rr = e / R, cc = e % R;
      int64_t i = r0 + rr;
      Yt[e] = (i < I) ? Y[i * Rp + cc] : 0.0f;
    }
    __syncthreads();
    if (g < groups) {
      for (int rr = g; rr < TR; rr += groups) {
        int64_t i = r0 + rr;
        if (i >= I) break;
        float sh = 0.0f, sl = 0.0f;
        for (int a = 0; a < R; ++a) {
          float y = Yt[rr * R + a];
          sh = fmaf(y, Phi[a * R + c], sh);
          sl = fmaf(y, Plo[a * R + c], sl);
        }
        float v = sh + sl;
        Uw[i * Rp + c] = v;
        acc += (double)(v * v);
      }
    }
    __syncthreads();
  }
  store_col_partials(g < groups ? acc : 0.0, R, groups, colpart + (int64_t)blockIdx.x * R);
}

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
    for (int j = 0; j < cnt; ++j) {
      float vj = __shfl_sync(CPD_FULL, v, j);
#pragma unroll
      for (int q = 0; q < CPD_MAX_RANK / 32; ++q) {
        int r = lane + 32 * q;
        if (32 * q < a.R) {
          float m = sg[q];
          for (int k = 0; k < a.N; ++k) {
            int ik = __shfl_sync(CPD_FULL, ii[k], j);
            m *= (r < a.R) ? a.U[k][(int64_t)ik * a.Rp + r] : 0.0f;
          }
          part32 = fmaf(vj, m, part32);
        }
      }
    }
    acc += (double)part32;
  }
  double s = block_sum_d(acc, red);
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
  size_t shm = (size_t)TR * R * sizeof(float);
  normalize_gram_kernel<<<h->gram_blocks, DTHREADS, shm, h->stream>>>(Uin, Uout, I, R, h->Rp, sigma, do_scale,
                                                                      h->Gpart);
  CPD_LAUNCH(h, "normalize_gram");
  gram_reduce_kernel<<<std::max(1, (R * (R + 1) / 2 + 255) / 256), 256, 0, h->stream>>>(h->Gpart, h->gram_blocks, R, G);
  CPD_LAUNCH(h, "gram_reduce");
  return CPD_OK;
}

cpd_status cpd_gram(cpd_ctx* h, const float* U, int64_t I, double* G) {
  return gram_from(h, U, (float*)U, I, nullptr, 0, G);
}

// Algorithm 1 lines 2-3: normalise the columns of the initial factors.
cpd_status cpd_renormalize_inputs(cpd_ctx* h) {
  const int R = h->R;
  for (int k = 0; k < h->N; ++k) {
    colsq_kernel<<<h->gram_blocks, DTHREADS, 0, h->stream>>>(h->U[k], h->dims[k], R, h->Rp, h->colsq);
    sigma_kernel<<<1, 128, 0, h->stream>>>(h->colsq, h->gram_blocks, R, h->sigma);
    CPD_LAUNCH(h, "colsq/sigma");
    cpd_status s = gram_from(h, h->U[k], h->U[k], h->dims[k], h->sigma, 1, h->G[k]);
    if (s != CPD_OK) return s;
  }
  return CPD_OK;
}

static cpd_status launch_pinv(cpd_ctx* h, const PinvJobs& jobs, int njobs) {
  PhaseTimer pt(h, CPD_PHASE_PINV);
  const int R = h->R;
  size_t shm = (size_t)R * R * sizeof(double);
  pinv_kernel<<<njobs, DTHREADS, shm, h->stream>>>(jobs, R);
  CPD_LAUNCH(h, "pinv");
  return CPD_OK;
}

// G = *_{k != mode} G_k into Gout and its pseudo-inverse into Pout.
cpd_status cpd_hadamard_pinv(cpd_ctx* h, int mode, double* Gout, double* Pout) {
  PinvJobs jobs;
  memset(&jobs, 0, sizeof(jobs));
  PinvJob& j = jobs.job[0];
  for (int k = 0; k < h->N; ++k)
    if (k != mode) j.in[j.nin++] = h->G[k];
  j.out_had = Gout;
  j.out_pinv = Pout;
  j.scratch = h->Gpart;   // 2 R^2 doubles at the front of the partial buffer
  return launch_pinv(h, jobs, 1);
}

cpd_status cpd_pinv_into(cpd_ctx* h, const double* G, double* P, double* B, int* tri) {
  PinvJobs jobs;
  memset(&jobs, 0, sizeof(jobs));
  jobs.job[0].in[0] = G;
  jobs.job[0].nin = 1;
  jobs.job[0].out_pinv = P;
  jobs.job[0].out_factor = B;
  jobs.job[0].out_tri = tri;
  jobs.job[0].scratch = h->Gpart;
  return launch_pinv(h, jobs, 1);
}

// U_mode = Y G^+ (G^+ already in h->Gnpinv), sigma, renormalise, Gram.
cpd_status cpd_solve_renorm(cpd_ctx* h, int mode, const float* Y, double* out_sigma) {
  const int R = h->R;
  const int64_t I = h->dims[mode];
  {
    PhaseTimer pt(h, CPD_PHASE_SOLVE);
    size_t shm = (size_t)(2 * R * R + TR * R) * sizeof(float);
    solve_kernel<<<h->gram_blocks, DTHREADS, shm, h->stream>>>(Y, h->Gnpinv, h->Uwork, I, R, h->Rp, h->colsq);
    CPD_LAUNCH(h, "solve");
    sigma_kernel<<<1, 128, 0, h->stream>>>(h->colsq, h->gram_blocks, R, h->sigma);
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
  if (h->nnz > 0) {
    fit_inner_kernel<<<nblk, 256, 0, h->stream>>>(h->idx, h->vals, h->nnz, a, h->sigma, h->colsq);
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
  size_t s1 = (size_t)TR * R * sizeof(float);
  size_t s2 = (size_t)R * R * sizeof(double);
  size_t s3 = (size_t)(2 * R * R + TR * R) * sizeof(float);
  CPD_CUDA(h, cudaFuncSetAttribute(normalize_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(s1, 1)));
  CPD_CUDA(h, cudaFuncSetAttribute(pinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(s2, 1)));
  CPD_CUDA(h, cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(s3, 1)));
  return CPD_OK;
}
