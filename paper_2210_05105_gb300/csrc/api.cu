// C ABI of libcpd (include/cpd.h): handle life cycle, the ALS round of
// Algorithm 1 captured as a CUDA graph, and the step-wise entry points.
#include "common.cuh"
#include <map>
#include <mutex>
#include <algorithm>
#include <cmath>
#include <cstring>

cpd_status cpd_sts_alloc(cpd_ctx* h);
cpd_status cpd_sts_fallback_count(cpd_ctx* h, int64_t* out);

// message of the last failed cpd_create on this thread (the handle is gone)
static thread_local std::string g_create_error;

cpd_status cpd_fail(cpd_ctx* h, cpd_status s, const std::string& msg) {
  if (h) h->last_error = msg;
  return s;
}

cpd_status cpd_cuda_check(cpd_ctx* h, cudaError_t e, const char* what) {
  cudaGetLastError();
  return cpd_fail(h, CPD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

__global__ void sumsq_kernel(const float* __restrict__ v, int64_t n, double* __restrict__ part) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x = (double)v[i];
    s = fma(x, x, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < 8; ++w) b += red[w];
    part[blockIdx.x] = b;
  }
}

__global__ void fill_kernel(double* p, int n, double v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void bump_kernel(unsigned long long* ctr) { *ctr += 1ull; }

// Algorithm 1's initial factors when the caller passes none: U_k[i, r]
// ~ N(0, 1) by the Box-Muller transform of two uniforms from Philox4x64-10,
// key (seed, 2), counter (i, r, k, 0): u1 = (top 53 bits of word 0 + 1) 2^-53
// in (0, 1], u2 = top 53 bits of word 1 times 2^-53,
// z = sqrt(-2 ln u1) cos(2 pi u2) in float64, rounded to float32.
__global__ void gauss_init_kernel(float* __restrict__ U, int64_t I, int R, int Rp, int k, unsigned long long seed) {
  const int64_t n = I * R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / R;
    const int r = (int)(e - i * R);
    unsigned long long c[4] = {(unsigned long long)i, (unsigned long long)r, (unsigned long long)k, 0ull};
    cpd_philox4x64(c, seed, CPD_STREAM_INIT);
    // u1 = (top 53 bits of word 0 + 1) 2^-53 in (0, 1], u2 = top 53 bits of
    // word 1 times 2^-53; z = sqrt(-2 ln u1) cos(2 pi u2) in float32 (the
    // float64 transcendentals run at 1/64 of the float32 rate): ln u1 as
    // log(u1) for u1 < 1/2 and log1p(-(1 - u1)) above, with 1 - u1 formed
    // exactly, so both branches keep float32 relative accuracy; cos(2 pi u2)
    // as cospi(2 u2).  Within a few float32 ulps of the binary64 definition.
    const unsigned long long a1 = (c[0] >> 11) + 1ull;                 // u1 2^53, in [1, 2^53]
    const float l = a1 < (1ull << 52) ? logf((float)((double)a1 * 0x1.0p-53))
                                      : log1pf(-(float)((double)((1ull << 53) - a1) * 0x1.0p-53));
    const float z = sqrtf(-2.0f * l) * cospif((float)((double)(c[1] >> 11) * 0x1.0p-52));
    U[i * Rp + r] = z;
  }
}

// One mode update of Algorithm 1 on the handle's stream.
// Pseudo-inverse of the Hadamard product of Grams for `mode` on the forked
// side stream of a captured sweep (it depends only on the factor Grams, so it
// overlaps the draws and the MTTKRP of the main branch).
cpd_status fork_pinv(cpd_ctx* h, int mode) {
  CPD_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
  CPD_CUDA(h, cudaStreamWaitEvent(h->side_stream, h->ev_fork, 0));
  if (h->opt.method == CPD_ARLS_LEV) {
    // the mode's MTTKRP buffers are cleared on the branch too (the previous
    // solve has consumed Y); the main branch waits for it before the probe
    cpd_status sc = cpd_clear_launch(h, mode, h->Y, h->side_stream);
    if (sc != CPD_OK) return sc;
    CPD_CUDA(h, cudaEventRecord(h->ev_clear, h->side_stream));
  }
  cudaStream_t main = h->stream;
  h->stream = h->side_stream;
  cpd_status s = cpd_hadamard_pinv(h, mode, h->Gn, h->Gnpinv, h->pinv_scratch2);
  h->stream = main;
  if (s != CPD_OK) return s;
  CPD_CUDA(h, cudaEventRecord(h->ev_join, h->side_stream));
  return CPD_OK;
}

// One mode update of Algorithm 1.  `forked`: G^+ of this mode was
// enqueued on the side stream and is joined before the solve.
cpd_status mode_update(cpd_ctx* h, int n, bool forked = false) {
  cpd_status s;
  if (!forked && (s = cpd_hadamard_pinv(h, n, h->Gn, h->Gnpinv)) != CPD_OK) return s;
  if (h->opt.method == CPD_EXACT) {
    if ((s = cpd_exact_mttkrp_launch(h, n, h->Y)) != CPD_OK) return s;
  } else {
    const int64_t J = h->opt.samples;
    if ((s = cpd_draw(h, n, J, h->sweep_ctr, 0, h->samp_idx, h->samp_p, h->samp_w)) != CPD_OK) return s;
    cudaEvent_t cleared = (forked && h->opt.method == CPD_ARLS_LEV) ? h->ev_clear : nullptr;
    if ((s = cpd_sampled_mttkrp_launch(h, n, h->samp_idx, h->samp_w, h->samp_p, J, h->Y, nullptr, cleared)) != CPD_OK)
      return s;
  }
  if (forked) CPD_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  if (h->opt.sketched_gram && h->opt.method != CPD_EXACT && (s = cpd_pinv_into(h, h->Gsk, h->Gnpinv)) != CPD_OK)
    return s;
  if ((s = cpd_solve_renorm(h, n, h->Y, nullptr)) != CPD_OK) return s;
  // the next mode's G^+ needs this mode's new Gram; fork it before the
  // sampler refresh so that the two overlap
  if (forked && n + 1 < h->N && (s = fork_pinv(h, n + 1)) != CPD_OK) return s;
  return cpd_refresh_sampler(h, n);
}

// One ALS round, captured.  For CP-ARLS-LEV and exact ALS the draws do not
// read G^+, so each mode's pseudo-inverse runs on a forked branch.
cpd_status one_sweep(cpd_ctx* h) {
  const bool fork = h->opt.method != CPD_STS_CP && !h->opt.sketched_gram;
  if (fork) {
    cpd_status s = fork_pinv(h, 0);
    if (s != CPD_OK) return s;
  }
  for (int n = 0; n < h->N; ++n) {
    cpd_status s = mode_update(h, n, fork);
    if (s != CPD_OK) return s;
  }
  bump_kernel<<<1, 1, 0, h->stream>>>(h->sweep_ctr);
  CPD_LAUNCH(h, "bump");
  return CPD_OK;
}

cpd_status read_status(cpd_ctx* h) {
  int hs = 0;
  CPD_CUDA(h, cudaMemcpyAsync(&hs, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CPD_CUDA(h, cudaStreamSynchronize(h->stream));
  if (hs != 0) {
    CPD_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    CPD_CUDA(h, cudaStreamSynchronize(h->stream));
    return cpd_fail(h, (cpd_status)hs, "device-side error latched by a kernel");
  }
  return CPD_OK;
}

bool valid_mode(cpd_ctx* h, int mode) { return h && mode >= 0 && mode < h->N; }

// copy a matrix with row stride `sp` floats to one with stride `dp`
cpd_status copy_rows(cpd_ctx* h, float* dst, int dp, const float* src, int sp, int64_t rows, int cols) {
  if (rows == 0) return CPD_OK;
  CPD_CUDA(h, cudaMemcpy2DAsync(dst, (size_t)dp * sizeof(float), src, (size_t)sp * sizeof(float),
                                (size_t)cols * sizeof(float), (size_t)rows, cudaMemcpyDefault, h->stream));
  return CPD_OK;
}

cpd_status create_impl(cpd_ctx* h, int32_t N, const int64_t* dims, int64_t nnz, const int32_t* idx,
                       const float* vals, const float* init) {
  cudaStream_t st = h->stream;
  const int R = h->R, Rp = h->Rp;
  cpd_status s;
  const cudaMemcpyKind kind = h->opt.input_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if ((s = cpd_alloc(h, &h->idx, (size_t)N * nnz)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->vals, (size_t)nnz)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->status, 1)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->counters, 8)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->sweep_ctr, 1)) != CPD_OK) return s;
  CPD_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(int), st));
  CPD_CUDA(h, cudaMemsetAsync(h->sweep_ctr, 0, sizeof(unsigned long long), st));
  if (nnz > 0) {
    CPD_CUDA(h, cudaMemcpyAsync(h->idx, idx, (size_t)N * nnz * sizeof(int32_t), kind, st));
    CPD_CUDA(h, cudaMemcpyAsync(h->vals, vals, (size_t)nnz * sizeof(float), kind, st));
  }
  if (h->opt.spmm_blocks_per_sm) h->tune_spmm_bps = h->opt.spmm_blocks_per_sm;
  h->hot_cap = cpd_spmm_hot_slots(h->Rp, 1);
  if ((s = cpd_spmm_init(h)) != CPD_OK) return s;
  if ((s = cpd_build_layouts(h)) != CPD_OK) return s;
  nnz = h->nnz;            // fewer when repeated coordinates were summed

  // ||T||^2
  h->gram_blocks = h->num_sms * 4;
  const int npairs = R * (R + 1) / 2;
  if ((s = cpd_alloc(h, &h->Gpart, std::max((size_t)h->gram_blocks * npairs, 2 * (size_t)R * R))) != CPD_OK)
    return s;
  if ((s = cpd_alloc(h, &h->fit_out, 4)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->pinv_scratch2, 2 * (size_t)R * R)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->colsq, (size_t)h->gram_blocks * R + 8)) != CPD_OK) return s;
  {
    sumsq_kernel<<<h->gram_blocks, 256, 0, st>>>(h->vals, nnz, h->colsq);
    CPD_LAUNCH(h, "sumsq");
    std::vector<double> part(h->gram_blocks);
    CPD_CUDA(h, cudaMemcpyAsync(part.data(), h->colsq, h->gram_blocks * sizeof(double), cudaMemcpyDeviceToHost, st));
    CPD_CUDA(h, cudaStreamSynchronize(st));
    double t = 0.0;
    for (double v : part) t += v;
    h->tnorm2 = t;
  }

  // factors and model state
  for (int k = 0; k < N; ++k) {
    if ((s = cpd_alloc(h, &h->U[k], (size_t)dims[k] * Rp)) != CPD_OK) return s;
    CPD_CUDA(h, cudaMemsetAsync(h->U[k], 0, (size_t)dims[k] * Rp * sizeof(float), st));
    if ((s = cpd_alloc(h, &h->G[k], (size_t)R * R)) != CPD_OK) return s;
  }
  int64_t off = 0;
  for (int k = 0; k < N; ++k) {
    if (init) {
      CPD_CUDA(h, cudaMemcpy2DAsync(h->U[k], (size_t)Rp * sizeof(float), init + off, (size_t)R * sizeof(float),
                                    (size_t)R * sizeof(float), (size_t)dims[k], kind, st));
    } else {
      const int g = (int)std::min<int64_t>(cpd_ceil_div(dims[k] * R, 256), (int64_t)h->num_sms * 8);
      gauss_init_kernel<<<g, 256, 0, st>>>(h->U[k], dims[k], R, Rp, k, h->opt.seed);
      CPD_LAUNCH(h, "gauss_init");
    }
    off += dims[k] * R;
  }
  if ((s = cpd_alloc(h, &h->sigma, (size_t)R)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->Gn, (size_t)R * R)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->Gsk, (size_t)R * R)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->Gnpinv, (size_t)R * R)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->Gnpinv_split, 2 * (size_t)R * R)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->Y, (size_t)h->Imax * Rp)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->Uwork, (size_t)h->Imax * Rp)) != CPD_OK) return s;

  // sampling and MTTKRP scratch
  h->Jcap = std::max<int64_t>(h->opt.samples, 1);
  if ((s = cpd_alloc(h, &h->samp_idx, (size_t)N * h->Jcap)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->samp_p, (size_t)h->Jcap)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->samp_w, (size_t)h->Jcap)) != CPD_OK) return s;
  uint32_t dcap = 64;
  while ((int64_t)dcap < 2 * h->Jcap) dcap <<= 1;
  h->dedup_mask = dcap - 1;
  if ((s = cpd_alloc(h, &h->dd_tag, dcap)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->dd_w, dcap)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->uq_slot, (size_t)h->Jcap)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->chunk_seg, (size_t)cpd_ceil_div(std::max<int64_t>(nnz, 1), 32) + 1)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->uq_off, (size_t)h->Jcap + 1)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->uq_beg, (size_t)h->Jcap + 1)) != CPD_OK) return s;
  if ((s = cpd_alloc(h, &h->H, (size_t)h->Jcap * Rp)) != CPD_OK) return s;

  if (h->opt.method == CPD_ARLS_LEV) {
    for (int k = 0; k < N; ++k) {
      if ((s = cpd_alloc(h, &h->Gkpinv[k], (size_t)R * R)) != CPD_OK) return s;
      if ((s = cpd_alloc(h, &h->ell[k], (size_t)dims[k])) != CPD_OK) return s;
      if ((s = cpd_alloc(h, &h->cdf[k], (size_t)dims[k])) != CPD_OK) return s;
      if ((s = cpd_alloc(h, &h->blk[k], (size_t)cpd_ceil_div(dims[k], 256))) != CPD_OK) return s;
    }
  }
  if (h->opt.method == CPD_STS_CP && (s = cpd_sts_alloc(h)) != CPD_OK) return s;
  if (h->opt.deterministic && (s = cpd_det_alloc(h)) != CPD_OK) return s;
  if ((s = cpd_rowsort_alloc(h)) != CPD_OK) return s;
  if ((s = cpd_dense_init(h)) != CPD_OK) return s;
  if ((s = cpd_sample_init(h)) != CPD_OK) return s;

  // Algorithm 1's initialisation: normalised factors, sigma = 1, sampler state
  if ((s = cpd_renormalize_inputs(h)) != CPD_OK) return s;
  fill_kernel<<<1, 128, 0, st>>>(h->sigma, R, 1.0);
  CPD_LAUNCH(h, "fill");
  for (int k = 0; k < N; ++k)
    if ((s = cpd_refresh_sampler(h, k)) != CPD_OK) return s;
  return read_status(h);
}

}  // namespace

// One captured ALS round of the handle on its current stream (used by the
// batch graph, which captures several handles on parallel branches).
// Error text of a failed call that returned no handle (cpd_last_error(NULL)).
void cpd_note_error(const std::string& msg) { g_create_error = msg; }

// Free one allocation of the handle before cpd_destroy (implicitly synchronises).
void cpd_free(cpd_ctx* h, void* p) {
  auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
  if (it == h->allocs.end()) return;
  h->allocs.erase(it);
  cudaFree(p);
}

cpd_status cpd_smem_attr(cpd_ctx* h, const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[std::make_pair(h->device, func)];
  const size_t want = std::max<size_t>(bytes, 48 * 1024);     // the default limit
  if (want <= cur) return CPD_OK;
  CPD_CUDA(h, cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want));
  cur = want;
  return CPD_OK;
}

cpd_status cpd_one_sweep(cpd_ctx* h) { return one_sweep(h); }

extern "C" {

cpd_status cpd_default_options(cpd_options* opt) {
  if (!opt) return CPD_ERR_INVALID_ARG;
  memset(opt, 0, sizeof(*opt));
  opt->method = CPD_ARLS_LEV;
  opt->rank = 8;
  opt->samples = 2000;
  opt->seed = 0;
  opt->leaf_rows = 0;
  opt->input_on_host = 0;
  return CPD_OK;
}

cpd_status cpd_create(int32_t N, const int64_t* dims, int64_t nnz, const int32_t* idx, const float* vals,
                      const float* init_factors, const cpd_options* opt, void* cuda_stream, cpd_handle* out) {
  if (!out) return CPD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!opt || !dims || N < 1 || N > CPD_MAX_MODES || nnz < 0 || nnz >= 0xffffffffll) return CPD_ERR_INVALID_ARG;
  if (opt->rank < 1 || opt->rank > CPD_MAX_RANK || opt->samples < 0) return CPD_ERR_INVALID_ARG;
  if (opt->method < CPD_ARLS_LEV || opt->method > CPD_EXACT) return CPD_ERR_INVALID_ARG;
  if (nnz > 0 && (!idx || !vals)) return CPD_ERR_INVALID_ARG;
  if (opt->method != CPD_EXACT && opt->samples < 1) return CPD_ERR_INVALID_ARG;
  {
    const int b = opt->spmm_blocks_per_sm;
    if (b != 0 && b != 1 && b != 2 && b != 4 && b != 8) return CPD_ERR_INVALID_ARG;
  }
  if (opt->duplicate_policy != 0 && opt->duplicate_policy != 1) return CPD_ERR_INVALID_ARG;
  if (opt->deterministic != 0 && opt->deterministic != 1) return CPD_ERR_INVALID_ARG;
  if (opt->deterministic && opt->method == CPD_EXACT) return CPD_ERR_INVALID_ARG;
  if (opt->nnz_sel_capacity < 0) return CPD_ERR_INVALID_ARG;
  // every column key (product of the other modes' dims) must stay below 2^64
  for (int k = 0; k < N; ++k)
    if (dims[k] < 1 || dims[k] > 0x7fffffffll) return CPD_ERR_INVALID_ARG;
  for (int n = 0; n < N; ++n) {
    long double prod = 1.0L;
    for (int k = 0; k < N; ++k)
      if (k != n) prod *= (long double)dims[k];
    if (prod >= 18446744073709551615.0L) return CPD_ERR_INVALID_ARG;
  }
  cpd_ctx* h = new cpd_ctx();
  h->opt = *opt;
  h->N = N;
  h->R = opt->rank;
  h->Rp = cpd_pad4(opt->rank);
  h->nnz = nnz;
  for (int k = 0; k < N; ++k) { h->dims[k] = dims[k]; h->Imax = std::max(h->Imax, dims[k]); }
  h->F = opt->leaf_rows > 0 ? opt->leaf_rows : opt->rank;
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  h->stream = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_clear, cudaEventDisableTiming) != cudaSuccess) {
    g_create_error = "stream or event creation failed";
    cpd_destroy(h);
    return CPD_ERR_CUDA;
  }
  cpd_status s = create_impl(h, N, dims, nnz, idx, vals, init_factors);
  if (s != CPD_OK) {
    g_create_error = h->last_error;
    cpd_destroy(h);
    return s;
  }
  *out = h;
  return CPD_OK;
}

cpd_status cpd_leverage_sample(cpd_handle h, int32_t mode, int64_t J, uint64_t sweep, int32_t* out_idx,
                               double* out_prob) {
  if (!valid_mode(h, mode) || J < 1 || J > h->Jcap || !out_idx || !out_prob) return CPD_ERR_INVALID_ARG;
  if (h->opt.method == CPD_EXACT) return cpd_fail(h, CPD_ERR_INVALID_ARG, "handle built for exact ALS");
  if (h->opt.method == CPD_STS_CP) {
    cpd_status s = cpd_hadamard_pinv(h, mode, h->Gn, h->Gnpinv);
    if (s != CPD_OK) return s;
  }
  return cpd_draw(h, mode, J, nullptr, sweep, out_idx, out_prob, nullptr);
}

cpd_status cpd_sampled_mttkrp(cpd_handle h, int32_t mode, const int32_t* idx, const double* w, int64_t J, float* Y,
                              int64_t* out_nnz_sel) {
  if (!valid_mode(h, mode) || J < 0 || J > h->Jcap || !Y || (J > 0 && (!idx || !w))) return CPD_ERR_INVALID_ARG;
  cpd_status s = cpd_sampled_mttkrp_launch(h, mode, idx, w, nullptr, J, h->Y, out_nnz_sel);
  if (s != CPD_OK) return s;
  return copy_rows(h, Y, h->R, h->Y, h->Rp, h->dims[mode], h->R);
}

cpd_status cpd_exact_mttkrp(cpd_handle h, int32_t mode, float* Y) {
  if (!valid_mode(h, mode) || !Y) return CPD_ERR_INVALID_ARG;
  cpd_status s = cpd_exact_mttkrp_launch(h, mode, h->Y);
  if (s != CPD_OK) return s;
  return copy_rows(h, Y, h->R, h->Y, h->Rp, h->dims[mode], h->R);
}

cpd_status cpd_gram_solve(cpd_handle h, int32_t mode, const float* Y, double* out_sigma) {
  if (!valid_mode(h, mode) || !Y) return CPD_ERR_INVALID_ARG;
  cpd_status s;
  if (h->Rp != h->R) CPD_CUDA(h, cudaMemsetAsync(h->Y, 0, (size_t)h->dims[mode] * h->Rp * sizeof(float), h->stream));
  if ((s = copy_rows(h, h->Y, h->Rp, Y, h->R, h->dims[mode], h->R)) != CPD_OK) return s;
  if (h->opt.sketched_gram && h->opt.method != CPD_EXACT) s = cpd_pinv_into(h, h->Gsk, h->Gnpinv);
  else s = cpd_hadamard_pinv(h, mode, h->Gn, h->Gnpinv);
  if (s != CPD_OK) return s;
  if ((s = cpd_solve_renorm(h, mode, h->Y, out_sigma)) != CPD_OK) return s;
  return cpd_refresh_sampler(h, mode);
}

cpd_status cpd_als_sweep(cpd_handle h, int32_t n_sweeps) {
  if (!h || n_sweeps < 0) return CPD_ERR_INVALID_ARG;
  if (n_sweeps == 0) return CPD_OK;
  if (!h->sweep_exec) {
    // capture on the private stream (the caller's may be the legacy stream,
    // which cannot be captured), replay on the caller's
    CPD_CUDA(h, cudaStreamSynchronize(h->stream));
    cudaStream_t saved = h->stream;
    const bool prof = h->profiling;
    h->profiling = false;
    h->stream = h->cap_stream;
    cudaError_t eb = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (eb != cudaSuccess) { h->stream = saved; return cpd_cuda_check(h, eb, "cudaStreamBeginCapture"); }
    cpd_status s = one_sweep(h);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    h->stream = saved;
    h->profiling = prof;
    if (s != CPD_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) return cpd_cuda_check(h, e, "cudaStreamEndCapture");
    h->sweep_graph = g;
    CPD_CUDA(h, cudaGraphInstantiate(&h->sweep_exec, g, 0));
  }
  for (int i = 0; i < n_sweeps; ++i) CPD_CUDA(h, cudaGraphLaunch(h->sweep_exec, h->stream));
  h->host_sweep += (unsigned long long)n_sweeps;
  return CPD_OK;
}

cpd_status cpd_fit(cpd_handle h, double* out_fit) {
  if (!h || !out_fit) return CPD_ERR_INVALID_ARG;
  cpd_status s = cpd_fit_launch(h, h->fit_out);
  if (s != CPD_OK) return s;
  double hv[2] = {0.0, 0.0};
  CPD_CUDA(h, cudaMemcpyAsync(hv, h->fit_out, sizeof(hv), cudaMemcpyDeviceToHost, h->stream));
  if ((s = read_status(h)) != CPD_OK) return s;
  const double resid2 = h->tnorm2 - 2.0 * hv[0] + hv[1];
  *out_fit = h->tnorm2 > 0.0 ? 1.0 - std::sqrt(std::max(resid2, 0.0)) / std::sqrt(h->tnorm2) : 0.0;
  return CPD_OK;
}

cpd_status cpd_get_factors(cpd_handle h, int32_t mode, float* dst) {
  if (!valid_mode(h, mode) || !dst) return CPD_ERR_INVALID_ARG;
  cpd_status s = copy_rows(h, dst, h->R, h->U[mode], h->Rp, h->dims[mode], h->R);
  if (s != CPD_OK) return s;
  return read_status(h);
}

cpd_status cpd_set_factors(cpd_handle h, int32_t mode, const float* src) {
  if (!valid_mode(h, mode) || !src) return CPD_ERR_INVALID_ARG;
  cpd_status s = copy_rows(h, h->U[mode], h->Rp, src, h->R, h->dims[mode], h->R);
  if (s != CPD_OK) return s;
  if ((s = cpd_gram(h, h->U[mode], h->dims[mode], h->G[mode])) != CPD_OK) return s;
  if ((s = cpd_refresh_sampler(h, mode)) != CPD_OK) return s;
  return read_status(h);
}

cpd_status cpd_get_sigma(cpd_handle h, double* dst) {
  if (!h || !dst) return CPD_ERR_INVALID_ARG;
  CPD_CUDA(h, cudaMemcpyAsync(dst, h->sigma, h->R * sizeof(double), cudaMemcpyDefault, h->stream));
  return read_status(h);
}

cpd_status cpd_get_arls_state(cpd_handle h, int32_t mode, double* ell, double* cdf) {
  if (!valid_mode(h, mode)) return CPD_ERR_INVALID_ARG;
  if (h->opt.method != CPD_ARLS_LEV) return cpd_fail(h, CPD_ERR_INVALID_ARG, "handle is not CP-ARLS-LEV");
  size_t bytes = (size_t)h->dims[mode] * sizeof(double);
  if (ell) CPD_CUDA(h, cudaMemcpyAsync(ell, h->ell[mode], bytes, cudaMemcpyDefault, h->stream));
  if (cdf) CPD_CUDA(h, cudaMemcpyAsync(cdf, h->cdf[mode], bytes, cudaMemcpyDefault, h->stream));
  return read_status(h);
}

cpd_status cpd_get_gram(cpd_handle h, int32_t mode, double* dst) {
  if (!valid_mode(h, mode) || !dst) return CPD_ERR_INVALID_ARG;
  CPD_CUDA(h, cudaMemcpyAsync(dst, h->G[mode], (size_t)h->R * h->R * sizeof(double), cudaMemcpyDefault, h->stream));
  return read_status(h);
}

static cpd_status drain_marks(cpd_ctx* h) {
  if (h->marks.empty()) return CPD_OK;
  CPD_CUDA(h, cudaStreamSynchronize(h->stream));
  for (auto& m : h->marks) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
      h->prof_ms[m.phase] += ms;
      h->prof_n[m.phase] += 1;
    }
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  h->marks.clear();
  return CPD_OK;
}

cpd_status cpd_profile(cpd_handle h, int32_t enable) {
  if (!h) return CPD_ERR_INVALID_ARG;
  cpd_status s = drain_marks(h);
  h->profiling = enable != 0;
  return s;
}

cpd_status cpd_profile_read(cpd_handle h, double* ms, int64_t* launches) {
  if (!h) return CPD_ERR_INVALID_ARG;
  cpd_status s = drain_marks(h);
  if (s != CPD_OK) return s;
  for (int p = 0; p < CPD_NUM_PHASES; ++p) {
    if (ms) ms[p] = h->prof_ms[p];
    if (launches) launches[p] = h->prof_n[p];
    h->prof_ms[p] = 0.0;
    h->prof_n[p] = 0;
  }
  return CPD_OK;
}

cpd_status cpd_sweep_kernel_count(cpd_handle h, int64_t* out) {
  if (!h || !out) return CPD_ERR_INVALID_ARG;
  *out = 0;
  if (!h->sweep_graph) return CPD_OK;
  size_t n = 0;
  CPD_CUDA(h, cudaGraphGetNodes(h->sweep_graph, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  CPD_CUDA(h, cudaGraphGetNodes(h->sweep_graph, nodes.data(), &n));
  int64_t k = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    CPD_CUDA(h, cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  *out = k;
  return CPD_OK;
}

cpd_status cpd_debug_gram_wait(cpd_handle h, int64_t wait_cycles, int32_t suppress_mma) {
  if (!h || wait_cycles < 0 || (suppress_mma != 0 && suppress_mma != 1)) return CPD_ERR_INVALID_ARG;
  if (suppress_mma && wait_cycles == 0) return CPD_ERR_INVALID_ARG;   // would wait the full ~2 s
  h->dbg_gram_wait = wait_cycles;
  h->dbg_gram_no_mma = suppress_mma;
  return CPD_OK;
}

cpd_status cpd_sts_rescans(cpd_handle h, int64_t* out) {
  if (!h || !out) return CPD_ERR_INVALID_ARG;
  cpd_status s = cpd_sts_fallback_count(h, out);
  if (s != CPD_OK) return s;
  return read_status(h);
}

cpd_status cpd_synchronize(cpd_handle h) {
  if (!h) return CPD_ERR_INVALID_ARG;
  return read_status(h);
}

const char* cpd_last_error(cpd_handle h) {
  if (!h) return g_create_error.c_str();
  return h->last_error.c_str();
}

void cpd_destroy(cpd_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (auto& m : h->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
  if (h->sweep_exec) cudaGraphExecDestroy(h->sweep_exec);
  if (h->sweep_graph) cudaGraphDestroy(h->sweep_graph);
  for (void* p : h->allocs) cudaFree(p);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_clear) cudaEventDestroy(h->ev_clear);
  delete h;
}

}  // extern "C"
