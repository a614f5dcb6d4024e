// Shared declarations of libcpd: the handle, device helpers and launchers.
// Written for sm_103a (GB300): 152 SMs, 32-wide warps, FP64 at 1/64 of FP32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>
#include "../../include/cpd.h"

#define CPD_WARP 32
#define CPD_FULL 0xffffffffu
#define CPD_EMPTY32 0xffffffffu
#define CPD_EMPTY64 0xffffffffffffffffull

// round-up helpers
__host__ __device__ static inline int64_t cpd_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int cpd_pad4(int r) { return (r + 3) & ~3; }

// Slot of the per-mode hash index: KRP-row key -> nonzero range [beg, beg+len)
// in the mode's key-sorted nonzero array.  16 bytes, one vector load.
struct __align__(16) FiberSlot {
  unsigned long long key;   // CPD_EMPTY64 when free
  uint32_t beg;
  uint32_t len;
};

// Per-mode layout (one matricization mat(T, n), Sec. 4.3): nonzeros sorted by
// their KRP-row key, packed (row i_n, value bits) pairs, plus the hash index.
struct ModeLayout {
  uint2* ent = nullptr;            // nnz: x = i_n, y = __float_as_uint(val)
  FiberSlot* table = nullptr;      // capacity = mask + 1 (power of two)
  unsigned long long mask = 0;
  int64_t n_fibers = 0;
  unsigned long long stride[CPD_MAX_MODES] = {0};  // key strides, 0 for mode n
  // Rows of mode n holding the most nonzeros ("hot" rows, hottest first);
  // their entries carry x = CPD_HOT_BIT | slot instead of the row, and the
  // SpMM accumulates them in shared memory before one flush per block.
  int32_t* hot_rows = nullptr;
  int n_hot = 0;
  uint32_t* row_code = nullptr;   // I_n: CPD_HOT_BIT | slot for hot rows, else the row's nonzero count
  bool row_sorted = false;        // the sampled SpMM sorts its nonzeros by output row (Y larger than L2)
};
#define CPD_HOT_BIT 0x80000000u
constexpr int CPD_HOT_MIN_COUNT = 256;   // a row with fewer nonzeros stays in the global path

// Device status codes are cpd_status values; 0 = fine.
struct cpd_ctx {
  int N = 0, R = 0, Rp = 0;   // Rp: row stride of factor storage (R rounded to 4)
  int64_t dims[CPD_MAX_MODES] = {0};
  int64_t nnz = 0, Imax = 0;
  cpd_options opt;
  cudaStream_t stream = nullptr;      // caller's stream (NULL: legacy default stream)
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture the sweep graph
  cudaStream_t side_stream = nullptr; // forked branch of the captured sweep
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_clear = nullptr;     // the forked branch has cleared the next MTTKRP's buffers
  double* pinv_scratch2 = nullptr;    // 2 R^2: scratch of the forked pseudo-inverse
  int device = 0, num_sms = 0;
  std::string last_error;

  // tensor in input order (for the fit and the exact MTTKRP)
  int32_t* idx = nullptr;   // N x nnz
  float* vals = nullptr;
  double tnorm2 = 0.0;      // ||T||_F^2
  ModeLayout mode[CPD_MAX_MODES];

  // model
  float* U[CPD_MAX_MODES] = {nullptr};      // I_k x Rp, padded columns zero
  double* G[CPD_MAX_MODES] = {nullptr};     // R x R Gram of U_k
  double* sigma = nullptr;                  // R

  // CP-ARLS-LEV state (Algorithm 2) per factor
  double* Gkpinv[CPD_MAX_MODES] = {nullptr};  // R x R
  double* ell[CPD_MAX_MODES] = {nullptr};     // I_k
  double* cdf[CPD_MAX_MODES] = {nullptr};     // I_k inclusive running sums
  double* blk[CPD_MAX_MODES] = {nullptr};     // per-block partial sums of ell

  // STS-CP state (Algorithm 4) per factor: heap of 2L node Grams
  int F = 0;
  int64_t L[CPD_MAX_MODES] = {0};
  // node v of factor k's tree at tree[k] + v * tree_stride: the packed upper
  // triangle (npad floats, R(R+1)/2 padded to 4); with tree_df the node holds
  // it twice, float32 hi then lo of a double-float (precision 0)
  float* tree[CPD_MAX_MODES] = {nullptr};
  bool tree_df = true;
  int tree_stride = 0;
  double* sts_ggt[CPD_MAX_MODES] = {nullptr}; // R x R: G^+ (*) Grams of factors drawn after k
  double* sts_Z = nullptr;                    // <G^+, G>_F
  float* sts_h = nullptr;                     // J x Rp running Hadamard products (J x 2Rp hi, lo with tree_df)
  int* sts_fallbacks = nullptr;               // leaves rescanned in double-float (counter)
  double* sts_q = nullptr;                    // Imax: row masses of the first factor drawn
  double* sts_cdf = nullptr;                  // Imax: their running sums
  double* sts_blk = nullptr;                  // block sums

  // per-update work buffers
  double* Gsk = nullptr;       // R x R Gram of the last draws (sketched-Gram solve)
  double* Gn = nullptr;        // R x R Hadamard of Grams for the solved mode
  double* Gnpinv = nullptr;    // R x R its pseudo-inverse
  float* Gnpinv_split = nullptr; // the same as float32 hi (R x R) then lo (R x R), for the solve
  double* Gpart = nullptr;     // Gram partial sums: gram_blocks x R x R
  int gram_blocks = 0;
  double* colsq = nullptr;     // column sum-of-squares partials: gram_blocks x R
  int32_t* samp_idx = nullptr; // N x J
  double* samp_p = nullptr;    // J
  double* samp_w = nullptr;    // J
  float* Y = nullptr;          // Imax x Rp
  float* Uwork = nullptr;      // Imax x Rp (unnormalised solve output)

  // sampled-MTTKRP scratch (sized from J)
  int64_t Jcap = 0;
  uint32_t dedup_mask = 0;
  uint32_t* dd_tag = nullptr;  // dedup capacity: fiber begin offset or EMPTY
  float* dd_w = nullptr;       // summed weight per distinct sampled column
  uint32_t* uq_slot = nullptr; // Jcap: dedup slot of each distinct column
  uint32_t* chunk_seg = nullptr; // ceil(nnz / 32): distinct column holding the first nonzero of each chunk
  uint32_t* uq_off = nullptr;  // Jcap: offset of each distinct column's nonzeros in the flat list
  uint32_t* uq_beg = nullptr;  // Jcap: first entry of each distinct column in the mode layout
  float* H = nullptr;          // Jcap x Rp: KRP row of each distinct column
  uint32_t* counters = nullptr;// words 0-1: one 64-bit (distinct columns << 32 | nnz_sel)
  int* status = nullptr;       // latched device error (cpd_status)
  double* fit_out = nullptr;   // 2 doubles: <T, T~>, ||T~||^2
  unsigned long long* sweep_ctr = nullptr;  // device sweep counter for graphs

  // graph of one ALS round
  cudaGraphExec_t sweep_exec = nullptr;
  cudaGraph_t sweep_graph = nullptr;
  unsigned long long host_sweep = 0;

  std::vector<void*> allocs;

  float2* lev_xs = nullptr;            // R(R+1)/2: the leverage kernel's coefficients (float32 hi + lo)

  // row-sorted sampled SpMM (R > 64, modes whose output Y exceeds 96 MB)
  int64_t rs_cap = 0;                  // selected nonzeros the sorted lists hold (multiple of 32)
  uint32_t* rs_cnt = nullptr;          // Imax + 1: per-row counts, counted down again by the scatter
  uint32_t* rs_off = nullptr;          // Imax + 1: row offsets (exclusive scan; total last)
  uint32_t* rs_bsum = nullptr;         // scan scratch
  uint4* rs_rec = nullptr;             // 2 rs_cap: 32-byte records (row, scale, column), sorted by row

  // deterministic downsampled MTTKRP (options.deterministic): sorted work
  // lists instead of floating-point atomics
  int64_t sel_cap = 0;                 // selected nonzeros a call may gather
  uint32_t* dslot = nullptr;           // Jcap: dedup slot of each draw (EMPTY: none)
  uint32_t* uq_len = nullptr;          // Jcap: nonzeros of each distinct column
  unsigned long long* dkeys = nullptr; // max(Jcap, sel_cap) sort keys, and the same again as scratch
  unsigned long long* dkeys2 = nullptr;
  uint32_t* dvals = nullptr;           // payloads, and scratch
  uint32_t* dvals2 = nullptr;
  uint32_t* dcounts = nullptr;         // radix-sort digit counts for max(Jcap, sel_cap)
  uint32_t* dlen = nullptr;            // Jcap + 1: column lengths in canonical order, then offsets
  uint32_t* dwords = nullptr;          // device counts: [0] selected nonzeros kept, [1] scan total
  uint32_t* sel_e = nullptr;           // sel_cap: layout entry of each canonical position
  uint32_t* sel_u = nullptr;           // sel_cap: distinct column of each canonical position
  float* dpart = nullptr;              // ceil(sel_cap / 256) x 2 x Rp run partial sums
  uint32_t* dflags = nullptr;          // ceil(sel_cap / 256) chunk flags

  // test hook of the tensor-core Gram's bounded waits (cpd_debug_gram_wait)
  long long dbg_gram_wait = 0;     // wait limit in clock cycles; 0 = the default (~2 s)
  int dbg_gram_no_mma = 0;         // 1: issue no MMA, so every wait runs out

  // launch shapes chosen by cpd_autotune
  int tune_spmm_bps = 2;    // SpMM blocks per SM (1024 threads each up to 2, then 2048 / bps)
  int hot_cap = 0;          // hot-row slots per mode kept by the layout
  int tune_sts_g = 16;      // lanes per draw in the STS walk

  // phase timers (cpd_profile)
  bool profiling = false;
  struct Mark { int phase; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  double prof_ms[CPD_NUM_PHASES] = {0};
  int64_t prof_n[CPD_NUM_PHASES] = {0};
};

// Bracket the launches between begin/end with events when profiling.
struct PhaseTimer {
  cpd_ctx* h; int phase; cudaEvent_t a = nullptr, b = nullptr;
  PhaseTimer(cpd_ctx* hh, int ph) : h(hh), phase(ph) {
    if (h->profiling) { cudaEventCreate(&a); cudaEventCreate(&b); cudaEventRecord(a, h->stream); }
  }
  ~PhaseTimer() {
    if (h->profiling) { cudaEventRecord(b, h->stream); h->marks.push_back({phase, a, b}); }
  }
};

// ---- error helpers -------------------------------------------------------
cpd_status cpd_fail(cpd_ctx* h, cpd_status s, const std::string& msg);
cpd_status cpd_cuda_check(cpd_ctx* h, cudaError_t e, const char* what);
#define CPD_CUDA(h, call) do { cudaError_t _e = (call); if (_e != cudaSuccess) return cpd_cuda_check((h), _e, #call); } while (0)
#define CPD_LAUNCH(h, what) do { cudaError_t _e = cudaGetLastError(); if (_e != cudaSuccess) return cpd_cuda_check((h), _e, what); } while (0)
template <typename T> cpd_status cpd_alloc(cpd_ctx* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) { cudaGetLastError(); return cpd_fail(h, CPD_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e)); }
  h->allocs.push_back((void*)*p);
  return CPD_OK;
}

// ---- device helpers ------------------------------------------------------
// Weight of a draw, w = 1 / (J p) (the diagonal of S^T S); a draw of
// probability 0 (a factor whose scores are all zero, so every KRP row is
// zero) gets weight 0 instead of an infinity.
__device__ __forceinline__ double cpd_weight(int64_t J, double p) { return p > 0.0 ? 1.0 / ((double)J * p) : 0.0; }

// Inverse CDF over non-negative running sums cdf[0..I): the smallest i with
// cdf[i] > t.  Non-negative doubles order as their bit patterns, so the
// search compares integers (no FP64 pipe).  If t >= the total C (u C rounded
// up to C), the first row whose running sum reaches C: the last row with a
// bin of nonzero width.  Requires C = cdf[I - 1] > 0 and finite.
__device__ __forceinline__ int64_t cpd_inverse_cdf(const double* __restrict__ cdf, int64_t I, double t) {
  const long long* cb = reinterpret_cast<const long long*>(cdf);
  const long long tb = __double_as_longlong(t);
  int64_t lo = 0, hi = I;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (cb[mid] > tb) hi = mid; else lo = mid + 1;
  }
  if (lo < I) return lo;
  const long long cbits = cb[I - 1];
  lo = 0; hi = I - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (cb[mid] >= cbits) hi = mid; else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ void cpd_set_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(CPD_FULL, v, o);
  return v;
}

// splitmix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom
// number generators", OOPSLA'14): hash of a KRP-row key to a table slot.
__device__ __forceinline__ unsigned long long cpd_mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): one block of 4 words.
__device__ __forceinline__ void cpd_philox4x64(unsigned long long c[4], unsigned long long k0,
                                               unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    unsigned long long x0 = hi1 ^ c[1] ^ k0, x2 = hi0 ^ c[3] ^ k1;
    c[0] = x0; c[1] = lo1; c[2] = x2; c[3] = lo0;
  }
}

// u(seed, stream; j, k, n, s) in [0, 1): top 53 bits of word 0 times 2^-53.
__device__ __forceinline__ double cpd_uniform(unsigned long long seed, unsigned long long stream,
                                              unsigned long long j, unsigned long long k,
                                              unsigned long long n, unsigned long long s) {
  unsigned long long c[4] = {j, k, n, s};
  cpd_philox4x64(c, seed, stream);
  return (double)(c[0] >> 11) * 0x1.0p-53;
}

// ---- double-float ("df64") accumulation on the float32 pipes ---------------
// GB300 issues float64 FMAs at 1/64 of the float32 rate, so the float64-exact
// Grams and leverage scores are accumulated as unevaluated sums hi + lo of two
// float32 with error-free transformations: Knuth's TwoSum and the FMA-based
// TwoProduct (Dekker; Ogita, Rump, Oishi, "Accurate sum and dot product",
// SIAM J. Sci. Comput. 2005).  The intrinsics keep the compiler from
// contracting or reassociating them.
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += x * y exactly up to the float32 rounding of lo.
__device__ __forceinline__ void df_fma(float& hi, float& lo, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float pe = __fmaf_rn(x, y, -p);
  float s, e;
  df_two_sum(hi, p, s, e);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}
// (hi, lo) += v for a float32 v
__device__ __forceinline__ void df_add(float& hi, float& lo, float v) {
  float s, e;
  df_two_sum(hi, v, s, e);
  hi = s;
  lo = __fadd_rn(lo, e);
}
// (h0, l0) += (h1, l1)
__device__ __forceinline__ void df_merge(float& h0, float& l0, float h1, float l1) {
  float s, e;
  df_two_sum(h0, h1, s, e);
  h0 = s;
  l0 = __fadd_rn(__fadd_rn(l0, l1), e);
}
__device__ __forceinline__ double df_value(float hi, float lo) { return (double)hi + (double)lo; }
// (hi, lo) := hi + lo renormalised so that |lo| <= ulp(hi) / 2 (Dekker's
// FastTwoSum; exact when |hi| >= |lo|)
__device__ __forceinline__ void df_renorm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}
// (ah, al) * (bh, bl) to ~2^-46 relative: exact leading product (TwoProduct)
// plus both cross terms; the lo * lo term is below the result's precision
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& rh, float& rl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  rh = p;
  rl = e;
  df_renorm(rh, rl);
}
// (ah, al) * b for a float32 b
__device__ __forceinline__ void df_mul_f(float ah, float al, float b, float& rh, float& rl) {
  const float p = __fmul_rn(ah, b);
  rl = __fmaf_rn(al, b, __fmaf_rn(ah, b, -p));
  rh = p;
  df_renorm(rh, rl);
}
// (sh, sl) += (ah, al) * (bh, bl): the Dot2 step of Ogita, Rump and Oishi
// with double-float operands (exact leading product, TwoSum into sh, all
// rounding errors and cross terms gathered in sl)
__device__ __forceinline__ void df_dot_step(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float pe = __fmaf_rn(ah, bh, -p);
  float s, e;
  df_two_sum(sh, p, s, e);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(e, __fmaf_rn(ah, bl, __fmaf_rn(al, bh, pe))));
}

// (sh, sl) += (xh, xl) * u for a float32 u: the Dot2 step with one
// double-float operand (exact leading product xh u, TwoSum into sh, the
// rounding errors and xl u gathered in sl)
__device__ __forceinline__ void df_dot_step_f(float& sh, float& sl, float xh, float xl, float u) {
  const float p = __fmul_rn(xh, u);
  const float pe = __fmaf_rn(xh, u, -p);
  float s, e;
  df_two_sum(sh, p, s, e);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(e, __fmaf_rn(xl, u, pe)));
}

#define CPD_STREAM_ARLS 0ull
#define CPD_STREAM_STS 1ull
#define CPD_STREAM_INIT 2ull

// ---- launchers implemented across the .cu files --------------------------
// layout.cu
cpd_status cpd_build_layouts(cpd_ctx* h);
// dense.cu
cpd_status cpd_renormalize_inputs(cpd_ctx* h);
cpd_status cpd_gram(cpd_ctx* h, const float* U, int64_t I, double* G);
// Raise (never lower) a kernel's dynamic shared-memory limit on the handle's
// device; the attribute is per function and shared by every handle.
cpd_status cpd_smem_attr(cpd_ctx* h, const void* func, size_t bytes);
int cpd_spmm_threads(int bps);
int cpd_spmm_hot_slots(int Rp, int bps);
cpd_status cpd_spmm_init(cpd_ctx* h);
void cpd_free(cpd_ctx* h, void* p);
size_t cpd_sts_tree_bytes(const cpd_ctx* h, int F);
bool cpd_sts_leaf_rows_valid(const cpd_ctx* h, int F);
cpd_status cpd_sts_set_leaf_rows(cpd_ctx* h, int F);
bool cpd_gram_tc_supported(const cpd_ctx* h);
cpd_status cpd_gram_tc_launch(cpd_ctx* h, const float* Uin, float* Uout, int64_t I, const double* sigma, int do_scale,
                              int* nblk);
cpd_status cpd_sketch_gram(cpd_ctx* h, int mode, const int32_t* idx, const double* w, int64_t J);
cpd_status cpd_hadamard_pinv(cpd_ctx* h, int mode, double* Gout, double* Pout, double* scratch = nullptr);
cpd_status cpd_pinv_into(cpd_ctx* h, const double* G, double* P);
cpd_status cpd_dense_init(cpd_ctx* h);
cpd_status cpd_solve_renorm(cpd_ctx* h, int mode, const float* Y, double* out_sigma);
cpd_status cpd_fit_launch(cpd_ctx* h, double* d_out);
// sample.cu
cpd_status cpd_refresh_sampler(cpd_ctx* h, int mode);
cpd_status cpd_sample_init(cpd_ctx* h);
bool cpd_sts_group_fits(cpd_ctx* h, int G);
cpd_status cpd_quadform_cdf(cpd_ctx* h, const float* U, int64_t I, const double* X, double* q, double* blk,
                            double* cdf);
cpd_status cpd_draw(cpd_ctx* h, int mode, int64_t J, const unsigned long long* d_sweep,
                    unsigned long long sweep, int32_t* out_idx, double* out_p, double* out_w);
// mttkrp.cu
cpd_status cpd_clear_launch(cpd_ctx* h, int mode, float* Y, cudaStream_t st);
cpd_status cpd_sampled_mttkrp_launch(cpd_ctx* h, int mode, const int32_t* idx, const double* w,
                                     const double* p, int64_t J, float* Y, int64_t* out_nnz_sel, cudaEvent_t cleared = nullptr);
cpd_status cpd_exact_mttkrp_launch(cpd_ctx* h, int mode, float* Y);
// scan.cu
cpd_status cpd_scan_u32(cpd_ctx* h, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total);
int64_t cpd_scan_u32_scratch(int64_t n);
cpd_status cpd_radix_init(cpd_ctx* h);
cpd_status cpd_scan_u32_buf(cpd_ctx* h, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                            uint32_t* bsum, cudaStream_t st);
cpd_status cpd_radix_sort_u64(cpd_ctx* h, unsigned long long* keys, uint32_t* vals, int64_t n, int bits,
                              unsigned long long* keys_tmp, uint32_t* vals_tmp);
cpd_status cpd_radix_sort_u64_dev(cpd_ctx* h, unsigned long long* keys, uint32_t* vals, int64_t cap,
                                  const uint32_t* n_dev, int bits, unsigned long long* keys_tmp, uint32_t* vals_tmp,
                                  uint32_t* counts, unsigned long long** out_k, uint32_t** out_v);
// det.cu (options.deterministic)
cpd_status cpd_det_alloc(cpd_ctx* h);
cpd_status cpd_rowsort_alloc(cpd_ctx* h);
cpd_status cpd_det_mttkrp(cpd_ctx* h, int mode, const double* w, int64_t J, float* Y, int64_t* out_nnz_sel);
