/*
 * cpd.h -- C ABI of libcpd: randomized sparse CP decomposition on one GB300.
 *
 * Method: V. Bharadwaj, O. A. Malik, R. Murray, A. Buluc, J. Demmel,
 * "Distributed-Memory Randomized Algorithms for Sparse Tensor CP
 * Decomposition" (arXiv 2210.05105).  Per mode n of each ALS round
 * (Algorithm 1) the library
 *   1. draws J rows of the Khatri-Rao product U_{!=n} (Eq. 3) by leverage
 *      scores: CP-ARLS-LEV (product of per-factor leverage scores, Appendix A,
 *      Algorithms 2-3) or STS-CP (exact leverage by a random walk on a binary
 *      tree of block Grams, Sec. 4.1 and Appendix B, Algorithms 4-5);
 *   2. computes the downsampled MTTKRP  Y = mat(T, n) S^T S U_{!=n}  (Eq. 7);
 *   3. solves  U_n = Y G^+  with G = *_{k != n} U_k^T U_k  (Eq. 4, Eq. 5) and
 *      renormalises the columns of U_n into sigma (Algorithm 1's mode update).
 *
 * Conventions shared by every entry point
 *   - Modes are 0-based; 1 <= N <= CPD_MAX_MODES.  Ranks 1 <= R <= CPD_MAX_RANK.
 *   - Factor U_k is I_k x R, row-major float32 with row stride R (the library
 *     keeps its own padded copy).
 *   - A "KRP row" of U_{!=n} is a tuple (i_k)_{k != n}; its linear key is
 *     sum_{k != n} i_k * prod_{k' < k, k' != n} I_k' (lowest mode fastest,
 *     the row order of Eq. 3).
 *   - Unless stated otherwise pointers are DEVICE pointers on the device that
 *     was current at cpd_create; calls are asynchronous on the handle's
 *     stream and return after enqueueing.
 *   - Host-checkable argument errors are returned at the call.  Errors found
 *     by kernels (index out of range, capacity overflow, a bounded wait that
 *     gave up) are latched in a device status word and returned by the next
 *     synchronising call (cpd_synchronize, cpd_fit, cpd_get_*).
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - Memory passed in stays owned by the caller; memory inside a handle is
 *     owned by the library and released by cpd_destroy.
 */
#ifndef CPD_H
#define CPD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPD_MAX_MODES 8
#define CPD_MAX_RANK 128

typedef struct cpd_ctx* cpd_handle;

typedef enum {
  CPD_OK = 0,
  CPD_ERR_INVALID_ARG = 1,       /* bad size, null pointer, unsupported option */
  CPD_ERR_OUT_OF_RANGE_INDEX = 2,/* a coordinate or sample index >= I_k or < 0 */
  CPD_ERR_DUPLICATE = 3,         /* two nonzeros share one coordinate */
  CPD_ERR_OOM = 4,               /* device allocation failed */
  CPD_ERR_CUDA = 5,              /* a CUDA runtime call failed; see cpd_last_error */
  CPD_ERR_CAPACITY = 6,          /* more samples / selected nonzeros than allocated */
  CPD_ERR_SINGULAR_GRAM = 7,     /* no pseudo-inverse of a Gram (Eq. 4): its eigensolver
                                    did not converge, i.e. the Gram held NaN or Inf */
  CPD_ERR_TIMEOUT = 8,           /* a bounded device-side wait gave up */
  CPD_ERR_NOT_FINITE = 9         /* NaN or Inf in values or factors */
} cpd_status;

typedef enum {
  CPD_ARLS_LEV = 0,  /* CP-ARLS-LEV: product of per-factor leverage scores */
  CPD_STS_CP = 1,    /* STS-CP: exact leverage scores by tree random walks */
  CPD_EXACT = 2      /* non-randomized ALS: full MTTKRP of Eq. 6 */
} cpd_method;

typedef struct {
  int32_t method;          /* cpd_method */
  int32_t rank;            /* R */
  int64_t samples;         /* J, draws per mode update (capacity for caller lists) */
  uint64_t seed;           /* Philox4x64-10 key word 0 for all draws */
  int32_t leaf_rows;       /* STS-CP rows per tree leaf F; 0: the smallest of 8, 16,
                              32 (below R) whose trees take at most 8 GB, else R */
  int32_t input_on_host;   /* 1: idx, vals, init_factors of cpd_create are host memory */
  int64_t nnz_sel_capacity; /* deterministic mode: most selected nonzeros one
                              downsampled MTTKRP may gather (its sorted work list is
                              sized from it); 0 = nnz.  More latches CPD_ERR_CAPACITY.
                              Otherwise, for R > 64: length of the row-sorted work
                              list (32 bytes an entry) of modes whose I_n x R output
                              exceeds 96 MB; 0 = min(nnz, 2^27).  Selected nonzeros
                              past it take the unsorted path (same result, no error) */
  int64_t reserved_i64[3];
  int32_t sketched_gram;   /* 0: solve with G = *_{k!=n} U_k^T U_k (Eq. 5, Sec. 4);
                              1: with the Gram of the sampled rows, sum_j w_j h_j h_j^T,
                              i.e. the normal equations of the downsampled problem
                              (Fig. 3 bottom, G~^+) */
  int32_t precision;       /* 0: Grams, leverage scores and G^+ accurate to float64
                              (the inverse-CDF draws then equal a float64 statement
                              of Algorithm 3 up to ties); 1: fast: accumulated in
                              float32, Grams on the tensor cores (draws may differ
                              near CDF boundaries; the fit stays within the
                              method's noise) */
  int32_t spmm_blocks_per_sm; /* launch shape of the sampled SpMM: blocks per SM in
                              {1, 2, 4, 8}, each holding an equal share of the SM's
                              shared memory for hot-row accumulation; 0 = default
                              (2); cpd_autotune may change it */
  int32_t duplicate_policy; /* repeated COO coordinates: 0 = rejected with
                              CPD_ERR_DUPLICATE; 1 = their values are summed into one
                              nonzero (the handle then holds fewer nonzeros) */
  int32_t deterministic;   /* 1: bitwise-repeatable runs.  The downsampled MTTKRP then
                              adds no floating-point value with an atomic: repeated
                              draws' weights are summed in draw order, and the
                              selected nonzeros are sorted by output row (stably,
                              in layout order) and reduced per row in that fixed
                              order.  Slower; CP-ARLS-LEV and STS-CP only (exact ALS:
                              CPD_ERR_INVALID_ARG).  0: atomics, faster, repeatable
                              to float32 rounding */
  int32_t reserved_i32[3];
} cpd_options;

/* Fill *opt with defaults: ARLS, R = 8, J = 2000, seed 0, leaf_rows 0 (the library picks F), device input. */
cpd_status cpd_default_options(cpd_options* opt);

/*
 * Build a handle for the N-mode sparse tensor given as COO (Sec. 2: a list of
 * (N+1)-tuples).
 *   dims          host, N entries, 1 <= I_k < 2^31; for every n the product of the
 *                 other modes' I_k must be < 2^64 (column keys are 64-bit).
 *   nnz           number of nonzeros, 0 <= nnz < 2^32 - 1.
 *   idx           N x nnz int32, mode-major (idx[k * nnz + e] = i_k of nonzero e).
 *   vals          nnz float32.
 *   init_factors  concatenated U_0 .. U_{N-1}, each I_k x R row-major float32
 *                 (the N(0,1) draws of Algorithm 1's initialisation), or NULL: the library
 *                 draws U_k[i, r] itself by the Box-Muller transform of two
 *                 uniforms from Philox4x64-10 with key (seed, 2) and counter
 *                 (i, r, k, 0): u1 = (top 53 bits of word 0 + 1) 2^-53,
 *                 u2 = top 53 bits of word 1 times 2^-53,
 *                 z = sqrt(-2 ln u1) cos(2 pi u2), evaluated in float32 (within
 *                 a few float32 ulps of the value in float64 rounded to float32).
 *   cuda_stream   cudaStream_t the handle enqueues on (NULL: legacy stream).
 * The library copies and re-sorts the inputs (one layout per matricization,
 * sorted by KRP-row key, with a hash index from key to its nonzeros, Sec. 4.3)
 * and normalises the factors (Algorithm 1's initialisation).  Coordinates must be
 * distinct (CPD_ERR_DUPLICATE otherwise).  Synchronises the stream.
 */
cpd_status cpd_create(int32_t N, const int64_t* dims, int64_t nnz,
                      const int32_t* idx, const float* vals,
                      const float* init_factors, const cpd_options* opt,
                      void* cuda_stream, cpd_handle* out);

/*
 * Draw J rows of U_{!=mode} with the handle's method (CP-ARLS-LEV:
 * Algorithm 3 with one processor; STS-CP: Algorithm 5 with one processor),
 * from the handle's current factors.  Uniform u(j, k) = Philox4x64-10 with
 * key (seed, stream) and counter (j, k, mode, sweep), top 53 bits of word 0
 * times 2^-53; stream 0 for CP-ARLS-LEV and 1 for STS-CP.
 *   out_idx   N x J int32 (row `mode` is written as -1).
 *   out_prob  J float64: probability of the drawn KRP row (ARLS: product of
 *             ell_k[i_k] / C_k; STS: exact leverage / <G^+, G>).
 * 1 <= J <= options.samples.
 */
cpd_status cpd_leverage_sample(cpd_handle h, int32_t mode, int64_t J, uint64_t sweep,
                               int32_t* out_idx, double* out_prob);

/*
 * Downsampled MTTKRP Y = mat(T, mode) S^T S U_{!=mode} (Eq. 7): draw j selects
 * the KRP row idx[:, j] with weight w[j] on the diagonal of S^T S; repeated
 * rows add their weights.  Y (I_mode x R float32, row-major) is overwritten.
 *   idx  N x J int32 (row `mode` ignored);  w  J float64.
 *   out_nnz_sel  device int64 or NULL: receives nnz(mat(T, mode) S^T), the
 *                nonzeros in the distinct sampled columns.
 * 0 <= J <= options.samples; indices out of range latch
 * CPD_ERR_OUT_OF_RANGE_INDEX and the draw is skipped.
 */
cpd_status cpd_sampled_mttkrp(cpd_handle h, int32_t mode, const int32_t* idx,
                              const double* w, int64_t J, float* Y,
                              int64_t* out_nnz_sel);

/*
 * Exact MTTKRP Y = mat(T, mode) U_{!=mode} (Eq. 6) over all nonzeros.
 * Y: I_mode x R float32, overwritten.
 */
cpd_status cpd_exact_mttkrp(cpd_handle h, int32_t mode, float* Y);

/*
 * Solve step of Algorithm 1 for `mode` given Y: U_mode := Y G^+ with
 * G = *_{k != mode} U_k^T U_k (Eq. 4, 5; pseudo-inverse by Cholesky, or by a
 * Jacobi eigendecomposition with eigenvalues <= R 2^-52 lambda_max dropped
 * when G is singular), sigma_r := ||U_mode[:, r]||, U_mode[:, r] /= sigma_r
 * (sigma_r = 0 leaves the column as is).  Then refreshes U_mode's Gram and
 * sampler (Algorithm 2 or 4).
 *   Y          I_mode x R float32 (may be the buffer given to cpd_sampled_mttkrp).
 *   out_sigma  R float64, or NULL.
 * With options.sketched_gram = 1 the Gram is that of the draws passed to the
 * last cpd_sampled_mttkrp call for this mode (sum_j w_j h_j h_j^T).
 */
cpd_status cpd_gram_solve(cpd_handle h, int32_t mode, const float* Y, double* out_sigma);

/*
 * n_sweeps ALS rounds (Algorithm 1's outer loop), each updating modes 0..N-1 in
 * order with sample, MTTKRP and solve; sweep s of the handle (counted from 0
 * at creation) uses counter word s.  The first call captures one round as a
 * CUDA graph; later rounds replay it.
 */
cpd_status cpd_als_sweep(cpd_handle h, int32_t n_sweeps);

/*
 * fit = 1 - ||T~ - T||_F / ||T||_F (Sec. 5.1) of the current model, computed
 * as ||T||^2 - 2 <T, T~> + sigma^T (*_k G_k) sigma in float64.  out_fit is a
 * HOST pointer.  Synchronises.
 */
cpd_status cpd_fit(cpd_handle h, double* out_fit);

/* Copy U_mode (I_mode x R float32 row-major) to / from dst / src, host or
 * device (any pointer cudaMemcpy accepts).  cpd_get_factors synchronises;
 * cpd_set_factors also refreshes the mode's Gram and sampler. */
cpd_status cpd_get_factors(cpd_handle h, int32_t mode, float* dst);
cpd_status cpd_set_factors(cpd_handle h, int32_t mode, const float* src);

/* Copy sigma (R float64) to dst, host or device.  Synchronises. */
cpd_status cpd_get_sigma(cpd_handle h, double* dst);

/*
 * Copy the CP-ARLS-LEV sampler state of `mode` (Algorithm 2): ell (I_mode
 * float64 leverage scores of U_mode alone) and cdf (I_mode float64 running
 * sums, cdf[I-1] = C); either pointer may be NULL.  Host or device.
 * Synchronises.  CPD_ERR_INVALID_ARG if the handle's method is not ARLS.
 */
cpd_status cpd_get_arls_state(cpd_handle h, int32_t mode, double* ell, double* cdf);

/* Copy the Gram U_mode^T U_mode (R x R float64).  Synchronises. */
cpd_status cpd_get_gram(cpd_handle h, int32_t mode, double* dst);

/*
 * Phase timers (profiling aid; the paper's runtime breakdown of Sec. 5.4 into
 * sampling, MTTKRP and post-processing).  While enabled, step-wise entry
 * points bracket each kernel class with CUDA events on the handle's stream;
 * captured sweeps (cpd_als_sweep) are not timed.  cpd_profile_read
 * synchronises, returns the accumulated milliseconds and launch counts per
 * phase (arrays of CPD_NUM_PHASES, either may be NULL) and clears them.
 */
typedef enum {
  CPD_PHASE_PINV = 0,      /* Hadamard of Grams and pseudo-inverse */
  CPD_PHASE_DRAW = 1,      /* leverage-score draws */
  CPD_PHASE_PROBE = 2,     /* sampled MTTKRP: hash lookup, merge, KRP rows */
  CPD_PHASE_SCAN = 3,      /* sampled MTTKRP: offsets of selected nonzeros */
  CPD_PHASE_SPMM = 4,      /* sampled MTTKRP: accumulation into Y */
  CPD_PHASE_SOLVE = 5,     /* Y G^+ and column norms */
  CPD_PHASE_GRAM = 6,      /* renormalisation and Gram */
  CPD_PHASE_SAMPLER = 7,   /* sampler rebuild (leverage + CDF, or tree) */
  CPD_PHASE_EXACT = 8,     /* exact MTTKRP */
  CPD_PHASE_CLEAR = 9,     /* clearing Y and per-call tables */
  CPD_NUM_PHASES = 10
} cpd_phase;
cpd_status cpd_profile(cpd_handle h, int32_t enable);
cpd_status cpd_profile_read(cpd_handle h, double* ms, int64_t* launches);

/* Number of kernel launches in one captured ALS round (0 before the first
 * cpd_als_sweep); memset and event nodes are not counted. */
cpd_status cpd_sweep_kernel_count(cpd_handle h, int64_t* out);

/*
 * Downsampled MTTKRP without any device allocation (no counterpart in the
 * paper): the same result as cpd_sampled_mttkrp, for callers that cannot
 * allocate.  Meant for
 * code that must not call cudaMalloc: code inside a framework whose memory
 * pool already owns the device memory, and latency-bound callers that cannot
 * accept the implicit device synchronisation of cudaMalloc / cudaFree.  It
 * needs no cpd_handle (creating one allocates): the caller passes the COO
 * tensor and the factor matrices directly, and one pass over the nonzeros
 * picks those whose column was drawn.
 *   N, dims (host), nnz, idx (N x nnz int32), vals    the tensor, laid out as for
 *            cpd_create (device memory; repeated coordinates simply add)
 *   factors  host array of N device pointers, U_k is I_k x R row-major float32;
 *            factors[mode] is not read and may be NULL
 *   samp_idx N x J int32 drawn KRP rows (row `mode` ignored); w J float64 weights
 *   Y        I_mode x R float32, overwritten
 *   status_out device int32, written by the GPU: 0 when every index was in
 *            range, else the OR of 1 (some draw had an index outside [0, I_k):
 *            that draw is skipped) and 2 (some nonzero had a coordinate
 *            outside [0, I_k): that nonzero is skipped)
 * Scratch: a fixed 2 MiB table in the library's static device memory, held on
 * every GPU that loads the library until the process exits; J is limited to
 * 65,536 (CPD_ERR_CAPACITY beyond).  The first call on a device looks up the
 * table's device address (cudaGetSymbolAddress).  All calls share the table
 * and it keeps the previous call's contents (each call clears it first), so
 * calls whose GPU work overlaps -- on different streams, or host threads --
 * race and must be serialised by the caller.  Asynchronous on cuda_stream.
 */
cpd_status cpd_sampled_mttkrp_noalloc(int32_t N, const int64_t* dims, int64_t nnz,
                                      const int32_t* idx, const float* vals,
                                      const float* const* factors, int32_t R, int32_t mode,
                                      const int32_t* samp_idx, const double* w, int64_t J,
                                      float* Y, int32_t* status_out, void* cuda_stream);

/*
 * Batched form: one CUDA graph holding one ALS round of each of T handles
 * (independent tensors, same device), assigned round-robin to `branches`
 * parallel graph branches so that small and uneven tensors run concurrently.
 * The handles must not be used on their own while a batch replays them.
 * Capturing synchronises the handles' streams; cpd_batch_sweep enqueues
 * n_sweeps replays on cuda_stream.  Destroying the batch leaves the handles.
 */
typedef struct cpd_batch_ctx* cpd_batch;
cpd_status cpd_batch_create(cpd_handle* handles, int32_t T, int32_t branches, void* cuda_stream,
                            cpd_batch* out);
cpd_status cpd_batch_sweep(cpd_batch b, int32_t n_sweeps);
cpd_status cpd_batch_synchronize(cpd_batch b);
void cpd_batch_destroy(cpd_batch b);

/*
 * Autotuner: times the candidates on the handle's own data and keeps the
 * fastest -- sampled-MTTKRP blocks per SM in {1, 2, 4, 8} and, for STS-CP,
 * the tree's leaf size F in {F, R, R/2, R/4, R/8} (trees of at most 8 GiB;
 * the trees are rebuilt, the sampling law does not depend on F) and lanes
 * per draw in the tree walk in {8, 16, 32}.  The model is not changed.
 * Drops the handle's captured round (recaptured on the next cpd_als_sweep);
 * call before building a batch.  out_choices: host int32[3] {blocks per SM,
 * lanes per draw, leaf rows F}, or NULL.  Synchronises.
 */
cpd_status cpd_autotune(cpd_handle h, int32_t* out_choices);

/*
 * STS-CP at precision 0 first scans a leaf's row masses in float32 with a
 * bound on their rounding error; a draw whose target lies within that bound
 * of a row boundary has its leaf rescanned in double-float (Sec. 4.1 leaf
 * scan of Algorithm 5).  *out (host) receives the number of such rescans
 * since cpd_create (0 for other methods or precision 1).  Synchronises.
 */
cpd_status cpd_sts_rescans(cpd_handle h, int64_t* out);

/*
 * Test hook of the bounded waits of the tensor-core Gram (precision 1, R <= 64):
 * sets their limit to wait_cycles SM clock cycles (0 restores the default,
 * ~2 s), and with suppress_mma = 1 the kernel issues no MMA, so that every
 * wait runs out.  The kernel then latches CPD_ERR_TIMEOUT (returned by the
 * next synchronising call), frees its tensor memory and writes zero partial
 * Grams; nothing is left in flight.  suppress_mma = 1 needs wait_cycles > 0.
 * Lets the timeout path be exercised without a device fault.
 */
cpd_status cpd_debug_gram_wait(cpd_handle h, int64_t wait_cycles, int32_t suppress_mma);

/* Wait for the handle's stream and return the first latched device error. */
cpd_status cpd_synchronize(cpd_handle h);

/* Text of the most recent error on this handle (static storage, never NULL). */
const char* cpd_last_error(cpd_handle h);

/* Release every allocation of the handle.  Synchronises.  NULL is a no-op. */
void cpd_destroy(cpd_handle h);

#ifdef __cplusplus
}
#endif

#endif /* CPD_H */
