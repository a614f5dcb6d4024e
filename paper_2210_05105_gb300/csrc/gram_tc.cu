// Tensor-core Gram G = U^T U (Eq. 5 operands) for the fast precision option,
// on the 5th-generation tensor cores (tcgen05.mma, accumulator in TMEM).
//
// Precision: every float32 entry is split exactly into three bfloat16 pieces,
// v = hi + mid + lo (8 + 8 + 8 significand bits), so each product of two
// pieces is exact in float32 and the only rounding is the tensor core's
// float32 accumulation, as in a float32 FMA loop.  With the pieces stacked as
// S = [hi^T; mid^T; lo^T] (3 Rp rows, K running over the rows of U), the MMA
// computes D = S S^T and G[a][b] is the sum of the 3 x 3 piece blocks of D.
//
// Per CTA (up to four per SM, persistent over 64-row tiles of U): one thread
// fetches each 64-row tile of U into shared memory with the Tensor Memory
// Accelerator (a 2D tensor map over U, cp.async.bulk.tensor, completion on an
// mbarrier; the next tile is in flight while the current one is staged);
// all threads then scale it (by 1 / sigma when renormalising, the scaled
// values written back as the new factor), split it and store the pieces in
// the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core
// matrix); one thread issues the MMAs and commits them to an mbarrier.  Two
// operand buffers let the next tile be staged while the tensor core reads the
// previous one.  At the end the
// accumulator is read with tcgen05.ld, the piece blocks are summed and the
// CTA's float64 partial Gram is written (reduced by gram_reduce_kernel).
//
// Every wait is bounded: a CTA whose MMAs do not complete within ~2 s sets
// CPD_ERR_TIMEOUT, waits once more (bounded) for them, frees its TMEM and
// writes a zero partial.  (cpd_debug_gram_wait shortens the limit and can
// suppress the MMAs, so that this path is tested without a fault.)
#include "common.cuh"
#include <cuda.h>           // CUtensorMap and cuTensorMapEncodeTiled's types (called through the runtime's entry point)
#include <cuda_bf16.h>
#include <algorithm>
#include <mutex>

namespace {

constexpr int GT_TK = 64;            // rows of U per tile (the MMA K of one stage)
constexpr int GT_THREADS = 256;
constexpr uint32_t GT_KC = GT_TK / 8;        // core matrices along K per tile
constexpr uint32_t GT_SBO = GT_KC * 128;     // bytes between 8-row groups
constexpr int GT_MAXW = 2;                   // work items per thread: Rp * GT_KC <= 512 (Rp <= 64)
constexpr long long GT_WAIT_CYCLES = 4000000000ll;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (between core matrices adjacent along K), stride byte offset
// (between adjacent 8-row groups), descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t gt_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ bool gt_wait(uint32_t bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__global__ void __launch_bounds__(GT_THREADS)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ Uin, float* __restrict__ Uout,
                   int64_t I, int R, int Rp, const double* __restrict__ sigma, int do_scale,
                   double* __restrict__ gpart, int* __restrict__ status, long long wait_limit, int issue_mma) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ __align__(8) unsigned long long tbar[2];      // TMA tile arrivals
  __shared__ uint32_t tmem_sh;
  __shared__ float inv[CPD_MAX_RANK];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int M3 = 3 * Rp;                         // rows of S
  const int MT = (M3 + 127) / 128;               // 128-row A tiles (1 or 2)
  const int NN = (M3 + 15) / 16 * 16;            // MMA N (rows of S used as B)
  const int COLS = (NN + 31) / 32 * 32;          // TMEM columns per A tile
  const uint32_t buf_bytes = (uint32_t)MT * 128u * GT_TK * 2u;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(MT * COLS)) ncols <<= 1;
  const bool write_back = Uout != Uin || do_scale;
  // raw float32 tiles (GT_TK x Rp, row-major as in U) written by the TMA,
  // after the two operand buffers
  float* raw = reinterpret_cast<float*>(gsm + 2 * (size_t)buf_bytes);
  const uint32_t raw_bytes = (uint32_t)GT_TK * (uint32_t)Rp * 4u;

  for (int r = t; r < CPD_MAX_RANK; r += GT_THREADS) {
    const double s = (do_scale && r < R) ? sigma[r] : 0.0;
    inv[r] = s > 0.0 ? (float)(1.0 / s) : 1.0f;
  }
  for (uint32_t e = t; e < 2u * buf_bytes / 16u; e += GT_THREADS) reinterpret_cast<uint4*>(gsm)[e] = make_uint4(0, 0, 0, 0);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  // kind::f16 instruction descriptor: D float32 (bit 4), A and B bfloat16
  // (bits 7, 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24 (M = 128)
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NN >> 3) << 17) | ((128u >> 4) << 24);
  const uint32_t base = smem_u32(gsm);
  const int64_t ntiles = (I + GT_TK - 1) / GT_TK;

  // the thread's work items (column r, 8-row group kg) of a tile: at most
  // GT_MAXW.  Tile tl goes to raw buffer tl's iteration parity: thread 0 arms
  // the buffer's mbarrier with the tile's byte count and issues the copy
  // (rows past I arrive as zeros: the tensor map's out-of-bounds fill).
  const int nwork = Rp * (int)GT_KC;
  auto fetch_tile = [&](int64_t tl, int rb) {
    const uint32_t bar = smem_u32(&tbar[rb]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(raw_bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(raw + (size_t)rb * GT_TK * Rp)),
        "l"(&tmap), "r"(0), "r"((int)(tl * GT_TK)), "r"(bar)
        : "memory");
  };
  if (t == 0 && (int64_t)blockIdx.x < ntiles) fetch_tile(blockIdx.x, 0);

  int it = 0;
  bool aborted = false;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    // the next tile's copy goes into the other raw buffer, consumed one
    // iteration ago (every thread passed the barrier after its staging)
    if (t == 0 && tile + gridDim.x < ntiles) fetch_tile(tile + gridDim.x, b ^ 1);
    bool ok = gt_wait(smem_u32(&tbar[b]), (uint32_t)(it >> 1) & 1u, wait_limit);       // this tile has arrived
    if (ok && it >= 2) ok = gt_wait(smem_u32(&mbar[b]), (uint32_t)((it - 2) >> 1) & 1u, wait_limit);   // MMAs of tile it-2 read buffer b
    if (__syncthreads_or(!ok)) { aborted = true; break; }
    const float* rt = raw + (size_t)b * GT_TK * Rp;
    unsigned char* buf = gsm + (size_t)b * buf_bytes;
    const int64_t k0 = tile * GT_TK;
#pragma unroll
    for (int wi = 0; wi < GT_MAXW; ++wi) {
      const int w = t + wi * GT_THREADS;
      if (w >= nwork) continue;
      const int r = w % Rp, kg = w / Rp;
      uint32_t ph[4], pm[4], pl[4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        float v[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int64_t k = k0 + kg * 8 + j + q;
          const float x = (r < R ? rt[(kg * 8 + j + q) * Rp + r] : 0.0f) * inv[r];
          if (write_back && k < I) Uout[k * Rp + r] = x;
          v[q] = x;
        }
        __nv_bfloat16 hi[2], mi[2], lo[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          hi[q] = __float2bfloat16_rn(v[q]);
          const float r1 = v[q] - __bfloat162float(hi[q]);     // exact
          mi[q] = __float2bfloat16_rn(r1);
          const float r2 = r1 - __bfloat162float(mi[q]);       // exact, <= 8 significant bits
          lo[q] = __float2bfloat16_rn(r2);
        }
        ph[j >> 1] = pack_bf16(hi[0], hi[1]);
        pm[j >> 1] = pack_bf16(mi[0], mi[1]);
        pl[j >> 1] = pack_bf16(lo[0], lo[1]);
      }
      // piece p of column r is row m = p Rp + r of S; its 8 K values form one
      // 16-byte row of core matrix (m / 8, kg)
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const int m = p * Rp + r;
        const uint4 val = p == 0 ? make_uint4(ph[0], ph[1], ph[2], ph[3])
                                 : (p == 1 ? make_uint4(pm[0], pm[1], pm[2], pm[3]) : make_uint4(pl[0], pl[1], pl[2], pl[3]));
        *reinterpret_cast<uint4*>(buf + ((uint32_t)(m >> 3) * GT_KC + (uint32_t)kg) * 128u + (uint32_t)(m & 7) * 16u) = val;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");    // generic-proxy stores -> tensor core
    __syncthreads();
    if (t == 0 && issue_mma) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t bb = base + (uint32_t)b * buf_bytes;
#pragma unroll 1
      for (int s = 0; s < GT_TK / 16; ++s) {
        const uint64_t bdesc = gt_desc(bb + (uint32_t)s * 256u, 128u, GT_SBO);
        for (int mt = 0; mt < MT; ++mt) {
          const uint64_t adesc = gt_desc(bb + (uint32_t)mt * 16u * GT_SBO + (uint32_t)s * 256u, 128u, GT_SBO);
          const uint32_t accum = (it > 0 || s > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + (uint32_t)(mt * COLS)),
              "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[b]))
                   : "memory");
    }
  }
  // the last commit covers every MMA this CTA issued
  bool ok = true;
  if (it > 0) ok = gt_wait(smem_u32(&mbar[(it - 1) & 1]), (uint32_t)((it - 1) >> 1) & 1u, wait_limit);
  // an aborted CTA may have a tile copy in flight (issued for iteration it +
  // 1 or not yet waited for at it): wait for it, bounded, before the buffers
  // are reused or the CTA exits
  if (aborted && t == 0) {
    const int64_t cur_tile = (int64_t)blockIdx.x + (int64_t)it * gridDim.x;
    gt_wait(smem_u32(&tbar[it & 1]), (uint32_t)(it >> 1) & 1u, wait_limit);
    if (cur_tile + gridDim.x < ntiles) gt_wait(smem_u32(&tbar[(it + 1) & 1]), (uint32_t)((it + 1) >> 1) & 1u, wait_limit);
  }
  const bool good = !__syncthreads_or(!ok) && !aborted;
  if (!good && t == 0) cpd_set_status(status, CPD_ERR_TIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // E[m][c] = sum over the three column pieces of D[m][q Rp + c]; warp w
  // reads TMEM lanes 32 (w % 4) .. + 31 of A tile w / 4
  float* E = reinterpret_cast<float*>(gsm);   // 3 Rp x Rp, over the operand buffers
  const bool have = good && it > 0;
  if (have) {
    const int quad = warp & 3, mt = warp >> 2;
    if (mt < MT) {
      const int m = mt * 128 + quad * 32 + lane;
      for (int c0 = 0; c0 < Rp; c0 += 4) {
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          uint32_t v0, v1, v2, v3;
          const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(mt * COLS + q * Rp + c0);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(v0), "=r"(v1), "=r"(v2), "=r"(v3)
                       : "r"(taddr)
                       : "memory");
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          acc[0] += __uint_as_float(v0);
          acc[1] += __uint_as_float(v1);
          acc[2] += __uint_as_float(v2);
          acc[3] += __uint_as_float(v3);
        }
        if (m < M3) {
#pragma unroll
          for (int c = 0; c < 4; ++c) E[m * Rp + c0 + c] = acc[c];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
  // G[a][b] = sum over the three row pieces of E[p Rp + a][b]
  const int npairs = R * (R + 1) / 2;
  double* out = gpart + (int64_t)blockIdx.x * npairs;
  for (int p = t; p < npairs; p += GT_THREADS) {
    int a = 0, rem = p;
    while (rem >= R - a) { rem -= R - a; ++a; }
    const int bc = a + rem;
    double s = 0.0;
    if (have)
      s = (double)E[a * Rp + bc] + (double)E[(Rp + a) * Rp + bc] + (double)E[(2 * Rp + a) * Rp + bc];
    out[p] = s;
  }
}

}  // namespace

bool cpd_gram_tc_supported(const cpd_ctx* h) { return h->opt.precision == 1 && h->Rp <= 64; }

size_t cpd_gram_tc_smem(int Rp) {
  const int M3 = 3 * Rp, MT = (M3 + 127) / 128;
  const size_t ops = 2 * (size_t)MT * 128 * GT_TK * 2;
  const size_t e = (size_t)M3 * Rp * sizeof(float);
  return (ops > e ? ops : e) + 2 * (size_t)GT_TK * Rp * sizeof(float);   // + the two raw TMA tiles
}

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  });
  return fn;
}
}  // namespace

// Partial Grams of U (rows scaled by 1 / sigma into Uout when do_scale) into
// h->Gpart, one per CTA; returns the number of partials in *nblk.
cpd_status cpd_gram_tc_launch(cpd_ctx* h, const float* Uin, float* Uout, int64_t I, const double* sigma, int do_scale,
                              int* nblk) {
  const size_t shm = cpd_gram_tc_smem(h->Rp);
  {
    const cpd_status st = cpd_smem_attr(h, (const void*)gram_tc_kernel, shm);
    if (st != CPD_OK) return st;
  }
  // several CTAs per SM hide the load latency of the staging; they share the
  // SM's 512 TMEM columns (a CTA whose allocation does not fit waits for one
  // that finishes), and there is one partial per CTA (h->Gpart holds
  // gram_blocks = 4 per SM)
  const int M3 = 3 * h->Rp, MT = (M3 + 127) / 128, COLS = ((M3 + 15) / 16 * 16 + 31) / 32 * 32;
  int ncols = 32;
  while (ncols < MT * COLS) ncols <<= 1;
  const int per_sm = std::max(1, std::min(4, 512 / ncols));
  const int grid = std::min(h->num_sms * per_sm, h->gram_blocks);
  const long long limit = h->dbg_gram_wait > 0 ? h->dbg_gram_wait : GT_WAIT_CYCLES;
  // 2D tensor map over U (Rp floats a row, 16-byte aligned rows: Rp is a
  // multiple of 4), boxes of GT_TK rows x Rp, rows past I read as zeros
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cpd_fail(h, CPD_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  CUtensorMap tmap;
  const cuuint64_t gdim[2] = {(cuuint64_t)h->Rp, (cuuint64_t)std::max<int64_t>(I, 1)};
  const cuuint64_t gstride[1] = {(cuuint64_t)h->Rp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)h->Rp, (cuuint32_t)GT_TK};
  const cuuint32_t estride[2] = {1, 1};
  const CUresult er = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(Uin), gdim, gstride, box,
                          estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (er != CUDA_SUCCESS) return cpd_fail(h, CPD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  gram_tc_kernel<<<grid, GT_THREADS, shm, h->stream>>>(tmap, Uin, Uout, I, h->R, h->Rp, sigma, do_scale, h->Gpart,
                                                       h->status, limit, h->dbg_gram_no_mma ? 0 : 1);
  CPD_LAUNCH(h, "gram_tc");
  *nblk = grid;
  return CPD_OK;
}
