// cpd_sampled_mttkrp_noalloc: the downsampled MTTKRP for callers that cannot
// allocate device memory.
//
// Who needs it: code that lives inside a framework whose caching allocator
// already owns the device memory and hands out no more, and latency-bound
// callers for which the implicit device synchronisation of cudaMalloc/cudaFree
// is unacceptable.
// They also may not hold a cpd_handle (creating one allocates), so this entry
// point works directly on the caller's COO tensor and factor matrices.
//
// Its only scratch is the file-scope table below, a fixed 2 MiB per device
// that every GPU loading the library keeps until the process exits.
#include "common.cuh"
#include <algorithm>
#include <cstring>
#include <mutex>

namespace {

constexpr int NA_MAX_SAMPLES = 65536;          // largest J accepted
constexpr int NA_SLOTS = 2 * NA_MAX_SAMPLES;   // power of two, load factor <= 1/2
constexpr int NA_MAX_DEVICES = 64;

struct __align__(16) NaSlot {
  unsigned long long key;   // KRP-row key or CPD_EMPTY64
  double w;                 // summed weight of the draws of that row
};

// Scratch shared by every call on this device.  Host code must not take its
// address directly (that is a host-side stand-in); it uses the device address
// fetched once per device with cudaGetSymbolAddress.
static __device__ __align__(256) NaSlot g_na_table[NA_SLOTS];

std::mutex g_na_mutex;
void* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

struct NaArgs {
  const float* U[CPD_MAX_MODES];
  int64_t dims[CPD_MAX_MODES];
  unsigned long long stride[CPD_MAX_MODES];
  int N, n, R;
};

__global__ void na_clear_kernel(NaSlot* __restrict__ table, float* __restrict__ Y, int64_t ny) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < NA_SLOTS; i += st) {
    table[i].key = CPD_EMPTY64;
    table[i].w = 0.0;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ny; i += st) Y[i] = 0.0f;
}

// S^T S as a hash map: each draw adds its weight to its KRP row's slot.
__global__ void na_insert_kernel(NaSlot* __restrict__ table, NaArgs a, const int32_t* __restrict__ sidx,
                                 const double* __restrict__ w, int64_t J, int* __restrict__ bad) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < J; j += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long key = 0;
    bool ok = true;
    for (int k = 0; k < a.N; ++k) {
      if (k == a.n) continue;
      const int32_t i = sidx[(int64_t)k * J + j];
      if (i < 0 || (int64_t)i >= a.dims[k]) ok = false;
      key += (unsigned long long)(ok ? i : 0) * a.stride[k];
    }
    if (!ok) { atomicOr(bad, 1); continue; }
    unsigned long long s = cpd_mix64(key) & (NA_SLOTS - 1);
    for (int probe = 0; probe < NA_SLOTS; ++probe) {
      const unsigned long long old = atomicCAS(&table[s].key, CPD_EMPTY64, key);
      if (old == CPD_EMPTY64 || old == key) {
        atomicAdd(&table[s].w, w[j]);
        break;
      }
      s = (s + 1) & (NA_SLOTS - 1);
    }
  }
}

// One pass over the nonzeros: a nonzero whose column was drawn adds
// w_col * val * (KRP row) to its output row; a warp takes 32 nonzeros.
// A nonzero with a coordinate outside [0, I_k) in any mode is skipped and
// latches bit 1 (value 2) of *bad, so no factor row or output row outside
// the caller's arrays is ever touched.
__global__ void na_accumulate_kernel(const NaSlot* __restrict__ table, NaArgs a, const int32_t* __restrict__ idx,
                                     const float* __restrict__ vals, int64_t nnz, float* __restrict__ Y,
                                     int* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c0 = warp * 32; c0 < nnz; c0 += nwarps * 32) {
    const int64_t e = c0 + lane;
    float scale = 0.0f;
    int32_t ii[CPD_MAX_MODES];
#pragma unroll
    for (int k = 0; k < CPD_MAX_MODES; ++k) ii[k] = (k < a.N && e < nnz) ? idx[(int64_t)k * nnz + e] : 0;
    bool in_range = e < nnz;
    for (int k = 0; k < a.N; ++k)
      if (ii[k] < 0 || (int64_t)ii[k] >= a.dims[k]) in_range = false;
    if (e < nnz && !in_range) atomicOr(bad, 2);
    if (in_range) {
      unsigned long long key = 0;
      for (int k = 0; k < a.N; ++k)
        if (k != a.n) key += (unsigned long long)ii[k] * a.stride[k];
      unsigned long long s = cpd_mix64(key) & (NA_SLOTS - 1);
      for (int probe = 0; probe < NA_SLOTS; ++probe) {
        const unsigned long long kk = table[s].key;
        if (kk == key) { scale = (float)(table[s].w * (double)vals[e]); break; }
        if (kk == CPD_EMPTY64) break;
        s = (s + 1) & (NA_SLOTS - 1);
      }
    }
    const unsigned hits = __ballot_sync(CPD_FULL, scale != 0.0f);
    for (unsigned m = hits; m; m &= m - 1) {
      const int j = __ffs(m) - 1;
      const float sj = __shfl_sync(CPD_FULL, scale, j);
      int32_t ij[CPD_MAX_MODES];
#pragma unroll
      for (int k = 0; k < CPD_MAX_MODES; ++k) ij[k] = __shfl_sync(CPD_FULL, ii[k], j);
      for (int r = lane; r < a.R; r += 32) {
        float v = sj;
        for (int k = 0; k < a.N; ++k)
          if (k != a.n) v *= a.U[k][(int64_t)ij[k] * a.R + r];
        atomicAdd(Y + (int64_t)ij[a.n] * a.R + r, v);
      }
    }
  }
}

}  // namespace

extern "C" cpd_status cpd_sampled_mttkrp_noalloc(int32_t N, const int64_t* dims, int64_t nnz, const int32_t* idx,
                                                 const float* vals, const float* const* factors, int32_t R,
                                                 int32_t mode, const int32_t* samp_idx, const double* w, int64_t J,
                                                 float* Y, int32_t* status_out, void* cuda_stream) {
  if (N < 1 || N > CPD_MAX_MODES || !dims || nnz < 0 || R < 1 || R > CPD_MAX_RANK || mode < 0 || mode >= N ||
      !factors || !Y || !status_out || J < 0 || (nnz > 0 && (!idx || !vals)) || (J > 0 && (!samp_idx || !w)))
    return CPD_ERR_INVALID_ARG;
  if (J > NA_MAX_SAMPLES) return CPD_ERR_CAPACITY;
  NaArgs a;
  memset(&a, 0, sizeof(a));
  long double prod = 1.0L;
  unsigned long long acc = 1;
  for (int k = 0; k < N; ++k) {
    if (dims[k] < 1 || dims[k] > 0x7fffffffll || (k != mode && !factors[k])) return CPD_ERR_INVALID_ARG;
    prod *= (long double)dims[k];
    a.U[k] = factors[k];
    a.dims[k] = dims[k];
    if (k != mode) { a.stride[k] = acc; acc *= (unsigned long long)dims[k]; }
  }
  if (prod >= 18446744073709551615.0L) return CPD_ERR_INVALID_ARG;
  a.N = N; a.n = mode; a.R = R;

  // once per device, with that device current: the device address of the table
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return CPD_ERR_CUDA;
  NaSlot* table = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_na_table) != cudaSuccess || !p) {
        cudaGetLastError();
        return CPD_ERR_CUDA;
      }
      g_na_ptr[dev] = p;
    }
    table = static_cast<NaSlot*>(g_na_ptr[dev]);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ny = dims[mode] * (int64_t)R;
  if (cudaMemsetAsync(status_out, 0, sizeof(int32_t), st) != cudaSuccess) return CPD_ERR_CUDA;
  na_clear_kernel<<<sms * 4, 256, 0, st>>>(table, Y, ny);
  if (J > 0)
    na_insert_kernel<<<(unsigned)std::min<int64_t>(cpd_ceil_div(J, 256), sms * 4), 256, 0, st>>>(
        table, a, samp_idx, w, J, status_out);
  if (nnz > 0) na_accumulate_kernel<<<sms * 8, 256, 0, st>>>(table, a, idx, vals, nnz, Y, status_out);
  if (cudaGetLastError() != cudaSuccess) return CPD_ERR_CUDA;
  return CPD_OK;
}
