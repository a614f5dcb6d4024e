// Many independent decompositions at once, and the launch-shape autotuner.
//
// cpd_batch captures one ALS round of each of T handles into a single CUDA
// graph whose branches run concurrently (handles are assigned round-robin to
// `branches` branches; within a handle the kernels stay in order).  Small or
// uneven tensors, each of which leaves most of the GPU idle, then fill it
// together, and one graph launch replaces T * ~40 kernel launches.
//
// cpd_autotune times the candidate launch shapes of the sampled MTTKRP and of
// the STS walk on the handle's own data (step-wise, on the current factors)
// and keeps the fastest.
#include "common.cuh"
#include <algorithm>
#include <vector>

cpd_status cpd_one_sweep(cpd_ctx* h);
cpd_status cpd_sts_refresh(cpd_ctx* h, int k);
void cpd_note_error(const std::string& msg);

struct cpd_batch_ctx {
  std::vector<cpd_ctx*> hs;
  cudaStream_t stream = nullptr;       // caller's (replay)
  cudaStream_t cap = nullptr;          // capture origin
  std::vector<cudaStream_t> br;        // branch streams
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string last_error;
};

static void batch_free(cpd_batch_ctx* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto e : b->ev_join) if (e) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (auto s : b->br) if (s) cudaStreamDestroy(s);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

static cpd_status capture_batch(cpd_batch_ctx* b) {
  for (auto h : b->hs)
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return CPD_ERR_CUDA;
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CPD_ERR_CUDA;
  cpd_status s = CPD_OK;
  if (cudaEventRecord(b->ev_fork, b->cap) != cudaSuccess) s = CPD_ERR_CUDA;
  for (size_t i = 0; i < b->br.size() && s == CPD_OK; ++i)
    if (cudaStreamWaitEvent(b->br[i], b->ev_fork, 0) != cudaSuccess) s = CPD_ERR_CUDA;
  for (size_t t = 0; t < b->hs.size() && s == CPD_OK; ++t) {
    cpd_ctx* h = b->hs[t];
    cudaStream_t saved = h->stream;
    const bool prof = h->profiling;
    h->profiling = false;
    h->stream = b->br[t % b->br.size()];
    s = cpd_one_sweep(h);
    h->stream = saved;
    h->profiling = prof;
    if (s != CPD_OK) b->last_error = h->last_error;
  }
  for (size_t i = 0; i < b->br.size(); ++i) {
    if (cudaEventRecord(b->ev_join[i], b->br[i]) != cudaSuccess && s == CPD_OK) s = CPD_ERR_CUDA;
    if (cudaStreamWaitEvent(b->cap, b->ev_join[i], 0) != cudaSuccess && s == CPD_OK) s = CPD_ERR_CUDA;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (s != CPD_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (s == CPD_OK) b->last_error = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return s != CPD_OK ? s : CPD_ERR_CUDA;
  }
  b->graph = g;
  const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
  if (ei != cudaSuccess) {
    b->last_error = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei);
    return CPD_ERR_CUDA;
  }
  return CPD_OK;
}

extern "C" {

cpd_status cpd_batch_create(cpd_handle* handles, int32_t T, int32_t branches, void* cuda_stream, cpd_batch* out) {
  if (!out || !handles || T < 1 || branches < 1) return CPD_ERR_INVALID_ARG;
  *out = nullptr;
  for (int t = 0; t < T; ++t)
    if (!handles[t] || handles[t]->device != handles[0]->device) return CPD_ERR_INVALID_ARG;
  cpd_batch_ctx* b = new cpd_batch_ctx();
  b->hs.assign(handles, handles + T);
  b->stream = (cudaStream_t)cuda_stream;
  const int K = std::min(branches, T);
  bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < K && ok; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    b->br.push_back(s);
    b->ev_join.push_back(e);
  }
  if (!ok) { batch_free(b); return CPD_ERR_CUDA; }
  cpd_status s = capture_batch(b);
  if (s != CPD_OK) {
    cpd_note_error("cpd_batch_create: " + (b->last_error.empty() ? std::string("graph capture failed") : b->last_error));
    batch_free(b);
    return s;
  }
  *out = b;
  return CPD_OK;
}

cpd_status cpd_batch_sweep(cpd_batch b, int32_t n_sweeps) {
  if (!b || n_sweeps < 0) return CPD_ERR_INVALID_ARG;
  for (int i = 0; i < n_sweeps; ++i)
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return CPD_ERR_CUDA;
  for (auto h : b->hs) h->host_sweep += (unsigned long long)n_sweeps;
  return CPD_OK;
}

cpd_status cpd_batch_synchronize(cpd_batch b) {
  if (!b) return CPD_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return CPD_ERR_CUDA;
  for (auto h : b->hs) {
    cpd_status s = cpd_synchronize(h);
    if (s != CPD_OK) return s;
  }
  return CPD_OK;
}

void cpd_batch_destroy(cpd_batch b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
}

// Times the candidates of each tunable on the handle's data and keeps the
// fastest: SpMM blocks per SM in {1, 2, 4, 8}; for STS-CP, the leaf size F
// in {F, R, R/2, R/4, R/8} and then lanes per draw in {8, 16, 32} (those
// that fit in shared memory).  Draws use sweep counter
// 2^62 + trial so they do not repeat the run's draws; the model is unchanged.
cpd_status cpd_autotune(cpd_handle h, int32_t* out_choices) {
  if (!h) return CPD_ERR_INVALID_ARG;
  if (h->opt.method == CPD_EXACT) {
    if (out_choices) { out_choices[0] = h->tune_spmm_bps; out_choices[1] = h->tune_sts_g; out_choices[2] = h->F; }
    return CPD_OK;
  }
  const int64_t J = h->opt.samples;
  cudaEvent_t a, z;
  CPD_CUDA(h, cudaEventCreate(&a));
  CPD_CUDA(h, cudaEventCreate(&z));
  auto time_modes = [&](bool draw_only, float* ms) -> cpd_status {
    CPD_CUDA(h, cudaEventRecord(a, h->stream));
    for (int n = 0; n < h->N; ++n) {
      cpd_status s;
      if (h->opt.method == CPD_STS_CP && (s = cpd_hadamard_pinv(h, n, h->Gn, h->Gnpinv)) != CPD_OK) return s;
      if ((s = cpd_draw(h, n, J, nullptr, (1ull << 62) + n, h->samp_idx, h->samp_p, h->samp_w)) != CPD_OK) return s;
      if (!draw_only &&
          (s = cpd_sampled_mttkrp_launch(h, n, h->samp_idx, h->samp_w, h->samp_p, J, h->Y, nullptr)) != CPD_OK)
        return s;
    }
    CPD_CUDA(h, cudaEventRecord(z, h->stream));
    CPD_CUDA(h, cudaEventSynchronize(z));
    CPD_CUDA(h, cudaEventElapsedTime(ms, a, z));
    return CPD_OK;
  };
  const bool prof = h->profiling;
  h->profiling = false;
  cpd_status st = CPD_OK;
  float best = 1e30f, ms = 0.0f;
  int best_bps = h->tune_spmm_bps;
  for (int bps : {1, 2, 4, 8}) {
    h->tune_spmm_bps = bps;
    for (int rep = 0; rep < 2 && st == CPD_OK; ++rep) st = time_modes(false, &ms);   // second run is timed
    if (st != CPD_OK) break;
    if (ms < best) { best = ms; best_bps = bps; }
  }
  h->tune_spmm_bps = best_bps;
  if (st == CPD_OK && h->opt.method == CPD_STS_CP) {
    // leaf rows F (Sec. 4.1: leaves of F rows): a shallower walk against a
    // longer leaf scan; each candidate rebuilds the trees (sampler refresh
    // and draws are timed), trees of at most 8 GiB and F >= R / 8
    auto time_sts = [&](float* ms) -> cpd_status {
      CPD_CUDA(h, cudaEventRecord(a, h->stream));
      for (int n = 0; n < h->N; ++n) {
        cpd_status s;
        if ((s = cpd_sts_refresh(h, n)) != CPD_OK) return s;
        if ((s = cpd_hadamard_pinv(h, n, h->Gn, h->Gnpinv)) != CPD_OK) return s;
        if ((s = cpd_draw(h, n, J, nullptr, (1ull << 62) + n, h->samp_idx, h->samp_p, h->samp_w)) != CPD_OK) return s;
      }
      CPD_CUDA(h, cudaEventRecord(z, h->stream));
      CPD_CUDA(h, cudaEventSynchronize(z));
      CPD_CUDA(h, cudaEventElapsedTime(ms, a, z));
      return CPD_OK;
    };
    const int F0 = h->F;
    int best_f = F0;
    best = 1e30f;
    std::vector<int> cands = {F0};
    for (int d = 1; d <= 8; d *= 2) {
      const int F = std::max(2, h->R / d);
      if (std::find(cands.begin(), cands.end(), F) == cands.end()) cands.push_back(F);
    }
    for (int F : cands) {
      if (!cpd_sts_leaf_rows_valid(h, F) || cpd_sts_tree_bytes(h, F) > (size_t(8) << 30)) continue;
      if (F != h->F && (st = cpd_sts_set_leaf_rows(h, F)) != CPD_OK) break;
      for (int rep = 0; rep < 2 && st == CPD_OK; ++rep) st = time_sts(&ms);
      if (st != CPD_OK) break;
      if (ms < best) { best = ms; best_f = F; }
    }
    if (st == CPD_OK && best_f != h->F) st = cpd_sts_set_leaf_rows(h, best_f);
  }
  if (st == CPD_OK && h->opt.method == CPD_STS_CP) {
    best = 1e30f;
    int best_g = h->tune_sts_g;
    for (int g : {8, 16, 32}) {
      if (!cpd_sts_group_fits(h, g)) continue;
      h->tune_sts_g = g;
      for (int rep = 0; rep < 2 && st == CPD_OK; ++rep) st = time_modes(true, &ms);
      if (st != CPD_OK) break;
      if (ms < best) { best = ms; best_g = g; }
    }
    h->tune_sts_g = best_g;
  }
  h->profiling = prof;
  cudaEventDestroy(a);
  cudaEventDestroy(z);
  if (st != CPD_OK) return st;
  // the captured round holds the old launch shapes
  if (h->sweep_exec) { cudaGraphExecDestroy(h->sweep_exec); h->sweep_exec = nullptr; }
  if (h->sweep_graph) { cudaGraphDestroy(h->sweep_graph); h->sweep_graph = nullptr; }
  if (out_choices) { out_choices[0] = h->tune_spmm_bps; out_choices[1] = h->tune_sts_g; out_choices[2] = h->F; }
  return cpd_synchronize(h);
}

}  // extern "C"
