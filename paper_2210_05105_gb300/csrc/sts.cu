// STS-CP sampler (Sec. 4.1, Appendix B, Algorithms 4-5).
#include "common.cuh"

cpd_status cpd_sts_refresh(cpd_ctx* h, int mode) {
  (void)mode;
  return cpd_fail(h, CPD_ERR_INVALID_ARG, "STS-CP sampler not available in this build");
}

cpd_status cpd_sts_draw(cpd_ctx* h, int mode, int64_t J, const unsigned long long* d_sweep,
                        unsigned long long sweep, int32_t* out_idx, double* out_p, double* out_w) {
  (void)mode; (void)J; (void)d_sweep; (void)sweep; (void)out_idx; (void)out_p; (void)out_w;
  return cpd_fail(h, CPD_ERR_INVALID_ARG, "STS-CP sampler not available in this build");
}

cpd_status cpd_sts_alloc(cpd_ctx* h) {
  (void)h;
  return CPD_OK;
}
