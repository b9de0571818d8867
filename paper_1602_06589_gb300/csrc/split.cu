// split.cu -- split-precision form (placeholder until the tcgen05 path lands).
#include "split.cuh"

namespace hsg {

int choose_slices(double target_rel_err, int override_slices) {
  if (override_slices > 0) return override_slices;
  (void)target_rel_err;
  return 6;
}
size_t split_workspace_bytes(int, int, int) { return 0; }
hsgen_status split_tapply(hsgen_ctx *ctx, const SplitCtx &, const Species &, const int *, int, const int *, int, int,
                          const double2 *, double2 *, long long, void *, int, cudaStream_t) {
  return set_err(ctx, HSGEN_ENOTSUP, "split form not available in this build");
}
hsgen_status split_hs(hsgen_ctx *ctx, const SplitCtx &, int, int, const double2 *, const double2 *, const double *,
                      long long, double2 *, double2 *, long long, int, bool, void *, int, cudaStream_t, cudaEvent_t) {
  return set_err(ctx, HSGEN_ENOTSUP, "split form not available in this build");
}
hsgen_status split_check_status(hsgen_ctx *, cudaStream_t) { return HSGEN_OK; }
hsgen_status split_batched(hsgen_ctx *, int, const int *, const double *const *, void *const *, void *const *,
                           const long long *, cudaStream_t) {
  return HSGEN_ENOTSUP;
}
void split_release(hsgen_ctx *) {}

}  // namespace hsg
