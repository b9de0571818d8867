// split.cuh -- the split-precision form of the contractions (a3, a4 via a5).
#pragma once

#include "internal.cuh"

namespace hsg {

constexpr int kMaxSlices = 8;

struct SplitCtx {
  long long wait_timeout_ns;
};

// Slices per operand for a target relative error (or the override when > 0).
int choose_slices(double target_rel_err, int override_slices);
// Bytes of device workspace the split form needs for one pass.
size_t split_workspace_bytes(int n_g, int chunk_depth, int slices);
// a3 in split form: X_a = T W_a for the atoms of one species.
hsgen_status split_tapply(hsgen_ctx *ctx, const SplitCtx &sc, const Species &sp, const int *d_atoms, int n_atoms,
                          const int *d_off, int row_base, int n_g, const double2 *W, double2 *X, long long ldw,
                          void *ws, int slices, cudaStream_t s);
// a4/a5 in split form: one triangle of H (+)= W^H X and S (+)= W^H diag(u) W.
hsgen_status split_hs(hsgen_ctx *ctx, const SplitCtx &sc, int n_g, int depth, const double2 *W, const double2 *X,
                      const double *urow, long long ldw, double2 *H, double2 *S, long long ld, int uplo,
                      bool accumulate, void *ws, int slices, cudaStream_t s, cudaEvent_t ev_after_slice);
// Reads the device status word of the last split launches (timeouts).
hsgen_status split_check_status(hsgen_ctx *ctx, cudaStream_t s);
// Batched k-points in one persistent launch; HSGEN_ENOTSUP when the context's
// form does not batch (the caller then loops over k-points).
hsgen_status split_batched(hsgen_ctx *ctx, int n_k, const int *n_g, const double *const *kvec, void *const *H,
                           void *const *S, const long long *ld, cudaStream_t s);
void split_release(hsgen_ctx *ctx);

}  // namespace hsg
