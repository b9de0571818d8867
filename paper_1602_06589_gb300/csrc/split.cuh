// split.cuh -- the split-precision form of the contractions (a3, a4 via a5).
//
// Every complex FP64 operand matrix is cut into s BF16 "slices" with one
// power-of-two scale per column: v = 2^(e - 7) (d_1 + 2^-8 d_2 + ... + 2^-8(s-1) d_s),
// integer digits |d_p| <= 128 (exact in BF16). A complex product P^H Q is
// then the sum over slice pairs p + q <= s + 1 of exact integer products
// D_p^T E_q computed on the tcgen05 tensor cores (BF16 inputs, FP32
// accumulation kept exact by bounding each accumulation chunk to 1024
// products of magnitude <= 2^14), gathered in an int64 fixed-point
// accumulator in tensor memory, and scaled back to FP64 once per tile.
#pragma once

#include "internal.cuh"

namespace hsg {

constexpr int kMaxSlices = 7;
constexpr int kMinModuli = 10;

// Slices per operand for a target relative error (or the override when > 0).
int choose_slices(double target_rel_err, int override_slices);
// Moduli (Ozaki scheme II) for a target relative error at complex depth K
// (or the override when > 0); 0 when no count up to the maximum meets it.
int choose_moduli(double target_rel_err, int override_moduli, long long K);
// The form of one pass over `depth` rows (see SplitPlan).
SplitPlan split_plan(const hsgen_ctx *ctx, int depth);
// Bytes of device workspace the split form needs for one pass over `chunk_depth` rows.
size_t split_workspace_bytes(const hsgen_ctx *ctx, int n_g, int chunk_depth);
// Tables of the moduli form in constant memory (once per device).
cudaError_t split_upload_tables();
// Slices the T matrices once per species (called by hsgen_set_atoms in split mode).
hsgen_status split_prepare_types(hsgen_ctx *ctx, int slices);
// Host outputs of the last pass: the H/S launches run group by group (groups
// of whole column bands, every depth segment of a group before the next
// group), and after each group the copy stream moves its finished columns
// (all ld rows of each) to the host buffers, so the copies overlap the
// remaining groups. Null: not copied here.
struct CopyOut {
  void *H = nullptr, *S = nullptr;
};
// One pass (one chunk of atoms [a0, a1)) of the split path: slice W, X = T W,
// slice X and U W, then one triangle of H (+)= W^H X and S (+)= (U W)^H W.
// phase_ev (or null): two events, recorded after X = T W and after the slicing.
hsgen_status split_chunk(hsgen_ctx *ctx, int n_g, int a0, int a1, const double2 *W, double2 *X, long long ldw,
                         double2 *H, double2 *S, long long ld, bool accumulate, void *ws, int slices,
                         cudaStream_t s, const cudaEvent_t *phase_ev, const CopyOut *co = nullptr);
// Makes `s` wait for the copies split_chunk queued on the copy stream.
hsgen_status split_join_copies(hsgen_ctx *ctx, cudaStream_t s);
// The device status word of the split launches (bounded waits): post queues
// a copy of it behind the work on `s` without waiting; poll reads the latest
// posted copy (wait: block until it has arrived; otherwise HSGEN_OK while it
// is still on its way) and returns HSGEN_ETIMEOUT, clearing the word, when a
// wait expired; check = post + poll with wait.
hsgen_status split_post_status(hsgen_ctx *ctx, cudaStream_t s);
hsgen_status split_poll_status(hsgen_ctx *ctx, bool wait);
hsgen_status split_check_status(hsgen_ctx *ctx, cudaStream_t s);
// Batched k-points in one persistent launch; HSGEN_ENOTSUP when not applicable
// (the caller then loops over k-points).
hsgen_status split_batched(hsgen_ctx *ctx, int n_k, const int *n_g, const double *const *kvec, void *const *H,
                           void *const *S, const long long *ld, cudaStream_t s);
void split_release(hsgen_ctx *ctx);
// C (+)= P^H Q, or C (+)= -(P^H Q) with `negate`, in the split form with
// `slices` slices: P is K x M and Q is K x N (complex column-major, leading
// dimensions ldp, ldq >= K), C is M x N (ldc >= M). uplo 'U' / 'L' (M == N):
// only that triangle's tiles and entries, diagonal imaginary parts set to 0;
// uplo 0: every entry. `ws` holds split_gemm_ws_bytes(M, N, K, slices) and
// must not be in use by earlier work still pending on another stream.
size_t split_gemm_ws_bytes(int M, int N, int K, int slices);
hsgen_status split_gemm(hsgen_ctx *ctx, int M, int N, int K, const double2 *P, long long ldp, const double2 *Q,
                        long long ldq, double2 *C, long long ldc, int uplo, bool accumulate, bool negate,
                        int slices, void *ws, cudaStream_t s);

}  // namespace hsg
