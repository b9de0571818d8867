// reduce.cu -- hand-off of H and S to the generalized eigensolver (Sec. 2.3,
// Eq. matrix_kohnsham: H c = eps S c with H, S Hermitian and S positive
// definite). S is factored in FP64, S = U^H U (opt.uplo 'U') or S = L L^H
// ('L'), in place in its triangle, and H is reduced in place to the standard
// problem H~ y = eps y, c = U^-1 y:
//   H~ = U^-H H U^-1   (= L^-1 H L^-H, the same matrix: the factor is unique),
// written in full and exactly Hermitian. The factorization (ZPOTRF) and the
// two triangular solves (ZTRSM) are cuSOLVER / cuBLAS calls in FP64; this file
// adds the checks, the Hermitian fill of H before the solves and the
// symmetrisation of the result.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cstdlib>
#include <string>
#include <vector>

#include "internal.cuh"
#include "split.cuh"

namespace hsg {
namespace {

// mode 0: the triangle opposite `uplo` takes the conjugate transpose of the
// `uplo` triangle; mode 1: both triangles take the average (M + M^H) / 2;
// in modes 0 and 1 diagonal imaginary parts become 0. mode 2: M becomes M^H
// (in place). A block takes the tile pair (bi, bj),
// (bj, bi) with bi <= bj: both tiles are read column-contiguously into shared
// memory, then each thread writes one (i, j), i <= j, and its mirror (the
// mirrored writes are strided; the solves around this dominate the time).
__global__ void hermitian_kernel(int n, double2 *M, long long ld, int uplo, int mode) {
  __shared__ double2 a[32][33], b[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;  // tile rows bi*32.., columns bj*32.., bi <= bj
  if (bi > bj) return;
  const int tx = threadIdx.x;
  for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
    const int r = bi * 32 + tx, c = bj * 32 + ty;  // (r, c) upper part, column c contiguous over r
    a[ty][tx] = (r < n && c < n) ? M[(size_t)c * ld + r] : make_double2(0.0, 0.0);
    const int r2 = bj * 32 + tx, c2 = bi * 32 + ty;  // (r2, c2) mirrored tile, lower part
    b[ty][tx] = (r2 < n && c2 < n) ? M[(size_t)c2 * ld + r2] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
    // upper element (i, j) = (bi*32 + tx, bj*32 + ty) = a[ty][tx];
    // its mirror (j, i) = (bj*32 + ty, bi*32 + tx) = b[tx][ty]
    const int i = bi * 32 + tx, j = bj * 32 + ty;
    if (i < n && j < n && i <= j) {
      const double2 up = a[ty][tx], lo = b[tx][ty];
      double2 vu, vl;  // new (i, j) and (j, i)
      if (mode == 2) {
        vu = make_double2(lo.x, -lo.y);
        vl = make_double2(up.x, -up.y);
      } else if (i == j) {
        vu = vl = make_double2(up.x, 0.0);
      } else {
        vu = (mode == 1) ? make_double2(0.5 * (up.x + lo.x), 0.5 * (up.y - lo.y))
                         : ((uplo == 'U') ? up : make_double2(lo.x, -lo.y));
        vl = make_double2(vu.x, -vu.y);
      }
      M[(size_t)j * ld + i] = vu;             // (i, j)
      if (i != j) M[(size_t)i * ld + j] = vl;  // (j, i)
    }
  }
}

cudaError_t launch_hermitian(int n, double2 *M, long long ld, int uplo, int mode, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned nb = (unsigned)((n + 31) / 32);
  hermitian_kernel<<<dim3(nb, nb), dim3(32, 8), 0, s>>>(n, M, ld, uplo, mode);
  return cudaGetLastError();
}

hsgen_status blas_err(hsgen_ctx *ctx, int code, const char *what) {
  return set_err(ctx, HSGEN_ECUDA, std::string(what) + " failed (status " + std::to_string(code) + ")");
}

// Split form of the reduction (upper triangle): blocks of kRedBlock rows;
// the diagonal blocks are factored and solved in FP64 (cuSOLVER / cuBLAS),
// the updates that carry ~all the flops run as BF16-slice products on the
// tensor cores (split_gemm) with kRedSlices slices, which give products to
// ~2e-15 relative, FP64's level.
// 256: at N_G 12 000, 1.13 s against 1.16 (192), 1.18 (128), 1.41 (512), 2.04 s (1024): smaller
// blocks shrink the FP64 diagonal-block solves, larger ones the updates' short depth
constexpr int kRedBlock = 256;  // default; HSGEN_REDUCE_BLOCK (64..4096, rounded to 64) overrides it
constexpr int kRedSlices = 7;

int reduce_block() {
  int nb = kRedBlock;
  if (const char *e = std::getenv("HSGEN_REDUCE_BLOCK")) nb = std::max(64, std::min(4096, std::atoi(e))) / 64 * 64;
  return nb;
}

// S = U^H U in place (upper triangle), right-looking: U11 = chol(A11),
// U12 = U11^-H A12, A22 -= U12^H U12.
hsgen_status potrf_split(hsgen_ctx *ctx, int n, int nb, double2 *S, long long ld, cuDoubleComplex *work, int lwork,
                         int *d_info, void *gws, cudaStream_t s) {
  cublasHandle_t blas = (cublasHandle_t)ctx->blas;
  cusolverDnHandle_t solver = (cusolverDnHandle_t)ctx->solver;
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0);
  for (int k = 0, blk = 0; k < n; k += nb, ++blk) {
    const int kb = std::min(nb, n - k), m = n - k - kb;
    cuDoubleComplex *Skk = (cuDoubleComplex *)(S + k + (size_t)k * ld);
    cusolverStatus_t se = cusolverDnZpotrf(solver, CUBLAS_FILL_MODE_UPPER, kb, Skk, (int)ld, work, lwork, d_info + blk);
    if (se != CUSOLVER_STATUS_SUCCESS) return blas_err(ctx, (int)se, "cusolverDnZpotrf");
    if (m == 0) break;
    double2 *U12 = S + k + (size_t)(k + kb) * ld;
    cublasStatus_t be = cublasZtrsm(blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_C, CUBLAS_DIAG_NON_UNIT,
                                    kb, m, &one, Skk, (int)ld, (cuDoubleComplex *)U12, (int)ld);
    if (be != CUBLAS_STATUS_SUCCESS) return blas_err(ctx, (int)be, "cublasZtrsm (panel)");
    hsgen_status st = split_gemm(ctx, m, m, kb, U12, ld, U12, ld, S + (k + kb) + (size_t)(k + kb) * ld, ld, 'U',
                                 true, true, kRedSlices, gws, s);
    if (st != HSGEN_OK) return st;
  }
  return HSGEN_OK;
}

// U^H X = B in place on B (n x n), U upper triangular; by block rows:
// X_k = U_kk^-H B_k, then B_rest -= U_{k,rest}^H X_k.
hsgen_status solve_left_split(hsgen_ctx *ctx, int n, int nb, const double2 *U, double2 *B, long long ld, void *gws,
                              cudaStream_t s) {
  cublasHandle_t blas = (cublasHandle_t)ctx->blas;
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0);
  for (int k = 0; k < n; k += nb) {
    const int kb = std::min(nb, n - k), m = n - k - kb;
    cublasStatus_t be = cublasZtrsm(blas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_C, CUBLAS_DIAG_NON_UNIT,
                                    kb, n, &one, (const cuDoubleComplex *)(U + k + (size_t)k * ld), (int)ld,
                                    (cuDoubleComplex *)(B + k), (int)ld);
    if (be != CUBLAS_STATUS_SUCCESS) return blas_err(ctx, (int)be, "cublasZtrsm (block)");
    if (m == 0) break;
    hsgen_status st = split_gemm(ctx, m, n, kb, U + k + (size_t)(k + kb) * ld, ld, B + k, ld, B + k + kb, ld, 0,
                                 true, true, kRedSlices, gws, s);
    if (st != HSGEN_OK) return st;
  }
  return HSGEN_OK;
}

}  // namespace

void reduce_release(hsgen_ctx *ctx) {
  if (ctx->solver) cusolverDnDestroy((cusolverDnHandle_t)ctx->solver);
  if (ctx->blas) cublasDestroy((cublasHandle_t)ctx->blas);
  if (ctx->ws_red.ptr) cudaFree(ctx->ws_red.ptr);
  if (ctx->h_info) cudaFreeHost(ctx->h_info);
  ctx->solver = ctx->blas = nullptr;
  ctx->ws_red = Workspace{};
  ctx->h_info = nullptr;
}

}  // namespace hsg

using namespace hsg;

extern "C" hsgen_status hsgen_reduce_generalized(hsgen_ctx *ctx, int n, void *H, void *S, long long ld,
                                                 void *cuda_stream) {
  if (!ctx) return HSGEN_EINVAL;
  if (n < 0) return set_err(ctx, HSGEN_EINVAL, "reduce: n < 0");
  if (n == 0) return HSGEN_OK;
  if (!H || !S) return set_err(ctx, HSGEN_EINVAL, "reduce: NULL pointer");
  if (ld < n) return set_err(ctx, HSGEN_EINVAL, "reduce: ld < n");
  if (ld > 0x7fffffffLL) return set_err(ctx, HSGEN_EINVAL, "reduce: ld above the 32-bit range of the solver");
  if (H == S) return set_err(ctx, HSGEN_EINVAL, "reduce: H and S alias");
  HSG_CUDA(ctx, cudaSetDevice(ctx->device));
  if (!is_device_ptr(H) || !is_device_ptr(S))
    return set_err(ctx, HSGEN_EINVAL, "reduce: H and S must be device pointers");
  if (on_other_device(H, ctx->device) || on_other_device(S, ctx->device))
    return set_err(ctx, HSGEN_EINVAL, "reduce: H or S lives on another GPU than the context's");
  hsgen_status pst = split_poll_status(ctx, false);  // an earlier build's expired wait
  if (pst != HSGEN_OK) return pst;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (!ctx->blas) {
    cublasHandle_t h = nullptr;
    cublasStatus_t e = cublasCreate(&h);
    if (e != CUBLAS_STATUS_SUCCESS) return blas_err(ctx, (int)e, "cublasCreate");
    ctx->blas = h;
  }
  if (!ctx->solver) {
    cusolverDnHandle_t h = nullptr;
    cusolverStatus_t e = cusolverDnCreate(&h);
    if (e != CUSOLVER_STATUS_SUCCESS) return blas_err(ctx, (int)e, "cusolverDnCreate");
    ctx->solver = h;
  }
  if (!ctx->h_info) HSG_CUDA(ctx, cudaMallocHost(&ctx->h_info, sizeof(int)));
  cublasHandle_t blas = (cublasHandle_t)ctx->blas;
  cusolverDnHandle_t solver = (cusolverDnHandle_t)ctx->solver;
  cublasStatus_t be = cublasSetStream(blas, s);
  if (be != CUBLAS_STATUS_SUCCESS) return blas_err(ctx, (int)be, "cublasSetStream");
  cusolverStatus_t se = cusolverDnSetStream(solver, s);
  if (se != CUSOLVER_STATUS_SUCCESS) return blas_err(ctx, (int)se, "cusolverDnSetStream");

  const int uplo = ctx->opt.uplo;
  const bool upper = uplo == 'U';
  const cublasFillMode_t fill = upper ? CUBLAS_FILL_MODE_UPPER : CUBLAS_FILL_MODE_LOWER;
  cuDoubleComplex *Sm = (cuDoubleComplex *)S, *Hm = (cuDoubleComplex *)H;
  if (ctx->opt.precision == HSGEN_SPLIT && upper) {
    // split form: S = U^H U blocked; Y = U^-H H; H~ = U^-H Y^H (= U^-H H U^-1, as H is Hermitian)
    const int nb = reduce_block();
    const int nblk = (n + nb - 1) / nb;
    int lwork = 0;
    se = cusolverDnZpotrf_bufferSize(solver, CUBLAS_FILL_MODE_UPPER, std::min(n, nb), Sm, (int)ld, &lwork);
    if (se != CUSOLVER_STATUS_SUCCESS) return blas_err(ctx, (int)se, "cusolverDnZpotrf_bufferSize");
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t work_bytes = al(sizeof(cuDoubleComplex) * (size_t)std::max(lwork, 1));
    const size_t info_bytes = al(sizeof(int) * (size_t)nblk);
    const size_t gemm_bytes = split_gemm_ws_bytes(n, n, std::min(n, nb), kRedSlices);
    hsgen_status st = ensure_ws(ctx, ctx->ws_red, work_bytes + info_bytes + gemm_bytes);
    if (st != HSGEN_OK) return st;
    char *base = (char *)ctx->ws_red.ptr;
    cuDoubleComplex *work = (cuDoubleComplex *)base;
    int *d_info = (int *)(base + work_bytes);
    void *gws = base + work_bytes + info_bytes;
    HSG_CUDA(ctx, cudaMemsetAsync(d_info, 0, sizeof(int) * nblk, s));
    HSG_CUDA(ctx, launch_hermitian(n, (double2 *)H, ld, uplo, 0, s));
    st = potrf_split(ctx, n, nb, (double2 *)S, ld, work, lwork, d_info, gws, s);
    if (st == HSGEN_OK) st = solve_left_split(ctx, n, nb, (const double2 *)S, (double2 *)H, ld, gws, s);
    if (st == HSGEN_OK) {
      HSG_CUDA(ctx, launch_hermitian(n, (double2 *)H, ld, uplo, 2, s));
      st = solve_left_split(ctx, n, nb, (const double2 *)S, (double2 *)H, ld, gws, s);
    }
    if (st == HSGEN_OK) HSG_CUDA(ctx, launch_hermitian(n, (double2 *)H, ld, uplo, 1, s));
    HSG_CUDA(ctx, cudaStreamSynchronize(s));
    if (st != HSGEN_OK) return st;
    st = split_check_status(ctx, s);
    if (st != HSGEN_OK) return st;
    std::vector<int> info(nblk);
    HSG_CUDA(ctx, cudaMemcpy(info.data(), d_info, sizeof(int) * nblk, cudaMemcpyDeviceToHost));
    for (int b = 0; b < nblk; ++b) {
      if (info[b] > 0)
        return set_err(ctx, HSGEN_ENUMERIC, "reduce: S is not positive definite (leading minor " +
                                                std::to_string(b * nb + info[b]) + ")");
      if (info[b] < 0)
        return set_err(ctx, HSGEN_ECUDA, "reduce: ZPOTRF argument " + std::to_string(-info[b]) + " invalid");
    }
    return HSGEN_OK;
  }
  int lwork = 0;
  se = cusolverDnZpotrf_bufferSize(solver, fill, n, Sm, (int)ld, &lwork);
  if (se != CUSOLVER_STATUS_SUCCESS) return blas_err(ctx, (int)se, "cusolverDnZpotrf_bufferSize");
  const size_t work_bytes = (sizeof(cuDoubleComplex) * (size_t)std::max(lwork, 1) + 255) / 256 * 256;
  hsgen_status st = ensure_ws(ctx, ctx->ws_red, work_bytes + 256);
  if (st != HSGEN_OK) return st;
  cuDoubleComplex *work = (cuDoubleComplex *)ctx->ws_red.ptr;
  int *d_info = (int *)((char *)ctx->ws_red.ptr + work_bytes);

  // H in full (only its `uplo` triangle is read), then S = U^H U (or L L^H)
  HSG_CUDA(ctx, launch_hermitian(n, (double2 *)H, ld, uplo, 0, s));
  se = cusolverDnZpotrf(solver, fill, n, Sm, (int)ld, work, lwork, d_info);
  if (se != CUSOLVER_STATUS_SUCCESS) return blas_err(ctx, (int)se, "cusolverDnZpotrf");
  // 'U': H <- U^-H H, then H <- H U^-1;  'L': H <- L^-1 H, then H <- H L^-H
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0);
  be = cublasZtrsm(blas, CUBLAS_SIDE_LEFT, fill, upper ? CUBLAS_OP_C : CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, n, n, &one,
                   Sm, (int)ld, Hm, (int)ld);
  if (be != CUBLAS_STATUS_SUCCESS) return blas_err(ctx, (int)be, "cublasZtrsm (left)");
  be = cublasZtrsm(blas, CUBLAS_SIDE_RIGHT, fill, upper ? CUBLAS_OP_N : CUBLAS_OP_C, CUBLAS_DIAG_NON_UNIT, n, n,
                   &one, Sm, (int)ld, Hm, (int)ld);
  if (be != CUBLAS_STATUS_SUCCESS) return blas_err(ctx, (int)be, "cublasZtrsm (right)");
  // exactly Hermitian: (H~ + H~^H) / 2
  HSG_CUDA(ctx, launch_hermitian(n, (double2 *)H, ld, uplo, 1, s));
  HSG_CUDA(ctx, cudaMemcpyAsync(ctx->h_info, d_info, sizeof(int), cudaMemcpyDeviceToHost, s));
  HSG_CUDA(ctx, cudaStreamSynchronize(s));
  const int info = *ctx->h_info;
  if (info > 0)
    return set_err(ctx, HSGEN_ENUMERIC,
                   "reduce: S is not positive definite (leading minor " + std::to_string(info) + ")");
  if (info < 0) return set_err(ctx, HSGEN_ECUDA, "reduce: ZPOTRF argument " + std::to_string(-info) + " invalid");
  return HSGEN_OK;
}
