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

#include <string>

#include "internal.cuh"

namespace hsg {
namespace {

// mode 0: the triangle opposite `uplo` takes the conjugate transpose of the
// `uplo` triangle; mode 1: both triangles take the average (M + M^H) / 2.
// Diagonal imaginary parts become 0. A block takes the tile pair (bi, bj),
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
      double2 v;
      if (i == j) {
        v = make_double2(up.x, 0.0);
      } else if (mode == 1) {
        v = make_double2(0.5 * (up.x + lo.x), 0.5 * (up.y - lo.y));
      } else {
        v = (uplo == 'U') ? up : make_double2(lo.x, -lo.y);
      }
      M[(size_t)j * ld + i] = v;                        // (i, j)
      if (i != j) M[(size_t)i * ld + j] = make_double2(v.x, -v.y);  // (j, i)
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
