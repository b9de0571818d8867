// reduce.cu -- hand-off of H and S to the generalized eigensolver (Sec. 2.3,
// Eq. matrix_kohnsham: H c = eps S c with H, S Hermitian and S positive
// definite). S is factored, S = U^H U (opt.uplo 'U') or S = L L^H ('L'), in
// place in its triangle, and H is reduced in place to the standard problem
// H~ y = eps y, c = U^-1 y:
//   H~ = U^-H H U^-1   (= L^-1 H L^-H, the same matrix: the factor is unique),
// written in full and exactly Hermitian.
//
// Everything runs in this library's kernels, blocked by nb rows (default
// 128), right-looking on the upper factor:
//   for each block row k:  U_kk = chol(S_kk) and D_k = U_kk^-1   (FP64, tiles of 32)
//                          U_k,rest = D_k^H S_k,rest              (a product)
//                          S_rest -= U_k,rest^H U_k,rest          (a product, upper triangle)
// and the two triangular solves Y = U^-H H, H~ = U^-H Y^H by block rows:
//   X_k = D_k^H B_k, B_rest -= U_k,rest^H X_k.
// The products run as 7-slice BF16 products on the tensor cores (split form,
// ~2e-15 relative, FP64's level) or as FP64 DMMA products (FP64 form); the
// diagonal blocks are factored and inverted in FP64 by tile kernels (32 x 32
// tiles: Cholesky of the diagonal tile and its inverse in one CTA, the row of
// tiles right of it, the trailing tiles, then the block's inverse by back
// substitution over tiles). The lower-triangle layout is factored through a
// conjugate-transposed copy of S in the upper layout.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <string>
#include <vector>

#include "internal.cuh"
#include "split.cuh"

namespace hsg {
namespace {

constexpr int TS = 32;  // tile of the diagonal-block kernels

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

// Cholesky of one diagonal tile (nt <= 32 rows, upper: A = U^H U) in place
// and its inverse Tinv = U^-1 (32 x 32, upper, zeros below). Only the upper
// triangle of the tile is read and written. A pivot that is not positive (or
// not finite) records the global row in `info` (the smallest one wins) and is
// replaced by 1 so that the rest stays finite.
__global__ void __launch_bounds__(TS * TS) chol_tile_kernel(double2 *A, long long ld, int nt, double2 *Tinv,
                                                           int row0, int *info) {
  __shared__ double2 a[TS][TS + 1];  // a[c][r] = A(r, c)
  __shared__ double2 x[TS][TS + 1];  // x[c][r] = Tinv(r, c)
  const int r = threadIdx.x, c = threadIdx.y;
  a[c][r] = (r < nt && c < nt && r <= c) ? A[(size_t)c * ld + r] : make_double2(0.0, 0.0);
  __syncthreads();
  for (int j = 0; j < nt; ++j) {
    if (r == 0 && c == 0) {
      double d = a[j][j].x;
      if (!(d > 0.0) || !isfinite(d)) {
        atomicMin(info, row0 + j + 1);
        d = 1.0;
      }
      a[j][j] = make_double2(sqrt(d), 0.0);
    }
    __syncthreads();
    if (r == j && c > j && c < nt) {  // row j of U
      const double inv = 1.0 / a[j][j].x;
      a[c][j] = make_double2(a[c][j].x * inv, a[c][j].y * inv);
    }
    __syncthreads();
    if (r > j && r <= c && c < nt) {  // S(r, c) -= conj(U(j, r)) U(j, c)
      const double2 u = a[r][j], v = a[c][j];
      a[c][r].x -= u.x * v.x + u.y * v.y;
      a[c][r].y -= u.x * v.y - u.y * v.x;
    }
    __syncthreads();
  }
  // inverse: column c of X = U^-1 by back substitution (one thread per column)
  if (c == 0 && r < TS) {
    const int col = r;
    for (int i = 0; i < TS; ++i) x[col][i] = make_double2(0.0, 0.0);
    if (col < nt) {
      x[col][col] = make_double2(1.0 / a[col][col].x, 0.0);
      for (int i = col - 1; i >= 0; --i) {
        double sr = 0.0, si = 0.0;
        for (int k = i + 1; k <= col; ++k) {  // U(i, k) X(k, col)
          const double2 u = a[k][i], v = x[col][k];
          sr += u.x * v.x - u.y * v.y;
          si += u.x * v.y + u.y * v.x;
        }
        const double inv = 1.0 / a[i][i].x;
        x[col][i] = make_double2(-sr * inv, -si * inv);
      }
    }
  }
  __syncthreads();
  if (r < nt && c < nt && r <= c) A[(size_t)c * ld + r] = a[c][r];
  Tinv[c * TS + r] = x[c][r];
}

// Row of tiles right of diagonal tile j: A_jc <- Tinv_j^H A_jc (blockIdx.x = c - j - 1).
__global__ void __launch_bounds__(TS * TS) tile_row_kernel(double2 *A, long long ld, int kb, int j,
                                                          const double2 *Tinv) {
  __shared__ double2 t[TS][TS + 1], b[TS][TS + 1];
  const int r = threadIdx.x, c = threadIdx.y;
  const int tc = j + 1 + blockIdx.x;
  const int rows = min(TS, kb - j * TS), cols = min(TS, kb - tc * TS);
  double2 *blk = A + (size_t)(tc * TS) * ld + j * TS;
  t[c][r] = Tinv[c * TS + r];
  b[c][r] = (r < rows && c < cols) ? blk[(size_t)c * ld + r] : make_double2(0.0, 0.0);
  __syncthreads();
  double sr = 0.0, si = 0.0;
  for (int k = 0; k <= r; ++k) {  // conj(Tinv(k, r)) B(k, c)
    const double2 u = t[r][k], v = b[c][k];
    sr += u.x * v.x + u.y * v.y;
    si += u.x * v.y - u.y * v.x;
  }
  if (r < rows && c < cols) blk[(size_t)c * ld + r] = make_double2(sr, si);
}

// Trailing tiles of the diagonal block: A_rc -= A_jr^H A_jc for j < r <= c
// (blockIdx.x enumerates the pairs); a diagonal tile keeps its lower part.
__global__ void __launch_bounds__(TS * TS) tile_update_kernel(double2 *A, long long ld, int kb, int j) {
  __shared__ double2 p[TS][TS + 1], q[TS][TS + 1];
  const int r = threadIdx.x, c = threadIdx.y;
  const int nt = (kb + TS - 1) / TS;
  int idx = blockIdx.x, tr = j + 1, tc = j + 1;
  for (tc = j + 1; tc < nt; ++tc) {  // pairs (tr, tc), j < tr <= tc, column by column
    const int cnt = tc - j;
    if (idx < cnt) {
      tr = j + 1 + idx;
      break;
    }
    idx -= cnt;
  }
  const int rows = min(TS, kb - tr * TS), cols = min(TS, kb - tc * TS), kd = min(TS, kb - j * TS);
  const double2 *Pj = A + (size_t)(tr * TS) * ld + j * TS;  // A_jr
  const double2 *Qj = A + (size_t)(tc * TS) * ld + j * TS;  // A_jc
  p[c][r] = (r < kd && c < rows) ? Pj[(size_t)c * ld + r] : make_double2(0.0, 0.0);
  q[c][r] = (r < kd && c < cols) ? Qj[(size_t)c * ld + r] : make_double2(0.0, 0.0);
  __syncthreads();
  double sr = 0.0, si = 0.0;
  for (int k = 0; k < kd; ++k) {  // conj(P(k, r)) Q(k, c)
    const double2 u = p[r][k], v = q[c][k];
    sr += u.x * v.x + u.y * v.y;
    si += u.x * v.y - u.y * v.x;
  }
  if (r < rows && c < cols && (tr != tc || r <= c)) {
    double2 *dst = A + (size_t)(tc * TS + c) * ld + tr * TS + r;
    const double2 o = *dst;
    *dst = make_double2(o.x - sr, o.y - si);
  }
}

// Inverse D = U^-1 of the factored diagonal block (kb x kb upper, tiles of
// 32): column of tiles c = blockIdx.x, from the diagonal tile up:
// D_cc = Tinv_c, D_rc = -Tinv_r sum_{r < k <= c} U_rk D_kc. D: ldd = kb,
// zeros below the diagonal.
__global__ void __launch_bounds__(TS * TS) block_inverse_kernel(const double2 *A, long long ld, int kb,
                                                               const double2 *Tinv, double2 *D, int ldd) {
  __shared__ double2 u[TS][TS + 1], v[TS][TS + 1];
  const int r = threadIdx.x, c = threadIdx.y;
  const int nt = (kb + TS - 1) / TS;
  const int tc = blockIdx.x;
  const int cols = min(TS, kb - tc * TS);
  for (int tr = nt - 1; tr > tc; --tr) {  // tiles below the diagonal: zero
    const int rows = min(TS, kb - tr * TS);
    if (r < rows && c < cols) D[(size_t)(tc * TS + c) * ldd + tr * TS + r] = make_double2(0.0, 0.0);
  }
  if (r < TS && c < cols && tc * TS + r < kb) {
    D[(size_t)(tc * TS + c) * ldd + tc * TS + r] = Tinv[(size_t)tc * TS * TS + c * TS + r];
  }
  __syncthreads();
  for (int tr = tc - 1; tr >= 0; --tr) {
    // acc = sum_{tr < k <= tc} U_{tr,k} D_{k,tc}
    double sr = 0.0, si = 0.0;
    for (int tk = tr + 1; tk <= tc; ++tk) {
      const int kd = min(TS, kb - tk * TS);
      u[c][r] = (c < kd) ? A[(size_t)(tk * TS + c) * ld + tr * TS + r] : make_double2(0.0, 0.0);  // U(tr*32+r, tk*32+c)
      v[c][r] = (r < kd && c < cols) ? D[(size_t)(tc * TS + c) * ldd + tk * TS + r] : make_double2(0.0, 0.0);
      __syncthreads();
      for (int k = 0; k < kd; ++k) {  // U(r, k) D(k, c)
        const double2 a = u[k][r], b = v[c][k];
        sr += a.x * b.x - a.y * b.y;
        si += a.x * b.y + a.y * b.x;
      }
      __syncthreads();
    }
    v[c][r] = make_double2(sr, si);  // the sum (both tiles are free again)
    u[c][r] = Tinv[(size_t)tr * TS * TS + c * TS + r];
    __syncthreads();
    double xr = 0.0, xi = 0.0;
    for (int k = r; k < TS; ++k) {  // -Tinv(r, k) acc(k, c), Tinv upper
      const double2 a = u[k][r], b = v[c][k];
      xr -= a.x * b.x - a.y * b.y;
      xi -= a.x * b.y + a.y * b.x;
    }
    if (c < cols) D[(size_t)(tc * TS + c) * ldd + tr * TS + r] = make_double2(xr, xi);
    __syncthreads();
  }
}

// Lower layout: dst(j, i) = conj(src(i, j)) for i >= j (the upper triangle of
// dst from the lower triangle of src), or, with to_lower, dst(i, j) =
// conj(src(j, i)) for i >= j (the lower triangle of dst from the upper of src).
__global__ void tri_transpose_kernel(int n, const double2 *src, double2 *dst, long long ld, int to_lower) {
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  if (i >= n || j >= n || i < j) return;
  if (to_lower) {
    const double2 v = src[(size_t)i * ld + j];
    dst[(size_t)j * ld + i] = make_double2(v.x, -v.y);
  } else {
    const double2 v = src[(size_t)j * ld + i];
    dst[(size_t)i * ld + j] = make_double2(v.x, -v.y);
  }
}

hsgen_status red_err(hsgen_ctx *ctx, cudaError_t e, const char *what) { return cuda_err(ctx, e, what); }

constexpr int kRedBlock = 128;  // default; HSGEN_REDUCE_BLOCK (32..1024, multiple of 32) overrides it
constexpr int kRedSlices = 7;

int reduce_block() {
  int nb = kRedBlock;
  if (const char *e = std::getenv("HSGEN_REDUCE_BLOCK")) nb = std::max(32, std::min(1024, std::atoi(e))) / 32 * 32;
  return nb;
}

struct RedWs {
  double2 *Dinv;   // inverses of the diagonal blocks, nb x nb each (ld nb), block k at k * nb * nb
  double2 *Tinv;   // tile inverses of the block being factored (nb / 32 tiles of 32 x 32)
  double2 *tmp;    // FP64 form: product output before it is copied back (nb x n)
  double2 *Scopy;  // lower layout: S in the upper layout
  int *info;
  void *gws;       // split products
  size_t bytes;
};

RedWs red_layout(void *base, int n, long long ld, int nb, bool split, bool lower) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const int nblk = (n + nb - 1) / nb;
  RedWs w;
  size_t o = 0;
  char *b = (char *)base;
  w.Dinv = (double2 *)(b + o);
  o += al(sizeof(double2) * (size_t)nblk * nb * nb);
  w.Tinv = (double2 *)(b + o);
  o += al(sizeof(double2) * (size_t)((nb + TS - 1) / TS) * TS * TS);
  w.tmp = (double2 *)(b + o);
  o += split ? 0 : al(sizeof(double2) * (size_t)nb * n);
  w.Scopy = (double2 *)(b + o);
  o += lower ? al(sizeof(double2) * (size_t)ld * n) : 0;
  w.info = (int *)(b + o);
  o += al(sizeof(int));
  w.gws = b + o;
  o += split ? split_gemm_ws_bytes(n, n, std::min(n, nb), kRedSlices) : 0;
  w.bytes = o;
  return w;
}

// C (+)= (+-) P^H Q (P: K x M, Q: K x N) in the chosen form. In the split
// form C may be Q itself (the operands are sliced before the product is
// formed); in the FP64 form an in-place product goes through w.tmp.
hsgen_status product(hsgen_ctx *ctx, bool split, int M, int N, int K, const double2 *P, long long ldp,
                     const double2 *Q, long long ldq, double2 *C, long long ldc, int uplo, bool accumulate,
                     bool negate, const RedWs &w, cudaStream_t s) {
  if (split)
    return split_gemm(ctx, M, N, K, P, ldp, Q, ldq, C, ldc, uplo, accumulate, negate, kRedSlices, w.gws, s);
  if (C == Q) {
    HSG_LAUNCH(ctx, launch_gemm_fp64(M, N, K, P, ldp, Q, ldq, w.tmp, M, uplo, 0, negate ? 1 : 0, s));
    HSG_CUDA(ctx, cudaMemcpy2DAsync(C, sizeof(double2) * ldc, w.tmp, sizeof(double2) * M, sizeof(double2) * M, N,
                                    cudaMemcpyDeviceToDevice, s));
    return HSGEN_OK;
  }
  HSG_LAUNCH(ctx, launch_gemm_fp64(M, N, K, P, ldp, Q, ldq, C, ldc, uplo, accumulate ? 1 : 0, negate ? 1 : 0, s));
  return HSGEN_OK;
}

// U_kk = chol(S_kk) in place and D = U_kk^-1 (kb x kb, ld kb), FP64 tile kernels.
hsgen_status factor_diag(hsgen_ctx *ctx, double2 *Skk, long long ld, int kb, int row0, double2 *D, const RedWs &w,
                         cudaStream_t s) {
  const int nt = (kb + TS - 1) / TS;
  const dim3 blk(TS, TS);
  for (int j = 0; j < nt; ++j) {
    const int tj = std::min(TS, kb - j * TS);
    double2 *Ajj = Skk + (size_t)(j * TS) * ld + j * TS;
    chol_tile_kernel<<<1, blk, 0, s>>>(Ajj, ld, tj, w.Tinv + (size_t)j * TS * TS, row0 + j * TS, w.info);
    HSG_LAUNCH(ctx, cudaGetLastError());
    if (j + 1 < nt) {
      tile_row_kernel<<<nt - 1 - j, blk, 0, s>>>(Skk, ld, kb, j, w.Tinv + (size_t)j * TS * TS);
      HSG_LAUNCH(ctx, cudaGetLastError());
      const int pairs = (nt - 1 - j) * (nt - j) / 2;
      tile_update_kernel<<<pairs, blk, 0, s>>>(Skk, ld, kb, j);
      HSG_LAUNCH(ctx, cudaGetLastError());
    }
  }
  block_inverse_kernel<<<nt, blk, 0, s>>>(Skk, ld, kb, w.Tinv, D, kb);
  HSG_LAUNCH(ctx, cudaGetLastError());
  return HSGEN_OK;
}

// S = U^H U in place (upper triangle), right-looking by blocks of nb.
hsgen_status potrf_blocked(hsgen_ctx *ctx, bool split, int n, int nb, double2 *S, long long ld, const RedWs &w,
                           cudaStream_t s) {
  for (int k = 0, blk = 0; k < n; k += nb, ++blk) {
    const int kb = std::min(nb, n - k), m = n - k - kb;
    double2 *Skk = S + k + (size_t)k * ld;
    double2 *D = w.Dinv + (size_t)blk * nb * nb;
    hsgen_status st = factor_diag(ctx, Skk, ld, kb, k, D, w, s);
    if (st != HSGEN_OK) return st;
    if (m == 0) break;
    double2 *U12 = S + k + (size_t)(k + kb) * ld;
    st = product(ctx, split, kb, m, kb, D, kb, U12, ld, U12, ld, 0, false, false, w, s);  // U12 = D^H S12
    if (st != HSGEN_OK) return st;
    st = product(ctx, split, m, m, kb, U12, ld, U12, ld, S + (k + kb) + (size_t)(k + kb) * ld, ld, 'U', true, true,
                 w, s);  // S22 -= U12^H U12
    if (st != HSGEN_OK) return st;
  }
  return HSGEN_OK;
}

// U^H X = B in place on B (n x n), U upper triangular with block inverses D_k:
// X_k = D_k^H B_k, then B_rest -= U_{k,rest}^H X_k.
hsgen_status solve_left_blocked(hsgen_ctx *ctx, bool split, int n, int nb, const double2 *U, double2 *B,
                                long long ld, const RedWs &w, cudaStream_t s) {
  for (int k = 0, blk = 0; k < n; k += nb, ++blk) {
    const int kb = std::min(nb, n - k), m = n - k - kb;
    const double2 *D = w.Dinv + (size_t)blk * nb * nb;
    hsgen_status st = product(ctx, split, kb, n, kb, D, kb, B + k, ld, B + k, ld, 0, false, false, w, s);
    if (st != HSGEN_OK) return st;
    if (m == 0) break;
    st = product(ctx, split, m, n, kb, U + k + (size_t)(k + kb) * ld, ld, B + k, ld, B + k + kb, ld, 0, true, true,
                 w, s);
    if (st != HSGEN_OK) return st;
  }
  return HSGEN_OK;
}

}  // namespace

void reduce_release(hsgen_ctx *ctx) {
  if (ctx->ws_red.ptr) cudaFree(ctx->ws_red.ptr);
  if (ctx->h_info) cudaFreeHost(ctx->h_info);
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
  if (ld > 0x7fffffffLL) return set_err(ctx, HSGEN_EINVAL, "reduce: ld above 2^31 - 1");
  if (H == S) return set_err(ctx, HSGEN_EINVAL, "reduce: H and S alias");
  HSG_CUDA(ctx, cudaSetDevice(ctx->device));
  if (!is_device_ptr(H) || !is_device_ptr(S))
    return set_err(ctx, HSGEN_EINVAL, "reduce: H and S must be device pointers");
  if (on_other_device(H, ctx->device) || on_other_device(S, ctx->device))
    return set_err(ctx, HSGEN_EINVAL, "reduce: H or S lives on another GPU than the context's");
  hsgen_status pst = split_poll_status(ctx, false);  // an earlier build's expired wait
  if (pst != HSGEN_OK) return pst;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (!ctx->h_info) HSG_CUDA(ctx, cudaMallocHost(&ctx->h_info, sizeof(int)));
  const int uplo = ctx->opt.uplo;
  const bool lower = uplo != 'U';
  const bool split = ctx->opt.precision == HSGEN_SPLIT;
  const int nb = reduce_block();
  if (split && !ctx->d_status) {
    HSG_CUDA(ctx, cudaMalloc(&ctx->d_status, sizeof(int)));
    HSG_CUDA(ctx, cudaMallocHost(&ctx->h_status, sizeof(int)));
    HSG_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
  }
  hsgen_status st = ensure_ws(ctx, ctx->ws_red, red_layout(nullptr, n, ld, nb, split, lower).bytes);
  if (st != HSGEN_OK) return st;
  const RedWs w = red_layout(ctx->ws_red.ptr, n, ld, nb, split, lower);
  ctx->launches = 0;
  const int big = INT_MAX;
  HSG_CUDA(ctx, cudaMemcpyAsync(w.info, &big, sizeof(int), cudaMemcpyHostToDevice, s));
  // S in the upper layout (the lower layout works on a conjugate-transposed copy)
  double2 *Su = (double2 *)S;
  if (lower) {
    Su = w.Scopy;
    const dim3 g((n + 31) / 32, (n + 7) / 8);
    tri_transpose_kernel<<<g, dim3(32, 8), 0, s>>>(n, (const double2 *)S, Su, ld, 0);
    HSG_LAUNCH(ctx, cudaGetLastError());
  }
  // S = U^H U; Y = U^-H H; H~ = U^-H Y^H (= U^-H H U^-1, as H is Hermitian)
  HSG_CUDA(ctx, launch_hermitian(n, (double2 *)H, ld, uplo, 0, s));
  st = potrf_blocked(ctx, split, n, nb, Su, ld, w, s);
  if (st == HSGEN_OK) st = solve_left_blocked(ctx, split, n, nb, Su, (double2 *)H, ld, w, s);
  if (st == HSGEN_OK) {
    HSG_CUDA(ctx, launch_hermitian(n, (double2 *)H, ld, uplo, 2, s));
    st = solve_left_blocked(ctx, split, n, nb, Su, (double2 *)H, ld, w, s);
  }
  if (st == HSGEN_OK) HSG_CUDA(ctx, launch_hermitian(n, (double2 *)H, ld, uplo, 1, s));
  if (st == HSGEN_OK && lower) {  // L = U^H into S's lower triangle
    const dim3 g((n + 31) / 32, (n + 7) / 8);
    tri_transpose_kernel<<<g, dim3(32, 8), 0, s>>>(n, Su, (double2 *)S, ld, 1);
    HSG_LAUNCH(ctx, cudaGetLastError());
  }
  HSG_CUDA(ctx, cudaMemcpyAsync(ctx->h_info, w.info, sizeof(int), cudaMemcpyDeviceToHost, s));
  HSG_CUDA(ctx, cudaStreamSynchronize(s));
  if (st != HSGEN_OK) return st;
  if (split) {
    st = split_check_status(ctx, s);
    if (st != HSGEN_OK) return st;
  }
  const int info = *ctx->h_info;
  if (info != big)
    return set_err(ctx, HSGEN_ENUMERIC,
                   "reduce: S is not positive definite (leading minor " + std::to_string(info) + ")");
  return HSGEN_OK;
}
