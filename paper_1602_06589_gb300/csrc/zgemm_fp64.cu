// zgemm_fp64.cu -- the FP64 form of the two contractions, on FP64 tensor cores
// (warp-level DMMA, mma.sync.m8n8k4.f64):
//
//  a3  X_a = T_a W_a for every atom (the per-atom zgemm/zhemm of Listings
//      alg:H_BB and alg:H_AA_nHPD, Sec. 4.4-4.6, with the four T blocks kept
//      together as one 2N_L x 2N_L Hermitian matrix);
//  a4  H = W^H X and S = W^H diag(u) W over the whole stacked depth
//      (Listings alg:S, alg:H_BB, alg:H_AA fused: W = [A;B] stacked over atoms
//      as in Fig. memorylayoutA, u = 1 on A rows and ||u_dot_l||^2 on B rows),
//      only the tiles of one triangle, H and S tiles sharing the W_i loads.
//
// Both are C = P^H Q with P (K x M) and Q (K x N) column-major complex (every
// column contiguous over the depth K); for a3 P = T_a (Hermitian, so T^H = T).
// Complex products use 4 real DMMAs: Re += Pr Qr + Pi Qi, Im += Pr Qi - Pi Qr.
#include "internal.cuh"

namespace hsg {

namespace {

constexpr int MT = 64, NT = 64, KT = 16;  // CTA tile (complex), depth step
constexpr int PADS = MT + 2;              // smem row stride in double2 (bank spread)
constexpr int NTHREADS = 256;             // 8 warps: 2 (m) x 4 (n), 32 x 16 each

__device__ __forceinline__ void dmma(double &d0, double &d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool pred) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  int n = pred ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Loads a KT x 64 complex tile (columns c0.., depth k0..) of a column-major
// matrix into smem laid out [k][col] with row stride PADS.
__device__ __forceinline__ void load_tile(double2 *sm, const double2 *__restrict__ G, long long ld, int c0,
                                          int ncols, int k0, int kmax) {
  for (int c = threadIdx.x; c < 64 * KT; c += NTHREADS) {
    int col = c / KT, k = c % KT;
    bool ok = (c0 + col < ncols) && (k0 + k < kmax);
    const double2 *src = ok ? G + (size_t)(c0 + col) * ld + (k0 + k) : G;
    cp_async16(sm + k * PADS + col, src, ok);
  }
}

// One CTA computes a 64 x 64 complex tile of C1 = P^H Q, or with UQ of
// C1 = P^H diag(u) Q (and, if DUAL, C2 = P^H diag(u) P restricted to the same
// rows/columns).
template <bool DUAL, bool UQ = false>
__device__ __forceinline__ void tile_mma(const double2 *__restrict__ P, long long ldp, const double2 *__restrict__ Q,
                                         long long ldq, const double *__restrict__ urow, int M, int N, int K, int i0,
                                         int j0, double (&acc1)[4][2][2][2], double (&acc2)[4][2][2][2],
                                         double2 *smem) {
  constexpr int STAGE = (DUAL ? 3 : 2) * KT * PADS;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int wm = warp / 4, wn = warp % 4;
  const int g = lane / 4, q = lane % 4;
  const int nk = (K + KT - 1) / KT;

  auto issue = [&](int kt, int buf) {
    double2 *s = smem + buf * STAGE;
    load_tile(s, P, ldp, i0, M, kt * KT, K);
    load_tile(s + KT * PADS, Q, ldq, j0, N, kt * KT, K);
    if (DUAL) load_tile(s + 2 * KT * PADS, P, ldp, j0, N, kt * KT, K);
    cp_async_commit();
  };
  if (nk > 0) issue(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    int buf = kt & 1;
    if (kt + 1 < nk) {
      issue(kt + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const double2 *sP = smem + buf * STAGE;
    const double2 *sQ = sP + KT * PADS;
    const double2 *sQ2 = sQ + KT * PADS;
#pragma unroll
    for (int kk = 0; kk < KT; kk += 4) {
      double2 a[4], b[2], b2[2];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) a[mt] = sP[(kk + q) * PADS + wm * 32 + mt * 8 + g];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) b[nt] = sQ[(kk + q) * PADS + wn * 16 + nt * 8 + g];
      if (UQ) {
        const int kg = kt * KT + kk + q;
        const double u = (kg < K) ? urow[kg] : 0.0;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) b[nt] = make_double2(b[nt].x * u, b[nt].y * u);
      }
      if (DUAL) {
        int kg = kt * KT + kk + q;
        double u = (kg < K) ? urow[kg] : 0.0;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          double2 v = sQ2[(kk + q) * PADS + wn * 16 + nt * 8 + g];
          b2[nt] = make_double2(v.x * u, v.y * u);
        }
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        double ar = a[mt].x, ai = a[mt].y, nai = -a[mt].y;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          dmma(acc1[mt][nt][0][0], acc1[mt][nt][0][1], ar, b[nt].x);
          dmma(acc1[mt][nt][0][0], acc1[mt][nt][0][1], ai, b[nt].y);
          dmma(acc1[mt][nt][1][0], acc1[mt][nt][1][1], ar, b[nt].y);
          dmma(acc1[mt][nt][1][0], acc1[mt][nt][1][1], nai, b[nt].x);
          if (DUAL) {
            dmma(acc2[mt][nt][0][0], acc2[mt][nt][0][1], ar, b2[nt].x);
            dmma(acc2[mt][nt][0][0], acc2[mt][nt][0][1], ai, b2[nt].y);
            dmma(acc2[mt][nt][1][0], acc2[mt][nt][1][1], ar, b2[nt].y);
            dmma(acc2[mt][nt][1][0], acc2[mt][nt][1][1], nai, b2[nt].x);
          }
        }
      }
    }
    __syncthreads();
  }
}

// Writes an accumulator set. Fragment layout of m8n8k4 f64: c0, c1 at
// row = lane/4, columns 2*(lane%4) + {0, 1}.
__device__ __forceinline__ void store_tile(double2 *C, long long ldc, int M, int N, int i0, int j0,
                                           const double (&acc)[4][2][2][2], int tri, int accumulate) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int wm = warp / 4, wn = warp % 4;
  const int g = lane / 4, q = lane % 4;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        int i = i0 + wm * 32 + mt * 8 + g;
        int j = j0 + wn * 16 + nt * 8 + 2 * q + e;
        if (i >= M || j >= N) continue;
        if (tri == 'U' && i > j) continue;
        if (tri == 'L' && i < j) continue;
        double re = acc[mt][nt][0][e], im = acc[mt][nt][1][e];
        double2 *dst = C + (size_t)j * ldc + i;
        if (accumulate) {
          double2 o = *dst;
          re += o.x;
          im += o.y;
        }
        if (tri && i == j) im = 0.0;
        *dst = make_double2(re, im);
      }
}

template <bool DUAL>
__device__ __forceinline__ void zero_acc(double (&acc)[4][2][2][2]) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int d = 0; d < 2; ++d) acc[a][b][c][d] = 0.0;
}

// a3: blockIdx.z = atom (of one species), (blockIdx.x, blockIdx.y) = (m, n) tile.
__global__ void __launch_bounds__(NTHREADS) tapply_kernel(int dpad, int n_g, const double2 *__restrict__ T,
                                                          const int *__restrict__ atoms, const int *__restrict__ off,
                                                          int row_base, const double2 *__restrict__ W,
                                                          double2 *__restrict__ X, long long ldw) {
  extern __shared__ double2 smem[];
  int a = atoms[blockIdx.z];
  int r0 = off[a] - row_base;
  double acc[4][2][2][2], dummy[4][2][2][2];
  zero_acc<false>(acc);
  tile_mma<false>(T, dpad, W + r0, ldw, nullptr, dpad, n_g, dpad, blockIdx.x * MT, blockIdx.y * NT, acc, dummy,
                  smem);
  store_tile(X + r0, ldw, dpad, n_g, blockIdx.x * MT, blockIdx.y * NT, acc, 0, 0);
}

// a4: one CTA per tile of the chosen triangle (linear index -> (bi, bj)).
// MODE 0: H = W^H X and S = W^H diag(u) W (W = P, X = Q); MODE 1: H = P^H Q
// only (S in the Legendre form, or H = Y^H Y of the HPD route); MODE 2:
// S = P^H diag(u) P only, into H's pointer (the HPD route's S).
template <int MODE>
__global__ void __launch_bounds__(NTHREADS) hs_kernel(int n_g, int depth, const double2 *__restrict__ W,
                                                      const double2 *__restrict__ X, const double *__restrict__ urow,
                                                      long long ldw, double2 *__restrict__ H, double2 *__restrict__ S,
                                                      long long ld, int uplo, int accumulate, BlockOwner own) {
  extern __shared__ double2 smem[];
  long long x = blockIdx.x;
  int hi = (int)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
  while ((long long)hi * (hi + 1) / 2 > x) --hi;
  while ((long long)(hi + 1) * (hi + 2) / 2 <= x) ++hi;
  int lo = (int)(x - (long long)hi * (hi + 1) / 2);  // lo <= hi
  int bi = (uplo == 'U') ? lo : hi, bj = (uplo == 'U') ? hi : lo;
  if (!own.owns((long long)bi * MT, (long long)bj * NT)) return;  // 64 x 64 tiles lie inside one block
  double acc1[4][2][2][2], acc2[4][2][2][2];
  zero_acc<true>(acc1);
  zero_acc<MODE == 0>(acc2);
  tile_mma<MODE == 0, MODE == 2>(W, ldw, MODE == 2 ? W : X, ldw, urow, n_g, n_g, depth, bi * MT, bj * NT, acc1, acc2,
                                 smem);
  store_tile(H, ld, n_g, n_g, bi * MT, bj * NT, acc1, uplo, accumulate);
  if (MODE == 0) store_tile(S, ld, n_g, n_g, bi * MT, bj * NT, acc2, uplo, accumulate);
}

// General C (+)= (+-) P^H Q (P: K x M, Q: K x N, C: M x N): one CTA per
// 64 x 64 tile (blockIdx.x row tile, blockIdx.y column tile); uplo 'U'
// computes only the tiles and entries i <= j (diagonal imaginary parts 0).
__global__ void __launch_bounds__(NTHREADS) gemm_kernel(int M, int N, int K, const double2 *__restrict__ P,
                                                        long long ldp, const double2 *__restrict__ Q, long long ldq,
                                                        double2 *__restrict__ C, long long ldc, int uplo,
                                                        int accumulate, int negate) {
  extern __shared__ double2 smem[];
  const int i0 = blockIdx.x * MT, j0 = blockIdx.y * NT;
  if (uplo == 'U' && i0 > j0 + NT - 1) return;
  double acc[4][2][2][2], dummy[4][2][2][2];
  zero_acc<false>(acc);
  tile_mma<false>(P, ldp, Q, ldq, nullptr, M, N, K, i0, j0, acc, dummy, smem);
  if (negate) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int d = 0; d < 2; ++d) acc[a][b][c][d] = -acc[a][b][c][d];
  }
  store_tile(C, ldc, M, N, i0, j0, acc, uplo, accumulate);
}

__global__ void mirror_kernel(int n, double2 *M, long long ld, int uplo) {
  int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  if (i >= n || j >= n) return;
  // destination (i, j) in the unwritten triangle takes conj of (j, i)
  bool dst = (uplo == 'U') ? (i > j) : (i < j);
  if (dst) {
    double2 v = M[(size_t)i * ld + j];
    M[(size_t)j * ld + i] = make_double2(v.x, -v.y);
  }
}

}  // namespace

cudaError_t launch_tapply_fp64(int dpad, int n_g, const double2 *T, const int *atoms, int n_atoms, const int *off,
                               int row_base, const double2 *W, double2 *X, long long ldw, cudaStream_t s) {
  if (n_g <= 0 || n_atoms <= 0) return cudaSuccess;
  size_t sm = sizeof(double2) * 2 * 2 * KT * PADS;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tapply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((dpad + MT - 1) / MT, (n_g + NT - 1) / NT, n_atoms);
  tapply_kernel<<<grid, NTHREADS, sm, s>>>(dpad, n_g, T, atoms, off, row_base, W, X, ldw);
  return cudaGetLastError();
}

cudaError_t launch_hs_fp64(int n_g, int depth, const double2 *W, const double2 *X, const double *urow, long long ldw,
                           double2 *H, double2 *S, long long ld, int uplo, int accumulate, const BlockOwner &own,
                           cudaStream_t s, bool gram) {
  if (n_g <= 0) return cudaSuccess;
  size_t sm = sizeof(double2) * 2 * 3 * KT * PADS;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(hs_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(hs_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(hs_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  long long nb = (n_g + MT - 1) / MT;
  long long ntiles = nb * (nb + 1) / 2;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const unsigned g = (unsigned)ntiles;
  if (gram) {  // H = X^H X (X = C^H W), then S = W^H diag(u) W
    hs_kernel<1><<<g, NTHREADS, sm, s>>>(n_g, depth, X, X, urow, ldw, H, nullptr, ld, uplo, accumulate, own);
    if (S) hs_kernel<2><<<g, NTHREADS, sm, s>>>(n_g, depth, W, W, urow, ldw, S, nullptr, ld, uplo, accumulate, own);
  } else if (S) {
    hs_kernel<0><<<g, NTHREADS, sm, s>>>(n_g, depth, W, X, urow, ldw, H, S, ld, uplo, accumulate, own);
  } else {
    hs_kernel<1><<<g, NTHREADS, sm, s>>>(n_g, depth, W, X, urow, ldw, H, S, ld, uplo, accumulate, own);
  }
  return cudaGetLastError();
}

cudaError_t launch_gemm_fp64(int M, int N, int K, const double2 *P, long long ldp, const double2 *Q, long long ldq,
                             double2 *C, long long ldc, int uplo, int accumulate, int negate, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  size_t sm = sizeof(double2) * 2 * 2 * KT * PADS;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((M + MT - 1) / MT, (N + NT - 1) / NT);
  gemm_kernel<<<grid, NTHREADS, sm, s>>>(M, N, K, P, ldp, Q, ldq, C, ldc, uplo, accumulate, negate);
  return cudaGetLastError();
}

cudaError_t launch_mirror(int n_g, double2 *M, long long ld, int uplo, cudaStream_t s) {
  if (n_g <= 0) return cudaSuccess;
  dim3 grid((n_g + 31) / 32, (n_g + 7) / 8);
  mirror_kernel<<<grid, dim3(32, 8), 0, s>>>(n_g, M, ld, uplo);
  return cudaGetLastError();
}

}  // namespace hsg
