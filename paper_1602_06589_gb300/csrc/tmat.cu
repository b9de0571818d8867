// tmat.cu -- T matrices of one species (App. A.2, Eqs. gaunt, nonsph_integrals
// and t_matrices), assembled on the device in FP64:
//
//   T^{[xy]}_{L',L} = sum_{l''} I^{(x,y)}_{l,l',l''} c_{m''} G_{L,L',(l'',m'')}
//                     + spherical diagonal,      m'' = m' - m,
//   G_{L,L',L''} = int Y*_{L'} Y_L Y_{L''} dOmega
//               = 2 pi delta_{m', m+m''} int_{-1}^{1} P_{L'} P_L P_{L''} dx,
//
// with P_L the orthonormal associated Legendre functions (Condon-Shortley
// phase). The x-integrand is a polynomial of degree <= l + l' + l'' <= 4 l_max,
// so Gauss-Legendre quadrature with n >= 2 l_max + 1 nodes is exact; the
// nodes come from Newton's iteration on P_n. c_{m''} = 1 (m'' >= 0),
// (-1)^{m''} (m'' < 0) makes the potential real and T Hermitian.
// Spherical diagonal: AA += E_l, BB += E_l ||u_dot_l||^2, AB += 1/2, BA += 1/2.
#include <cmath>

#include "internal.cuh"

namespace hsg {

// Recurrence coefficient a_lm = sqrt((4l^2 - 1) / (l^2 - m^2)) (computed inline:
// this kernel runs once per species).
__device__ __forceinline__ double rec_a(int l, int m) {
  return sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
}

// Gauss-Legendre nodes and weights on [-1, 1].
__global__ void gauss_legendre_kernel(int n, double *x, double *w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double z = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
  double pp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    pp = n * (z * p1 - p0) / (z * z - 1.0);
    double dz = p1 / pp;
    z -= dz;
    if (fabs(dz) < 1e-16) break;
  }
  {  // derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    pp = n * (z * p1 - p0) / (z * z - 1.0);
  }
  x[i] = z;
  w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
}

// tab[node][l][m] = Pbar_lm(x_node), l <= lt, 0 <= m <= l (orthonormal incl. 1/sqrt(2 pi)).
__global__ void legendre_table_kernel(int n, const double *x, int lt, double *tab) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  double ct = x[g], st = sqrt(1.0 - ct * ct);
  double *T = tab + (size_t)g * kLTab * kLTab;
  for (int l = 0; l <= lt; ++l)
    for (int m = 0; m <= l; ++m) {
      double v;
      if (m == l)
        v = (l == 0) ? 0.28209479177387814347 : -sqrt((2.0 * l + 1.0) / (2.0 * l)) * st * T[(l - 1) * kLTab + l - 1];
      else if (m == l - 1)
        v = sqrt(2.0 * m + 3.0) * ct * T[(l - 1) * kLTab + m];
      else
        v = rec_a(l, m) * (ct * T[(l - 1) * kLTab + m] - T[(l - 2) * kLTab + m] / rec_a(l - 1, m));
      T[l * kLTab + m] = v;
    }
}

struct TParams {
  int lmax;     // species l_max: strides of the radial integrals I[l][l'][l'']
  int nl;       // N_L of the T built here (the contraction's, (lc+1)^2)
  int lns;      // l_nonsph: Gaunt part only for l, l' <= lns (Fig. Tmat_structure)
  int dpad, nq;
  const double *I[4];  // uu, uud, udu, udud on the device
  const double *el, *un2;
};

__device__ __forceinline__ double pbar(const double *tab, int g, int l, int m) {
  double v = tab[(size_t)g * kLTab * kLTab + l * kLTab + (m < 0 ? -m : m)];
  return (m < 0 && (m & 1)) ? -v : v;  // Pbar_{l,-m} = (-1)^m Pbar_{l,m}
}

__global__ void tmatrix_kernel(TParams p, const double *__restrict__ xw, const double *__restrict__ tab,
                               double2 *__restrict__ T) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.nl * p.nl) return;
  int Lp = idx / p.nl, L = idx % p.nl;
  int lp = (int)floor(sqrt((double)Lp) + 1e-9), l = (int)floor(sqrt((double)L) + 1e-9);
  if ((lp + 1) * (lp + 1) <= Lp) ++lp;
  if ((l + 1) * (l + 1) <= L) ++l;
  int mp = Lp - lp * lp - lp, m = L - l * l - l, mpp = mp - m;
  const double *w = xw + p.nq;  // weights follow the nodes
  int n3 = 2 * p.lmax + 1;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int lo = lp > l ? lp - l : l - lp;
  for (int lpp = lo; lpp <= l + lp && l <= p.lns && lp <= p.lns; lpp += 2) {
    if ((mpp < 0 ? -mpp : mpp) > lpp) continue;
    double q = 0.0;
    for (int g = 0; g < p.nq; ++g) q += w[g] * pbar(tab, g, lp, mp) * pbar(tab, g, l, m) * pbar(tab, g, lpp, mpp);
    double G = 6.283185307179586477 * q;
    double c = (mpp >= 0) ? 1.0 : ((mpp & 1) ? -1.0 : 1.0);
    size_t ii = ((size_t)l * (p.lmax + 1) + lp) * n3 + lpp;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] += p.I[k][ii] * c * G;
  }
  if (L == Lp) {
    acc[0] += p.el[l];
    acc[1] += 0.5;
    acc[2] += 0.5;
    acc[3] += p.el[l] * p.un2[l];
  }
  // blocks: 0 = AA (rows A, cols A), 1 = AB (rows A, cols B), 2 = BA, 3 = BB
  int rb[4] = {0, 0, p.nl, p.nl}, cb[4] = {0, p.nl, 0, p.nl};
#pragma unroll
  for (int k = 0; k < 4; ++k) T[(size_t)(rb[k] + Lp) + (size_t)(cb[k] + L) * p.dpad] = make_double2(acc[k], 0.0);
}

cudaError_t launch_tmatrix(const Species &sp, double2 *d_T, double *scratch, cudaStream_t s) {
  // scratch layout: nodes[nq], weights[nq], I[4][n], el[lmax+1], un2[lmax+1], table[nq][kLTab^2]
  cudaError_t e;
  size_t bytesT = sizeof(double2) * (size_t)sp.dpad * sp.dpad;
  if ((e = cudaMemsetAsync(d_T, 0, bytesT, s)) != cudaSuccess) return e;
  if (!sp.T_override.empty()) {
    // Caller-supplied Hermitian T (2N_L x 2N_L, column-major) placed into the padded block.
    int n = 2 * sp.nl;
    return cudaMemcpy2DAsync(d_T, sizeof(double2) * sp.dpad, sp.T_override.data(), sizeof(double2) * n,
                             sizeof(double2) * n, n, cudaMemcpyHostToDevice, s);
  }
  int nq = 2 * sp.lmax + 2;
  size_t nI = (size_t)(sp.lmax + 1) * (sp.lmax + 1) * (2 * sp.lmax + 1);
  double *xw = scratch;
  double *dI = xw + 2 * nq;
  double *del = dI + 4 * nI;
  double *dun2 = del + (sp.lmax + 1);
  double *tab = dun2 + (sp.lmax + 1);
  for (int k = 0; k < 4; ++k)
    if ((e = cudaMemcpyAsync(dI + k * nI, sp.I[k].data(), sizeof(double) * nI, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return e;
  if ((e = cudaMemcpyAsync(del, sp.el.data(), sizeof(double) * (sp.lmax + 1), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(dun2, sp.un2.data(), sizeof(double) * (sp.lmax + 1), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  gauss_legendre_kernel<<<1, 64, 0, s>>>(nq, xw, xw + nq);
  legendre_table_kernel<<<1, 64, 0, s>>>(nq, xw, 2 * sp.lmax, tab);
  TParams p;
  p.lmax = sp.lmax;
  p.nl = sp.nlc;
  p.lns = sp.lns;
  p.dpad = sp.dpad;
  p.nq = nq;
  for (int k = 0; k < 4; ++k) p.I[k] = dI + k * nI;
  p.el = del;
  p.un2 = dun2;
  int nt = sp.nlc * sp.nlc;
  tmatrix_kernel<<<(nt + 127) / 128, 128, 0, s>>>(p, xw, tab, d_T);
  return cudaGetLastError();
}

// HPD test of a species' T (Sec. 4.6.2-4.6.3: the Cholesky factorization whose
// status routes an atom's H contribution): the n x n leading block of C (the
// contraction's rows of T, lower triangle read; leading dimension ld) is
// factored in place as T = C C^H, C lower triangular with a real positive
// diagonal, column by column (right-looking) by one CTA. *info = 0 when every
// pivot is positive and finite; otherwise k, the order of the first leading
// minor that is not positive definite (LAPACK potrf's status), and C keeps
// only its first k - 1 columns. The strict upper triangle is zeroed.
__global__ void __launch_bounds__(1024) cholesky_kernel(int n, int ld, double2 *C, int *info) {
  __shared__ double s_piv;
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = C[j + (size_t)j * ld].x;
      if (!(d > 0.0) || !isfinite(d))
        s_bad = j + 1;
      else
        s_piv = sqrt(d);
    }
    __syncthreads();
    if (s_bad) break;
    const double c = s_piv;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double2 v = C[i + (size_t)j * ld];
      C[i + (size_t)j * ld] = make_double2(v.x / c, v.y / c);
    }
    if (threadIdx.x == 0) C[j + (size_t)j * ld] = make_double2(c, 0.0);
    __syncthreads();
    // trailing lower triangle: C_rq -= C_rj conj(C_qj), j < q <= r < n
    const int m = n - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int q = j + 1 + e / m, r = j + 1 + e % m;
      if (r < q) continue;
      const double2 a = C[r + (size_t)j * ld], b = C[q + (size_t)j * ld];
      double2 t = C[r + (size_t)q * ld];
      t.x -= a.x * b.x + a.y * b.y;
      t.y -= a.y * b.x - a.x * b.y;
      C[r + (size_t)q * ld] = t;
    }
    __syncthreads();
  }
  const int bad = s_bad;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int r = e % n, q = e / n;
    if (r < q || (bad && q >= bad - 1)) C[r + (size_t)q * ld] = make_double2(0.0, 0.0);
  }
  if (threadIdx.x == 0) *info = bad;
}

cudaError_t launch_cholesky(const Species &sp, const double2 *d_T, double2 *d_C, int *d_info, cudaStream_t s) {
  const int n = 2 * sp.nlc;
  cudaError_t e = cudaMemsetAsync(d_C, 0, sizeof(double2) * (size_t)sp.dpad * sp.dpad, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy2DAsync(d_C, sizeof(double2) * sp.dpad, d_T, sizeof(double2) * sp.dpad, sizeof(double2) * n, n,
                        cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  cholesky_kernel<<<1, 1024, 0, s>>>(n, sp.dpad, d_C, d_info);
  return cudaGetLastError();
}

}  // namespace hsg
