// coef.cu -- matching coefficients A, B (App. A.1, Eqs. def_a_tensor and
// def_b_tensor) on the device, in FP64.
//
//   A_{(l,m),a,t} = 4 pi / (W_l sqrt(Omega)) i^l e^{i K_t.x_a} Y*_lm(R_a K^_t)
//                   [u_dot K j_l'(r_MT K) - u_dot' j_l(r_MT K)]
//   B_{(l,m),a,t} = same prefactor [-u K j_l'(r_MT K) + u' j_l(r_MT K)]
//
// Step 1 (radial kernel, one thread per species and plane wave): j_l and j_l'
// of x = |K_t| r_MT, by the continued fraction for j_{L+1}/j_L followed by
// downward recurrence normalised with j_0 = sin x / x (or j_1), upward
// recurrence when x > l_max + 1, and a short power series for tiny x. The
// radial factors f_A, f_B times 4 pi/(W_l sqrt(Omega)) are stored per l.
//
// Step 2 (coefficient kernel, one thread per atom and plane wave): the
// orthonormal associated Legendre functions by the standard three-term
// recurrence in l for every m (Condon-Shortley phase included), e^{i m phi}
// by complex multiplication, the structure phase e^{i K.x_a}, and the writes
// of A and B into column t of W = [A_a; B_a] stacked over atoms (the layout
// of Fig. memorylayoutA: column t contiguous over the depth).
#include <cmath>

#include "internal.cuh"

namespace hsg {

// a_lm = sqrt((4l^2-1)/(l^2-m^2)) and b_lm = a_lm / a_{l-1,m}, l <= 2*kLmaxMax.
__constant__ double c_alm[kLTab * kLTab];
__constant__ double c_blm[kLTab * kLTab];
__constant__ double c_pmm[kLTab];   // sqrt((2m+1)/(2m)), m >= 1
__constant__ double c_pm1[kLTab];   // sqrt(2m+3)

cudaError_t upload_tables() {
  double a[kLTab * kLTab] = {0}, b[kLTab * kLTab] = {0}, pmm[kLTab] = {0}, pm1[kLTab] = {0};
  for (int l = 0; l < kLTab; ++l)
    for (int m = 0; m + 2 <= l; ++m) {
      a[l * kLTab + m] = std::sqrt((4.0 * l * l - 1.0) / (double(l) * l - double(m) * m));
      double am1 = (l - 1 > m) ? std::sqrt((4.0 * (l - 1) * (l - 1) - 1.0) /
                                           (double(l - 1) * (l - 1) - double(m) * m))
                               : std::sqrt(2.0 * m + 3.0);  // a_{m+1,m} = sqrt(2m+3)
      b[l * kLTab + m] = a[l * kLTab + m] / am1;
    }
  for (int m = 1; m < kLTab; ++m) pmm[m] = std::sqrt((2.0 * m + 1.0) / (2.0 * m));
  for (int m = 0; m < kLTab; ++m) pm1[m] = std::sqrt(2.0 * m + 3.0);
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(c_alm, a, sizeof(a))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_blm, b, sizeof(b))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_pmm, pmm, sizeof(pmm))) != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_pm1, pm1, sizeof(pm1));
}

// ---------------------------------------------------------------------------
// Spherical Bessel functions j_0..j_{n} (n = lmax + 1) of x > 0.
// ---------------------------------------------------------------------------
__device__ void sph_bessel_upto(int n, double x, double *j) {
  if (x < 1e-6) {
    // j_l(x) = x^l / (2l+1)!! (1 - x^2 / (2(2l+3)) + ...)
    double p = 1.0, df = 1.0;
    for (int l = 0; l <= n; ++l) {
      if (l > 0) { p *= x; df *= (2.0 * l + 1.0); }
      j[l] = p / df * (1.0 - x * x / (2.0 * (2.0 * l + 3.0)));
    }
    return;
  }
  double s, c;
  sincos(x, &s, &c);
  double j0 = s / x;
  if (x > (double)n) {
    j[0] = j0;
    if (n >= 1) j[1] = s / (x * x) - c / x;
    for (int l = 1; l < n; ++l) j[l + 1] = (2.0 * l + 1.0) / x * j[l] - j[l - 1];
    return;
  }
  // rho_l = j_l / j_{l-1} = x / (2l+1 - x rho_{l+1}), evaluated from far above.
  int top = n + 1 + 40 + (int)x;
  double rho = 0.0;
  for (int l = top; l >= n + 1; --l) rho = x / (2.0 * l + 1.0 - x * rho);
  // j_{n+1} / j_n = rho; recurse down with j_n = 1.
  double jp1 = rho, jc = 1.0;
  j[n] = 1.0;
  for (int l = n; l >= 1; --l) {
    double jm1 = (2.0 * l + 1.0) / x * jc - jp1;
    jp1 = jc;
    jc = jm1;
    j[l - 1] = jc;
  }
  double j1 = s / (x * x) - c / x;
  double scale = (fabs(j0) >= fabs(j1)) ? j0 / j[0] : j1 / j[1];
  for (int l = 0; l <= n; ++l) j[l] *= scale;
}

__global__ void radial_kernel(int n_g, const double *__restrict__ kvec, int n_types,
                              const RadialParams *__restrict__ rp, double2 *__restrict__ F) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int ty = blockIdx.y;
  if (t >= n_g || ty >= n_types) return;
  const RadialParams &p = rp[ty];
  double kx = kvec[3 * t], ky = kvec[3 * t + 1], kz = kvec[3 * t + 2];
  double kn = sqrt(kx * kx + ky * ky + kz * kz);
  double x = kn * p.rmt;
  double j[kLmaxMax + 2], dj[kLmaxMax + 1];
  int n = p.lmax + 1;
  if (x == 0.0) {
    for (int l = 0; l <= n; ++l) j[l] = (l == 0) ? 1.0 : 0.0;
    for (int l = 0; l < n; ++l) dj[l] = 0.0;  // |K| j_l'(0) = 0
  } else {
    sph_bessel_upto(n, x, j);
    for (int l = 0; l < n; ++l) dj[l] = kn * ((double)l / x * j[l] - j[l + 1]);  // |K| j_l'(x)
  }
  double2 *out = F + ((size_t)ty * n_g + t) * kRadStride;
  for (int l = 0; l < n; ++l) {
    double fa = p.udot[l] * dj[l] - p.dudot[l] * j[l];
    double fb = -p.u[l] * dj[l] + p.du[l] * j[l];
    out[l] = make_double2(p.pre[l] * fa, p.pre[l] * fb);
  }
}

cudaError_t launch_radial(int n_g, const double *kvec, int n_types, const RadialParams *d_rp, double2 *F,
                          cudaStream_t s) {
  if (n_g <= 0) return cudaSuccess;
  dim3 grid((n_g + 127) / 128, n_types);
  radial_kernel<<<grid, 128, 0, s>>>(n_g, kvec, n_types, d_rp, F);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Coefficient kernel: one thread per (plane wave t, atom of the species).
// ---------------------------------------------------------------------------
template <int LMAX>
__global__ void __launch_bounds__(128) coef_kernel(int n_g, const double *__restrict__ kvec,
                                                   const double2 *__restrict__ F, const int *__restrict__ atoms,
                                                   const double *__restrict__ pos, const double *__restrict__ rot,
                                                   const int *__restrict__ off, int row_base, int dpad,
                                                   double2 *__restrict__ W, long long ldw) {
  constexpr int NL = (LMAX + 1) * (LMAX + 1);
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_g) return;
  int a = atoms[blockIdx.y];
  double kx = kvec[3 * t], ky = kvec[3 * t + 1], kz = kvec[3 * t + 2];
  double kn = sqrt(kx * kx + ky * ky + kz * kz);
  double hx = 0.0, hy = 0.0, hz = 1.0;
  if (kn > 0.0) {
    double r = 1.0 / kn;
    hx = kx * r; hy = ky * r; hz = kz * r;
  }
  const double *R = rot + 9 * a;
  double vx = R[0] * hx + R[1] * hy + R[2] * hz;
  double vy = R[3] * hx + R[4] * hy + R[5] * hz;
  double vz = R[6] * hx + R[7] * hy + R[8] * hz;
  double vn = sqrt(vx * vx + vy * vy + vz * vz);
  double ct = vz / vn;
  double rho = sqrt(vx * vx + vy * vy);
  double st = rho / vn;
  double cp = 1.0, sp = 0.0;
  if (rho > 0.0) { cp = vx / rho; sp = vy / rho; }
  // structure phase e^{i K.x_a}
  const double *xa = pos + 3 * a;
  double ps, pc;
  sincos(kx * xa[0] + ky * xa[1] + kz * xa[2], &ps, &pc);

  double2 *out = W + (size_t)t * ldw + (off[a] - row_base);
  const double2 *Ft = F + (size_t)t * kRadStride;

  double p1[LMAX + 1], p2[LMAX + 1];   // Pbar_{l-1,m}, Pbar_{l-2,m}
  double er[LMAX + 1], ei[LMAX + 1];   // e^{i m phi}
  er[0] = 1.0; ei[0] = 0.0;
#pragma unroll
  for (int m = 1; m <= LMAX; ++m) {
    er[m] = er[m - 1] * cp - ei[m - 1] * sp;
    ei[m] = er[m - 1] * sp + ei[m - 1] * cp;
  }
#pragma unroll
  for (int l = 0; l <= LMAX; ++l) {
    double pl[LMAX + 1];
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      double v;
      if (m == l) {
        v = (l == 0) ? 0.28209479177387814347 : -c_pmm[l] * st * p1[l - 1];
      } else if (m == l - 1) {
        v = c_pm1[m] * ct * p1[m];
      } else {
        v = c_alm[l * kLTab + m] * ct * p1[m] - c_blm[l * kLTab + m] * p2[m];
      }
      pl[m] = v;
    }
    // c = pre_l f * i^l * e^{i K.x}
    double2 f = Ft[l];
    double qr, qi;  // i^l e^{iKx}
    switch (l & 3) {
      case 0: qr = pc; qi = ps; break;
      case 1: qr = -ps; qi = pc; break;
      case 2: qr = -pc; qi = -ps; break;
      default: qr = ps; qi = -pc; break;
    }
    double aR = f.x * qr, aI = f.x * qi, bR = f.y * qr, bI = f.y * qi;
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      double gAr = aR * pl[m], gAi = aI * pl[m], gBr = bR * pl[m], gBi = bI * pl[m];
      // conj(Y_lm) = Pbar (er - i ei); conj(Y_{l,-m}) = (-1)^m Pbar (er + i ei)
      int L = l * l + l + m;
      out[L] = make_double2(gAr * er[m] + gAi * ei[m], gAi * er[m] - gAr * ei[m]);
      out[NL + L] = make_double2(gBr * er[m] + gBi * ei[m], gBi * er[m] - gBr * ei[m]);
      if (m > 0) {
        double sg = (m & 1) ? -1.0 : 1.0;
        int Ln = l * l + l - m;
        out[Ln] = make_double2(sg * (gAr * er[m] - gAi * ei[m]), sg * (gAi * er[m] + gAr * ei[m]));
        out[NL + Ln] = make_double2(sg * (gBr * er[m] - gBi * ei[m]), sg * (gBi * er[m] + gBr * ei[m]));
      }
    }
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      p2[m] = p1[m];
      p1[m] = pl[m];
    }
  }
  for (int r = 2 * NL; r < dpad; ++r) out[r] = make_double2(0.0, 0.0);
}

cudaError_t launch_coefficients(int lmax, int n_g, const double *kvec, const double2 *F_type, const int *atoms,
                                int n_atoms, const double *pos, const double *rot, const int *off, int row_base,
                                int dpad, double2 *W, long long ldw, cudaStream_t s) {
  if (n_g <= 0 || n_atoms <= 0) return cudaSuccess;
  dim3 grid((n_g + 127) / 128, n_atoms);
#define HSG_COEF_CASE(L)                                                                                   \
  case L:                                                                                                  \
    coef_kernel<L><<<grid, 128, 0, s>>>(n_g, kvec, F_type, atoms, pos, rot, off, row_base, dpad, W, ldw); \
    break;
  switch (lmax) {
    HSG_COEF_CASE(0) HSG_COEF_CASE(1) HSG_COEF_CASE(2) HSG_COEF_CASE(3) HSG_COEF_CASE(4) HSG_COEF_CASE(5)
    HSG_COEF_CASE(6) HSG_COEF_CASE(7) HSG_COEF_CASE(8) HSG_COEF_CASE(9) HSG_COEF_CASE(10)
    default: return cudaErrorInvalidValue;
  }
#undef HSG_COEF_CASE
  return cudaGetLastError();
}

}  // namespace hsg
