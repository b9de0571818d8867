/*
 * hsref.c -- ORACLE (test infrastructure only): plain FP64 CPU implementation
 * of the muffin-tin H and S of the FLAPW method. Only tests/, the smoke check
 * and the benchmark's CPU-baseline leg load it. See hsref.h for conventions.
 *
 * Everything is written out from the definitions, in the paper's order:
 *   j_l, j_l'          -- spherical Bessel functions (App. A.1)
 *   Y_lm               -- explicit associated-Legendre sum (App. A.1)
 *   G_{L,L',L''}       -- Racah formula for 3j symbols (Eq. gaunt)
 *   T^{[..]}           -- Eq. t_matrices
 *   A, B               -- Eqs. def_a_tensor, def_b_tensor
 *   S, H               -- Eqs. def_overlap, def_hamilton, in the matrix form of
 *                         Sec. 4 (S = sum_a A^H A + B^H U B,
 *                         H = sum_a [A;B]^H T_a [A;B])
 * No blocking or reordering beyond evaluating x = T_a w first.
 */
#include "hsref.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI_L 3.141592653589793238462643383279502884L

int hsref_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Spherical Bessel functions (App. A.1: j_l from the Rayleigh expansion).  */
/* x == 0: exact limits. x < 1e-3: power series. x > lmax+1: upward         */
/* recurrence from j_0 = sin x / x, j_1 = sin x / x^2 - cos x / x (stable   */
/* for l < x). Otherwise Miller's downward recurrence normalised by j_0 or  */
/* j_1 (whichever is larger). Derivative: j_l' = (l/x) j_l - j_{l+1}.       */
/* ------------------------------------------------------------------------ */
int hsref_sbessel(int lmax, double x, double *j, double *dj) {
  if (lmax < 0 || lmax > 60) return 1;
  int L = lmax + 1;
  double jj[64];
  if (x == 0.0) {
    for (int l = 0; l <= lmax; ++l) {
      j[l] = (l == 0) ? 1.0 : 0.0;
      dj[l] = (l == 1) ? 1.0 / 3.0 : 0.0;
    }
    return 0;
  }
  if (fabs(x) < 1e-3) {
    double xl = 1.0, dfact = 1.0; /* x^l, (2l+1)!! */
    for (int l = 0; l <= L; ++l) {
      if (l > 0) {
        xl *= x;
        dfact *= (2.0 * l + 1.0);
      }
      double t = 1.0, s = 1.0;
      for (int k = 1; k < 12; ++k) {
        t *= (-0.5 * x * x) / (k * (2.0 * l + 2.0 * k + 1.0));
        s += t;
      }
      jj[l] = xl / dfact * s;
    }
  } else if (x > (double)L) {
    jj[0] = sin(x) / x;
    jj[1] = sin(x) / (x * x) - cos(x) / x;
    for (int l = 1; l < L; ++l) jj[l + 1] = (2.0 * l + 1.0) / x * jj[l] - jj[l - 1];
  } else {
    int start = L + 30 + (int)x;
    double f[256];
    f[start + 1] = 0.0;
    f[start] = 1e-30;
    for (int l = start; l >= 1; --l) {
      f[l - 1] = (2.0 * l + 1.0) / x * f[l] - f[l + 1];
      if (fabs(f[l - 1]) > 1e250)
        for (int q = l - 1; q <= start + 1; ++q) f[q] *= 1e-250;
    }
    double j0 = sin(x) / x, j1 = sin(x) / (x * x) - cos(x) / x;
    double sc = (fabs(j0) >= fabs(j1)) ? j0 / f[0] : j1 / f[1];
    for (int l = 0; l <= L; ++l) jj[l] = f[l] * sc;
  }
  for (int l = 0; l <= lmax; ++l) {
    j[l] = jj[l];
    dj[l] = (double)l / x * jj[l] - jj[l + 1];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Spherical harmonics by the explicit sum for the associated Legendre      */
/* function (Condon-Shortley phase included):                               */
/*   P_l^m(x) = (-1)^m (1-x^2)^{m/2} 2^{-l}                                 */
/*              sum_k (-1)^k (2l-2k)! / (k! (l-k)! (l-2k-m)!) x^{l-2k-m}    */
/*   Y_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m(cos th) e^{i m phi}     */
/* evaluated in long double.                                                */
/* ------------------------------------------------------------------------ */
static long double factl(int n) {
  long double f = 1.0L;
  for (int i = 2; i <= n; ++i) f *= (long double)i;
  return f;
}

int hsref_ylm(int lmax, const double *v, double *Y) {
  if (lmax < 0 || lmax > 30) return 1;
  long double x = v[0], y = v[1], z = v[2];
  long double r = sqrtl(x * x + y * y + z * z);
  long double ct, st, phi;
  if (r == 0.0L) {
    ct = 1.0L;
    st = 0.0L;
    phi = 0.0L;
  } else {
    ct = z / r;
    st = sqrtl(x * x + y * y) / r;
    phi = atan2l(y, x);
  }
  for (int l = 0; l <= lmax; ++l) {
    for (int m = 0; m <= l; ++m) {
      long double s = 0.0L;
      for (int k = 0; 2 * k <= l - m; ++k) {
        long double term = factl(2 * l - 2 * k) / (factl(k) * factl(l - k) * factl(l - 2 * k - m));
        long double p = 1.0L;
        for (int e = 0; e < l - 2 * k - m; ++e) p *= ct;
        s += ((k & 1) ? -term : term) * p;
      }
      long double sm = 1.0L;
      for (int e = 0; e < m; ++e) sm *= st;
      long double plm = ((m & 1) ? -1.0L : 1.0L) * sm * s / powl(2.0L, l);
      long double nrm = sqrtl((2.0L * l + 1.0L) / (4.0L * PI_L) * factl(l - m) / factl(l + m));
      long double re = nrm * plm * cosl(m * phi), im = nrm * plm * sinl(m * phi);
      int ip = l * l + l + m, in = l * l + l - m;
      Y[2 * ip] = (double)re;
      Y[2 * ip + 1] = (double)im;
      if (m > 0) {
        long double sg = (m & 1) ? -1.0L : 1.0L; /* Y_{l,-m} = (-1)^m conj(Y_lm) */
        Y[2 * in] = (double)(sg * re);
        Y[2 * in + 1] = (double)(-sg * im);
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Wigner 3j symbol, Racah formula.                                         */
/* ------------------------------------------------------------------------ */
double hsref_wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (abs(m1) > j1 || abs(m2) > j2 || abs(m3) > j3) return 0.0;
  long double tri = factl(j1 + j2 - j3) * factl(j1 - j2 + j3) * factl(-j1 + j2 + j3) / factl(j1 + j2 + j3 + 1);
  long double pre = sqrtl(tri * factl(j1 + m1) * factl(j1 - m1) * factl(j2 + m2) * factl(j2 - m2) *
                          factl(j3 + m3) * factl(j3 - m3));
  int kmin = 0;
  if (j2 - j3 - m1 > kmin) kmin = j2 - j3 - m1;
  if (j1 - j3 + m2 > kmin) kmin = j1 - j3 + m2;
  int kmax = j1 + j2 - j3;
  if (j1 - m1 < kmax) kmax = j1 - m1;
  if (j2 + m2 < kmax) kmax = j2 + m2;
  long double s = 0.0L;
  for (int k = kmin; k <= kmax; ++k) {
    long double d = factl(k) * factl(j3 - j2 + k + m1) * factl(j3 - j1 + k - m2) * factl(j1 + j2 - j3 - k) *
                    factl(j1 - k - m1) * factl(j2 - k + m2);
    s += ((k & 1) ? -1.0L : 1.0L) / d;
  }
  int ph = j1 - j2 - m3;
  long double sg = (((ph % 2) + 2) % 2) ? -1.0L : 1.0L;
  return (double)(sg * pre * s);
}

/* G_{L,L',L''} = int Y*_{l'm'} Y_{lm} Y_{l''m''} dOmega.
 * With Y*_{l'm'} = (-1)^{m'} Y_{l',-m'} and the three-Y integral
 * sqrt((2l+1)(2l''+1)(2l'+1)/(4 pi)) (l l'' l'; 0 0 0) (l l'' l'; m m'' -m'). */
double hsref_gaunt(int l, int m, int lp, int mp, int lpp, int mpp) {
  if (m + mpp != mp) return 0.0;
  if (((l + lp + lpp) & 1) || lpp < abs(l - lp) || lpp > l + lp) return 0.0;
  if (abs(m) > l || abs(mp) > lp || abs(mpp) > lpp) return 0.0;
  double w0 = hsref_wigner3j(l, lpp, lp, 0, 0, 0);
  if (w0 == 0.0) return 0.0;
  double w = hsref_wigner3j(l, lpp, lp, m, mpp, -mp);
  double pre = sqrt((2.0 * l + 1.0) * (2.0 * lpp + 1.0) * (2.0 * lp + 1.0) / (4.0 * M_PI));
  double sg = (mp & 1) ? -1.0 : 1.0;
  return sg * pre * w0 * w;
}

/* ------------------------------------------------------------------------ */
/* T matrices, Eq. t_matrices:                                              */
/*  T^{[xy]}_{L',L} = sum_{l''} I^{(x,y)}_{l,l',l''} c_{m'-m}               */
/*                    G_{L,L',(l'',m'-m)} + spherical diagonal              */
/* ------------------------------------------------------------------------ */
static double cpot(int mpp) { return (mpp >= 0) ? 1.0 : ((mpp & 1) ? -1.0 : 1.0); }

int hsref_T(const hsref_type *ty, double *T) {
  int lmax = ty->lmax, nl = (lmax + 1) * (lmax + 1), n = 2 * nl, n3 = 2 * lmax + 1;
  if (ty->T_override) {
    memcpy(T, ty->T_override, sizeof(double) * 2 * (size_t)n * n);
    return 0;
  }
  memset(T, 0, sizeof(double) * 2 * (size_t)n * n);
  const double *Ixy[2][2] = {{ty->I_uu, ty->I_uud}, {ty->I_udu, ty->I_udud}}; /* [x][y] */
  /* Sec. 3.1 (Fig. Tmat_structure): the non-spherical (Gaunt) part is dense for
   * l, l' <= l_nonsph only; the spherical diagonal below runs to lmax */
  const int lns = ty->lmax_nonsph < lmax ? ty->lmax_nonsph : lmax;
  for (int lp = 0; lp <= lmax; ++lp)
    for (int mp = -lp; mp <= lp; ++mp)
      for (int l = 0; l <= lmax; ++l)
        for (int m = -l; m <= l; ++m) {
          int Lp = lp * lp + lp + mp, L = l * l + l + m, mpp = mp - m;
          double acc[2][2] = {{0, 0}, {0, 0}};
          for (int lpp = abs(l - lp); lpp <= l + lp && l <= lns && lp <= lns; ++lpp) {
            if ((l + lp + lpp) & 1) continue;
            if (abs(mpp) > lpp) continue;
            double g = hsref_gaunt(l, m, lp, mp, lpp, mpp) * cpot(mpp);
            for (int x = 0; x < 2; ++x)
              for (int y = 0; y < 2; ++y)
                acc[x][y] += Ixy[x][y][((size_t)l * (lmax + 1) + lp) * n3 + lpp] * g;
          }
          if (Lp == L) {
            acc[0][0] += ty->e_l[l];
            acc[1][1] += ty->e_l[l] * ty->udot_norm2[l];
            acc[0][1] += 0.5;
            acc[1][0] += 0.5;
          }
          for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) {
              size_t row = (size_t)x * nl + Lp, col = (size_t)y * nl + L;
              T[2 * (row + col * n)] = acc[x][y];
            }
        }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* HPD test of a species' T (Sec. 4.6.2-4.6.3, Listings alg:H_AA_HPD and    */
/* alg:H_AA_dynamic): the Cholesky factorisation T = C C^H (C lower         */
/* triangular, real positive diagonal) attempted column by column, reading  */
/* the lower triangle of T only. The status follows LAPACK potrf, whose     */
/* error code the paper branches on: 0 when every pivot is positive (T is   */
/* HPD and C its factor); k > 0 when the k-th pivot is not positive or not  */
/* finite, i.e. the leading minor of order k is not positive definite.     */
/* ------------------------------------------------------------------------ */
int hsref_cholesky(int n, const double *T, long long ld, double *C) {
  const double complex *A = (const double complex *)T;
  double complex *L = (double complex *)calloc((size_t)n * n + 1, sizeof(double complex));
  if (!L) return -1;
  int info = 0;
  for (int j = 0; j < n && !info; ++j) {
    double d = creal(A[j + (size_t)j * ld]);
    for (int k = 0; k < j; ++k) {
      double complex c = L[j + (size_t)k * n];
      d -= creal(c) * creal(c) + cimag(c) * cimag(c);
    }
    if (!(d > 0.0) || !isfinite(d)) {
      info = j + 1;
      break;
    }
    const double cjj = sqrt(d);
    L[j + (size_t)j * n] = cjj;
    for (int i = j + 1; i < n; ++i) {
      double complex v = A[i + (size_t)j * ld];
      for (int k = 0; k < j; ++k) v -= L[i + (size_t)k * n] * conj(L[j + (size_t)k * n]);
      L[i + (size_t)j * n] = v / cjj;
    }
  }
  if (C) memcpy(C, L, sizeof(double complex) * (size_t)n * n);
  free(L);
  return info;
}

/* ------------------------------------------------------------------------ */
/* Matching coefficients, Eqs. def_a_tensor / def_b_tensor:                 */
/*  A_{L,a,t} = 4 pi/(W_l sqrt(Omega)) i^l e^{i K_t.x_a} Y*_L(R_a K^_t)     */
/*              [u_dot K j_l'(R K) - u_dot' j_l(R K)]                        */
/*  B_{L,a,t} = same prefactor [-u K j_l'(R K) + u' j_l(R K)]               */
/*  W_l = u_dot u' - u u_dot' (or the caller's W_l when one is given).      */
/* ------------------------------------------------------------------------ */
static void coef_column(const hsref_system *sys, int atom, const double *K, double complex *w) {
  const hsref_type *ty = &sys->types[sys->type_of_atom[atom]];
  int lmax = ty->lmax, nl = (lmax + 1) * (lmax + 1);
  const double *x = sys->pos + 3 * atom, *R = sys->rot + 9 * atom;
  double kn = sqrt(K[0] * K[0] + K[1] * K[1] + K[2] * K[2]);
  double kh[3] = {0.0, 0.0, 1.0};
  if (kn > 0.0) {
    kh[0] = K[0] / kn;
    kh[1] = K[1] / kn;
    kh[2] = K[2] / kn;
  }
  double v[3];
  for (int i = 0; i < 3; ++i) v[i] = R[3 * i] * kh[0] + R[3 * i + 1] * kh[1] + R[3 * i + 2] * kh[2];
  double Y[2 * 121 * 4];
  hsref_ylm(lmax, v, Y);
  double jl[64], djl[64];
  hsref_sbessel(lmax, kn * ty->rmt, jl, djl);
  double kx = K[0] * x[0] + K[1] * x[1] + K[2] * x[2];
  double complex phase = cos(kx) + I * sin(kx);
  for (int l = 0; l <= lmax; ++l) {
    double W = ty->wronskian ? ty->wronskian[l] : ty->udot[l] * ty->du[l] - ty->u[l] * ty->dudot[l];
    double fa = ty->udot[l] * kn * djl[l] - ty->dudot[l] * jl[l];
    double fb = -ty->u[l] * kn * djl[l] + ty->du[l] * jl[l];
    double complex il = (l % 4 == 0) ? 1.0 : (l % 4 == 1) ? I : (l % 4 == 2) ? -1.0 : -I;
    double complex pre = 4.0 * M_PI / (W * sqrt(sys->omega)) * il * phase;
    for (int m = -l; m <= l; ++m) {
      int L = l * l + l + m;
      double complex yc = Y[2 * L] - I * Y[2 * L + 1];
      w[L] = pre * yc * fa;
      w[nl + L] = pre * yc * fb;
    }
  }
}

int hsref_coefficients(const hsref_system *sys, int atom, int n_g, const double *kvec, double *W) {
  if (atom < 0 || atom >= sys->n_atoms || n_g < 0) return 1;
  int nl2 = 2 * (sys->types[sys->type_of_atom[atom]].lmax + 1) * (sys->types[sys->type_of_atom[atom]].lmax + 1);
#pragma omp parallel for schedule(static)
  for (int t = 0; t < n_g; ++t) coef_column(sys, atom, kvec + 3 * t, (double complex *)W + (size_t)t * nl2);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Depth layout: for every atom a, rows [A_a ; B_a] (2 N_La rows), stacked  */
/* over atoms in order. w holds W (the coefficients), x = T_a w per atom,   */
/* y = diag(1, ||u_dot_l||^2) w per atom.                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int depth;
  int *off;        /* [n_atoms] row offset of atom a   */
  double **T;      /* [n_types] T matrices              */
} layout_t;

static int make_layout(const hsref_system *sys, layout_t *lay) {
  lay->off = (int *)malloc(sizeof(int) * (sys->n_atoms + 1));
  lay->T = (double **)calloc(sys->n_types, sizeof(double *));
  if (!lay->off || !lay->T) return 1;
  int d = 0;
  for (int a = 0; a < sys->n_atoms; ++a) {
    int lm = sys->types[sys->type_of_atom[a]].lmax;
    lay->off[a] = d;
    d += 2 * (lm + 1) * (lm + 1);
  }
  lay->off[sys->n_atoms] = d;
  lay->depth = d;
  for (int tt = 0; tt < sys->n_types; ++tt) {
    int n = 2 * (sys->types[tt].lmax + 1) * (sys->types[tt].lmax + 1);
    lay->T[tt] = (double *)malloc(sizeof(double) * 2 * (size_t)n * n);
    if (!lay->T[tt]) return 1;
    hsref_T(&sys->types[tt], lay->T[tt]);
  }
  return 0;
}

static void free_layout(const hsref_system *sys, layout_t *lay) {
  if (lay->T)
    for (int tt = 0; tt < sys->n_types; ++tt) free(lay->T[tt]);
  free(lay->T);
  free(lay->off);
}

/* Column t of W, X = T W and Y = U W over the whole depth. */
static void wxy_column(const hsref_system *sys, const layout_t *lay, const double *K, double complex *w,
                       double complex *x, double complex *y) {
  for (int a = 0; a < sys->n_atoms; ++a) {
    int ti = sys->type_of_atom[a];
    const hsref_type *ty = &sys->types[ti];
    int nl = (ty->lmax + 1) * (ty->lmax + 1), n = 2 * nl;
    double complex *wa = w + lay->off[a], *xa = x + lay->off[a], *ya = y + lay->off[a];
    coef_column(sys, a, K, wa);
    const double complex *T = (const double complex *)lay->T[ti];
    for (int r = 0; r < n; ++r) {
      double complex s = 0.0;
      for (int c = 0; c < n; ++c) s += T[r + (size_t)c * n] * wa[c];
      xa[r] = s;
    }
    for (int l = 0; l <= ty->lmax; ++l)
      for (int m = -l; m <= l; ++m) {
        int L = l * l + l + m;
        ya[L] = wa[L];
        ya[nl + L] = ty->udot_norm2[l] * wa[nl + L];
      }
  }
}

/* sum_k conj(p_k) q_k, plain or compensated (Ogita-Rump-Oishi Dot2 on the
 * real and imaginary sums separately). */
static inline void two_prod(double a, double b, double *p, double *e) {
  *p = a * b;
  *e = fma(a, b, -*p);
}
static inline void two_sum(double a, double b, double *s, double *e) {
  *s = a + b;
  double z = *s - a;
  *e = (a - (*s - z)) + (b - z);
}

static double complex cdot(const double complex *p, const double complex *q, int n, int compensated) {
  if (!compensated) {
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < n; ++k) {
      double pr = creal(p[k]), pi = cimag(p[k]), qr = creal(q[k]), qi = cimag(q[k]);
      sr += pr * qr + pi * qi;
      si += pr * qi - pi * qr;
    }
    return sr + I * si;
  }
  double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0, h, r, q2;
  for (int k = 0; k < n; ++k) {
    double pr = creal(p[k]), pi = cimag(p[k]), qr = creal(q[k]), qi = cimag(q[k]);
    two_prod(pr, qr, &h, &r); two_sum(sr, h, &sr, &q2); cr += q2 + r;
    two_prod(pi, qi, &h, &r); two_sum(sr, h, &sr, &q2); cr += q2 + r;
    two_prod(pr, qi, &h, &r); two_sum(si, h, &si, &q2); ci += q2 + r;
    two_prod(-pi, qr, &h, &r); two_sum(si, h, &si, &q2); ci += q2 + r;
  }
  return (sr + cr) + I * (si + ci);
}

int hsref_build_HS(const hsref_system *sys, int n_g, const double *kvec, double *H, double *S, long long ld,
                   int full, int compensated) {
  if (n_g < 0 || ld < n_g) return 1;
  if (n_g == 0) return 0;
  layout_t lay = {0};
  if (make_layout(sys, &lay)) {
    free_layout(sys, &lay);
    return 2;
  }
  int D = lay.depth;
  double complex *w = (double complex *)malloc(sizeof(double complex) * (size_t)D * n_g);
  double complex *x = (double complex *)malloc(sizeof(double complex) * (size_t)D * n_g);
  double complex *y = (double complex *)malloc(sizeof(double complex) * (size_t)D * n_g);
  if (!w || !x || !y) {
    free(w); free(x); free(y);
    free_layout(sys, &lay);
    return 2;
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (int t = 0; t < n_g; ++t)
    wxy_column(sys, &lay, kvec + 3 * t, w + (size_t)t * D, x + (size_t)t * D, y + (size_t)t * D);
  double complex *Hc = (double complex *)H, *Sc = (double complex *)S;
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < n_g; ++t) {
    int tp_end = full ? n_g - 1 : t;
    for (int tp = 0; tp <= tp_end; ++tp) {
      Hc[tp + (size_t)t * ld] = cdot(w + (size_t)tp * D, x + (size_t)t * D, D, compensated);
      Sc[tp + (size_t)t * ld] = cdot(w + (size_t)tp * D, y + (size_t)t * D, D, compensated);
    }
  }
  free(w); free(x); free(y);
  free_layout(sys, &lay);
  return 0;
}

int hsref_HS_entries(const hsref_system *sys, int n_g, const double *kvec, int n_pairs, const int *rows,
                     const int *cols, double *H, double *S, int compensated) {
  if (n_pairs < 0) return 1;
  for (int p = 0; p < n_pairs; ++p)
    if (rows[p] < 0 || rows[p] >= n_g || cols[p] < 0 || cols[p] >= n_g) return 1;
  layout_t lay = {0};
  if (make_layout(sys, &lay)) {
    free_layout(sys, &lay);
    return 2;
  }
  int D = lay.depth;
  /* distinct columns that are needed */
  int *slot = (int *)malloc(sizeof(int) * (size_t)(n_g > 0 ? n_g : 1));
  int *cols_u = (int *)malloc(sizeof(int) * (size_t)(2 * n_pairs + 1));
  for (int t = 0; t < n_g; ++t) slot[t] = -1;
  int nu = 0;
  for (int p = 0; p < n_pairs; ++p) {
    if (slot[rows[p]] < 0) { slot[rows[p]] = nu; cols_u[nu++] = rows[p]; }
    if (slot[cols[p]] < 0) { slot[cols[p]] = nu; cols_u[nu++] = cols[p]; }
  }
  double complex *w = (double complex *)malloc(sizeof(double complex) * (size_t)D * (nu + 1));
  double complex *x = (double complex *)malloc(sizeof(double complex) * (size_t)D * (nu + 1));
  double complex *y = (double complex *)malloc(sizeof(double complex) * (size_t)D * (nu + 1));
#pragma omp parallel for schedule(dynamic, 1)
  for (int u = 0; u < nu; ++u)
    wxy_column(sys, &lay, kvec + 3 * cols_u[u], w + (size_t)u * D, x + (size_t)u * D, y + (size_t)u * D);
  double complex *Hc = (double complex *)H, *Sc = (double complex *)S;
#pragma omp parallel for schedule(static)
  for (int p = 0; p < n_pairs; ++p) {
    int a = slot[rows[p]], b = slot[cols[p]];
    Hc[p] = cdot(w + (size_t)a * D, x + (size_t)b * D, D, compensated);
    Sc[p] = cdot(w + (size_t)a * D, y + (size_t)b * D, D, compensated);
  }
  free(w); free(x); free(y); free(slot); free(cols_u);
  free_layout(sys, &lay);
  return 0;
}

static double cnorm(const double complex *p, int n) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) s += creal(p[k]) * creal(p[k]) + cimag(p[k]) * cimag(p[k]);
  return sqrt(s);
}

int hsref_HS_columns(const hsref_system *sys, int n_g, const double *kvec, int n_cols, const int *cols,
                     double *H, double *S, double *wnorm, double *xnorm, double *ynorm) {
  if (n_g < 0 || n_cols < 0) return 1;
  for (int c = 0; c < n_cols; ++c)
    if (cols[c] < 0 || cols[c] >= n_g) return 1;
  layout_t lay = {0};
  if (make_layout(sys, &lay)) {
    free_layout(sys, &lay);
    return 2;
  }
  int D = lay.depth;
  /* W for every plane wave (the rows), X = T W and Y = U W for the columns */
  double complex *w = (double complex *)malloc(sizeof(double complex) * (size_t)D * (n_g + 1));
  double complex *wc = (double complex *)malloc(sizeof(double complex) * (size_t)D * (n_cols + 1));
  double complex *x = (double complex *)malloc(sizeof(double complex) * (size_t)D * (n_cols + 1));
  double complex *y = (double complex *)malloc(sizeof(double complex) * (size_t)D * (n_cols + 1));
  if (!w || !wc || !x || !y) {
    free(w); free(wc); free(x); free(y);
    free_layout(sys, &lay);
    return 2;
  }
#pragma omp parallel for schedule(dynamic, 8)
  for (int t = 0; t < n_g; ++t)
    for (int a = 0; a < sys->n_atoms; ++a) coef_column(sys, a, kvec + 3 * t, w + (size_t)t * D + lay.off[a]);
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < n_cols; ++c)
    wxy_column(sys, &lay, kvec + 3 * cols[c], wc + (size_t)c * D, x + (size_t)c * D, y + (size_t)c * D);
  double complex *Hc = (double complex *)H, *Sc = (double complex *)S;
#pragma omp parallel for schedule(static)
  for (long long e = 0; e < (long long)n_g * n_cols; ++e) {
    int tp = (int)(e % n_g), c = (int)(e / n_g);
    Hc[e] = cdot(w + (size_t)tp * D, x + (size_t)c * D, D, 0);
    Sc[e] = cdot(w + (size_t)tp * D, y + (size_t)c * D, D, 0);
  }
  for (int t = 0; t < n_g && wnorm; ++t) wnorm[t] = cnorm(w + (size_t)t * D, D);
  for (int c = 0; c < n_cols; ++c) {
    if (xnorm) xnorm[c] = cnorm(x + (size_t)c * D, D);
    if (ynorm) ynorm[c] = cnorm(y + (size_t)c * D, D);
  }
  free(w); free(wc); free(x); free(y);
  free_layout(sys, &lay);
  return 0;
}

int hsref_HS_brute(const hsref_system *sys, int n_g, const double *kvec, double *H, double *S, long long ld) {
  if (n_g < 0 || ld < n_g) return 1;
  layout_t lay = {0};
  if (make_layout(sys, &lay)) {
    free_layout(sys, &lay);
    return 2;
  }
  int D = lay.depth;
  double complex *w = (double complex *)malloc(sizeof(double complex) * (size_t)D * (n_g + 1));
#pragma omp parallel for schedule(static)
  for (int t = 0; t < n_g; ++t)
    for (int a = 0; a < sys->n_atoms; ++a) coef_column(sys, a, kvec + 3 * t, w + (size_t)t * D + lay.off[a]);
  double complex *Hc = (double complex *)H, *Sc = (double complex *)S;
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < n_g; ++t)
    for (int tp = 0; tp < n_g; ++tp) {
      double complex h = 0.0, s = 0.0;
      for (int a = 0; a < sys->n_atoms; ++a) {
        int ti = sys->type_of_atom[a];
        const hsref_type *ty = &sys->types[ti];
        int nl = (ty->lmax + 1) * (ty->lmax + 1), n = 2 * nl;
        const double complex *T = (const double complex *)lay.T[ti];
        const double complex *wp = w + (size_t)tp * D + lay.off[a], *wt = w + (size_t)t * D + lay.off[a];
        for (int r = 0; r < n; ++r)
          for (int c = 0; c < n; ++c) h += conj(wp[r]) * T[r + (size_t)c * n] * wt[c];
        for (int l = 0; l <= ty->lmax; ++l)
          for (int m = -l; m <= l; ++m) {
            int L = l * l + l + m;
            s += conj(wp[L]) * wt[L] + ty->udot_norm2[l] * conj(wp[nl + L]) * wt[nl + L];
          }
      }
      Hc[tp + (size_t)t * ld] = h;
      Sc[tp + (size_t)t * ld] = s;
    }
  free(w);
  free_layout(sys, &lay);
  return 0;
}
