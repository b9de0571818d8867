/*
 * hsref.h -- ORACLE (test infrastructure only).
 *
 * Plain, slow, FP64 CPU implementation of the muffin-tin Hamiltonian H and
 * overlap S of the FLAPW method (Di Napoli, Peise, Hrywniak, Bientinesi,
 * "High-performance generation of the Hamiltonian and Overlap matrices in
 * FLAPW methods"). It exists to check the CUDA library and is used only by
 * the tests, by the smoke check and by the benchmark's CPU-baseline leg. It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Conventions (readings of the paper where it is silent or inconsistent):
 *  - Y_lm orthonormal with the Condon-Shortley phase, Y_{l,-m} = (-1)^m Y_lm^*.
 *  - R_a is a proper 3x3 rotation (row-major) acting on column vectors.
 *  - K = 0: the direction is taken as z; only l = 0 survives.
 *  - The potential is real: V = sum_{l''} v_{l''} sum_{m''} c_{m''} Y_{l''m''}
 *    with c_{m''} = 1 (m'' >= 0) and (-1)^{m''} (m'' < 0), so T is Hermitian.
 *  - Spherical diagonal of T: AA += E_l, BB += E_l ||u_dot_l||^2,
 *    AB += 1/2, BA += 1/2 (the Hermitian part of the paper's 1 / 0).
 *  - Matrix index: row t' is the conjugated side, column t the plain side.
 *  - All complex arrays are interleaved (re, im) doubles.
 */
#ifndef HSREF_ORACLE_H
#define HSREF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int lmax;
  double rmt;
  const double *u, *du, *udot, *dudot; /* [lmax+1] values at rmt           */
  const double *udot_norm2;            /* [lmax+1] ||u_dot_l||^2            */
  const double *e_l;                   /* [lmax+1]                          */
  const double *I_uu, *I_uud, *I_udu, *I_udud; /* [lmax+1][lmax+1][2lmax+1] */
  const double *T_override; /* NULL, or (2N_L)^2 complex, column-major      */
  int lmax_nonsph;          /* l_nonsph (Sec. 3.1, Fig. Tmat_structure): the */
                            /* Gaunt sum enters T only for l, l' <= l_nonsph */
                            /* (l_nonsph >= lmax: everywhere)                */
  const double *wronskian;  /* NULL, or [lmax+1] W_l given by the caller and */
                            /* used in App. A.1's prefactor as it is          */
} hsref_type;

typedef struct {
  double omega;
  int n_types;
  const hsref_type *types;
  int n_atoms;
  const int *type_of_atom;
  const double *pos; /* [n_atoms][3] Cartesian       */
  const double *rot; /* [n_atoms][9] row-major       */
} hsref_system;

/* Spherical Bessel j_l(x) and j_l'(x), l = 0..lmax. */
int hsref_sbessel(int lmax, double x, double *j, double *dj);
/* Y_lm(v/|v|) for all l <= lmax, m = -l..l at index l*l + l + m. */
int hsref_ylm(int lmax, const double *v, double *Y);
/* Wigner 3j symbol by the Racah formula. */
double hsref_wigner3j(int j1, int j2, int j3, int m1, int m2, int m3);
/* Gaunt coefficient G_{L,L',L''} = int Y*_{L'} Y_L Y_{L''} dOmega (Eq. gaunt). */
double hsref_gaunt(int l, int m, int lp, int mp, int lpp, int mpp);
/* T = [[T^AA, T^AB], [T^BA, T^BB]] (2N_L x 2N_L, column-major) (Eq. t_matrices). */
int hsref_T(const hsref_type *ty, double *T);
/* Cholesky factorisation T = C C^H of an n x n Hermitian matrix (lower
 * triangle of T read, leading dimension ld; C: n x n, column-major, lower,
 * or NULL). Returns 0 (T is HPD) or k > 0, the order of the first leading
 * minor that is not positive definite (the status of LAPACK potrf); -1 when
 * out of memory. Sec. 4.6.2-4.6.3: the HPD test that routes a species. */
int hsref_cholesky(int n, const double *T, long long ld, double *C);
/* W_a = [A_a; B_a]: out[t][2N_L] (column t contiguous) (Eqs. def_a_tensor/def_b_tensor). */
int hsref_coefficients(const hsref_system *sys, int atom, int n_g, const double *kvec, double *W);
/* Full H and S (column-major, leading dimension ld). full=0: upper triangle
 * only (i <= j), lower part left untouched; full=1: every entry computed.
 * compensated=1 uses compensated (Dot2) summation for every entry. */
int hsref_build_HS(const hsref_system *sys, int n_g, const double *kvec, double *H, double *S,
                   long long ld, int full, int compensated);
/* Entries H[rows[p], cols[p]] and S[...] only. */
int hsref_HS_entries(const hsref_system *sys, int n_g, const double *kvec, int n_pairs,
                     const int *rows, const int *cols, double *H, double *S, int compensated);
/* Whole columns: H[:, cols[c]] and S[:, cols[c]] for every row 0..n_g-1
 * (H, S: n_g x n_cols, column-major, leading dimension n_g). Optional
 * (NULL to skip): wnorm[n_g] = ||w_t|| of every row's coefficient column,
 * xnorm[n_cols] = ||T w|| and ynorm[n_cols] = ||U w|| of the chosen columns
 * (the Cauchy-Schwarz scales of an entry's dot product). */
int hsref_HS_columns(const hsref_system *sys, int n_g, const double *kvec, int n_cols, const int *cols,
                     double *H, double *S, double *wnorm, double *xnorm, double *ynorm);
/* The quadruple sum of Eq. def_hamilton / def_overlap with no intermediate
 * product (tiny inputs only). */
int hsref_HS_brute(const hsref_system *sys, int n_g, const double *kvec, double *H, double *S,
                   long long ld);
/* Number of OpenMP threads the oracle uses. */
int hsref_threads(void);

#ifdef __cplusplus
}
#endif
#endif
