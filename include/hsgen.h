/*
 * hsgen.h -- C ABI of the GB300 (sm_103a) muffin-tin H/S generator.
 *
 * For one k-point (or a batch of k-points) the library computes the
 * muffin-tin parts of the FLAPW Hamiltonian H and overlap S of Di Napoli,
 * Peise, Hrywniak, Bientinesi, "High-performance generation of the
 * Hamiltonian and Overlap matrices in FLAPW methods":
 *
 *   A_{L,a,t}, B_{L,a,t}   matching coefficients          (App. A.1,
 *                          Eqs. def_a_tensor, def_b_tensor)
 *   T_a = [[T^AA, T^AB], [T^BA, T^BB]]                     (App. A.2,
 *                          Eqs. gaunt, nonsph_integrals, t_matrices)
 *   S = sum_a A_a^H A_a + B_a^H U_a B_a                    (Sec. 4, Eq. S;
 *                          Eq. def_overlap)
 *   H = sum_a [A_a;B_a]^H T_a [A_a;B_a]                    (Sec. 4, Eq. H;
 *                          Eq. def_hamilton)
 *
 * Every step runs in CUDA kernels on the device given to hsgen_create.
 * There is no CPU fallback: without a usable sm_103a device every entry
 * point that computes returns HSGEN_ECUDA.
 *
 * Conventions (readings of the paper where it is silent or inconsistent):
 *  - Y_lm orthonormal with the Condon-Shortley phase (Y_{l,-m} = (-1)^m Y_lm^*).
 *  - R_a is a proper rotation acting on column vectors: Y_lm(R_a K^_t).
 *  - K_t = 0: only l = 0 survives (j_l(0) = delta_l0, |K| j_l'(0) = 0).
 *  - The potential is real (Eq. pot_harm with coefficient 1 for m'' >= 0 and
 *    (-1)^{m''} for m'' < 0), so T is Hermitian. The spherical diagonal adds
 *    E_l to AA, E_l ||u_dot_l||^2 to BB and 1/2 to both AB and BA (the
 *    Hermitian part of the paper's "1" and "0").
 *  - U = diag(||u_dot_l||^2) over the B rows (Eq. def_overlap).
 *  - Matrix entry (t', t): t' is the conjugated (row) side, t the column.
 *  - Complex numbers are two consecutive doubles (re, im); matrices are
 *    column-major with a leading dimension (Sec. 4.1 storage format).
 *
 * Errors: every function returns a status and never aborts, throws across
 * the ABI or traps the device; hsgen_last_error() gives the message.
 * Threading: one context must not be used by two host threads at once, and
 * calls on one context are ordered (they share device workspaces): issue
 * them on one stream, or synchronise between streams.
 * Buffers on another GPU than the context's are rejected (HSGEN_EINVAL).
 * Environment (tuning only; results move at the rounding level at most;
 * read by hsgen_create, and hsgen_autotune picks the first five per shape):
 *  HSGEN_KSEG_BLOCKS   the split form's depth segment, in 64-deep blocks;
 *  HSGEN_TILE_BAND     the split form's tile band, in 64-column blocks;
 *  HSGEN_CRT_ORDER     0 or 1, the order of the moduli kernel's work units;
 *  HSGEN_L2_HINT       0 or 8, the L2 priority of its operand loads;
 *  HSGEN_CRT_GEOMETRY  0 or 1, its pipeline stage geometry;
 *  HSGEN_CRT_RECON     1 (default): the moduli form's reconstruction of H
 *                      and S in a kernel of its own, 0: inside the
 *                      contraction's last launch;
 *  HSGEN_WS_BYTES      the split form's workspace budget, which sets the
 *                      passes over the atoms when opt.atom_chunk is 0
 *                      (default 176e9);
 *  HSGEN_BATCH_BYTES   the operand-memory budget of one batched group;
 *  HSGEN_REDUCE_BLOCK  the block rows of hsgen_reduce_generalized
 *                      (default 128).
 * Fault injection (tests): HSGEN_FAIL_ALLOC=1 makes every growth of a
 * library workspace fail as an out-of-memory cudaMalloc would (the call
 * returns HSGEN_ENOMEM; the context stays usable once the variable is unset).
 */
#ifndef HSGEN_H
#define HSGEN_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hsgen_ctx hsgen_ctx;

typedef enum {
  HSGEN_OK = 0,
  HSGEN_EINVAL = 1,   /* invalid argument (NULL, size, range, layout)          */
  HSGEN_ENOMEM = 2,   /* device or host allocation failed                      */
  HSGEN_ECUDA = 3,    /* CUDA runtime/driver error, or no usable sm_103a device */
  HSGEN_ETIMEOUT = 4, /* a bounded device wait gave up; results are invalid    */
  HSGEN_ENOTSUP = 5,  /* option combination not supported                      */
  HSGEN_ENUMERIC = 6  /* |W_l| too small, NaN/Inf input, non-Hermitian T,     */
                      /* S not positive definite (hsgen_reduce_generalized)    */
} hsgen_status;

enum { HSGEN_FP64 = 0, HSGEN_SPLIT = 1 };
enum { HSGEN_S_CONTRACTION = 0, HSGEN_S_LEGENDRE = 1 };
/* How the split form cuts an FP64 product into BF16 tensor-core products (no
 * counterpart in the paper, which is all FP64):
 *  HSGEN_SCHEME_SLICES: s slices per operand, s(s+1)/2 products (Ozaki
 *    scheme I);
 *  HSGEN_SCHEME_MODULI: every operand column rounded to integers of 2-norm
 *    at most 2^B, one product per modulus, exact integer result by the
 *    Chinese remainder theorem (Ozaki scheme II), 10..14 moduli;
 *  HSGEN_SCHEME_AUTO: moduli when a count of at most 14 meets target_rel_err
 *    (and no slice count is forced), otherwise slices. */
enum { HSGEN_SCHEME_AUTO = 0, HSGEN_SCHEME_SLICES = 1, HSGEN_SCHEME_MODULI = 2 };
/* How an atom's contribution to H is formed (Sec. 4.6.2-4.6.3, Listings
 * alg:H_AA_HPD and alg:H_AA_dynamic):
 *  HSGEN_H_TW: X_a = T W_a and H += W_a^H X_a for every atom;
 *  HSGEN_H_HPD: hsgen_set_atoms factors each species' T (the rows the
 *    contraction uses) as T = C C^H; a species whose factorization succeeds
 *    (LAPACK potrf status 0, hsgen_T_factor) takes Y_a = C^H W_a and
 *    H += Y_a^H Y_a, the others X = T W as above. The paper tests T^[AA] only,
 *    because its H_AA is a separate product; here T's four blocks stay one
 *    matrix, so the test covers all of it. Passes over the atoms are split
 *    where the route changes (order atoms by species to keep them few). */
enum { HSGEN_H_TW = 0, HSGEN_H_HPD = 1 };

typedef struct {
  int precision;            /* HSGEN_FP64 (default) or HSGEN_SPLIT                  */
  double target_rel_err;    /* split form: error the slice count is chosen for      */
                            /* (default 1e-12, relative Frobenius)                  */
  int slices;               /* split form: slices per operand, 0 = from the target  */
  int uplo;                 /* 'U' (default): i <= j written; 'L': i >= j written   */
  int fill_full;            /* 1: also write the other triangle (Hermitian mirror)  */
  int atom_chunk;           /* atoms per pass over the depth, 0 = the library's     */
                            /* choice: as few passes as fit HSGEN_WS_BYTES (split   */
                            /* form; of two, the last as large as fits), else all   */
  long long wait_timeout_ns; /* limit of every device-side wait (default 2e9)       */
  int s_form;               /* HSGEN_S_CONTRACTION (default): S = sum_a A^H A +    */
                            /* B^H U B in the chosen precision; HSGEN_S_LEGENDRE:  */
                            /* the m-summed form of Sec. 3.1 (Eq. overlap_no_m) in */
                            /* FP64, used when all K_t lie on one lattice k + G,   */
                            /* otherwise the contraction (see hsgen_stats.s_form)  */
  int scheme;               /* split form: HSGEN_SCHEME_* (default AUTO)            */
  int moduli;               /* split form, moduli scheme: 10..14, 0 = from the      */
                            /* target and the depth                                 */
  int h_form;               /* HSGEN_H_TW (default) or HSGEN_H_HPD                  */
} hsgen_options;

/* Radial data of one atom species (App. A.1 and A.2). All arrays are host
 * pointers, read during hsgen_set_atoms and copied; the caller keeps
 * ownership. Index of I: ((l * (lmax+1)) + l') * (2 lmax + 1) + l'', with
 * I^{(x,y)}_{l,l',l''} = int x_{l'} v_{l''} y_l r^2 dr (Eq. nonsph_integrals). */
typedef struct {
  int lmax;                         /* 0..10                                   */
  double rmt;                       /* muffin-tin radius r_MT (> 0)            */
  const double *u, *du;             /* [lmax+1] u_l(r_MT), u_l'(r_MT)          */
  const double *udot, *dudot;       /* [lmax+1] u_dot_l(r_MT), u_dot_l'(r_MT)  */
  const double *wronskian;          /* [lmax+1] W_l, or NULL: computed as      */
                                    /* u_dot u' - u u_dot' (App. A.1)          */
  const double *udot_norm2;         /* [lmax+1] ||u_dot_l||^2 (> 0)            */
  const double *e_l;                /* [lmax+1] E_l                            */
  const double *I_uu, *I_uud;       /* I^{(u,u)}, I^{(u,u_dot)}                */
  const double *I_udu, *I_udud;     /* I^{(u_dot,u)}, I^{(u_dot,u_dot)}        */
  const double *T_override;         /* NULL, or (2N_L)^2 complex, column-major */
                                    /* Hermitian T used instead of Eq.         */
                                    /* t_matrices (rows/cols: A then B)        */
  int lmax_nonsph;                  /* l_nonsph (Sec. 3.1, Fig. Tmat_structure):*/
                                    /* the Gaunt part of T only for l, l' <=   */
                                    /* it, the spherical diagonal to lmax;     */
                                    /* < 0 or >= lmax: lmax. With s_form       */
                                    /* HSGEN_S_LEGENDRE the contraction then   */
                                    /* covers l <= l_nonsph only and H's       */
                                    /* spherical tail is added in the Legendre */
                                    /* form (every K_t must be on one lattice  */
                                    /* k + G: HSGEN_ENOTSUP otherwise)         */
} hsgen_type;

typedef struct {
  double ms_coefficients;  /* a1: radial factors + A/B coefficient kernel      */
  double ms_tapply;        /* a3: X = T W                                       */
  double ms_slice;         /* a5: split-form slicing (0 for FP64)               */
  double ms_contract;      /* a4/a5: H and S contraction                        */
  double ms_total;         /* whole last call, device time                      */
  double flops_algorithmic;/* algorithmic flops of the last call (all k-points) */
  int precision;           /* form used by the last call                        */
  int slices;              /* slices per operand used (split form)              */
  int n_kpoints;           /* k-points in the last call                         */
  long long workspace_bytes; /* device workspace currently held                 */
  long long kernel_launches; /* kernels the last call launched                   */
  int s_form;              /* how the last call built S (HSGEN_S_*)             */
  double ms_s;             /* S in the Legendre form (0 otherwise)              */
  int kseg_blocks;         /* split form: depth segment (64-deep blocks) in use */
  int tile_band;           /* split form: column blocks per tile band in use    */
  double ms_upload;        /* host inputs/outputs: K_t upload and zeroing of    */
                           /* the device staging of H, S, before the build      */
  double ms_download;      /* host outputs: copy-out time after the build ends  */
                           /* (the part not overlapped with the last tiles)     */
  int scheme;              /* split form of the last pass: HSGEN_SCHEME_SLICES  */
                           /* or HSGEN_SCHEME_MODULI                            */
  int moduli;              /* moduli used (moduli scheme)                       */
  int bits;                /* moduli scheme: B, the operand columns' integer    */
                           /* 2-norm bound 2^B                                  */
  int products;            /* BF16 products per FP64 product of the contraction */
  int atom_chunks;         /* passes over the atoms (a6) of the last build      */
  double tuned_rel_err;    /* hsgen_autotune: relative Frobenius error of the   */
                           /* chosen form against a 7-slice build (0: not       */
                           /* measured)                                         */
  int stage_geometry;      /* moduli scheme: pipeline stages of its kernel, 0:  */
                           /* three of two 64-deep blocks, 1: two of three      */
  int unit_order;          /* moduli scheme: order of its (tile, modulus) work  */
                           /* units, 0: every modulus of a tile before the next */
                           /* tile, 1: every tile of a modulus before the next  */
                           /* modulus                                           */
  int l2_hint;             /* moduli scheme: L2 priority of its operand loads,  */
                           /* 0: normal, 8: the column operand (re-read by the  */
                           /* next waves of a band) evict-last                  */
  int hpd_species;         /* species on the HPD route (opt.h_form HSGEN_H_HPD) */
} hsgen_stats;

/* Fills *opt with the defaults listed above. */
hsgen_status hsgen_default_options(hsgen_options *opt);

/* Creates a context on CUDA device `cuda_device` (must be sm_103). opt may be
 * NULL (defaults). *out receives the context, NULL on failure. */
hsgen_status hsgen_create(hsgen_ctx **out, int cuda_device, const hsgen_options *opt);

/* Sets the crystal (Sec. 2.2, App. A.1): lattice rows a1,a2,a3 in bohr
 * (lattice[9], row-major), cell volume omega (> 0), the species and the atoms
 * (type_of_atom[n_atoms] in [0,n_types), pos[n_atoms][3] Cartesian,
 * rot[n_atoms][9] row-major proper rotations). Host pointers, deep-copied.
 * Assembles the T matrices on the device (a2). Synchronous. */
hsgen_status hsgen_set_atoms(hsgen_ctx *ctx, const double *lattice, double omega, int n_types,
                             const hsgen_type *types, int n_atoms, const int *type_of_atom,
                             const double *pos, const double *rot);

/* Builds H and S for one k-point: kvec[n_g][3] are the Cartesian vectors
 * K_t = k + G_t (host or device pointer). H and S are complex128 column-major
 * n_g x n_g with leading dimension ld >= n_g: device pointers (written on
 * `cuda_stream`, a cudaStream_t or NULL for the default stream; only the
 * triangle named by opt.uplo is written unless opt.fill_full; with a device
 * kvec the call returns without waiting for the device, in both forms) or
 * host pointers (computed in a library-owned device buffer and copied back in
 * full, ld x n_g entries: the other triangle is zero unless opt.fill_full;
 * the call returns after the copy; in the split form the copies of finished
 * column bands run on a library-owned stream while the last tiles are
 * computed). Diagonal imaginary parts are set to 0.
 * Bounded waits (split form): every device-side wait of the tensor-core
 * kernels gives up after opt.wait_timeout_ns and records it in a status word
 * instead of trapping. A call that returns before its work is done cannot see
 * that word; it is read, and HSGEN_ETIMEOUT returned (the results of the call
 * that launched the expired wait are then invalid), by hsgen_synchronize, by
 * hsgen_get_stats, by this call itself when it waits (host inputs or
 * outputs), and by the next build or reduction on the context once the
 * earlier work has finished. */
hsgen_status hsgen_build_HS(hsgen_ctx *ctx, int n_g, const double *kvec, void *H, void *S, long long ld,
                            void *cuda_stream);

/* Within one k-point, the part of hsgen_build_HS that one process of an
 * nprow x npcol process grid owns in the 2-D block-cyclic layout of a
 * distributed dense eigensolver (the paper's outlook, Sec. 5: distributed
 * dense linear algebra): block (I, J) of block x block entries belongs to
 * process (I mod nprow, J mod npcol). Writes exactly the entries of opt.uplo's
 * triangle inside this process's (myrow, mycol) blocks of the full-size
 * device buffers H and S (ld >= n_g) and leaves every other entry as it was;
 * those entries are bit for bit the ones hsgen_build_HS writes, so the union
 * over the grid is the whole build. Only the contraction's tiles are split
 * (each process forms the coefficients of all plane waves, a few percent of
 * the build). block: a multiple of 256. Device pointers only; not with
 * opt.fill_full or S in the Legendre form (HSGEN_ENOTSUP). Asynchronous like
 * hsgen_build_HS. */
hsgen_status hsgen_build_HS_blocks(hsgen_ctx *ctx, int n_g, const double *kvec, void *H, void *S, long long ld,
                                   int block, int nprow, int npcol, int myrow, int mycol, void *cuda_stream);

/* Builds H and S for n_k k-points in one go (one H, S per k-point, Sec. 2.3):
 * n_g[k], kvec[k] (host pointers to [n_g[k]][3]), H[k], S[k] device
 * pointers with leading dimension ld[k]. The whole kernel sequence is
 * captured in a CUDA graph and replayed while sizes and pointers stay the
 * same. The contraction tiles of a group of k-points (up to HSGEN_BATCH_BYTES
 * of operand planes, default 96 GiB for slices and 12 GiB of residue planes
 * and stores for moduli) run in one persistent launch over a grouped tile
 * queue.
 * The FP64 form loops over hsgen_build_HS. */
hsgen_status hsgen_build_HS_batched(hsgen_ctx *ctx, int n_k, const int *n_g, const double *const *kvec,
                                    void *const *H, void *const *S, const long long *ld, void *cuda_stream);

/* Inspection of single steps (same kernels as hsgen_build_HS):
 * W = [A_a; B_a] stacked over atoms (a1) into W (device, complex, column t at
 * W + t*ldw, rows at the offsets hsgen_depth_layout reports, padding rows 0). */
hsgen_status hsgen_coefficients(hsgen_ctx *ctx, int n_g, const double *kvec, void *W, long long ldw,
                                void *cuda_stream);
/* Same result as hsgen_coefficients, for callers that must not have the
 * library allocate device memory (no counterpart in the paper). Code running
 * under another framework's memory manager may find the GPU's memory already
 * reserved, and latency-critical loops cannot accept the device
 * synchronisation a cudaMalloc can cause; hsgen_coefficients may call
 * cudaMalloc to grow its workspace, this function never does (nor cudaFree,
 * nor any allocating routine). Its scratch (the radial factors) is a fixed
 * 16 MiB array in device memory that belongs to the loaded library and is
 * held on every GPU that uses it until the process exits (under the CUDA
 * runtime's default lazy loading the 16 MiB are taken on a device at the
 * first call of this function there, not when the library is loaded); it
 * limits n_types * n_g to 95325, larger requests return HSGEN_EINVAL without
 * launching anything. kvec and W must be device pointers on the context's
 * GPU (HSGEN_EINVAL otherwise); the call is asynchronous on `cuda_stream`.
 * The first call on a device looks up the array's device address (once per
 * device, again after that device's context was replaced, e.g. by
 * cudaDeviceReset); make that first call before capturing the stream into a
 * graph. All calls, from every
 * context, share the one array: calls whose kernels overlap on the GPU (on
 * different streams, or from different host threads) race and must be
 * ordered by the caller. Nothing needs clearing between calls: every entry
 * read is written earlier in the same call. */
hsgen_status hsgen_coefficients_noalloc(hsgen_ctx *ctx, int n_g, const double *kvec, void *W, long long ldw,
                                        void *cuda_stream);
/* T of species `type` (a2) copied into T (host, (2N_L)^2 complex, column-major),
 * with the l_nonsph structure of Fig. Tmat_structure. */
hsgen_status hsgen_T_matrix(hsgen_ctx *ctx, int type, double *T);
/* Cholesky factor of species `type`'s T (Sec. 4.6.2-4.6.3; set by
 * hsgen_set_atoms when opt.h_form is HSGEN_H_HPD, HSGEN_EINVAL otherwise):
 * *info receives the status of the factorization (0: T is Hermitian positive
 * definite; k > 0: the leading minor of order k is not, as LAPACK potrf
 * reports it) and C (host, (2N_L')^2 complex, column-major, or NULL) the
 * lower factor C with T = C C^H (for k > 0, its first k - 1 columns, zeros
 * elsewhere). N_L' = N_L, or (l_nonsph + 1)^2 with S in the Legendre form
 * (the rows the contraction uses). */
hsgen_status hsgen_T_factor(hsgen_ctx *ctx, int type, double *C, int *info);
/* Row offsets of the atoms in the depth of W (offsets[n_atoms+1], host); the
 * block of atom a is offsets[a] .. offsets[a] + 2 N_La (A rows, then B rows),
 * followed by zero rows up to offsets[a+1]. */
hsgen_status hsgen_depth_layout(hsgen_ctx *ctx, int *offsets, int capacity);

/* Autotuner of the split form (no counterpart in the paper), on this
 * k-point. (1) The form: with device outputs and neither a scheme nor a
 * count forced in the options, it builds H and S once with 7 slices (~2e-15)
 * as the reference, then measures the relative Frobenius error of candidate
 * forms over the whole triangle: for each scheme (moduli 10..14, slices
 * 5..7) the smallest count within half of opt.target_rel_err, searched from
 * the a-priori choice; of the two, the faster build on this GPU is kept
 * (hsgen_stats tuned_rel_err reports its error). (2) The schedule: times builds for
 * depth-segment lengths {64, 96, 128, 192, 256} blocks of 64 (moduli scheme:
 * {64, 128, 256} in modulus-major unit order and 32 in tile-major order;
 * tile band 16), then tile bands {8, 32} with the best segment, then, for
 * the moduli scheme, the other L2 priority of its operand loads and its
 * kernel's other stage geometry (hsgen_stats unit_order, l2_hint,
 * stage_geometry). The choices stay in the
 * context for later builds (batched ones use the schedule) and H and S are
 * left built with them. Same arguments as hsgen_build_HS; synchronous; about
 * ten to fifteen builds long. The FP64 form has nothing to tune: it builds
 * once and returns HSGEN_OK. */
hsgen_status hsgen_autotune(hsgen_ctx *ctx, int n_g, const double *kvec, void *H, void *S, long long ld,
                            void *cuda_stream);

/* Hand-off to the generalized eigensolver (Sec. 2.3, Eq. matrix_kohnsham:
 * H c = eps S c; no counterpart in the paper's H/S generation itself). H, S:
 * device pointers, complex128 column-major n x n with leading dimension
 * ld >= n (ld < 2^31), Hermitian with their opt.uplo triangle given (as
 * hsgen_build_HS writes them; the other triangle is not read); S must be
 * positive definite (the full problem's S: the muffin-tin part this library
 * builds plus the interstitial part the caller adds). In place and in FP64:
 * S's opt.uplo triangle becomes the Cholesky factor (U with S = U^H U for
 * 'U', L with S = L L^H for 'L'; the other triangle is left as it was) and H
 * becomes H~ = U^-H H U^-1 (= L^-1 H L^-H), written in full and exactly
 * Hermitian, so that H~ y = eps y and c = U^-1 y (= L^-H y). Everything
 * runs in the library's own kernels, blocked by HSGEN_REDUCE_BLOCK rows
 * (default 128): the diagonal blocks' Cholesky factors and inverses in FP64
 * tile kernels; the panel and trailing updates and the two triangular solves
 * as products with those inverses, 7-slice BF16 products on the tensor cores
 * with opt.precision HSGEN_SPLIT (FP64-level accuracy) or FP64 DMMA products
 * otherwise; the lower layout works on a conjugate-transposed copy. Runs on
 * `cuda_stream` and returns when it is done. HSGEN_ENUMERIC when S is not
 * positive definite: the leading minor that failed is named in
 * hsgen_last_error, and H and S are then overwritten with partial results
 * (the call still runs to its end, so both must be rebuilt);
 * HSGEN_EINVAL for host pointers, aliasing or bad sizes. */
hsgen_status hsgen_reduce_generalized(hsgen_ctx *ctx, int n, void *H, void *S, long long ld, void *cuda_stream);

/* Statistics of the last call (waits for its device work). Returns
 * HSGEN_ETIMEOUT, with the stats filled in all the same, when a bounded wait
 * of an earlier split-form call expired (see hsgen_build_HS). */
hsgen_status hsgen_get_stats(hsgen_ctx *ctx, hsgen_stats *stats);
/* Waits for `cuda_stream` and reports the bounded-wait status of the split
 * form's work queued on it: HSGEN_ETIMEOUT when a wait expired since the last
 * report (no counterpart in the paper). */
hsgen_status hsgen_synchronize(hsgen_ctx *ctx, void *cuda_stream);
const char *hsgen_last_error(const hsgen_ctx *ctx);
/* Releases the context and its device memory. NULL-safe. */
void hsgen_destroy(hsgen_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HSGEN_H */
