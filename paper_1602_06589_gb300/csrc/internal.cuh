// internal.cuh -- shared declarations of the hsgen CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "hsgen.h"

namespace hsg {

constexpr int kLmaxMax = 10;                    // largest l_max per species
constexpr int kLTab = 2 * kLmaxMax + 1;         // Legendre table extent (l'' <= 2 l_max)
constexpr int kRadStride = kLmaxMax + 1;        // F[type][t][l] stride

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Species data kept by the context.
struct Species {
  int lmax = 0, nl = 0;            // l_max, N_L = (lmax+1)^2
  int lns = 0;                     // l_nonsph: the Gaunt part of T is dense for l, l' <= lns
  // The contraction's view of the species: l_max lc and N_L nlc = (lc+1)^2 of
  // the coefficient rows it multiplies (lc = lns when S is in the Legendre form,
  // which then also adds H's spherical tail lns < l <= lmax; lc = lmax otherwise),
  // its depth block dpad (2 nlc rows; padded to 8 in the FP64 form) and T (d_T).
  int lc = 0, nlc = 0, dpad = 0;
  double rmt = 0.0;
  std::vector<double> u, du, udot, dudot, wr, un2, el;
  std::vector<double> I[4];        // uu, uud, udu, udud
  std::vector<double> T_override;  // empty or (2N_L)^2 complex (interleaved), col-major
  double *d_T = nullptr;           // contraction block of T: dpad x dpad complex col-major (ld = dpad)
  // split form: BF16 slices of T (planes re, im per slice) and column exponents.
  // T is stored once per depth shift d = 0, 2, .., 62 (32 copies), each
  // t_kspan deep with T's rows at [d, d + dpad) and zeros elsewhere, so that
  // X = T W of an atom whose depth offset is d mod 64 reads whole 64-deep
  // blocks of W.
  void *d_Tsl = nullptr;
  int *d_Texp = nullptr;
  int t_kspan = 0;
  int t_real = 0;                  // imaginary part of T identically zero
  // HPD route (option h_form HSGEN_H_HPD, Sec. 4.6.2-4.6.3): the Cholesky
  // factor C of the contraction block of T (T = C C^H, lower, dpad x dpad) and
  // the status of its factorization (0: HPD); a routed species multiplies its
  // atoms' W by C^H instead of T, and its H contribution is (C^H W)^H (C^H W).
  double *d_C = nullptr;
  int hpd_info = -1;
  bool routed = false;
  // the matrix P of the T-apply step X = P^H W (T is Hermitian: P = T)
  const double *apply_matrix() const { return routed ? d_C : d_T; }
};

// Per-species radial parameters read by the radial-factor kernel.
struct RadialParams {
  int lmax;
  double rmt;
  double u[kLmaxMax + 1], du[kLmaxMax + 1], udot[kLmaxMax + 1], dudot[kLmaxMax + 1];
  double pre[kLmaxMax + 1];  // 4 pi / (W_l sqrt(Omega))
};

struct Workspace {
  void *ptr = nullptr;
  size_t bytes = 0;
};

// Split form of one pass: slices (Ozaki scheme I: s(s+1)/2 BF16 products per
// FP64 product) or moduli (Ozaki scheme II: one BF16 product per modulus on
// b-bit integer operands). `slices` is also the slice count of T and of
// X = T W in either form.
enum { kSchemeSlices = 1, kSchemeModuli = 2 };

// 2-D block-cyclic ownership of H and S blocks (block x block entries) over
// an nprow x npcol process grid: this process (myrow, mycol) owns block
// (I, J) when I % nprow == myrow and J % npcol == mycol. block = 0: all.
struct BlockOwner {
  int block = 0, nprow = 1, npcol = 1, myrow = 0, mycol = 0;
  __host__ __device__ bool owns(long long row, long long col) const {
    return block == 0 || ((row / block) % nprow == myrow && (col / block) % npcol == mycol);
  }
  bool operator==(const BlockOwner &o) const {
    return block == o.block && nprow == o.nprow && npcol == o.npcol && myrow == o.myrow && mycol == o.mycol;
  }
};
struct SplitPlan {
  int scheme = kSchemeSlices;
  int slices = 0, nmod = 0, bits = 0;
};

}  // namespace hsg

struct hsgen_ctx {
  int device = 0;
  hsgen_options opt{};
  std::string err;
  bool have_system = false;
  double lattice[9]{};
  double omega = 0.0;
  std::vector<hsg::Species> types;
  std::vector<int> toa;
  std::vector<double> pos, rot;
  std::vector<int> off;             // depth offset of each atom (n_atoms + 1)
  int depth = 0;                    // total padded depth
  std::vector<std::vector<int>> atoms_of_type;
  // device copies of the system
  int *d_toa = nullptr, *d_off = nullptr, *d_atoms_by_type = nullptr;
  std::vector<int> atoms_by_type_start;  // start of each species' list in d_atoms_by_type
  double *d_pos = nullptr, *d_rot = nullptr;
  double *d_urow = nullptr;         // per depth row: 1 (A), ||u_dot_l||^2 (B), 0 (padding)
  hsg::RadialParams *d_radial = nullptr;
  // workspaces
  hsg::Workspace ws_main;           // W, X, radial factors, kvec copy, split slices
  hsg::Workspace ws_out;            // device H/S staging when the caller passes host pointers
  hsg::Workspace ws_leg;            // S in the Legendre form: coordinates, structure factors, tables
  hsg::Workspace ws_ref;            // autotuner: the reference H and S it measures errors against
  hsg::Workspace ws_red;            // generalized-eigenproblem reduction: block inverses, products, status
  int *h_info = nullptr;            // pinned host copy of the factorization status
  int split_slices = 0;             // slices the species' T were cut into
  int *d_status = nullptr;          // device status word of the split kernels
  int *h_status = nullptr;          // pinned host copy
  cudaEvent_t status_ev = nullptr;  // marks the arrival of the latest copy in h_status
  bool status_pending = false;      // a copy of the status word is queued and not yet read
  void *d_tiles = nullptr;          // split form: tile list of one triangle (int2 row/column blocks)
  int tiles_n = -1, tiles_uplo = 0;
  long long tiles_count = 0;
  int kseg_blocks = 128;            // split form: k-blocks (64 deep) per H/S launch
  int tile_band = 16;               // split form: column blocks per band of the tile order
  int tiles_band = 0;               // band the cached tile list was built with
  int tiles_bn = 0;                 // tile width (complex columns) of that list
  hsg::SplitPlan last_plan;         // split form of the last pass
  hsg::BlockOwner owner;            // blocks of H and S the current build writes
  hsg::BlockOwner tiles_owner;      // ownership the cached tile list was built for
  int auto_chunk = 0;               // atoms per pass chosen by the library (0: all), see atom_chunk
  int last_chunk = 0;               // two library-chosen passes: atoms of the (larger) last one, 0: equal passes
  int crt_geom = 0;                 // moduli kernel's stage geometry (0: 3 x 2 k-blocks, 1: 2 x 3)
  int crt_order = 1;                // moduli kernel's unit order (0: tile-major, 1: modulus-major)
  int l2_hint = 8;                  // moduli kernel's L2 priorities of its A and B loads (8: B evict-last)
  int crt_recon_apart = 1;          // moduli form: reconstruction in a kernel of its own (0: in the contraction)
  std::vector<int2> tiles_host;     // host copy of that list (column bands of the overlapped copies)
  cudaStream_t copy_stream = nullptr;  // host outputs: copies of finished column bands
  cudaEvent_t copy_ev = nullptr;       // orders each copy after the launch that finished its bands
  hsg::Workspace ws_batch;          // batched k-points: per-k slices, tables, shared scratch
  cudaGraphExec_t batch_exec = nullptr;  // captured kernel sequence of the last batch
  cudaStream_t capture_stream = nullptr; // private stream the batch sequence is captured on
  std::vector<long long> batch_key;      // what that graph was captured for
  // timing
  cudaEvent_t ev[10]{};
  bool events_ready = false;
  // per pass over an atom chunk: start, coefficients done, X = T W done,
  // slicing done, contraction done (5 events per chunk, created on demand)
  std::vector<cudaEvent_t> chunk_ev;
  int chunks_timed = 0;
  hsgen_stats stats{};
  long long launches = 0;           // kernels launched by the current call
  int phase_used[8]{};
};

namespace hsg {

// ---- error helpers ---------------------------------------------------------
// True for device (or managed) memory.
bool is_device_ptr(const void *p);
// True for device memory of a GPU other than `device`.
bool on_other_device(const void *p, int device);
// Grows a library workspace to at least `bytes` (contents not kept).
hsgen_status ensure_ws(hsgen_ctx *ctx, Workspace &w, size_t bytes);
// Frees the reduction's handles and buffers.
void reduce_release(hsgen_ctx *ctx);
hsgen_status set_err(hsgen_ctx *ctx, hsgen_status st, const std::string &msg);
hsgen_status cuda_err(hsgen_ctx *ctx, cudaError_t e, const char *what);
#define HSG_CUDA(ctx, call)                                         \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return hsg::cuda_err((ctx), e_, #call);  \
  } while (0)
// A launch wrapper call that starts one kernel (counted for the stats).
#define HSG_LAUNCH(ctx, call) \
  do {                        \
    HSG_CUDA(ctx, call);      \
    ++(ctx)->launches;        \
  } while (0)

// ---- kernels (launch wrappers) ---------------------------------------------
// a0/a1: per-species radial factors F[type][t][l] = pre_l * (f_A, f_B)(|K_t| r_MT).
cudaError_t launch_radial(int n_g, const double *kvec, int n_types, const RadialParams *d_rp, double2 *F,
                          cudaStream_t s);
// a1: W[t][off_a + ...] = [A_a; B_a] for the atoms in `atoms` (one species).
cudaError_t launch_coefficients(int lmax, int n_g, const double *kvec, const double2 *F_type, const int *atoms,
                                int n_atoms, const double *pos, const double *rot, const int *off,
                                int row_base, int dpad, double2 *W, long long ldw, cudaStream_t s);
// S in the m-summed (Legendre) form (Sec. 3.1, Eq. overlap_no_m): the plan
// holds each plane wave's integer reciprocal-lattice coordinates relative to
// K_0 (shifted to start at 0) and the box of their differences; `ok` is false
// when the K_t do not lie on one lattice k + G or the tables would be too large.
struct LegendrePlan {
  bool ok = false;
  std::vector<int> nco;  // 3 per plane wave
  int span[3] = {0, 0, 0}, dim[3] = {1, 1, 1};
  long long cells = 1;
  int lmax = 0;
  bool tail = false;  // some species' contraction stops below its l_max: add H's spherical tail
};
bool legendre_plan(const hsgen_ctx *ctx, int n_g, const double *kvec_host, LegendrePlan &p);
size_t legendre_ws_bytes(const hsgen_ctx *ctx, int n_g, const LegendrePlan &p);
// Writes the opt.uplo triangle of S (device, ld) from the radial factors F of
// this k-point (F[type][t][l], as launch_radial writes them) and, when the plan
// has a tail, adds H's spherical rows beyond each species' contraction into H;
// ws holds legendre_ws_bytes. Asynchronous on s (host tables are staged by the copies).
// S_host (pinned host, same ld; upper triangle only): S's finished column
// groups are copied there on ctx->copy_stream while later groups compute.
// The two halves of legendre_S, for graph capture: the host-table uploads and
// kernel attributes (before a capture), then the kernel launches (capturable
// when S_host is null).
hsgen_status legendre_upload(hsgen_ctx *ctx, int n_g, const LegendrePlan &p, void *ws, cudaStream_t s);
hsgen_status legendre_launch(hsgen_ctx *ctx, int n_g, const double *kvec_dev, const double2 *F,
                             const LegendrePlan &p, void *ws, double2 *S, double2 *H, long long ld, cudaStream_t s,
                             void *S_host = nullptr);
hsgen_status legendre_S(hsgen_ctx *ctx, int n_g, const double *kvec_dev, const double2 *F, const LegendrePlan &p,
                        void *ws, double2 *S, double2 *H, long long ld, cudaStream_t s, void *S_host = nullptr);
// a2: T matrix of one species (device, dpad x dpad complex, column-major).
cudaError_t launch_tmatrix(const Species &sp, double2 *d_T, double *scratch, cudaStream_t s);
// Cholesky factor of the species' T into d_C and its status into *d_info (device).
cudaError_t launch_cholesky(const Species &sp, const double2 *d_T, double2 *d_C, int *d_info, cudaStream_t s);
// Recurrence tables in constant memory (called once per device).
cudaError_t upload_tables();
// a3: X_a = T_type W_a for all atoms of one species (FP64 DMMA).
cudaError_t launch_tapply_fp64(int dpad, int n_g, const double2 *T, const int *atoms, int n_atoms,
                               const int *off, int row_base, const double2 *W, double2 *X, long long ldw,
                               cudaStream_t s);
// a4: upper (or lower) triangle of H += W^H X and S += W^H diag(u) W (FP64 DMMA);
// gram (the HPD route, X = C^H W): H += X^H X instead.
cudaError_t launch_hs_fp64(int n_g, int depth, const double2 *W, const double2 *X, const double *urow,
                           long long ldw, double2 *H, double2 *S, long long ld, int uplo, int accumulate,
                           const BlockOwner &own, cudaStream_t s, bool gram = false);
// C (+)= (+-) P^H Q in FP64 (DMMA): P is K x M, Q is K x N (complex, column-major), C is M x N;
// uplo 'U': only the entries i <= j (diagonal imaginary parts set to 0); C must not overlap P or Q.
cudaError_t launch_gemm_fp64(int M, int N, int K, const double2 *P, long long ldp, const double2 *Q, long long ldq,
                             double2 *C, long long ldc, int uplo, int accumulate, int negate, cudaStream_t s);
// Mirror the written triangle into the other one (fill_full) and clear diagonal imaginary parts.
cudaError_t launch_mirror(int n_g, double2 *M, long long ld, int uplo, cudaStream_t s);

}  // namespace hsg
