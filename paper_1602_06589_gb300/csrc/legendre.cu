// legendre.cu -- S in the m-summed (Legendre) form, the reduction the paper
// describes for FLEUR (Sec. 3.1, Eq. overlap_no_m).
//
// Summing conj(Y_lm(R K^_t)) Y_lm(R K^_t') over m gives (2l+1)/(4 pi)
// P_l(K^_t . K^_t') (the rotation drops out), so with the radial factors
// F_A, F_B of App. A.1 (prefactor 4 pi / (W_l sqrt(Omega)) included)
//
//   S_{t t'} = sum_tau SF_tau(n_t' - n_t) sum_{l <= lmax_tau} (2l+1)/(4 pi) P_l(K^_t . K^_t')
//              [F_A(tau,l,t) F_A(tau,l,t') + ||u_dot_l||^2 F_B(tau,l,t) F_B(tau,l,t')],
//
// where SF_tau(dn) = sum over the atoms of species tau of exp(2 pi i dn . f_a)
// (f_a fractional coordinates) is the per-species phase sum: K_t' - K_t =
// sum_j dn_j b_j for the integer reciprocal-lattice coordinates n_t of the
// plane waves, so the atom sum depends on t, t' only through dn and is
// tabulated once per k-point over the box of differences. Per entry this is
// ~170 FP64 operations instead of 16 sum_a N_L flops of the contraction.
//
// With l_nonsph < l_max (Sec. 3.1, Fig. Tmat_structure) T is diagonal in L
// for l > l_nonsph, with the spherical 2 x 2 block [[E_l, 1/2], [1/2,
// E_l ||u_dot_l||^2]] (reading R1) coupling A and B of the same L; the same
// m-sum turns H's part from those rows into
//   H_tail = sum_tau SF_tau sum_{l_c < l <= l_max} (2l+1)/(4 pi) P_l sum_{x,y} T^{xy}_l F_x(t) F_y(t'),
// which the same pass adds into H (the contraction covers l <= l_c).
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace hsg {

namespace {

constexpr int TILE = 32;        // rows x columns of S per CTA
constexpr int LTHREADS = 512;   // 32 rows x 16 column groups, 2 columns per thread
constexpr double kInv4Pi = 0.07957747154594766788;
// Bonnet recurrence coefficients ((2l-1)/l, (l-1)/l), l = 0..10
__constant__ double2 c_bonnet[kLmaxMax + 1] = {
    {0.0, 0.0}, {1.0, 0.0}, {1.5, 0.5}, {5.0 / 3.0, 2.0 / 3.0}, {1.75, 0.75}, {1.8, 0.8},
    {11.0 / 6.0, 5.0 / 6.0}, {13.0 / 7.0, 6.0 / 7.0}, {1.875, 0.875}, {17.0 / 9.0, 8.0 / 9.0}, {1.9, 0.9}};

// SF[idx * n_types + tau], idx = (i1 * d2 + i2) * d3 + i3 for dn = (i1 - s1, i2 - s2, i3 - s3).
__global__ void sfactor_kernel(int d1, int d2, int d3, int s1, int s2, int s3, int n_types,
                               const int *__restrict__ atoms_by_type, const int *__restrict__ type_start,
                               const double *__restrict__ frac, double2 *__restrict__ SF) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)d1 * d2 * d3) return;
  const int i3 = (int)(idx % d3);
  const long long r = idx / d3;
  const int i2 = (int)(r % d2), i1 = (int)(r / d2);
  const double n1 = i1 - s1, n2 = i2 - s2, n3 = i3 - s3;
  for (int ty = 0; ty < n_types; ++ty) {
    double sr = 0.0, si = 0.0;
    for (int k = type_start[ty]; k < type_start[ty + 1]; ++k) {
      const double *f = frac + 3 * atoms_by_type[k];
      double q = n1 * f[0] + n2 * f[1] + n3 * f[2];
      q -= rint(q);  // exp(2 pi i q) depends on q mod 1
      double sn, cs;
      sincospi(2.0 * q, &sn, &cs);
      sr += cs;
      si += sn;
    }
    SF[idx * n_types + ty] = make_double2(sr, si);
  }
}

// One CTA per TILE x TILE tile of the chosen triangle. TAIL: also add H's
// spherical tail (htab[(tau, l)] = (T^AA, T^AB), (T^BA, T^BB) times (2l+1)/(4 pi),
// zero for l <= l_c) into H.
template <int LMAX, bool TAIL>
__global__ void __launch_bounds__(LTHREADS) legendre_s_kernel(
    int n_g, const double *__restrict__ K, const int *__restrict__ nco, const double2 *__restrict__ F, int n_types,
    const int *__restrict__ lmax_of, const double2 *__restrict__ wts, const double2 *__restrict__ htab,
    const double2 *__restrict__ SF, int d2, int d3, int s1, int s2, int s3, double2 *__restrict__ S,
    double2 *__restrict__ H, long long ld, int uplo, long long x0) {
  constexpr int NLP = LMAX + 1;
  extern __shared__ double2 smem[];
  const int nlf = n_types * NLP;
  double2 *rowF = smem;              // [TILE][n_types][NLP], scaled by the weights
  double2 *colF = smem + TILE * nlf; // [TILE][n_types][NLP]
  double2 *rowH = colF + TILE * nlf; // TAIL: [TILE][n_types][NLP], transformed by the tail's T blocks
  __shared__ double rK[TILE][3], cK[TILE][3];
  __shared__ int rN[TILE][3], cN[TILE][3];

  const long long x = x0 + blockIdx.x;  // tiles in order of hi (the column block for 'U')
  int hi = (int)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
  while ((long long)hi * (hi + 1) / 2 > x) --hi;
  while ((long long)(hi + 1) * (hi + 2) / 2 <= x) ++hi;
  const int lo = (int)(x - (long long)hi * (hi + 1) / 2);  // lo <= hi
  const int bi = (uplo == 'U') ? lo : hi, bj = (uplo == 'U') ? hi : lo;
  const int r0 = bi * TILE, c0 = bj * TILE;

  for (int i = threadIdx.x; i < TILE * nlf; i += LTHREADS) {
    const int tt = i / nlf, rem = i - tt * nlf, ty = rem / NLP, l = rem - ty * NLP;
    double2 fr = make_double2(0.0, 0.0), fc = make_double2(0.0, 0.0), fh = make_double2(0.0, 0.0);
    if (l <= lmax_of[ty]) {  // entries above a species' l_max are never read from F
      const double2 w = wts[ty * NLP + l];
      const int tr = r0 + tt, tc = c0 + tt;
      if (tr < n_g) {
        const double2 f = F[((size_t)ty * n_g + tr) * kRadStride + l];
        fr = make_double2(f.x * w.x, f.y * w.y);
        if (TAIL) {  // (sum_x T^{xA} F_x, sum_x T^{xB} F_x)
          const double2 ha = htab[2 * (ty * NLP + l)], hb = htab[2 * (ty * NLP + l) + 1];
          fh = make_double2(fma(ha.x, f.x, hb.x * f.y), fma(ha.y, f.x, hb.y * f.y));
        }
      }
      if (tc < n_g) fc = F[((size_t)ty * n_g + tc) * kRadStride + l];
    }
    rowF[i] = fr;
    colF[i] = fc;
    if (TAIL) rowH[i] = fh;
  }
  if (threadIdx.x < 2 * TILE) {
    const int side = threadIdx.x / TILE, tt = threadIdx.x % TILE;
    const int t = (side ? c0 : r0) + tt;
    double h[3] = {0.0, 0.0, 1.0};  // K = 0: direction taken as z (only l = 0 survives)
    int nn[3] = {0, 0, 0};
    if (t < n_g) {
      const double kx = K[3 * t], ky = K[3 * t + 1], kz = K[3 * t + 2];
      const double kn = sqrt(kx * kx + ky * ky + kz * kz);
      if (kn > 0.0) {
        h[0] = kx / kn;
        h[1] = ky / kn;
        h[2] = kz / kn;
      }
      nn[0] = nco[3 * t];
      nn[1] = nco[3 * t + 1];
      nn[2] = nco[3 * t + 2];
    }
    for (int d = 0; d < 3; ++d) {
      if (side) {
        cK[tt][d] = h[d];
        cN[tt][d] = nn[d];
      } else {
        rK[tt][d] = h[d];
        rN[tt][d] = nn[d];
      }
    }
  }
  __syncthreads();

  const int tr = threadIdx.x & (TILE - 1), cg = threadIdx.x >> 5;
  const int row = r0 + tr;
  int col[2];
  double P[2][NLP];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int tc = cg + 16 * j;
    col[j] = c0 + tc;
    double ct = rK[tr][0] * cK[tc][0] + rK[tr][1] * cK[tc][1] + rK[tr][2] * cK[tc][2];
    ct = fmin(1.0, fmax(-1.0, ct));
    P[j][0] = 1.0;
    if constexpr (LMAX >= 1) P[j][1] = ct;
#pragma unroll
    for (int l = 2; l <= LMAX; ++l)  // Bonnet: l P_l = (2l-1) x P_{l-1} - (l-1) P_{l-2}
      P[j][l] = fma(c_bonnet[l].x * ct, P[j][l - 1], -c_bonnet[l].y * P[j][l - 2]);
  }
  double2 acc[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
  double2 acch[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
  for (int ty = 0; ty < n_types; ++ty) {
    double g[2] = {0.0, 0.0}, gh[2] = {0.0, 0.0};
    const double2 *rf = rowF + tr * nlf + ty * NLP;
    const double2 *rh = rowH + tr * nlf + ty * NLP;
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
      const double2 a = rf[l];
      double2 ah;
      if (TAIL) ah = rh[l];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const double2 b = colF[(cg + 16 * j) * nlf + ty * NLP + l];
        g[j] = fma(P[j][l], fma(a.x, b.x, a.y * b.y), g[j]);
        if (TAIL) gh[j] = fma(P[j][l], fma(ah.x, b.x, ah.y * b.y), gh[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int tc = cg + 16 * j;
      const long long idx = ((long long)(cN[tc][0] - rN[tr][0] + s1) * d2 + (cN[tc][1] - rN[tr][1] + s2)) * d3 +
                            (cN[tc][2] - rN[tr][2] + s3);
      const double2 sf = SF[idx * n_types + ty];
      acc[j].x = fma(g[j], sf.x, acc[j].x);
      acc[j].y = fma(g[j], sf.y, acc[j].y);
      if (TAIL) {
        acch[j].x = fma(gh[j], sf.x, acch[j].x);
        acch[j].y = fma(gh[j], sf.y, acch[j].y);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const bool keep = row < n_g && col[j] < n_g && ((uplo == 'U') ? row <= col[j] : row >= col[j]);
    if (!keep) continue;
    double2 v = acc[j];
    if (row == col[j]) v.y = 0.0;
    S[(size_t)col[j] * ld + row] = v;
    if (TAIL) {
      double2 h = H[(size_t)col[j] * ld + row];
      h.x += acch[j].x;
      h.y = (row == col[j]) ? 0.0 : h.y + acch[j].y;
      H[(size_t)col[j] * ld + row] = h;
    }
  }
}

template <int L>
cudaError_t launch_s_lmax(int n_g, const double *K, const int *nco, const double2 *F, int n_types, const int *lmax_of,
                          const double2 *wts, const double2 *htab, const double2 *SF, const int d[3], const int sp[3],
                          double2 *S, double2 *H, long long ld, int uplo, long long x0, long long ntiles,
                          cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (H) {
    const size_t sm = sizeof(double2) * 3 * TILE * n_types * (L + 1);
    legendre_s_kernel<L, true><<<(unsigned)ntiles, LTHREADS, sm, s>>>(
        n_g, K, nco, F, n_types, lmax_of, wts, htab, SF, d[1], d[2], sp[0], sp[1], sp[2], S, H, ld, uplo, x0);
  } else {
    const size_t sm = sizeof(double2) * 2 * TILE * n_types * (L + 1);
    legendre_s_kernel<L, false><<<(unsigned)ntiles, LTHREADS, sm, s>>>(
        n_g, K, nco, F, n_types, lmax_of, wts, htab, SF, d[1], d[2], sp[0], sp[1], sp[2], S, H, ld, uplo, x0);
  }
  return cudaGetLastError();
}

}  // namespace

bool legendre_plan(const hsgen_ctx *ctx, int n_g, const double *K, LegendrePlan &p) {
  p.ok = false;
  p.nco.assign(3 * (size_t)std::max(n_g, 0), 0);
  if (n_g <= 0) return false;
  // integer coordinates n_t with K_t - K_0 = sum_j n_tj b_j, i.e. n_tj = a_j . (K_t - K_0) / (2 pi)
  const double *A = ctx->lattice;
  int mn[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
  for (int t = 0; t < n_g; ++t) {
    const double dk[3] = {K[3 * t] - K[0], K[3 * t + 1] - K[1], K[3 * t + 2] - K[2]};
    for (int j = 0; j < 3; ++j) {
      const double v = (A[3 * j] * dk[0] + A[3 * j + 1] * dk[1] + A[3 * j + 2] * dk[2]) / (2.0 * M_PI);
      const double r = std::nearbyint(v);
      if (!(std::fabs(v - r) <= 1e-6) || std::fabs(r) > 1e6) return false;  // not a lattice of K_0
      const int n = (int)r;
      p.nco[3 * t + j] = n;
      mn[j] = std::min(mn[j], n);
      mx[j] = std::max(mx[j], n);
    }
  }
  long long cells = 1;
  for (int j = 0; j < 3; ++j) {
    p.span[j] = mx[j] - mn[j];
    p.dim[j] = 2 * p.span[j] + 1;
    cells *= p.dim[j];
  }
  for (int t = 0; t < n_g; ++t)
    for (int j = 0; j < 3; ++j) p.nco[3 * t + j] -= mn[j];
  p.cells = cells;
  const size_t nt = ctx->types.size();
  if ((double)cells * nt * sizeof(double2) > 1.0 * (1ull << 30)) return false;  // table above 1 GiB
  int lm = 0;
  p.tail = false;
  for (const auto &sp : ctx->types) {
    lm = std::max(lm, sp.lmax);
    p.tail = p.tail || sp.lc < sp.lmax;
  }
  p.lmax = lm;
  if (sizeof(double2) * (p.tail ? 3 : 2) * TILE * nt * (lm + 1) > 200 * 1024)
    return false;  // staging above the kernel's limit
  p.ok = true;
  return true;
}

size_t legendre_ws_bytes(const hsgen_ctx *ctx, int n_g, const LegendrePlan &p) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t nt = ctx->types.size(), na = ctx->toa.size();
  // the regions leg_ws() carves, in its order
  return al(sizeof(int) * 3 * (size_t)n_g) + al(sizeof(double2) * (size_t)p.cells * nt) +
         al(sizeof(double2) * nt * (kLmaxMax + 1)) + al(sizeof(double2) * 2 * nt * (kLmaxMax + 1)) +
         al(sizeof(int) * nt) + al(sizeof(int) * (nt + 1)) + al(sizeof(double) * 3 * na);
}

namespace {

constexpr int kLegSmemMax = 200 * 1024;  // staging limit legendre_plan enforces

template <int L>
cudaError_t set_smem_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e =
      cudaFuncSetAttribute(legendre_s_kernel<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLegSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(legendre_s_kernel<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kLegSmemMax);
  if (e == cudaSuccess) done = true;
  return e;
}

struct LegWs {
  int *n, *lmax, *tstart;
  double2 *sf, *w, *h;
  double *frac;
};

LegWs leg_ws(const hsgen_ctx *ctx, int n_g, const LegendrePlan &p, void *ws) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const int nt = (int)ctx->types.size();
  char *b = (char *)ws;
  LegWs L;
  L.n = (int *)b;
  b += al(sizeof(int) * 3 * (size_t)n_g);
  L.sf = (double2 *)b;
  b += al(sizeof(double2) * (size_t)p.cells * nt);
  L.w = (double2 *)b;
  b += al(sizeof(double2) * nt * (kLmaxMax + 1));
  L.h = (double2 *)b;
  b += al(sizeof(double2) * 2 * nt * (kLmaxMax + 1));
  L.lmax = (int *)b;
  b += al(sizeof(int) * nt);
  L.tstart = (int *)b;
  b += al(sizeof(int) * (nt + 1));
  L.frac = (double *)b;
  return L;
}

}  // namespace

hsgen_status legendre_upload(hsgen_ctx *ctx, int n_g, const LegendrePlan &p, void *ws, cudaStream_t s) {
  const int nt = (int)ctx->types.size(), na = (int)ctx->toa.size();
  const LegWs L = leg_ws(ctx, n_g, p, ws);
  // host tables: weights (2l+1)/(4 pi) and ||u_dot_l||^2 (2l+1)/(4 pi) at stride lmax+1,
  // species l_max, species starts in the per-species atom list, fractional coordinates
  const int NLP = p.lmax + 1;
  std::vector<double2> w((size_t)nt * NLP, make_double2(0.0, 0.0));
  std::vector<double2> h(2 * (size_t)nt * NLP, make_double2(0.0, 0.0));
  std::vector<int> lmax(nt), tstart(ctx->atoms_by_type_start.begin(), ctx->atoms_by_type_start.end());
  for (int t = 0; t < nt; ++t) {
    const Species &sp = ctx->types[t];
    lmax[t] = sp.lmax;
    for (int l = 0; l <= sp.lmax; ++l) {
      const double c = (2.0 * l + 1.0) * kInv4Pi;
      w[(size_t)t * NLP + l] = make_double2(c, c * sp.un2[l]);
      if (l > sp.lc) {  // H's spherical tail: (T^AA, T^AB), (T^BA, T^BB) of l, times c
        h[2 * ((size_t)t * NLP + l)] = make_double2(c * sp.el[l], c * 0.5);
        h[2 * ((size_t)t * NLP + l) + 1] = make_double2(c * 0.5, c * sp.el[l] * sp.un2[l]);
      }
    }
  }
  // fractional coordinates: x = sum_j f_j a_j, i.e. f = x A^{-1} with A's rows a_j
  const double *A = ctx->lattice;
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  const double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det,
                         (A[1] * A[5] - A[2] * A[4]) / det, (A[5] * A[6] - A[3] * A[8]) / det,
                         (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                         (A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det,
                         (A[0] * A[4] - A[1] * A[3]) / det};
  std::vector<double> frac(3 * (size_t)na);
  for (int a = 0; a < na; ++a)
    for (int j = 0; j < 3; ++j)
      frac[3 * a + j] = ctx->pos[3 * a] * inv[j] + ctx->pos[3 * a + 1] * inv[3 + j] + ctx->pos[3 * a + 2] * inv[6 + j];
  // kernel attribute first (not a stream operation: must not happen inside a graph capture)
  cudaError_t ea = cudaErrorInvalidValue;
  switch (p.lmax) {
#define HSG_LEG_ATTR(LM) \
  case LM:               \
    ea = set_smem_attr<LM>(); \
    break;
    HSG_LEG_ATTR(0) HSG_LEG_ATTR(1) HSG_LEG_ATTR(2) HSG_LEG_ATTR(3) HSG_LEG_ATTR(4) HSG_LEG_ATTR(5)
    HSG_LEG_ATTR(6) HSG_LEG_ATTR(7) HSG_LEG_ATTR(8) HSG_LEG_ATTR(9) HSG_LEG_ATTR(10)
#undef HSG_LEG_ATTR
    default: break;
  }
  HSG_CUDA(ctx, ea);
  // pageable sources: each copy has been staged when it returns
  HSG_CUDA(ctx, cudaMemcpyAsync(L.n, p.nco.data(), sizeof(int) * 3 * (size_t)n_g, cudaMemcpyHostToDevice, s));
  HSG_CUDA(ctx, cudaMemcpyAsync(L.w, w.data(), sizeof(double2) * w.size(), cudaMemcpyHostToDevice, s));
  HSG_CUDA(ctx, cudaMemcpyAsync(L.h, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice, s));
  HSG_CUDA(ctx, cudaMemcpyAsync(L.lmax, lmax.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, s));
  HSG_CUDA(ctx, cudaMemcpyAsync(L.tstart, tstart.data(), sizeof(int) * (nt + 1), cudaMemcpyHostToDevice, s));
  HSG_CUDA(ctx, cudaMemcpyAsync(L.frac, frac.data(), sizeof(double) * frac.size(), cudaMemcpyHostToDevice, s));
  return HSGEN_OK;
}

hsgen_status legendre_launch(hsgen_ctx *ctx, int n_g, const double *K_dev, const double2 *F, const LegendrePlan &p,
                             void *ws, double2 *S, double2 *H, long long ld, cudaStream_t s, void *S_host) {
  const int nt = (int)ctx->types.size();
  const LegWs L = leg_ws(ctx, n_g, p, ws);
  {
    const unsigned blocks = (unsigned)((p.cells + 255) / 256);
    sfactor_kernel<<<blocks, 256, 0, s>>>(p.dim[0], p.dim[1], p.dim[2], p.span[0], p.span[1], p.span[2], nt,
                                          ctx->d_atoms_by_type, L.tstart, L.frac, L.sf);
    HSG_CUDA(ctx, cudaGetLastError());
    ++ctx->launches;
  }
  const long long nb = (n_g + TILE - 1) / TILE;
  const long long ntiles = nb * (nb + 1) / 2;
  auto launch = [&](long long x0, long long cnt) -> hsgen_status {
    cudaError_t e = cudaErrorInvalidValue;
    switch (p.lmax) {
#define HSG_LEG_CASE(LM)                                                                                         \
  case LM:                                                                                                       \
    e = launch_s_lmax<LM>(n_g, K_dev, L.n, F, nt, L.lmax, L.w, L.h, L.sf, p.dim, p.span, S,                    \
                          p.tail ? H : nullptr, ld, ctx->opt.uplo, x0, cnt, s);                                \
    break;
      HSG_LEG_CASE(0) HSG_LEG_CASE(1) HSG_LEG_CASE(2) HSG_LEG_CASE(3) HSG_LEG_CASE(4) HSG_LEG_CASE(5)
      HSG_LEG_CASE(6) HSG_LEG_CASE(7) HSG_LEG_CASE(8) HSG_LEG_CASE(9) HSG_LEG_CASE(10)
#undef HSG_LEG_CASE
      default: break;
    }
    HSG_CUDA(ctx, e);
    ++ctx->launches;
    return HSGEN_OK;
  };
  if (!S_host || ctx->opt.uplo != 'U') return launch(0, ntiles);
  // Host output of S (upper triangle): the tiles of column block j are
  // x in [j(j+1)/2, (j+1)(j+2)/2), so launches over whole column blocks,
  // about 1/16 of the tiles each, leave finished columns that the copy
  // stream moves to the host while the next launches compute.
  if (!ctx->copy_stream) HSG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  if (!ctx->copy_ev) HSG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->copy_ev, cudaEventDisableTiming));
  const long long want = std::max<long long>(1, (ntiles + 15) / 16);
  for (long long j0 = 0; j0 < nb;) {
    long long j1 = j0 + 1;
    while (j1 < nb && j1 * (j1 + 1) / 2 - j0 * (j0 + 1) / 2 < want) ++j1;
    const long long x0 = j0 * (j0 + 1) / 2, x1 = j1 * (j1 + 1) / 2;
    hsgen_status st = launch(x0, x1 - x0);
    if (st != HSGEN_OK) return st;
    const long long c0 = j0 * TILE, c1 = std::min<long long>(n_g, j1 * TILE);
    HSG_CUDA(ctx, cudaEventRecord(ctx->copy_ev, s));
    HSG_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_ev, 0));
    HSG_CUDA(ctx, cudaMemcpyAsync((double2 *)S_host + c0 * ld, S + c0 * ld, sizeof(double2) * (c1 - c0) * ld,
                                  cudaMemcpyDeviceToHost, ctx->copy_stream));
    j0 = j1;
  }
  return HSGEN_OK;
}

hsgen_status legendre_S(hsgen_ctx *ctx, int n_g, const double *K_dev, const double2 *F, const LegendrePlan &p,
                        void *ws, double2 *S, double2 *H, long long ld, cudaStream_t s, void *S_host) {
  hsgen_status st = legendre_upload(ctx, n_g, p, ws, s);
  if (st != HSGEN_OK) return st;
  return legendre_launch(ctx, n_g, K_dev, F, p, ws, S, H, ld, s, S_host);
}

}  // namespace hsg
