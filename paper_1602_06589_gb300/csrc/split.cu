// split.cu -- split-precision form of a3 (X = T W) and a4 (H, S) on the
// tcgen05 tensor cores of sm_103a.
//
// Slicing (a5, part 1): every column of a complex FP64 operand gets one
// power-of-two scale 2^e with all |re|, |im| < 2^e; each real value v becomes
// the integer N = round(v 2^(7 + 8(s-1) - e)) (|N| <= 2^(7+8(s-1))), cut into
// balanced base-256 digits d_1 .. d_s, |d_p| <= 128, stored as BF16 planes
// (exact). The integer work uses the IEEE bit pattern directly, so no FP64
// arithmetic is spent on it.
//
// Products (a5, part 2): C = P^H Q is, in real form,
//   Re C = Pr^T Qr + Pi^T Qi,   Im C = Pr^T Qi - Pi^T Qr.
// One tile is 128 output rows x 64 complex columns. The "r half" multiplies
// A = Pr with the B block [Qr | Qi], the "i half" A = Pi with [Qi | -Qr] (a
// negated plane is stored), so both halves add into the same [Re | Im] FP32
// accumulator of 128 TMEM columns.
// For a slice pair (p, q) the products are integers of magnitude <= 2^14; a
// chunk of 1024 of them sums exactly in FP32 (|sum| <= 2^24). After each
// chunk the epilogue warps move the FP32 accumulator into an int64 fixed-point
// accumulator held in registers, weighting pair (p, q) by 2^(-8(p+q-2)); pairs
// with p + q > s + 1 are dropped (Ozaki-style truncation). After the last
// chunk the tile is scaled by 2^(e_i + f_j - 14 - F) into FP64.
//
// Class pairs: the weight classes g = p + q are taken two at a time (g, g+1).
// For a slice p of A, one M = 128, N = 256 MMA multiplies it with the B blocks
// of q = g - p and q' = g + 1 - p side by side, into a 256-column accumulator
// [class g | class g+1]; where only one of the two pairs exists the MMA has
// N = 128. An N = 256 MMA does twice the work of an N = 128 one per issue,
// which keeps the tensor core busy where 128 x 128 MMAs are issue-bound.
//
// CTA pairs: a tile is 256 output rows x 64 complex columns, computed by two
// CTAs (a cluster of 2 on two SMs) with M = 256 tcgen05 MMAs of cta_group::2.
// Each CTA loads its own 128 rows of A and its half of B (the class-g block in
// CTA 0, the class-(g+1) block in CTA 1), so an SM takes in 32 KB of operands
// per 64-deep block instead of 48 KB; the leader CTA issues the MMAs, which
// read both CTAs' shared memory and write each CTA's 128 rows into its own
// tensor memory.
//
// Kernel roles (384 threads per CTA, one CTA per SM, persistent over tiles):
//   warps 0-7   epilogue (TMEM lane quadrant = warp % 4, real or imaginary half)
//   warp 8      TMA producer (cp.async.bulk.tensor, 128B swizzle, 3 stages of 2 k-blocks)
//   warp 9      TMEM allocator; tcgen05.mma issuer in the leader CTA
//   warps 10-11 idle (their registers go to the epilogue)
// Every wait is bounded (wait_timeout_ns); on expiry the kernel records an
// error word, drains its own copies and MMAs (again bounded), frees TMEM and
// returns, and the host reports HSGEN_ETIMEOUT.
#include <cuda.h>  // CUtensorMap and enums; the encoder is fetched from the driver at run time
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "split.cuh"

namespace hsg {

namespace {

constexpr int kMaxProb = 4;
constexpr int kTShiftStep = 2;                // atoms start on even depth rows (2 N_L rows each)
constexpr int kTShifts = 64 / kTShiftStep;    // depth shifts 0, 2, .., 62 of the per-atom T copies
// BM: rows of A per CTA (one TMA box); BMT: rows of a tile (a CTA pair)
constexpr int BM = 128, BMT = 256, BN = 64, BK = 64;
// A pipeline stage holds KPS 64-deep k-blocks: large stages keep the fixed
// cost of each barrier round trip small next to the bytes moved.
constexpr int KPS = 2;
constexpr int NST = 3;
constexpr int A_BYTES = 16384;                 // one k-block of A: 128x64 bf16 (this CTA's rows)
constexpr int B_BYTES = 16384;                 // one k-block of this CTA's half of B: 128x64 bf16
constexpr int STAGE_A = KPS * A_BYTES;         // A k-blocks of a stage, then its B k-blocks
constexpr int STAGE_BYTES = KPS * (A_BYTES + B_BYTES);
// warps 0-7 epilogue (warpgroups 0, 1), warp 8 TMA, warp 9 MMA, warps 10-11 idle
// (warpgroup 2, which hands its registers to the epilogue)
constexpr int NTHREADS = 384;
constexpr int WARP_TMA = 8, WARP_MMA = 9;
// Register split (setmaxnreg): the CTA is launched with 168 registers per
// thread (65536 / 384 rounded down to 8), 384 x 168 = 64512 in all;
// warpgroup 2 drops to 72 and the two epilogue warpgroups rise to 216:
// 256 x 216 + 128 x 72 = 64512, so the epilogue's int64 sums need no spills.
constexpr int REG_LAUNCH = 168, REG_EPI = 216, REG_AUX = 72;
static_assert(2 * 128 * REG_EPI + 128 * REG_AUX <= NTHREADS * REG_LAUNCH, "register split exceeds the launch");
constexpr int NACC = 2;                 // FP32 accumulator buffers of 256 TMEM columns
constexpr int SMEM_BYTES = NST * STAGE_BYTES + 1024 + 256;  // 197888 <= 232448 (227 KiB)
constexpr uint32_t TMEM_COLS = 512;
// tcgen05 kind::f16 instruction descriptors: D f32, A bf16, B bf16, both K-major, M = 256 (CTA pair), N = 256 or 128.
constexpr uint32_t IDESC_N256 = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((256u >> 4) << 24);
constexpr uint32_t IDESC_N128 = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((256u >> 4) << 24);

enum : int { ERR_TIMEOUT_PRODUCER = 1, ERR_TIMEOUT_MMA = 2, ERR_TIMEOUT_EPILOGUE = 4 };

struct GemmProblem {
  int M, N, K;              // output rows, output complex columns, complex depth
  int a_pps, b_pps;         // planes per slice of the A and B slice arrays
  int a_nkb, b_nkb;         // k-blocks per plane of the A and B slice arrays
  int kb_begin;             // first k-block of this problem's depth range (both operands)
  int a_real;               // A has a zero imaginary part: skip the i half
  int uplo;                 // 0, 'U' or 'L' (tile set and write mask)
  int accumulate;           // C += result instead of C = result
  int F;                    // fixed-point fractional bits of the wide accumulator
  const int *expA, *expB;   // per A column (output row) / per B column exponents
  double2 *C;
  long long ldc;
  const int *atoms;         // batch mode: atom of each batch item
  const int *off;           // depth offset of each atom
  int row_base;             // depth offset of the chunk
  int n_batch, nbm, nbn;    // batch items, row blocks, column blocks
  int a_shift_planes;       // batch mode: A planes per depth shift (the shifted copies of T)
  const int2 *tile_list;    // triangle mode: (row block, column block) of every tile, L2-friendly order
  long long tile_begin;     // first global tile index of this problem
  // moduli form: per-tile residue store (one byte per output and modulus),
  // the problem's first slot in it, and whether this launch starts / ends the depth
  unsigned char *res;
  long long res_base;
  int seg_first, seg_last;
};

// Moduli form (Ozaki scheme II): pairwise coprime moduli m_i <= 256, CRT
// weights c_i = (M / m_i) ((M / m_i)^-1 mod m_i) mod M as 128-bit integers
// (lo, hi), M = prod m_i, and 2^64 / M for the quotient estimate.
constexpr int kMaxModuli = 14;
struct CrtConsts {
  int n;
  int m[kMaxModuli];
  float inv_m[kMaxModuli];
  unsigned long long c_lo[kMaxModuli], c_hi[kMaxModuli];
  unsigned long long M_lo, M_hi, Mh_lo, Mh_hi;  // M and M / 2
  float q_scale;
};

struct GemmParams {
  CUtensorMap mapA[kMaxProb];
  CUtensorMap mapB[kMaxProb];
  GemmProblem prob[kMaxProb];
  // grouped launches (many k-points): problems and maps in device memory
  // (gmap[2i] = A map, gmap[2i+1] = B map of problem i); null: use the arrays above
  const GemmProblem *gprob;
  const CUtensorMap *gmap;
  int nprob;
  long long ntiles;
  int s;
  int *status;
  unsigned long long timeout_ns;
  CrtConsts crt;  // moduli form only
  int crt_order;  // moduli form: 0 tile-major units, 1 modulus-major (see crt_unit)
  int l2_hint;    // moduli form: L2 priority of A (bits 0-1) and B (bits 2-3) loads: 0 normal, 1 first, 2 last
  int recon_apart;  // moduli form: the launch that ends the depth leaves the reconstruction to crt_reconstruct_kernel
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when `timeout_ns` elapsed without the phase completing.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, unsigned long long timeout_ns) {
  if (mbar_try(a, parity)) return true;
  uint64_t t0 = gtime();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try(a, parity)) return true;
    if (gtime() - t0 > timeout_ns) return false;
  }
}
// Both CTAs of a pair load into their own shared memory and signal the
// leader CTA's barrier (`mbar` is a shared::cluster address).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t mbar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];"
      ::"r"(dst), "l"((uint64_t)map), "r"(mbar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
// The same load with an L2 eviction-priority hint (a policy from createpolicy).
__device__ __forceinline__ void tma_load_3d_hint(uint32_t dst, const CUtensorMap *map, uint32_t mbar, int c0, int c1,
                                                 int c2, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4, %5}], [%2], %6;"
      ::"r"(dst), "l"((uint64_t)map), "r"(mbar), "r"(c0), "r"(c1), "r"(c2), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ uint32_t map_rank(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Tensor memory of a CTA pair: one warp of each CTA takes part in allocation,
// permit release and deallocation; the leader CTA issues the MMAs, which read
// A and B from both CTAs' shared memory and write both CTAs' tensor memory.
__device__ __forceinline__ void tc_alloc(uint32_t dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// arrives on the barrier at offset `mbar` in both CTAs of the pair once the
// MMAs issued so far have completed
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
               ::"r"(mbar), "h"((uint16_t)3)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// One lane of the (converged) warp; the warp's other lanes skip the guarded
// block. Issuing tcgen05/TMA work this way keeps the surrounding bookkeeping
// warp-uniform, so descriptors stay in uniform registers and the issue loop
// keeps up with the tensor core.
__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile("{\n .reg .b32 r;\n .reg .pred p;\n elect.sync r|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(pred));
  return pred != 0;
}
// Bounded wait of a whole converged warp with a warp-uniform verdict: every
// lane polls the barrier (try_wait with a suspend-time hint) until the phase
// completes or the global-timer deadline passes.
// `Cluster`: acquire at cluster scope (arrivals released by the peer CTA).
template <bool Cluster = false>
__device__ __forceinline__ bool warp_wait(uint32_t a, uint32_t parity, unsigned long long timeout_ns) {
  uint32_t ok;
  if (Cluster)
    asm volatile(
        "{\n .reg .pred P1;\n .reg .u64 t, dl;\n"
        " mov.u64 t, %%globaltimer;\n add.u64 dl, t, %3;\n"
        "WARP_WAIT_LOOP:\n"
        " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 P1, [%1], %2, 1000000;\n"
        " @P1 bra WARP_WAIT_DONE;\n"
        " mov.u64 t, %%globaltimer;\n setp.lt.u64 P1, t, dl;\n @P1 bra WARP_WAIT_LOOP;\n"
        "WARP_WAIT_DONE:\n selp.u32 %0, 1, 0, P1;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "l"(timeout_ns)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred P1;\n .reg .u64 t, dl;\n"
        " mov.u64 t, %%globaltimer;\n add.u64 dl, t, %3;\n"
        "WARP_WAIT_LOOP:\n"
        " mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2, 1000000;\n"
        " @P1 bra WARP_WAIT_DONE;\n"
        " mov.u64 t, %%globaltimer;\n setp.lt.u64 P1, t, dl;\n @P1 bra WARP_WAIT_LOOP;\n"
        "WARP_WAIT_DONE:\n selp.u32 %0, 1, 0, P1;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "l"(timeout_ns)
        : "memory");
  return __all_sync(0xffffffffu, ok) != 0;
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of 1024 B.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset 16 B (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // SWIZZLE_128B
  return d;
}

// ---------------------------------------------------------------------------
// Tile schedule (identical in every role)
// ---------------------------------------------------------------------------
struct Tile {
  int prob, m0, n0, b_k0, c_row0, nkb, a_p0;
};

__device__ __forceinline__ const GemmProblem &problem(const GemmParams &P, int i) {
  return P.gprob ? P.gprob[i] : P.prob[i];
}
__device__ __forceinline__ const CUtensorMap *map_a(const GemmParams &P, int i) {
  return P.gprob ? &P.gmap[2 * i] : &P.mapA[i];
}
__device__ __forceinline__ const CUtensorMap *map_b(const GemmParams &P, int i) {
  return P.gprob ? &P.gmap[2 * i + 1] : &P.mapB[i];
}

__device__ __forceinline__ Tile decode_tile(const GemmParams &P, long long t) {
  int pi = 0, hi = P.nprob;  // last problem with tile_begin <= t
  while (hi - pi > 1) {
    const int mid = (pi + hi) >> 1;
    if (problem(P, mid).tile_begin <= t) pi = mid; else hi = mid;
  }
  const GemmProblem &pr = problem(P, pi);
  long long lt = t - pr.tile_begin;
  Tile ti;
  ti.prob = pi;
  int bi, bj, koff = 0;
  if (pr.tile_list) {
    const int2 bij = pr.tile_list[lt];
    bi = bij.x;
    bj = bij.y;
  } else {
    long long per = (long long)pr.nbm * pr.nbn;
    int b = (int)(lt / per);
    int rem = (int)(lt % per);
    bi = rem % pr.nbm;
    bj = rem / pr.nbm;
    koff = pr.off[pr.atoms[b]] - pr.row_base;  // a multiple of kTShiftStep
  }
  ti.m0 = bi * BMT;
  ti.n0 = bj * BN;
  // B starts at the 64-deep block holding the atom's first row; A is the copy
  // of T shifted down by the rest (zero rows elsewhere)
  ti.b_k0 = koff & ~(BK - 1);
  ti.a_p0 = ((koff & (BK - 1)) / kTShiftStep) * pr.a_shift_planes;
  ti.c_row0 = koff;
  ti.nkb = (pr.K + BK - 1) / BK;
  return ti;
}

// The accumulation schedule of one tile, identical in every role: chunk kc
// covers complex k-blocks [kc*ckb, min(nkb, (kc+1)*ckb)); within it the class
// pairs (g, g+1), g = 2, 4, ... <= s + 1, go in order, and within a class pair
// the units p = 1 .. units(g) (slice p of A times slices g - p and g + 1 - p of
// B). Up to `ppc` units share a chunk when their products still fit the
// 1024-product exactness bound (short depths, e.g. X = T W).
struct Sched {
  int s, nkb, ckb, nkc, halves, ppc;
  __device__ Sched(const GemmProblem &pr, const Tile &ti, int s_) : s(s_) {
    nkb = ti.nkb;
    halves = pr.a_real ? 1 : 2;
    ckb = pr.a_real ? 16 : 8;
    nkc = (nkb + ckb - 1) / ckb;
    const int per_pair = (nkb < ckb ? nkb : ckb) * BK * halves;  // products per output and pair
    ppc = (nkc == 1) ? max(1, 1024 / per_pair) : 1;
  }
  // units of the class pair based at g
  __device__ __forceinline__ int units(int g) const { return (g + 1 <= s + 1) ? g : s; }
  // which accumulator halves unit p of class pair g writes: bit 0 class g, bit 1 class g + 1
  __device__ __forceinline__ int mask(int g, int p) const { return (g + 1 > s + 1) ? 1 : (p < g ? 3 : 2); }
};

// ---------------------------------------------------------------------------
// The persistent split GEMM kernel
// ---------------------------------------------------------------------------
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    split_gemm_kernel(const __grid_constant__ GemmParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *bars = (uint64_t *)(smem + NST * STAGE_BYTES);
  uint32_t *tmem_slot = (uint32_t *)(bars + 2 * NST + 2 * NACC + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * NST, accf0 = empty0 + 8 * NST,
                 acce0 = accf0 + 8 * NACC, tdown = acce0 + 8 * NACC;
  const uint32_t sbase = smem_u32(smem);
  const unsigned long long tmo = P.timeout_ns;
  // CTA pair: rank 0 (leader) issues the MMAs; its `full` barriers count both
  // CTAs' copies and its `acce` barriers both CTAs' epilogue warps
  const uint32_t rank = cta_rank();
  const bool leader = rank == 0;
  const uint32_t lead_full0 = map_rank(full0, 0), lead_acce0 = map_rank(acce0, 0);
  const long long pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    for (int i = 0; i < NACC; ++i) {
      mbar_init(accf0 + 8 * i, 1);
      mbar_init(acce0 + 8 * i, 16);  // one arrival per epilogue warp of either CTA
    }
    mbar_init(tdown, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == WARP_MMA) {
    tc_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers exist before either signals the other's
  tc_fence_after();
  const uint32_t tbase = *tmem_slot;
  const int S = P.s;
  // teardown waits: long enough for copies and MMAs already issued to finish
  const unsigned long long drain = tmo > 1000000000ull ? tmo : 1000000000ull;
  if (warp == WARP_TMA) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_AUX));
    // ------------------------------ TMA producer ------------------------------
    uint32_t it = 0;
    bool ok = true;
    for (long long t = pair; t < P.ntiles && ok; t += npairs) {
      const Tile ti = decode_tile(P, t);
      const GemmProblem &pr = problem(P, ti.prob);
      const Sched sc(pr, ti, S);
      const CUtensorMap *mA = map_a(P, ti.prob), *mB = map_b(P, ti.prob);
      for (int kc = 0; kc < sc.nkc && ok; ++kc) {
        const int kb0 = kc * sc.ckb, kb1 = min(sc.nkb, kb0 + sc.ckb);
        for (int g = 2; g <= S + 1 && ok; g += 2) {
          const int nu = sc.units(g);
          for (int pb = 1; pb <= nu && ok; pb += sc.ppc) {
            const int pe = min(nu, pb + sc.ppc - 1);
            for (int p = pb; p <= pe && ok; ++p) {
              const int m = sc.mask(g, p);
              const int q0 = g - p, q1 = g + 1 - p;  // B slices of the two classes
              for (int kb = kb0; kb < kb1 && ok; kb += KPS) {
                const int nk = min(KPS, kb1 - kb);
                // both CTAs' bytes, expected on the leader's barrier
                const uint32_t bytes = nk * (2 * A_BYTES + (m == 3 ? 2 * B_BYTES : B_BYTES));
                for (int h = 0; h < sc.halves; ++h, ++it) {
                  const int st = it % NST;
                  const uint32_t round = it / NST;
                  if (!warp_wait(empty0 + 8 * st, (round & 1) ^ 1, tmo)) {
                    if (lane == 0) atomicOr(P.status, ERR_TIMEOUT_PRODUCER);
                    ok = false;
                    break;
                  }
                  const uint32_t sA0 = sbase + st * STAGE_BYTES;
                  const uint32_t mbar = lead_full0 + 8 * st;
                  const int pa = ti.a_p0 + (p - 1) * pr.a_pps + h;
                  const int kbA = pr.kb_begin + kb;
                  const int kbB = pr.kb_begin + ti.b_k0 / BK + kb;  // b_k0 is a multiple of 64
                  if (elect_one()) {
                    if (leader) mbar_expect_tx(full0 + 8 * st, bytes);
                    for (int j = 0; j < nk; ++j) {
                      const uint32_t sA = sA0 + j * A_BYTES, sB = sA0 + STAGE_A + j * B_BYTES;
                      tma_load_3d(sA, mA, mbar, 0, ti.m0 + (int)rank * BM, pa * pr.a_nkb + kbA + j);
                      // The pair's B operand is split by rows between the CTAs. N = 256:
                      // rows [0, 128) class g (CTA 0), [128, 256) class g + 1 (CTA 1), each
                      // [plane h | plane h + 1] = [re | im] (h = 0) or [im | -re] (h = 1).
                      // N = 128 (one class): plane h in CTA 0, plane h + 1 in CTA 1.
                      if (m == 3) {
                        const int pq = ((rank ? q1 : q0) - 1) * pr.b_pps + h;
                        tma_load_3d(sB, mB, mbar, 0, ti.n0, pq * pr.b_nkb + kbB + j);
                        tma_load_3d(sB + 8192, mB, mbar, 0, ti.n0, (pq + 1) * pr.b_nkb + kbB + j);
                      } else {
                        const int pq = ((m == 1 ? q0 : q1) - 1) * pr.b_pps + h + (int)rank;
                        tma_load_3d(sB, mB, mbar, 0, ti.n0, pq * pr.b_nkb + kbB + j);
                      }
                    }
                  }
                  __syncwarp();
                }
              }
            }
          }
        }
      }
    }
    // no copy may still be in flight at teardown: the latest use of every
    // stage must have landed in both CTAs (bounded; the leader's barriers
    // count both, and the final cluster barrier holds the peer until then)
    for (int st = 0; st < NST && leader; ++st) {
      if (it <= (uint32_t)st) break;
      const uint32_t j = st + NST * ((it - 1 - st) / NST);
      if (!warp_wait(full0 + 8 * st, (j / NST) & 1, drain) && lane == 0) atomicOr(P.status, ERR_TIMEOUT_PRODUCER);
    }
  } else if (warp == WARP_MMA) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_AUX));
    if (leader) {
    // ------------------------------ MMA issuer --------------------------------
    const uint64_t descA0 = desc_sw128(sbase), descB0 = desc_sw128(sbase + STAGE_A);
    uint32_t it = 0, cc = 0;
    bool ok = true;
    for (long long t = pair; t < P.ntiles && ok; t += npairs) {
      const Tile ti = decode_tile(P, t);
      const GemmProblem &pr = problem(P, ti.prob);
      const Sched sc(pr, ti, S);
      for (int kc = 0; kc < sc.nkc && ok; ++kc) {
        const int kb0 = kc * sc.ckb, kb1 = min(sc.nkb, kb0 + sc.ckb);
        for (int g = 2; g <= S + 1 && ok; g += 2) {
          const int nu = sc.units(g);
          for (int pb = 1; pb <= nu && ok; pb += sc.ppc, ++cc) {
            const int pe = min(nu, pb + sc.ppc - 1);
            const int buf = cc % NACC;
            const uint32_t use = cc / NACC;
            if (!warp_wait<true>(acce0 + 8 * buf, (use & 1) ^ 1, tmo)) {
              if (lane == 0) atomicOr(P.status, ERR_TIMEOUT_MMA);
              ok = false;
              break;
            }
            tc_fence_after();
            // the chunk's first unit writes every accumulator half the chunk uses
            // (units with both classes come before the single-class unit p = g)
            uint32_t accum = 0;
            for (int p = pb; p <= pe && ok; ++p) {
              const int m = sc.mask(g, p);
              const uint32_t idesc = (m == 3) ? IDESC_N256 : IDESC_N128;
              const uint32_t dacc = tbase + buf * 256 + (m == 2 ? 128 : 0);
              for (int kb = kb0; kb < kb1 && ok; kb += KPS) {
                const int nk = min(KPS, kb1 - kb);
                for (int h = 0; h < sc.halves; ++h, ++it) {
                  const int st = it % NST;
                  if (!warp_wait(full0 + 8 * st, (it / NST) & 1, tmo)) {
                    if (lane == 0) atomicOr(P.status, ERR_TIMEOUT_MMA);
                    ok = false;
                    break;
                  }
                  tc_fence_after();
                  const uint64_t da = descA0 + (uint64_t)(st * (STAGE_BYTES >> 4));
                  const uint64_t db = descB0 + (uint64_t)(st * (STAGE_BYTES >> 4));
                  if (elect_one()) {
                    for (int j = 0; j < nk; ++j) {
#pragma unroll
                      for (int kk = 0; kk < BK / 16; ++kk)
                        tc_mma(dacc, da + (uint64_t)(j * (A_BYTES >> 4)) + 2 * kk,
                               db + (uint64_t)(j * (B_BYTES >> 4)) + 2 * kk, idesc, (accum | j | kk) ? 1u : 0u);
                    }
                    tc_commit(empty0 + 8 * st);
                  }
                  __syncwarp();
                  accum = 1;
                }
              }
            }
            if (ok) {
              if (elect_one()) tc_commit(accf0 + 8 * buf);
              __syncwarp();
            }
          }
        }
      }
    }
    // every MMA issued has completed before TMEM is released (bounded)
    if (elect_one()) tc_commit(tdown);
    __syncwarp();
    if (!warp_wait(tdown, 0, drain) && lane == 0) atomicOr(P.status, ERR_TIMEOUT_MMA);
    }
  } else if (warp < WARP_TMA) {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_EPI));
    // ------------------------------ epilogue ----------------------------------
    // Eight warps: warp w reads TMEM lane quadrant w % 4 (rows), and half hf of
    // the accumulator columns (hf 0: real parts, hf 1: imaginary parts of the
    // tile's 64 complex columns). The int64 fixed-point sums live in registers
    // for the whole tile.
    const int qd = warp & 3;
    const int hf = warp >> 2;
    const uint32_t lane_off = (uint32_t)(qd * 32) << 16;
    uint32_t cc = 0;
    bool ok = true;
    for (long long t = pair; t < P.ntiles && ok; t += npairs) {
      const Tile ti = decode_tile(P, t);
      const GemmProblem &pr = problem(P, ti.prob);
      const Sched sc(pr, ti, S);
      long long acc[64];
#pragma unroll
      for (int u = 0; u < 64; ++u) acc[u] = 0;
      for (int kc = 0; kc < sc.nkc && ok; ++kc)
        for (int g = 2; g <= S + 1 && ok; g += 2) {
          const int nu = sc.units(g);
          for (int pb = 1; pb <= nu && ok; pb += sc.ppc, ++cc) {
            const int buf = cc % NACC;
            const uint32_t use = cc / NACC;
            // one lane waits, the whole warp follows its verdict (the TMEM loads
            // below are warp-collective)
            int got = 0;
            if (lane == 0) got = mbar_wait(accf0 + 8 * buf, use & 1, tmo) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) {
              if (lane == 0) atomicOr(P.status, ERR_TIMEOUT_EPILOGUE);
              ok = false;
              break;
            }
            tc_fence_after();
            const int m = sc.mask(g, pb);  // accumulator halves written in this chunk
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              if (!((m >> c) & 1)) continue;
              const int sh = pr.F - 8 * (g + c - 2);
              const int ish = sh > 0 ? sh : 0;
              const float fsc = (sh < 0) ? __int_as_float((127 + sh) << 23) : 1.0f;
              const uint32_t tacc = tbase + lane_off + buf * 256 + c * 128 + hf * 64;
              uint32_t v[32];
#pragma unroll
              for (int half = 0; half < 2; ++half) {
                tc_ld32(tacc + half * 32, v);
                tc_wait_ld();
#pragma unroll
                for (int u = 0; u < 32; ++u)
                  acc[half * 32 + u] += (long long)__float2int_rn(__uint_as_float(v[u]) * fsc) << ish;
              }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(lead_acce0 + 8 * buf);
          }
        }
      if (!ok) break;
      // ---- tile output: int64 fixed point -> FP64, scaled by 2^(eA + eB - 14 - F)
      const int row = ti.m0 + (int)rank * BM + qd * 32 + lane;  // row within the problem
      if (row < pr.M && !pr.tile_list) {
        // Batched X = T W tiles (short, written once): problem fields and
        // column exponents go to registers first, so no load waits behind a
        // store to C. The H/S tiles keep the loop below, whose slower,
        // interleaved stores spread the read-modify-write of H and S over
        // time: the fast form made the H/S contraction 20 % slower (the
        // tiles of a wave finish together and their bursts collide).
        const int eA = pr.expA[row];
        const int ncol = pr.N, uplo = pr.uplo, F = pr.F;
        const bool acc_old = pr.accumulate != 0;
        const long long ldc = pr.ldc;
        const int *expB = pr.expB;
        const long long grow = (long long)ti.c_row0 + row;  // row in C
        double *Cd = (double *)pr.C + 2 * grow + hf;
#pragma unroll
        for (int u0 = 0; u0 < 64; u0 += 16) {
          // previous values and exponents first (independent loads in flight together), then the stores
          double old[16];
          int eb[16];
          bool keep[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int col = ti.n0 + u0 + u;
            keep[u] = col < ncol && !(uplo == 'U' && row > col) && !(uplo == 'L' && row < col);
            eb[u] = keep[u] ? expB[col] : 0;
            old[u] = (keep[u] && acc_old) ? Cd[2 * (size_t)col * ldc] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            if (!keep[u]) continue;
            const int col = ti.n0 + u0 + u;
            const int e = eA + eb[u] - 14 - F;
            const double scl =
                (e > -1022 && e < 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
            double x = __ll2double_rn(acc[u0 + u]) * scl + old[u];
            if (hf == 1 && uplo && row == col) x = 0.0;
            Cd[2 * (size_t)col * ldc] = x;
          }
        }
      } else if (row < pr.M) {
        const int eA = pr.expA[row];
        const long long grow = (long long)ti.c_row0 + row;  // row in C
        double *Cd = (double *)pr.C + 2 * grow + hf;
#pragma unroll
        for (int u0 = 0; u0 < 64; u0 += 16) {
          // previous values first (independent loads in flight together), then the stores
          double old[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int col = ti.n0 + u0 + u;
            const bool keep = col < pr.N && !(pr.uplo == 'U' && row > col) && !(pr.uplo == 'L' && row < col);
            old[u] = (keep && pr.accumulate) ? Cd[2 * (size_t)col * pr.ldc] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int col = ti.n0 + u0 + u;
            const bool keep = col < pr.N && !(pr.uplo == 'U' && row > col) && !(pr.uplo == 'L' && row < col);
            if (!keep) continue;
            const int e = eA + pr.expB[col] - 14 - pr.F;
            const double scl =
                (e > -1022 && e < 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
            double x = __ll2double_rn(acc[u0 + u]) * scl + old[u];
            if (hf == 1 && pr.uplo && row == col) x = 0.0;
            Cd[2 * (size_t)col * pr.ldc] = x;
          }
        }
      }
    }
  } else {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_AUX));
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // the leader's MMAs and both CTAs' copies are complete
  tc_fence_after();
  if (warp == WARP_MMA) tc_dealloc(tbase, TMEM_COLS);
}

// ---------------------------------------------------------------------------
// The moduli form (Ozaki scheme II) of the H/S contraction
// ---------------------------------------------------------------------------
// Every operand column is integerised once, N = round(v 2^(b - e)) with one
// power-of-two scale per column (|N| <= 2^b), and stored as its balanced
// residues r_i = N mod m_i (|r_i| <= 128, exact in BF16) for n pairwise
// coprime moduli m_i <= 256. The integer product C' = P'^H Q' is then known
// from its residues C' mod m_i = (sum_k r_i(P) r_i(Q)) mod m_i: one BF16
// product per modulus instead of s(s+1)/2 slice pairs. b is the largest value
// with 4 K 2^(2b) < M = prod m_i (K = complex depth), so the balanced
// representative of C' in [-M/2, M/2) is C' itself (Chinese remainder
// theorem); only the rounding of P and Q to b-bit integers is an error.
//
// Tiles are 256 output rows x 128 complex columns (CTA pair, M = 256): every
// MMA is N = 256, the B operand [Qr | Qi] (r half) or [Qi | -Qr] (i half)
// split by rows between the two CTAs. Per modulus the depth runs in chunks
// of 1024 products (exact in FP32) into one of two TMEM accumulators; the
// epilogue adds each chunk into int32 sums in registers, reduces them mod m_i
// at the end of the modulus and keeps the residue bytes in a per-tile store
// in global memory, added mod m_i across depth segments (separate launches).
// The launch that ends the depth reconstructs C' from the residues (128-bit
// integers), scales it to FP64 and writes (or adds) the tile of H or S.
constexpr int BNC = 128;  // complex output columns of a moduli-form tile
// the moduli kernel's stage geometries, as template arguments (k-blocks per
// stage, stages, k-blocks per accumulation chunk): <2, 3, 8> and <3, 2, 6>; a
// chunk holds at most 1024 products (exact in FP32)

__device__ __forceinline__ Tile decode_tile_crt(const GemmParams &P, long long t, long long &slot) {
  int pi = 0, hi = P.nprob;
  while (hi - pi > 1) {
    const int mid = (pi + hi) >> 1;
    if (problem(P, mid).tile_begin <= t) pi = mid; else hi = mid;
  }
  const GemmProblem &pr = problem(P, pi);
  const long long lt = t - pr.tile_begin;
  const int2 bij = pr.tile_list[lt];
  Tile ti;
  ti.prob = pi;
  ti.m0 = bij.x * BMT;
  ti.n0 = bij.y * BNC;
  ti.b_k0 = 0;
  ti.a_p0 = 0;
  ti.c_row0 = 0;
  ti.nkb = (pr.K + BK - 1) / BK;
  slot = pr.res_base + lt;
  return ti;
}

__device__ __forceinline__ void ld_v4(const uint4 *p, uint32_t (&w)[4]) {
  asm volatile("ld.global.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p)
               : "memory");
}
// Asynchronous prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void st_v4(uint4 *p, const uint32_t (&w)[4]) {
  asm volatile("st.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
               : "memory");
}


// a mod m for 0 <= a < 2^31, 2 <= m <= 256: the float quotient is within 3
// of the true one (rounding of a, of 1/m and of the product), then corrected
__device__ __forceinline__ int mod_small(int a, int m, float inv_m) {
  const int q = __float2int_rz(__int2float_rz(a) * inv_m);
  int r = a - q * m;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r = (r < 0) ? r + m : r;
    r = (r >= m) ? r - m : r;
  }
  return r;
}

// One entry of the moduli form from its residues (byte b of word q of each
// modulus's 16-byte group): C' = sum_i r_i c_i mod M in 32-bit limbs (one
// 32 x 32 -> 64-bit multiply-add per limb and modulus; each limb sum < 2^44),
// the quotient by M (< 2^12) estimated from the high word and corrected once,
// the balanced representative, then |C'| 2^e as a double built from its bits
// (the top 53 bits, rounded half up on the next one; integer work only).
__device__ __forceinline__ double crt_value(const uint4 (&rv)[kMaxModuli], int NM, int q, int b, const CrtConsts &c,
                                            int e) {
  unsigned long long L0 = 0, L1 = 0, L2 = 0, L3 = 0;
  const bool limb3 = (c.M_hi >> 32) != 0;  // M < 2^96 (up to 12 moduli): every c_i's fourth limb is 0
#pragma unroll
  for (int i = 0; i < kMaxModuli; ++i) {
    if (i >= NM) break;
    const uint32_t word = (q == 0) ? rv[i].x : (q == 1) ? rv[i].y : (q == 2) ? rv[i].z : rv[i].w;
    const uint32_t r = (word >> (8 * b)) & 0xFFu;
    L0 += (unsigned long long)r * (uint32_t)c.c_lo[i];
    L1 += (unsigned long long)r * (uint32_t)(c.c_lo[i] >> 32);
    L2 += (unsigned long long)r * (uint32_t)c.c_hi[i];
    if (limb3) L3 += (unsigned long long)r * (uint32_t)(c.c_hi[i] >> 32);
  }
  L1 += L0 >> 32;
  L2 += L1 >> 32;
  L3 += L2 >> 32;  // the sum is below 14 x 255 x M < 2^123
  unsigned __int128 sum = ((unsigned __int128)((L3 << 32) | (uint32_t)L2) << 64) | ((L1 << 32) | (uint32_t)L0);
  const float qf = (float)((L3 << 32) | (uint32_t)L2) * c.q_scale - 0.5f;
  const uint32_t q0 = qf > 0.f ? (uint32_t)qf : 0u;
  {
    unsigned long long t = (unsigned long long)q0 * (uint32_t)c.M_lo;
    const uint32_t p0 = (uint32_t)t;
    t = (t >> 32) + (unsigned long long)q0 * (uint32_t)(c.M_lo >> 32);
    const uint32_t p1 = (uint32_t)t;
    t = (t >> 32) + (unsigned long long)q0 * (uint32_t)c.M_hi;
    const uint32_t p2 = (uint32_t)t;
    t = (t >> 32) + (unsigned long long)q0 * (uint32_t)(c.M_hi >> 32);
    sum -= ((unsigned __int128)((t << 32) | p2) << 64) | (((unsigned long long)p1 << 32) | p0);
  }
  const unsigned __int128 Mv = ((unsigned __int128)c.M_hi << 64) | c.M_lo;
  const unsigned __int128 Mh = ((unsigned __int128)c.Mh_hi << 64) | c.Mh_lo;
  if (sum >= Mv) sum -= Mv;
  const bool neg = sum > Mh;
  const unsigned __int128 mag = neg ? Mv - sum : sum;
  const unsigned long long mh = (unsigned long long)(mag >> 64), ml = (unsigned long long)mag;
  if (!(mh | ml)) return 0.0;
  const int nb = mh ? 128 - __clzll((long long)mh) : 64 - __clzll((long long)ml);  // bit length
  const int sh = nb - 54;                                                          // keep 54 bits
  unsigned long long top;
  if (sh <= 0)
    top = ml << (-sh);
  else if (sh < 64)
    top = (ml >> sh) | (mh << (64 - sh));
  else
    top = mh >> (sh - 64);
  unsigned long long mant = (top + 1) >> 1;  // 53 bits, or 2^53 after rounding up
  int ex = nb - 1 + e;
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  double x = (ex > -1023 && ex < 1024)
                 ? __longlong_as_double((long long)(((unsigned long long)(ex + 1023) << 52) |
                                                    (mant & 0xFFFFFFFFFFFFFull)))
                 : ldexp((double)mant, ex - 52);
  return neg ? -x : x;
}

// The work of a CTA pair is its tiles t = pair, pair + npairs, .. times the
// n moduli, in units (modulus i, tile t). Tile-major order (0) runs every
// modulus of a tile before its next tile, so the operands a wave of tiles
// shares are fetched again for every modulus; modulus-major order (1) runs all
// of the pair's tiles for modulus 0, then for modulus 1, .., so consecutive
// waves of the grid work on one modulus and share its operand blocks in L2.
// Either way the last unit of a tile is its last modulus, where the launch
// that ends the depth reconstructs the tile from the residues the same
// threads stored for the earlier moduli.
__device__ __forceinline__ void crt_unit(long long u, int nm, long long my_tiles, long long pair, long long npairs,
                                         int order, int &i, long long &t) {
  long long k;
  if (order == 1) {
    i = (int)(u / my_tiles);
    k = u - (long long)i * my_tiles;
  } else {
    k = u / nm;
    i = (int)(u - k * nm);
  }
  t = pair + k * npairs;
}

template <int KPS_, int NST_, int CKB_>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    crt_gemm_kernel(const __grid_constant__ GemmParams P) {
  // stage geometry: KPS_ k-blocks per stage, NST_ stages, CKB_ k-blocks per chunk
  constexpr int KPS = KPS_, NST = NST_, CKB = CKB_;
  constexpr int STAGE_A = KPS * A_BYTES, STAGE_BYTES = KPS * (A_BYTES + B_BYTES);
  static_assert(CKB % KPS == 0 && CKB * BK * 2 <= 1024 && NST * STAGE_BYTES + 1024 + 256 <= SMEM_BYTES,
                "stage geometry");
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *bars = (uint64_t *)(smem + NST * STAGE_BYTES);
  uint32_t *tmem_slot = (uint32_t *)(bars + 2 * NST + 2 * NACC + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * NST, accf0 = empty0 + 8 * NST,
                 acce0 = accf0 + 8 * NACC, tdown = acce0 + 8 * NACC;
  const uint32_t sbase = smem_u32(smem);
  const unsigned long long tmo = P.timeout_ns;
  const uint32_t rank = cta_rank();
  const bool leader = rank == 0;
  const uint32_t lead_full0 = map_rank(full0, 0), lead_acce0 = map_rank(acce0, 0);
  const long long pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int NM = P.crt.n;
  const long long my_tiles = P.ntiles > pair ? (P.ntiles - 1 - pair) / npairs + 1 : 0;
  const long long nunits = my_tiles * NM;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    for (int i = 0; i < NACC; ++i) {
      mbar_init(accf0 + 8 * i, 1);
      mbar_init(acce0 + 8 * i, 16);
    }
    mbar_init(tdown, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == WARP_MMA) {
    tc_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  const uint32_t tbase = *tmem_slot;
  const unsigned long long drain = tmo > 1000000000ull ? tmo : 1000000000ull;
  if (warp == WARP_TMA) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_AUX));
    // ------------------------------ TMA producer ------------------------------
    uint32_t it = 0;
    bool ok = true;
    auto policy = [](int h) {
      return h == 1 ? policy_evict_first() : h == 2 ? policy_evict_last() : policy_evict_normal();
    };
    const uint64_t polA = policy(P.l2_hint & 3), polB = policy((P.l2_hint >> 2) & 3);
    for (long long un = 0; un < nunits && ok; ++un) {
      int i;
      long long t, slot;
      crt_unit(un, NM, my_tiles, pair, npairs, P.crt_order, i, t);
      const Tile ti = decode_tile_crt(P, t, slot);
      const GemmProblem &pr = problem(P, ti.prob);
      const CUtensorMap *mA = map_a(P, ti.prob), *mB = map_b(P, ti.prob);
      for (int kb = 0; kb < ti.nkb && ok; kb += KPS) {
        const int nk = min(KPS, ti.nkb - kb);
        const uint32_t bytes = nk * 2 * (A_BYTES + B_BYTES);
        for (int h = 0; h < 2; ++h, ++it) {
          const int st = it % NST;
          const uint32_t round = it / NST;
          if (!warp_wait(empty0 + 8 * st, (round & 1) ^ 1, tmo)) {
            if (lane == 0) atomicOr(P.status, ERR_TIMEOUT_PRODUCER);
            ok = false;
            break;
          }
          const uint32_t sA0 = sbase + st * STAGE_BYTES;
          const uint32_t mbar = lead_full0 + 8 * st;
          const int pa = i * pr.a_pps + h;
          // B rows [0, 128) in CTA 0, [128, 256) in CTA 1: [re | im] (h = 0), [im | -re] (h = 1)
          const int pb = i * pr.b_pps + h + (int)rank;
          const int kbA = pr.kb_begin + kb;
          if (elect_one()) {
            if (leader) mbar_expect_tx(full0 + 8 * st, bytes);
            for (int j = 0; j < nk; ++j) {
              tma_load_3d_hint(sA0 + j * A_BYTES, mA, mbar, 0, ti.m0 + (int)rank * BM, pa * pr.a_nkb + kbA + j, polA);
              tma_load_3d_hint(sA0 + STAGE_A + j * B_BYTES, mB, mbar, 0, ti.n0, pb * pr.b_nkb + kbA + j, polB);
            }
          }
          __syncwarp();
        }
      }
    }
    for (int st = 0; st < NST && leader; ++st) {
      if (it <= (uint32_t)st) break;
      const uint32_t j = st + NST * ((it - 1 - st) / NST);
      if (!warp_wait(full0 + 8 * st, (j / NST) & 1, drain) && lane == 0) atomicOr(P.status, ERR_TIMEOUT_PRODUCER);
    }
  } else if (warp == WARP_MMA) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_AUX));
    if (leader) {
      // ------------------------------ MMA issuer --------------------------------
      const uint64_t descA0 = desc_sw128(sbase), descB0 = desc_sw128(sbase + STAGE_A);
      uint32_t it = 0, cc = 0;
      bool ok = true;
      for (long long un = 0; un < nunits && ok; ++un) {
        int i;
        long long t, slot;
        crt_unit(un, NM, my_tiles, pair, npairs, P.crt_order, i, t);
        (void)i;
        const Tile ti = decode_tile_crt(P, t, slot);
        for (int kc0 = 0; kc0 < ti.nkb && ok; kc0 += CKB, ++cc) {
          const int kc1 = min(ti.nkb, kc0 + CKB);
          const int buf = cc % NACC;
          const uint32_t use = cc / NACC;
          if (!warp_wait<true>(acce0 + 8 * buf, (use & 1) ^ 1, tmo)) {
            if (lane == 0) atomicOr(P.status, ERR_TIMEOUT_MMA);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dacc = tbase + buf * 256;
          uint32_t accum = 0;
          for (int kb = kc0; kb < kc1 && ok; kb += KPS) {
            const int nk = min(KPS, kc1 - kb);
            for (int h = 0; h < 2; ++h, ++it) {
              const int st = it % NST;
              if (!warp_wait(full0 + 8 * st, (it / NST) & 1, tmo)) {
                if (lane == 0) atomicOr(P.status, ERR_TIMEOUT_MMA);
                ok = false;
                break;
              }
              tc_fence_after();
              const uint64_t da = descA0 + (uint64_t)(st * (STAGE_BYTES >> 4));
              const uint64_t db = descB0 + (uint64_t)(st * (STAGE_BYTES >> 4));
              if (elect_one()) {
                for (int j = 0; j < nk; ++j) {
#pragma unroll
                  for (int kk = 0; kk < BK / 16; ++kk)
                    tc_mma(dacc, da + (uint64_t)(j * (A_BYTES >> 4)) + 2 * kk,
                           db + (uint64_t)(j * (B_BYTES >> 4)) + 2 * kk, IDESC_N256, (accum | j | kk) ? 1u : 0u);
                }
                tc_commit(empty0 + 8 * st);
              }
              __syncwarp();
              accum = 1;
            }
          }
          if (ok) {
            if (elect_one()) tc_commit(accf0 + 8 * buf);
            __syncwarp();
          }
        }
      }
      if (elect_one()) tc_commit(tdown);
      __syncwarp();
      if (!warp_wait(tdown, 0, drain) && lane == 0) atomicOr(P.status, ERR_TIMEOUT_MMA);
    }
  } else if (warp < WARP_TMA) {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_EPI));
    // ------------------------------ epilogue ----------------------------------
    // Warp w: TMEM lane quadrant w % 4 (rows), accumulator half hf = w / 4
    // (hf 0: real parts, hf 1: imaginary parts of the tile's 128 columns);
    // each thread holds the int32 sums of its row's 128 values. (Giving each
    // thread the real and imaginary parts of 64 columns, for 16-byte stores
    // of whole entries, made the launch that reconstructs H and S slower.)
    const int qd = warp & 3;
    const int hf = warp >> 2;
    const uint32_t lane_off = (uint32_t)(qd * 32) << 16;
    uint32_t cc = 0;
    bool ok = true;
    for (long long un = 0; un < nunits && ok; ++un) {
      int i;
      long long t, slot;
      crt_unit(un, NM, my_tiles, pair, npairs, P.crt_order, i, t);
      const Tile ti = decode_tile_crt(P, t, slot);
      const GemmProblem &pr = problem(P, ti.prob);
      const int nkc = (ti.nkb + CKB - 1) / CKB;
      // this thread's 128 residue bytes of modulus i
      auto res_ptr = [&](int i) {
        return (uint4 *)(pr.res + ((((size_t)slot * NM + i) * 2 + rank) * 256 + threadIdx.x) * 128);
      };
      {
        int acc[128];
#pragma unroll
        for (int u = 0; u < 128; ++u) acc[u] = 0;
        for (int kc = 0; kc < nkc && ok; ++kc, ++cc) {
          const int buf = cc % NACC;
          const uint32_t use = cc / NACC;
          // the residues this unit adds to: one 128-byte line per thread, 4 KB
          // per warp, brought into L2 one chunk ahead of their read
          if (!pr.seg_first && kc == max(0, nkc - 2) && lane == 0) prefetch_l2(res_ptr(i), 32 * 128);
          int got = 0;
          if (lane == 0) got = mbar_wait(accf0 + 8 * buf, use & 1, tmo) ? 1 : 0;
          got = __shfl_sync(0xffffffffu, got, 0);
          if (!got) {
            if (lane == 0) atomicOr(P.status, ERR_TIMEOUT_EPILOGUE);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t tacc = tbase + lane_off + buf * 256 + hf * 128;
          uint32_t v[16];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            tc_ld16(tacc + q * 16, v);
            tc_wait_ld();
#pragma unroll
            for (int u = 0; u < 16; ++u) acc[q * 16 + u] += __float2int_rn(__uint_as_float(v[u]));
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(lead_acce0 + 8 * buf);
        }
        if (!ok) break;
        // end of modulus i in this launch: sums mod m_i, added to the residues
        // of the earlier depth segments
        const int m = P.crt.m[i];
        const float inv = P.crt.inv_m[i];
        const int off = m << 22;  // makes every sum non-negative (|sum| <= 256 x 128 products x 2^14)
#pragma unroll
        for (int u = 0; u < 128; ++u) acc[u] = mod_small(acc[u] + off, m, inv);
        uint4 *rp = res_ptr(i);
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          // ordered loads and stores: one 16-byte group of residues in flight at a time
          uint32_t w[4] = {0u, 0u, 0u, 0u};
          if (!pr.seg_first) ld_v4(rp + g, w);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t outw = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              int r = acc[g * 16 + q * 4 + b] + (int)((w[q] >> (8 * b)) & 0xFFu);
              r = (r >= m) ? r - m : r;
              outw |= (uint32_t)r << (8 * b);
            }
            w[q] = outw;
          }
          st_v4(rp + g, w);
        }
      }
      if (!ok) break;
      if (!pr.seg_last || i != NM - 1 || P.recon_apart) continue;
      // ---- last segment: C' from its residues (CRT), scaled to FP64 by 2^(eA + eB - 2B)
      const int row = ti.m0 + (int)rank * BM + qd * 32 + lane;
      if (row >= pr.M) continue;
      const int eA = pr.expA[row];
      double *Cd = (double *)pr.C + 2 * (long long)row + hf;
      for (int g = 0; g < 8; ++g) {
        uint4 rv[kMaxModuli];
#pragma unroll
        for (int i = 0; i < kMaxModuli; ++i)
          if (i < NM) rv[i] = res_ptr(i)[g];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int col = ti.n0 + g * 16 + u;
          const bool keep = col < pr.N && !(pr.uplo == 'U' && row > col) && !(pr.uplo == 'L' && row < col);
          if (!keep) continue;
          double x = crt_value(rv, NM, u >> 2, u & 3, P.crt, eA + pr.expB[col] - pr.F);
          double *dst = Cd + 2 * (size_t)col * pr.ldc;
          if (pr.accumulate) x += *dst;
          if (hf == 1 && pr.uplo && row == col) x = 0.0;
          *dst = x;
        }
      }
    }
  } else {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_AUX));
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  if (warp == WARP_MMA) tc_dealloc(tbase, TMEM_COLS);
}

// The reconstruction of the moduli form as a kernel of its own, after the
// launch that ends the depth (same parameters): block (t, rank, g) takes the
// 16 columns [16 g, 16 g + 16) of tile t's rows [128 rank, 128 rank + 128);
// thread (warp w, lane) is the thread of the contraction's epilogue that
// stored the residues of row 32 (w % 4) + lane, part w / 4 (real, imaginary).
// With many blocks per SM the loads of the residues and of H, S overlap,
// where the contraction's eight epilogue warps would leave the MMA waiting.
__global__ void __launch_bounds__(256, 3) crt_reconstruct_kernel(const __grid_constant__ GemmParams P) {
  const long long t = blockIdx.x;
  const int rank = blockIdx.y, g = blockIdx.z;
  long long slot;
  const Tile ti = decode_tile_crt(P, t, slot);
  const GemmProblem &pr = problem(P, ti.prob);
  if (!pr.seg_last) return;
  const int NM = P.crt.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qd = warp & 3, hf = warp >> 2;
  const int row = ti.m0 + rank * BM + qd * 32 + lane;
  if (row >= pr.M) return;
  const int eA = pr.expA[row];
  double *Cd = (double *)pr.C + 2 * (long long)row + hf;
  uint4 rv[kMaxModuli];
#pragma unroll
  for (int i = 0; i < kMaxModuli; ++i)
    if (i < NM)
      rv[i] = ((const uint4 *)(pr.res + ((((size_t)slot * NM + i) * 2 + rank) * 256 + threadIdx.x) * 128))[g];
#pragma unroll 1
  for (int u = 0; u < 16; ++u) {
    const int col = ti.n0 + g * 16 + u;
    const bool keep = col < pr.N && !(pr.uplo == 'U' && row > col) && !(pr.uplo == 'L' && row < col);
    if (!keep) continue;
    double x = crt_value(rv, NM, u >> 2, u & 3, P.crt, eA + pr.expB[col] - pr.F);
    double *dst = Cd + 2 * (size_t)col * pr.ldc;
    if (pr.accumulate) x += *dst;
    if (hf == 1 && pr.uplo && row == col) x = 0.0;
    *dst = x;
  }
}

// ---------------------------------------------------------------------------
// Slicing kernel: one CTA per column.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long to_fixed(double v, int shift) {
  const long long b = __double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0;  // zero or subnormal: far below every scale in use
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const int t = E - 1075 + shift;
  long long N;
  if (t >= 0) {
    N = m << t;  // t <= 2 because |v| < 2^e
  } else {
    const int r = -t;
    N = (r > 62) ? 0 : ((m + (1LL << (r - 1))) >> r);
  }
  return (b < 0) ? -N : N;
}

// Output layout (k-blocked): plane P, column c, depth k at
//   dst[P * plane_stride + ((k / 64) * ncols + c) * 64 + k % 64],
// so one 64-deep block of 128 consecutive columns is 16 KB of contiguous memory.
__global__ void __launch_bounds__(256) slice_kernel(const double2 *__restrict__ src, long long lds, int K,
                                                    const double *__restrict__ urow, int s, int planes,
                                                    __nv_bfloat16 *__restrict__ dst, long long ldk, int ncols,
                                                    long long plane_stride, int *__restrict__ expo) {
  const int col = blockIdx.x;
  const double2 *c = src + (size_t)col * lds;
  __shared__ double red[8];
  __shared__ int e_sh;
  double mx = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double2 v = c[k];
    const double u = urow ? urow[k] : 1.0;
    mx = fmax(mx, fmax(fabs(v.x * u), fabs(v.y * u)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    const int e = (m > 0.0) ? ilogb(m) + 1 : 0;
    e_sh = e;
    expo[col] = e;
  }
  __syncthreads();
  const int shift = 7 + 8 * (s - 1) - e_sh;
  for (int k = threadIdx.x; k < (int)ldk; k += blockDim.x) {
    __nv_bfloat16 *out = dst + ((size_t)(k >> 6) * ncols + col) * 64 + (k & 63);
    long long Nr = 0, Ni = 0;
    if (k < K) {
      double2 v = c[k];
      if (urow) {
        const double u = urow[k];
        v.x *= u;
        v.y *= u;
      }
      Nr = to_fixed(v.x, shift);
      Ni = to_fixed(v.y, shift);
    }
    for (int p = s; p >= 1; --p) {
      int dr, di;
      if (p > 1) {
        dr = (int)((Nr << 56) >> 56);
        di = (int)((Ni << 56) >> 56);
        Nr = (Nr - dr) >> 8;
        Ni = (Ni - di) >> 8;
      } else {
        dr = (int)Nr;
        di = (int)Ni;
      }
      __nv_bfloat16 *base = out + (size_t)(p - 1) * planes * plane_stride;
      base[0] = __float2bfloat16_rn((float)dr);
      base[plane_stride] = __float2bfloat16_rn((float)di);
      if (planes == 3) base[2 * plane_stride] = __float2bfloat16_rn((float)-dr);
    }
  }
}

// Moduli form: residues of the integers N = round(v 2^f), with one power of
// two 2^f per column chosen from the column's 2-norm: f is the largest value
// with 2^f ||v|| (1 + 1e-9) + 0.5 sqrt(2K) <= 2^B, so the rounded column has
// ||N||_2 <= 2^B (every part is off by at most 1/2; the factor covers the
// rounding of the norm). The column's exponent e = B - f is stored (v ~ N
// 2^(e - B), as with a scale from the column's largest entry). For every
// modulus the balanced residues |r| <= 128, exact in BF16, are written as BF16
// planes in the k-blocked layout of slice_kernel; plane i * planes + {0, 1, 2}
// holds re, im, -re of modulus i. |N| <= 2^B <= 2^47 is cut into four 12-bit
// pieces, exact in FP32, so |N| mod m = sum_j piece_j (2^12j mod m) mod m is
// formed in FP32 (every partial sum is an integer below 2^22, exact) with a
// quotient rounded by the 1.5 2^23 shift: full-rate FP32 work, no integer
// division and no conversion instruction. Each thread takes two consecutive
// depth rows (one 4-byte store per plane).
__constant__ float c_pow12[kMaxModuli][3];  // 2^12, 2^24, 2^36 mod m_i

// One output of residue_kernel: the column's values weighted by urow (or not),
// their planes (re, im, and -re for planes == 3) and per-column exponents.
struct ResidueOut {
  const double *urow;
  int planes;
  __nv_bfloat16 *dst;
  int *expo;
};

// One or two outputs from one read of the source column (W's residues and
// U W's: the column is read once for both norms and once for both residues).
__global__ void __launch_bounds__(256) residue_kernel(const double2 *__restrict__ src, long long lds, int K, int b,
                                                      CrtConsts crt, long long ldk, int ncols, long long plane_stride,
                                                      ResidueOut o0, ResidueOut o1, int nout) {
  const int col = blockIdx.x;
  const double2 *c = src + (size_t)col * lds;
  __shared__ double red[2][8];
  __shared__ int e_sh[2];
  double ss[2] = {0.0, 0.0};  // sums of squares of the (weighted) column
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double2 v = c[k];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const double *urow = o ? o1.urow : o0.urow;
      if (o < nout) {
        const double u = urow ? urow[k] : 1.0;
        ss[o] = fma(v.x * u, v.x * u, fma(v.y * u, v.y * u, ss[o]));
      }
    }
  }
#pragma unroll
  for (int o = 0; o < 2; ++o) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) ss[o] += __shfl_xor_sync(0xffffffffu, ss[o], d);
    if ((threadIdx.x & 31) == 0) red[o][threadIdx.x >> 5] = ss[o];
  }
  __syncthreads();
  if (threadIdx.x < (unsigned)nout) {
    const int o = threadIdx.x;
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[o][w];
    int e = 0;
    if (t > 1e-280) {  // below: a zero column (or one that rounds to zero at any usable scale)
      const double room = ldexp(1.0, b) - 0.5 * sqrt(2.0 * (double)K);
      e = b - ilogb(room / (sqrt(t) * (1.0 + 1e-9)));
    }
    e_sh[o] = e;
    (o ? o1.expo : o0.expo)[col] = e;
  }
  __syncthreads();
  constexpr float kShift = 12582912.0f;  // 1.5 2^23: adding and subtracting it rounds to an integer
  for (int k = 2 * threadIdx.x; k < (int)ldk; k += 2 * blockDim.x) {  // ldk is a multiple of 64
    double2 v[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (k + h < K) v[h] = c[k + h];
    for (int o = 0; o < nout; ++o) {
      const ResidueOut &out_o = o ? o1 : o0;
      const int shift = b - e_sh[o];
      // (row, re/im): |N| in four exact FP32 pieces, and the sign
      float pc[4][4];
      bool ng[4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        long long N[2] = {0, 0};
        if (k + h < K) {
          double2 w = v[h];
          if (out_o.urow) {
            const double u = out_o.urow[k + h];
            w.x *= u;
            w.y *= u;
          }
          N[0] = to_fixed(w.x, shift);
          N[1] = to_fixed(w.y, shift);
        }
#pragma unroll
        for (int z = 0; z < 2; ++z) {
          const int q = 2 * z + h;
          ng[q] = N[z] < 0;
          const unsigned long long a = ng[q] ? (unsigned long long)(-N[z]) : (unsigned long long)N[z];
#pragma unroll
          for (int j = 0; j < 4; ++j)
            pc[q][j] = __int_as_float(0x4B000000 | (int)((a >> (12 * j)) & 0xFFFu)) - 8388608.0f;
        }
      }
      __nv_bfloat16 *out = out_o.dst + ((size_t)(k >> 6) * ncols + col) * 64 + (k & 63);
      for (int i = 0; i < crt.n; ++i) {
        const float m = (float)crt.m[i], inv = crt.inv_m[i], half = 0.5f * m;
        const float c12 = c_pow12[i][0], c24 = c_pow12[i][1], c36 = c_pow12[i][2];
        float r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float a = __fmaf_rn(pc[q][3], c36, __fmaf_rn(pc[q][2], c24, __fmaf_rn(pc[q][1], c12, pc[q][0])));
          const float qt = __fmaf_rn(a, inv, kShift) - kShift;  // a / m rounded, within one of the floor
          float x = __fmaf_rn(-qt, m, a);                       // |N| mod m, up to one m off: |x| < 0.51 m
          x = ng[q] ? -x : x;                                    // N mod m, up to one m off
          x = (x > half) ? x - m : x;                            // balanced: |x| <= m / 2 <= 128
          r[q] = (x < -half) ? x + m : x;
        }
        __nv_bfloat162 *base = (__nv_bfloat162 *)(out + (size_t)i * out_o.planes * plane_stride);
        base[0] = __floats2bfloat162_rn(r[0], r[1]);  // re of rows k, k + 1
        *(__nv_bfloat162 *)((__nv_bfloat16 *)base + plane_stride) = __floats2bfloat162_rn(r[2], r[3]);
        if (out_o.planes == 3)
          *(__nv_bfloat162 *)((__nv_bfloat16 *)base + 2 * plane_stride) = __floats2bfloat162_rn(-r[0], -r[1]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// 3D map over k-blocked bf16 planes: dim0 = 64 (depth inside a block),
// dim1 = column, dim2 = plane * nkb + k-block; boxes of 64 x box_rows x 1.
bool make_map(CUtensorMap *m, const void *base, long long nkb, long long ncols, long long nplanes, int box_rows) {
  EncodeTiledFn fn = encoder();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)BK, (cuuint64_t)ncols, (cuuint64_t)(nkb * nplanes)};
  cuuint64_t strides[2] = {(cuuint64_t)BK * 2, (cuuint64_t)(ncols * BK * 2)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int fixed_point_bits(int K) {
  // |accumulator| <= 2K * 2^14 * 2^F * (1 + 2^-7): keep it below 2^62; group-2
  // contributions (< 2^24 << F) must also fit, hence F <= 38.
  int lg = 0;
  while ((1LL << lg) < 2LL * K + 1) ++lg;
  return std::max(0, std::min(38, 47 - lg));
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

// CTA pairs that can be resident at once (one pair per two SMs).
int max_pairs() {
  static int n = 0;
  if (!n) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * (num_sms() / 2));
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, (const void *)split_gemm_kernel, &cfg) != cudaSuccess || c <= 0) {
      cudaGetLastError();
      c = num_sms() / 2;
    }
    n = std::max(1, c);
  }
  return n;
}

// Shared-memory attribute of both tensor-core kernels (once per process; set
// before any stream capture).
cudaError_t gemm_attrs() {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(split_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(crt_gemm_kernel<2, 3, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(crt_gemm_kernel<3, 2, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return cudaSuccess;
}

cudaError_t launch_gemm(GemmParams &P, cudaStream_t s) {
  cudaError_t e = gemm_attrs();
  if (e != cudaSuccess) return e;
  if (P.ntiles <= 0) return cudaSuccess;
  const long long pairs = std::min<long long>(P.ntiles, max_pairs());
  split_gemm_kernel<<<(unsigned)(2 * pairs), NTHREADS, SMEM_BYTES, s>>>(P);
  return cudaGetLastError();
}

// last_seg: some problem of this launch ends the depth (its tiles are then
// reconstructed by crt_reconstruct_kernel when P.recon_apart is set).
cudaError_t launch_crt(GemmParams &P, int geom, cudaStream_t s, bool last_seg) {
  cudaError_t e = gemm_attrs();
  if (e != cudaSuccess) return e;
  if (P.ntiles <= 0) return cudaSuccess;
  const long long pairs = std::min<long long>(P.ntiles, max_pairs());
  if (geom == 1)
    crt_gemm_kernel<3, 2, 6><<<(unsigned)(2 * pairs), NTHREADS, SMEM_BYTES, s>>>(P);
  else
    crt_gemm_kernel<2, 3, 8><<<(unsigned)(2 * pairs), NTHREADS, SMEM_BYTES, s>>>(P);
  if (P.recon_apart && last_seg) {
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    crt_reconstruct_kernel<<<dim3((unsigned)P.ntiles, 2, BNC / 16), 256, 0, s>>>(P);
  }
  return cudaGetLastError();
}

cudaError_t launch_residue(const double2 *src, long long lds, int K, const double *urow, int b, const CrtConsts &crt,
                           int planes, __nv_bfloat16 *dst, long long ldk, long long plane_stride, int *expo,
                           int ncols, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  const ResidueOut o0{urow, planes, dst, expo};
  residue_kernel<<<ncols, 256, 0, st>>>(src, lds, K, b, crt, ldk, ncols, plane_stride, o0, o0, 1);
  return cudaGetLastError();
}

// W's residues (3 planes) and U W's (2 planes, rows weighted by urow) from one read of W.
cudaError_t launch_residue_w_uw(const double2 *W, long long lds, int K, const double *urow, int b,
                                const CrtConsts &crt, __nv_bfloat16 *Wr, int *expW, __nv_bfloat16 *Yr, int *expY,
                                long long ldk, long long plane_stride, int ncols, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  const ResidueOut o0{nullptr, 3, Wr, expW}, o1{urow, 2, Yr, expY};
  residue_kernel<<<ncols, 256, 0, st>>>(W, lds, K, b, crt, ldk, ncols, plane_stride, o0, o1, 2);
  return cudaGetLastError();
}

// ---- moduli form: constants --------------------------------------------------
// pairwise coprime moduli <= 256 (2^8, 3.5.17, 11.23, 251, 13.19, then primes
// and 7.31), largest first: n of them give M = prod m_i of about 7.9 n bits
constexpr int kModuli[kMaxModuli] = {256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199};
// A-priori error model of the moduli form (relative Frobenius error of H
// and S for columns scaled to 2-norm 2^B, depth K): kCrtErr sqrt(2K) 2^-B,
// the worst case of columns whose entries are all of one size (each then
// keeps B - log2(sqrt(2K)) bits; measured 2.3-2.5 x 2^-bits with a scale from
// the largest entry), with a little margin. Coefficient columns hold their
// norm in a few large entries and do much better: 1.1e-11 at B = 39 on the
// one-atom workload (K = 50), and for W^H (T W) at K = 30976 (a numpy
// emulation of the rounding) 2.6e-11, 1.6e-12, 2.1e-13 for B = 39, 43, 46,
// 0.06 sqrt(2K) 2^-B. hsgen_autotune measures instead of using the model.
constexpr double kCrtErr = 3.0;

unsigned __int128 crt_M(int n) {
  unsigned __int128 M = 1;
  for (int i = 0; i < n; ++i) M *= (unsigned __int128)kModuli[i];
  return M;
}

// Norm bits B of n moduli: the largest B <= 47 with 2^(2B+1) < M. With both
// operands' columns of 2-norm <= 2^B, every real and imaginary part of the
// integer product is a dot product of two real vectors of those norms, so
// |C'| <= 2^(2B) < M / 2 (Cauchy-Schwarz) and C' is the balanced
// representative of its residues (Chinese remainder theorem). 47 keeps every
// |N| <= 2^47 within the residue kernel's four 12-bit pieces.
int crt_bits(int n) {
  const unsigned __int128 M = crt_M(n);
  int b = 0;
  while (b < 47 && ((unsigned __int128)1 << (2 * (b + 1) + 1)) < M) ++b;
  return b;
}

int inv_mod(int a, int m) {  // a^-1 mod m (gcd(a, m) = 1)
  int t = 0, nt = 1, r = m, nr = a % m;
  while (nr) {
    const int q = r / nr;
    int x = t - q * nt;
    t = nt;
    nt = x;
    x = r - q * nr;
    r = nr;
    nr = x;
  }
  return t < 0 ? t + m : t;
}

CrtConsts make_crt(int n) {
  CrtConsts c;
  std::memset(&c, 0, sizeof(c));
  c.n = n;
  const unsigned __int128 M = crt_M(n);
  for (int i = 0; i < n; ++i) {
    const int m = kModuli[i];
    const unsigned __int128 Mi = M / (unsigned)m;
    const int y = inv_mod((int)(Mi % (unsigned)m), m);
    const unsigned __int128 ci = (Mi * (unsigned)y) % M;
    c.m[i] = m;
    c.inv_m[i] = 1.0f / (float)m;
    c.c_lo[i] = (unsigned long long)ci;
    c.c_hi[i] = (unsigned long long)(ci >> 64);
  }
  c.M_lo = (unsigned long long)M;
  c.M_hi = (unsigned long long)(M >> 64);
  c.Mh_lo = (unsigned long long)(M >> 1);
  c.Mh_hi = (unsigned long long)(M >> 65);
  c.q_scale = (float)(18446744073709551616.0 / (double)M);
  return c;
}

// 2^12, 2^24 and 2^36 mod m_i for the residue kernel (constant memory, once per device)
cudaError_t upload_crt_table() {
  float tab[kMaxModuli][3];
  for (int i = 0; i < kMaxModuli; ++i) {
    const long long m = kModuli[i];
    for (int j = 0; j < 3; ++j) tab[i][j] = (float)((1LL << (12 * (j + 1))) % m);
  }
  return cudaMemcpyToSymbol(c_pow12, tab, sizeof(tab));
}

cudaError_t launch_slice(const double2 *src, long long lds, int K, const double *urow, int s, int planes,
                         __nv_bfloat16 *dst, long long ldk, long long plane_stride, int *expo, int ncols,
                         cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  slice_kernel<<<ncols, 256, 0, st>>>(src, lds, K, urow, s, planes, dst, ldk, ncols, plane_stride, expo);
  return cudaGetLastError();
}

struct SplitWs {
  __nv_bfloat16 *Wsl, *Xsl, *Ysl;
  int *expW, *expX, *expY;
  long long ldk;
  size_t bytes;
};

SplitWs split_ws_layout(void *base, int n_g, int depth, int s) {
  SplitWs w;
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t r = o;
    o += (b + 1023) / 1024 * 1024;
    return r;
  };
  w.ldk = round_up(std::max(depth, 1), BK);
  size_t plane = (size_t)n_g * w.ldk * sizeof(__nv_bfloat16);
  size_t oW = take(plane * 3 * s), oX = take(plane * 3 * s), oY = take(plane * 2 * s);
  size_t oe = take(sizeof(int) * 3 * (size_t)n_g);
  w.bytes = o;
  char *b = (char *)base;
  w.Wsl = (__nv_bfloat16 *)(b + oW);
  w.Xsl = (__nv_bfloat16 *)(b + oX);
  w.Ysl = (__nv_bfloat16 *)(b + oY);
  w.expW = (int *)(b + oe);
  w.expX = w.expW + n_g;
  w.expY = w.expX + n_g;
  return w;
}

// Tiles of one triangle, in bands of `band` column blocks: within a band all
// row blocks in order, so the ~one wave of tiles that runs at a time shares a
// few A row blocks and `band` B column blocks through L2.
std::vector<int2> tri_tiles(int n, int uplo, int band, int bn = BN) {
  const int kBand = std::max(1, band);
  const int nbm = (n + BMT - 1) / BMT, nbn = (n + bn - 1) / bn;
  std::vector<int2> out;
  for (int b0 = 0; b0 < nbn; b0 += kBand) {
    const int b1 = std::min(nbn, b0 + kBand);
    for (int bi = 0; bi < nbm; ++bi)
      for (int bj = b0; bj < b1; ++bj) {
        const bool valid = (uplo == 'U') ? (bi * BMT <= bj * bn + bn - 1) : (bi * BMT + BMT - 1 >= bj * bn);
        if (valid) out.push_back(make_int2(bi, bj));
      }
  }
  return out;
}

// X_a = T_a W_a for the atoms [a0, a1) (one launch per kMaxProb species).
hsgen_status tapply_split(hsgen_ctx *ctx, int n_g, int a0, int a1, const __nv_bfloat16 *Wsl, long long ldk,
                          const int *expW, double2 *X, long long ldw, int slices, cudaStream_t s) {
  const int row_base = ctx->off[a0];
  std::vector<int> species;
  std::vector<std::pair<int, int>> ranges;
  for (int t = 0; t < (int)ctx->types.size(); ++t) {
    const auto &lst = ctx->atoms_of_type[t];
    int lo = 0;
    while (lo < (int)lst.size() && lst[lo] < a0) ++lo;
    int hi = lo;
    while (hi < (int)lst.size() && lst[hi] < a1) ++hi;
    if (hi > lo) {
      species.push_back(t);
      ranges.push_back({lo, hi});
    }
  }
  for (size_t b0 = 0; b0 < species.size(); b0 += kMaxProb) {
    GemmParams P;
    std::memset(&P, 0, sizeof(P));
    P.s = slices;
    P.status = ctx->d_status;
    P.timeout_ns = (unsigned long long)ctx->opt.wait_timeout_ns;
    long long tiles = 0;
    int np = 0;
    for (size_t b = b0; b < species.size() && np < kMaxProb; ++b, ++np) {
      const Species &sp = ctx->types[species[b]];
      GemmProblem &pr = P.prob[np];
      pr.M = sp.dpad;
      pr.N = n_g;
      pr.K = sp.t_kspan;
      pr.kb_begin = 0;
      pr.a_pps = 2;
      pr.b_pps = 3;
      pr.a_real = sp.t_real;
      pr.uplo = 0;
      pr.accumulate = 0;
      pr.F = fixed_point_bits(sp.t_kspan);
      pr.expA = sp.d_Texp;
      pr.expB = expW;
      pr.C = X;
      pr.ldc = ldw;
      pr.atoms = ctx->d_atoms_by_type + ctx->atoms_by_type_start[species[b]] + ranges[b].first;
      pr.off = ctx->d_off;
      pr.row_base = row_base;
      pr.n_batch = ranges[b].second - ranges[b].first;
      pr.nbm = (sp.dpad + BMT - 1) / BMT;
      pr.nbn = (n_g + BN - 1) / BN;
      pr.tile_list = nullptr;
      pr.tile_begin = tiles;
      tiles += (long long)pr.n_batch * pr.nbm * pr.nbn;
      pr.a_nkb = sp.t_kspan / BK;
      pr.b_nkb = (int)(ldk / BK);
      pr.a_shift_planes = 2 * slices;
      if (!make_map(&P.mapA[np], sp.d_Tsl, pr.a_nkb, sp.dpad, 2LL * slices * kTShifts, BM) ||
          !make_map(&P.mapB[np], Wsl, pr.b_nkb, n_g, 3LL * slices, BN))
        return set_err(ctx, HSGEN_ECUDA, "split: cuTensorMapEncodeTiled failed (T-apply)");
    }
    P.nprob = np;
    P.ntiles = tiles;
    HSG_LAUNCH(ctx, launch_gemm(P, s));
  }
  return HSGEN_OK;
}

// One H problem (H = W^H X) and one S problem (S = (U W)^H W) of one k-point
// over the depth segment [kb0, kb0 + seg) of 64-deep blocks; S == nullptr:
// the H problem only (S is built in the Legendre form).
bool hs_problems(GemmProblem *pr, CUtensorMap *mA, CUtensorMap *mB, int n_g, long long ldk, int kb0, int seg,
                 bool accumulate, int uplo, const __nv_bfloat16 *Wsl, const __nv_bfloat16 *Xsl,
                 const __nv_bfloat16 *Ysl, const int *expW, const int *expX, const int *expY, double2 *H, double2 *S,
                 long long ld, const int2 *tiles, long long ntiles, long long tile_begin, int slices, bool gram) {
  // gram (HPD route, X = C^H W): H = X^H X, X's planes on both sides; S unchanged
  const __nv_bfloat16 *Wsl0 = Wsl;
  const int *expW0 = expW;
  if (gram) {
    Wsl = Xsl;
    expW = expX;
  }
  for (int k = 0; k < (S ? 2 : 1); ++k) {
    GemmProblem &q = pr[k];
    std::memset(&q, 0, sizeof(q));
    q.M = n_g;
    q.N = n_g;
    q.K = seg * BK;
    q.kb_begin = kb0;
    q.a_pps = (k == 0) ? 3 : 2;
    q.b_pps = 3;
    q.a_real = 0;
    q.uplo = uplo;
    q.accumulate = (accumulate || kb0 > 0) ? 1 : 0;
    q.F = fixed_point_bits(seg * BK);
    q.expA = (k == 0) ? expW : expY;
    q.expB = (k == 0) ? expX : expW0;
    q.C = (k == 0) ? H : S;
    q.ldc = ld;
    q.n_batch = 1;
    q.nbm = (n_g + BMT - 1) / BMT;
    q.nbn = (n_g + BN - 1) / BN;
    q.tile_list = tiles;
    q.tile_begin = tile_begin + k * ntiles;
    q.a_nkb = q.b_nkb = (int)(ldk / BK);
    const void *a = (k == 0) ? (const void *)Wsl : (const void *)Ysl;
    const void *b = (k == 0) ? (const void *)Xsl : (const void *)Wsl0;
    if (!make_map(&mA[k], a, q.a_nkb, n_g, (long long)q.a_pps * slices, BM) ||
        !make_map(&mB[k], b, q.b_nkb, n_g, 3LL * slices, BN))
      return false;
  }
  return true;
}

// Moduli form, one H problem (H = W^H X) and one S problem (S = (U W)^H W)
// over the depth segment [kb0, kb0 + seg): residue planes per modulus W 3,
// X 3, U W 2; the residue store holds the H tiles' slots, then the S tiles'.
bool crt_problems(GemmProblem *pr, CUtensorMap *mA, CUtensorMap *mB, int n_g, long long ldk, int kb0, int seg,
                  int nkb_all, bool accumulate, int uplo, const __nv_bfloat16 *Wr, const __nv_bfloat16 *Xr,
                  const __nv_bfloat16 *Yr, const int *expW, const int *expX, const int *expY, double2 *H, double2 *S,
                  long long ld, const int2 *tiles, long long ntiles, long long tile_begin, long long slot0,
                  long long slots_per_matrix, unsigned char *store, int nmod, int bits, bool gram) {
  for (int k = 0; k < (S ? 2 : 1); ++k) {
    GemmProblem &q = pr[k];
    std::memset(&q, 0, sizeof(q));
    q.M = n_g;
    q.N = n_g;
    q.K = seg * BK;
    q.kb_begin = kb0;
    q.a_pps = (k == 0) ? 3 : 2;
    q.b_pps = 3;
    q.uplo = uplo;
    q.accumulate = accumulate ? 1 : 0;
    q.F = 2 * bits;
    // gram (HPD route, X = C^H W): H = X^H X, X's residues on both sides
    q.expA = (k == 0) ? (gram ? expX : expW) : expY;
    q.expB = (k == 0) ? expX : expW;
    q.C = (k == 0) ? H : S;
    q.ldc = ld;
    q.n_batch = 1;
    q.nbm = (n_g + BMT - 1) / BMT;
    q.nbn = (n_g + BNC - 1) / BNC;
    q.tile_list = tiles;
    q.tile_begin = tile_begin + k * ntiles;
    q.a_nkb = q.b_nkb = (int)(ldk / BK);
    q.res = store;
    q.res_base = k * slots_per_matrix + slot0;
    q.seg_first = kb0 == 0;
    q.seg_last = kb0 + seg >= nkb_all;
    const void *a = (k == 0) ? (gram ? (const void *)Xr : (const void *)Wr) : (const void *)Yr;
    const void *b = (k == 0) ? (const void *)Xr : (const void *)Wr;
    if (!make_map(&mA[k], a, q.a_nkb, n_g, (long long)q.a_pps * nmod, BM) ||
        !make_map(&mB[k], b, q.b_nkb, n_g, 3LL * nmod, BNC))
      return false;
  }
  return true;
}

long long crt_tile_count(int n, int uplo) {
  // BNC-wide tiles of one triangle (the band only reorders them)
  return (long long)tri_tiles(n, uplo, 1 << 20, BNC).size();
}

struct CrtWs {
  __nv_bfloat16 *Wr, *Xr, *Yr;
  int *expW, *expX, *expY;
  unsigned char *store;
  long long ldk;
  size_t bytes;
};

CrtWs crt_ws_layout(void *base, int n_g, int depth, int nmod, long long slots) {
  CrtWs w;
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t r = o;
    o += (b + 1023) / 1024 * 1024;
    return r;
  };
  w.ldk = round_up(std::max(depth, 1), BK);
  const size_t plane = (size_t)n_g * w.ldk * sizeof(__nv_bfloat16);
  const size_t oW = take(plane * 3 * nmod), oX = take(plane * 3 * nmod), oY = take(plane * 2 * nmod);
  const size_t oe = take(sizeof(int) * 3 * (size_t)n_g);
  const size_t os = take((size_t)slots * nmod * 65536);
  w.bytes = o;
  char *b = (char *)base;
  w.Wr = (__nv_bfloat16 *)(b + oW);
  w.Xr = (__nv_bfloat16 *)(b + oX);
  w.Yr = (__nv_bfloat16 *)(b + oY);
  w.expW = (int *)(b + oe);
  w.expX = w.expW + n_g;
  w.expY = w.expX + n_g;
  w.store = (unsigned char *)(b + os);
  return w;
}

}  // namespace

int choose_moduli(double target_rel_err, int override_moduli, long long K) {
  if (override_moduli > 0) return std::max(kMinModuli, std::min(override_moduli, kMaxModuli));
  for (int n = kMinModuli; n <= kMaxModuli; ++n)
    if (kCrtErr * std::sqrt(2.0 * (double)std::max(K, 1LL)) * std::ldexp(1.0, -crt_bits(n)) <= target_rel_err)
      return n;
  return 0;
}

SplitPlan split_plan(const hsgen_ctx *ctx, int depth) {
  SplitPlan p;
  p.slices = choose_slices(ctx->opt.target_rel_err, ctx->opt.slices);
  p.scheme = kSchemeSlices;
  p.nmod = 0;
  p.bits = 0;
  const int want = ctx->opt.scheme;
  if (want == HSGEN_SCHEME_MODULI || (want == HSGEN_SCHEME_AUTO && ctx->opt.slices == 0)) {
    int n = choose_moduli(ctx->opt.target_rel_err, ctx->opt.moduli, depth);
    if (n == 0 && want == HSGEN_SCHEME_MODULI) n = kMaxModuli;
    if (n > 0) {
      p.scheme = kSchemeModuli;
      p.nmod = n;
      p.bits = crt_bits(n);
    }
  }
  return p;
}

cudaError_t split_upload_tables() { return upload_crt_table(); }

int choose_slices(double target_rel_err, int override_slices) {
  if (override_slices > 0) return std::min(override_slices, kMaxSlices);
  // relative Frobenius error observed per slice count on coefficient data,
  // with a factor ~3 of margin (8 bits per slice)
  static const double err[kMaxSlices + 1] = {1, 1, 1, 5e-6, 3e-8, 1e-10, 5e-13, 3e-15};
  for (int s = 3; s <= kMaxSlices; ++s)
    if (err[s] <= target_rel_err) return s;
  return kMaxSlices;
}

// ---------------------------------------------------------------------------
// Generic C (+)= (+-) P^H Q in the split form (used by the eigenproblem
// reduction): P is K x M, Q is K x N, complex column-major; C is M x N.
// ---------------------------------------------------------------------------
namespace {

struct GemmWs {
  __nv_bfloat16 *Psl, *Qsl;
  int *expP, *expQ;
  double *neg;
  int2 *tiles;
  size_t bytes;
};

GemmWs gemm_ws_layout(void *base, int M, int N, int K, int slices) {
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t ldk = (size_t)((K + BK - 1) / BK) * BK;
  const size_t nbm = (M + BMT - 1) / BMT, nbn = (N + BN - 1) / BN;
  char *b = (char *)base;
  GemmWs w;
  size_t o = 0;
  w.Psl = (__nv_bfloat16 *)(b + o);
  o += al(sizeof(__nv_bfloat16) * 2 * slices * (size_t)M * ldk);
  w.Qsl = (__nv_bfloat16 *)(b + o);
  o += al(sizeof(__nv_bfloat16) * 3 * slices * (size_t)N * ldk);
  w.expP = (int *)(b + o);
  o += al(sizeof(int) * (size_t)M);
  w.expQ = (int *)(b + o);
  o += al(sizeof(int) * (size_t)N);
  w.neg = (double *)(b + o);
  o += al(sizeof(double) * ldk);
  w.tiles = (int2 *)(b + o);
  o += al(sizeof(int2) * nbm * nbn);
  w.bytes = o;
  return w;
}

}  // namespace

size_t split_gemm_ws_bytes(int M, int N, int K, int slices) {
  return gemm_ws_layout(nullptr, M, N, K, slices).bytes;
}

hsgen_status split_gemm(hsgen_ctx *ctx, int M, int N, int K, const double2 *P, long long ldp, const double2 *Q,
                        long long ldq, double2 *C, long long ldc, int uplo, bool accumulate, bool negate,
                        int slices, void *ws, cudaStream_t s) {
  if (M <= 0 || N <= 0) return HSGEN_OK;
  if (K <= 0 || ldp < K || ldq < K || ldc < M || slices < 1 || slices > kMaxSlices || (uplo && M != N))
    return set_err(ctx, HSGEN_EINVAL, "split_gemm: bad sizes");
  if (!ctx->d_status) {
    HSG_CUDA(ctx, cudaMalloc(&ctx->d_status, sizeof(int)));
    HSG_CUDA(ctx, cudaMallocHost(&ctx->h_status, sizeof(int)));
    HSG_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
  }
  GemmWs w = gemm_ws_layout(ws, M, N, K, slices);
  const long long ldk = (long long)((K + BK - 1) / BK) * BK;
  const double *urow = nullptr;
  if (negate) {
    std::vector<double> minus(ldk, -1.0);
    HSG_CUDA(ctx, cudaMemcpyAsync(w.neg, minus.data(), sizeof(double) * ldk, cudaMemcpyHostToDevice, s));
    urow = w.neg;
  }
  // P as the left operand (planes re, im; negated through the row weights), Q as the right (re, im, -re)
  HSG_LAUNCH(ctx, launch_slice(P, ldp, K, urow, slices, 2, w.Psl, ldk, (long long)M * ldk, w.expP, M, s));
  HSG_LAUNCH(ctx, launch_slice(Q, ldq, K, nullptr, slices, 3, w.Qsl, ldk, (long long)N * ldk, w.expQ, N, s));
  std::vector<int2> tl;
  if (uplo) {
    tl = tri_tiles(M, uplo, 16);
  } else {
    const int nbm = (M + BMT - 1) / BMT, nbn = (N + BN - 1) / BN;
    for (int b0 = 0; b0 < nbn; b0 += 16)
      for (int bi = 0; bi < nbm; ++bi)
        for (int bj = b0; bj < std::min(nbn, b0 + 16); ++bj) tl.push_back(make_int2(bi, bj));
  }
  HSG_CUDA(ctx, cudaMemcpyAsync(w.tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice, s));
  GemmParams G;
  std::memset(&G, 0, sizeof(G));
  G.s = slices;
  G.status = ctx->d_status;
  G.timeout_ns = (unsigned long long)ctx->opt.wait_timeout_ns;
  GemmProblem &q = G.prob[0];
  q.M = M;
  q.N = N;
  q.K = (int)ldk;
  q.kb_begin = 0;
  q.a_pps = 2;
  q.b_pps = 3;
  q.a_real = 0;
  q.uplo = uplo;
  q.accumulate = accumulate ? 1 : 0;
  q.F = fixed_point_bits((int)ldk);
  q.expA = w.expP;
  q.expB = w.expQ;
  q.C = C;
  q.ldc = ldc;
  q.n_batch = 1;
  q.nbm = (M + BMT - 1) / BMT;
  q.nbn = (N + BN - 1) / BN;
  q.tile_list = w.tiles;
  q.tile_begin = 0;
  q.a_nkb = q.b_nkb = (int)(ldk / BK);
  if (!make_map(&G.mapA[0], w.Psl, q.a_nkb, M, 2LL * slices, BM) ||
      !make_map(&G.mapB[0], w.Qsl, q.b_nkb, N, 3LL * slices, BN))
    return set_err(ctx, HSGEN_ECUDA, "split_gemm: cuTensorMapEncodeTiled failed");
  G.nprob = 1;
  G.ntiles = (long long)tl.size();
  HSG_LAUNCH(ctx, launch_gemm(G, s));
  return HSGEN_OK;
}

size_t split_workspace_bytes(const hsgen_ctx *ctx, int n_g, int chunk_depth) {
  const SplitPlan pl = split_plan(ctx, chunk_depth);
  if (pl.scheme == kSchemeModuli)
    return crt_ws_layout(nullptr, n_g, chunk_depth, pl.nmod, 2 * crt_tile_count(n_g, ctx->opt.uplo)).bytes;
  return split_ws_layout(nullptr, n_g, chunk_depth, pl.slices).bytes;
}

hsgen_status split_prepare_types(hsgen_ctx *ctx, int slices) {
  if (!ctx->d_status) {
    HSG_CUDA(ctx, cudaMalloc(&ctx->d_status, sizeof(int)));
    HSG_CUDA(ctx, cudaMallocHost(&ctx->h_status, sizeof(int)));
    HSG_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
  }
  for (auto &sp : ctx->types) {
    if (sp.d_Tsl) cudaFree(sp.d_Tsl);
    if (sp.d_Texp) cudaFree(sp.d_Texp);
    sp.d_Tsl = nullptr;
    sp.d_Texp = nullptr;
    // shifted copies of T (FP64, kspan x dpad each), then their slices
    sp.t_kspan = round_up(sp.dpad + BK - kTShiftStep, BK);
    const size_t span = (size_t)sp.t_kspan * sp.dpad;
    double2 *Tsh = nullptr;
    HSG_CUDA(ctx, cudaMalloc(&Tsh, sizeof(double2) * span * kTShifts));
    HSG_CUDA(ctx, cudaMemset(Tsh, 0, sizeof(double2) * span * kTShifts));
    // (the matrix P of X = P^H W: T, or its Cholesky factor C on the HPD route)
    for (int d = 0; d < kTShifts; ++d)
      HSG_CUDA(ctx, cudaMemcpy2D(Tsh + d * span + kTShiftStep * d, sizeof(double2) * sp.t_kspan, sp.apply_matrix(),
                                 sizeof(double2) * sp.dpad, sizeof(double2) * sp.dpad, sp.dpad,
                                 cudaMemcpyDeviceToDevice));
    HSG_CUDA(ctx, cudaMalloc(&sp.d_Tsl, span * 2 * slices * kTShifts * sizeof(__nv_bfloat16)));
    HSG_CUDA(ctx, cudaMalloc(&sp.d_Texp, sizeof(int) * sp.dpad));
    for (int d = 0; d < kTShifts; ++d)
      HSG_CUDA(ctx, launch_slice(Tsh + d * span, sp.t_kspan, sp.t_kspan, nullptr, slices, 2,
                                 (__nv_bfloat16 *)sp.d_Tsl + d * span * 2 * slices, sp.t_kspan, (long long)span,
                                 sp.d_Texp, sp.dpad, 0));
    HSG_CUDA(ctx, cudaDeviceSynchronize());
    cudaFree(Tsh);
    // does it have an imaginary part?
    std::vector<double2> h((size_t)sp.dpad * sp.dpad);
    HSG_CUDA(ctx, cudaMemcpy(h.data(), sp.apply_matrix(), sizeof(double2) * h.size(), cudaMemcpyDeviceToHost));
    sp.t_real = 1;
    for (auto &v : h)
      if (v.y != 0.0) {
        sp.t_real = 0;
        break;
      }
  }
  HSG_CUDA(ctx, cudaDeviceSynchronize());
  ctx->split_slices = slices;
  return HSGEN_OK;
}

hsgen_status split_chunk(hsgen_ctx *ctx, int n_g, int a0, int a1, const double2 *W, double2 *X, long long ldw,
                         double2 *H, double2 *S, long long ld, bool accumulate, void *ws, int slices,
                         cudaStream_t s, const cudaEvent_t *phase_ev, const CopyOut *co) {
  if (ctx->split_slices != slices) {
    hsgen_status st = split_prepare_types(ctx, slices);
    if (st != HSGEN_OK) return st;
  }
  const int row_base = ctx->off[a0];
  const int cdepth = ctx->off[a1] - row_base;
  const int uplo = ctx->opt.uplo;
  const SplitPlan pl = split_plan(ctx, cdepth);
  const bool crt = pl.scheme == kSchemeModuli;
  ctx->last_plan = pl;
  // moduli form: residue planes and the residue store; slice form: slice planes
  const long long slots = crt ? crt_tile_count(n_g, uplo) : 0;
  const CrtWs cw = crt ? crt_ws_layout(ws, n_g, cdepth, pl.nmod, 2 * slots) : CrtWs{};
  const SplitWs w = crt ? SplitWs{} : split_ws_layout(ws, n_g, cdepth, slices);
  const long long ldk = crt ? cw.ldk : w.ldk;
  int *expW = crt ? cw.expW : w.expW;
  // W's slices for X = T W (in the moduli form they sit in X's residue
  // region, which is written only after X = T W)
  __nv_bfloat16 *Wsl = crt ? cw.Xr : w.Wsl;
  const long long plane = (long long)n_g * ldk;
  const unsigned long long tmo = (unsigned long long)ctx->opt.wait_timeout_ns;
  // (1) W slices: planes re, im, -re (used as the left operand of H and the right of X and S)
  HSG_LAUNCH(ctx, launch_slice(W, ldw, cdepth, nullptr, slices, 3, Wsl, ldk, plane, expW, n_g, s));
  // (2) X_a = T W_a, species by species (up to kMaxProb per launch)
  {
    hsgen_status st = tapply_split(ctx, n_g, a0, a1, Wsl, ldk, expW, X, ldw, slices, s);
    if (st != HSGEN_OK) return st;
  }
  if (phase_ev) HSG_CUDA(ctx, cudaEventRecord(phase_ev[0], s));
  // (3) the operands of the contraction: X (right operand of H), W (left of
  // H, right of S) and U W (left of S), as residues or slices. A pass on the
  // HPD route (Sec. 4.6.2) holds Y = C^H W in X and forms H = Y^H Y: W is then
  // an operand of S only, and without S its residues are not needed.
  const bool gram = ctx->types[ctx->toa[a0]].routed;
  const CrtConsts cc = crt ? make_crt(pl.nmod) : CrtConsts{};
  if (crt) {
    HSG_LAUNCH(ctx, launch_residue(X, ldw, cdepth, nullptr, pl.bits, cc, 3, cw.Xr, ldk, plane, cw.expX, n_g, s));
    if (S)
      HSG_LAUNCH(ctx, launch_residue_w_uw(W, ldw, cdepth, ctx->d_urow + row_base, pl.bits, cc, cw.Wr, cw.expW, cw.Yr,
                                          cw.expY, ldk, plane, n_g, s));
    else if (!gram)
      HSG_LAUNCH(ctx, launch_residue(W, ldw, cdepth, nullptr, pl.bits, cc, 3, cw.Wr, ldk, plane, cw.expW, n_g, s));
  } else {
    HSG_LAUNCH(ctx, launch_slice(X, ldw, cdepth, nullptr, slices, 3, w.Xsl, ldk, plane, w.expX, n_g, s));
    if (S)
      HSG_LAUNCH(ctx, launch_slice(W, ldw, cdepth, ctx->d_urow + row_base, slices, 2, w.Ysl, ldk, plane, w.expY,
                                   n_g, s));
  }
  if (phase_ev) HSG_CUDA(ctx, cudaEventRecord(phase_ev[1], s));
  // (4) H = W^H X and S = (U W)^H W over one triangle
  {
    const int bn = crt ? BNC : BN;
    // tiles in bands of tile_band 64-column blocks (the same width in columns for either tile)
    const int band = crt ? std::max(1, ctx->tile_band * BN / BNC) : ctx->tile_band;
    if (ctx->tiles_n != n_g || ctx->tiles_uplo != uplo || ctx->tiles_band != band || ctx->tiles_bn != bn ||
        !(ctx->tiles_owner == ctx->owner)) {
      std::vector<int2> tl = tri_tiles(n_g, uplo, band, bn);
      if (ctx->owner.block) {  // only the tiles of this process's blocks (a tile lies inside one block)
        std::vector<int2> mine;
        for (const int2 &t : tl)
          if (ctx->owner.owns((long long)t.x * BMT, (long long)t.y * bn)) mine.push_back(t);
        tl.swap(mine);
      }
      if (ctx->d_tiles) cudaFree(ctx->d_tiles);
      ctx->d_tiles = nullptr;
      ctx->tiles_n = -1;
      HSG_CUDA(ctx, cudaMalloc(&ctx->d_tiles, sizeof(int2) * std::max<size_t>(tl.size(), 1)));
      HSG_CUDA(ctx, cudaMemcpy(ctx->d_tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice));
      ctx->tiles_host = tl;
      ctx->tiles_n = n_g;
      ctx->tiles_uplo = uplo;
      ctx->tiles_band = band;
      ctx->tiles_bn = bn;
      ctx->tiles_owner = ctx->owner;
      ctx->tiles_count = (long long)tl.size();
    }
    if (ctx->tiles_count == 0) return HSGEN_OK;
    const int nkb_all = (int)(ldk / BK);
    // moduli form: at most 256 k-blocks per launch (32 chunks of exact FP32
    // sums keep the epilogue's int32 sums below 2^29)
    const int seg_kb = crt ? std::max(1, std::min(ctx->kseg_blocks, 256)) : std::max(1, ctx->kseg_blocks);
    const long long per = ctx->tiles_count;
    // one launch: the tiles [t0, t0 + cnt) of the list, of H (and S), over
    // the depth segment [kb0, kb0 + seg)
    auto launch_seg = [&](long long t0, long long cnt, int kb0) -> hsgen_status {
      const int seg = std::min(seg_kb, nkb_all - kb0);
      GemmParams P;
      std::memset(&P, 0, sizeof(P));
      P.s = slices;
      P.status = ctx->d_status;
      P.timeout_ns = tmo;
      P.nprob = S ? 2 : 1;
      P.ntiles = P.nprob * cnt;
      if (crt) {
        P.crt = cc;
        P.crt_order = ctx->crt_order;
        P.l2_hint = ctx->l2_hint;
        P.recon_apart = ctx->crt_recon_apart;
        if (!crt_problems(P.prob, P.mapA, P.mapB, n_g, ldk, kb0, seg, nkb_all, accumulate, uplo, cw.Wr, cw.Xr,
                          cw.Yr, cw.expW, cw.expX, cw.expY, H, S, ld, (const int2 *)ctx->d_tiles + t0, cnt, 0, t0,
                          slots, cw.store, pl.nmod, pl.bits, gram))
          return set_err(ctx, HSGEN_ECUDA, "split: cuTensorMapEncodeTiled failed (H/S, moduli)");
        HSG_LAUNCH(ctx, launch_crt(P, ctx->crt_geom, s, kb0 + seg >= nkb_all));
        if (P.recon_apart && kb0 + seg >= nkb_all) ++ctx->launches;  // crt_reconstruct_kernel
        return HSGEN_OK;
      }
      if (!hs_problems(P.prob, P.mapA, P.mapB, n_g, ldk, kb0, seg, accumulate, uplo, w.Wsl, w.Xsl, w.Ysl, w.expW,
                       w.expX, w.expY, H, S, ld, (const int2 *)ctx->d_tiles + t0, cnt, 0, slices, gram))
        return set_err(ctx, HSGEN_ECUDA, "split: cuTensorMapEncodeTiled failed (H/S)");
      HSG_LAUNCH(ctx, launch_gemm(P, s));
      return HSGEN_OK;
    };
    if (!co || (!co->H && !(S && co->S))) {
      // The depth is cut into segments run as separate launches that add into
      // H and S (slices) or into the residue store (moduli): shorter tiles keep
      // the CTAs of one wave close together in k, so the A and B blocks they
      // share stay in L2.
      for (int kb0 = 0; kb0 < nkb_all; kb0 += seg_kb) {
        hsgen_status st = launch_seg(0, per, kb0);
        if (st != HSGEN_OK) return st;
      }
      return HSGEN_OK;
    }
    // Host outputs: the same launches in column-band-group-major order (all
    // depth segments of one group of whole bands, at least a few waves of
    // tiles, then the next), so a group's finished columns go to the host on
    // the copy stream while the later groups compute.
    if (!ctx->copy_stream) HSG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    if (!ctx->copy_ev) HSG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->copy_ev, cudaEventDisableTiming));
    const long long min_tiles = 4 * max_pairs();
    const int bandw = std::max(1, ctx->tiles_band);
    const std::vector<int2> &tl = ctx->tiles_host;
    if ((long long)tl.size() != per) return set_err(ctx, HSGEN_EINVAL, "split: tile list out of date");
    for (long long t0 = 0; t0 < per;) {
      long long t1 = t0;
      while (t1 < per) {
        const int band = tl[t1].y / bandw;
        while (t1 < per && tl[t1].y / bandw == band) ++t1;
        if (t1 - t0 >= min_tiles) break;
      }
      for (int kb0 = 0; kb0 < nkb_all; kb0 += seg_kb) {
        hsgen_status st = launch_seg(t0, t1 - t0, kb0);
        if (st != HSGEN_OK) return st;
      }
      // the group holds every tile of columns [c0, c1)
      const long long c0 = (long long)(tl[t0].y / bandw) * bandw * bn;
      const long long c1 = std::min<long long>(n_g, (long long)(tl[t1 - 1].y / bandw + 1) * bandw * bn);
      HSG_CUDA(ctx, cudaEventRecord(ctx->copy_ev, s));
      HSG_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_ev, 0));
      for (int k = 0; k < 2; ++k) {
        void *dst = (k == 0) ? co->H : (S ? co->S : nullptr);
        const double2 *src = (k == 0) ? H : S;
        if (dst)
          HSG_CUDA(ctx, cudaMemcpyAsync((double2 *)dst + c0 * ld, src + c0 * ld, sizeof(double2) * (c1 - c0) * ld,
                                        cudaMemcpyDeviceToHost, ctx->copy_stream));
      }
      t0 = t1;
    }
  }
  return HSGEN_OK;
}

hsgen_status split_join_copies(hsgen_ctx *ctx, cudaStream_t s) {
  if (!ctx->copy_stream) return HSGEN_OK;
  HSG_CUDA(ctx, cudaEventRecord(ctx->copy_ev, ctx->copy_stream));
  HSG_CUDA(ctx, cudaStreamWaitEvent(s, ctx->copy_ev, 0));
  return HSGEN_OK;
}

hsgen_status split_post_status(hsgen_ctx *ctx, cudaStream_t s) {
  if (!ctx->d_status) return HSGEN_OK;
  if (!ctx->status_ev) HSG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->status_ev, cudaEventDisableTiming));
  HSG_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  HSG_CUDA(ctx, cudaEventRecord(ctx->status_ev, s));
  ctx->status_pending = true;
  return HSGEN_OK;
}

hsgen_status split_poll_status(hsgen_ctx *ctx, bool wait) {
  if (!ctx->status_pending) return HSGEN_OK;
  if (wait) {
    HSG_CUDA(ctx, cudaEventSynchronize(ctx->status_ev));
  } else {
    const cudaError_t e = cudaEventQuery(ctx->status_ev);
    if (e == cudaErrorNotReady) {
      cudaGetLastError();
      return HSGEN_OK;
    }
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaEventQuery(status word)");
  }
  ctx->status_pending = false;
  const int st = *ctx->h_status;
  if (st != 0) {
    *ctx->h_status = 0;
    // error path only: clear the word before any later launch can read it
    HSG_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
    HSG_CUDA(ctx, cudaDeviceSynchronize());
    return set_err(ctx, HSGEN_ETIMEOUT,
                   "split kernel: a bounded device wait expired (status " + std::to_string(st) +
                       "); the results of the call that launched it are invalid");
  }
  return HSGEN_OK;
}

hsgen_status split_check_status(hsgen_ctx *ctx, cudaStream_t s) {
  hsgen_status st = split_post_status(ctx, s);
  if (st != HSGEN_OK) return st;
  return split_poll_status(ctx, true);
}

// Many k-points (one H, S per k-point, Sec. 2.3): per k-point the cheap steps (radial factors,
// coefficients, slicing, X = T W) fill that k-point's slice buffers; then one
// persistent grouped launch per depth segment runs the H and S tiles of every
// k-point of a group (uneven N_G and mixed l_max share one tile queue). The
// whole kernel sequence is captured once into a CUDA graph and replayed while
// the batch (sizes and output pointers) stays the same.
hsgen_status split_batched(hsgen_ctx *ctx, int n_k, const int *n_g, const double *const *kvec, void *const *H,
                           void *const *S, const long long *ld, cudaStream_t s) {
  if (ctx->opt.precision != HSGEN_SPLIT) return HSGEN_ENOTSUP;
  const int na = (int)ctx->toa.size();
  if (ctx->opt.atom_chunk > 0 && ctx->opt.atom_chunk < na) return HSGEN_ENOTSUP;
  if (!ctx->have_system) return set_err(ctx, HSGEN_EINVAL, "build_HS_batched: no system set");
  if (ctx->opt.fill_full) return HSGEN_ENOTSUP;
  // one pass over all atoms: every species on one H route (HPD route: H = Y^H Y)
  const bool gram = ctx->types[ctx->toa[0]].routed;
  for (const auto &sp : ctx->types)
    if (sp.routed != gram) return HSGEN_ENOTSUP;
  for (int k = 0; k < n_k; ++k) {
    if (n_g[k] < 0 || ld[k] < n_g[k] || (n_g[k] > 0 && (!kvec[k] || !H[k] || !S[k])))
      return set_err(ctx, HSGEN_EINVAL, "build_HS_batched: bad size, leading dimension or pointer");
    if (n_g[k] > 0) {
      for (int i = 0; i < 3 * n_g[k]; ++i)
        if (!std::isfinite(kvec[k][i])) return set_err(ctx, HSGEN_ENUMERIC, "build_HS_batched: non-finite kvec");
    }
  }
  const int slices = choose_slices(ctx->opt.target_rel_err, ctx->opt.slices);
  // the form of the whole batch (every k-point has the same depth)
  const SplitPlan pl = split_plan(ctx, ctx->depth);
  const bool crt = pl.scheme == kSchemeModuli;
  const int units = crt ? pl.nmod : slices;  // planes per operand part: moduli or slices
  const CrtConsts cc = crt ? make_crt(pl.nmod) : CrtConsts{};
  const int bn = crt ? BNC : BN;
  const int tband = crt ? std::max(1, ctx->tile_band * BN / BNC) : ctx->tile_band;
  ctx->last_plan = pl;
  if (ctx->split_slices != slices) {
    hsgen_status st = split_prepare_types(ctx, slices);
    if (st != HSGEN_OK) return st;
  }
  HSG_CUDA(ctx, gemm_attrs());
  // S in the Legendre form: every k-point must lie on its lattice k + G
  // (otherwise the caller's k-point loop takes over, per k-point)
  const bool leg = ctx->opt.s_form == HSGEN_S_LEGENDRE;
  std::vector<LegendrePlan> plans(leg ? n_k : 0);
  for (int k = 0; k < (leg ? n_k : 0); ++k)
    if (n_g[k] > 0 && !legendre_plan(ctx, n_g[k], kvec[k], plans[k])) return HSGEN_ENOTSUP;
  const int depth = ctx->depth;
  const long long ldk = round_up(depth, BK);
  const int nt = (int)ctx->types.size();
  const int uplo = ctx->opt.uplo;
  const int nkb_all = (int)(ldk / BK);
  const int seg_kb = crt ? std::max(1, std::min(ctx->kseg_blocks, 256)) : std::max(1, ctx->kseg_blocks);
  const int nseg = (nkb_all + seg_kb - 1) / seg_kb;
  auto al = [](size_t b) { return (b + 1023) / 1024 * 1024; };
  // ---- plan: groups of k-points whose slices fit the budget
  // slices: groups of k-points up to 96 GiB of planes share each launch;
  // moduli: up to 12 GiB of residue planes and stores (about three k-points
  // of N_G ~3300: 6.02 ms per k-point against 6.21 with one k-point and 6.15
  // with eleven per launch)
  size_t budget = (size_t)(crt ? 12 : 96) << 30;
  if (const char *e = std::getenv("HSGEN_BATCH_BYTES")) budget = (size_t)std::max(1.0, std::atof(e));
  // per k-point: 8 planes per slice or modulus (W 3, X 3, U W 2), and in the
  // moduli form its residue store (H and S tiles)
  std::vector<size_t> kslice(n_k), kstore(n_k, 0);
  std::vector<long long> kslots(n_k, 0);
  int max_ng = 1;
  long long sum_ng = 0;
  for (int k = 0; k < n_k; ++k) {
    kslice[k] = al((size_t)8 * units * n_g[k] * ldk * sizeof(__nv_bfloat16));
    if (crt && n_g[k] > 0) {
      kslots[k] = crt_tile_count(n_g[k], uplo);
      kstore[k] = al((size_t)2 * kslots[k] * pl.nmod * 65536);
      kslice[k] += kstore[k];
    }
    max_ng = std::max(max_ng, n_g[k]);
    sum_ng += n_g[k];
  }
  std::vector<std::pair<int, int>> groups;
  for (int k = 0; k < n_k;) {
    size_t acc = 0;
    int k1 = k;
    while (k1 < n_k && (k1 == k || acc + kslice[k1] <= budget)) acc += kslice[k1++];
    groups.push_back({k, k1});
    k = k1;
  }
  // ---- tile lists per k-point (host) and table sizes
  std::vector<std::vector<int2>> tl(n_k);
  size_t n_tl = 0;
  for (int k = 0; k < n_k; ++k) {
    if (n_g[k] > 0) tl[k] = tri_tiles(n_g[k], uplo, tband, bn);
    n_tl += tl[k].size();
  }
  // ---- workspace layout
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t r = o;
    o += al(b);
    return r;
  };
  const size_t o_kv = take(sizeof(double) * 3 * (size_t)std::max<long long>(sum_ng, 1));
  // radial factors: one scratch reused k-point by k-point, or (Legendre form,
  // which reads them after the group's contraction) one region per k-point
  const size_t o_F = take(sizeof(double2) * (size_t)nt * (leg ? (size_t)std::max<long long>(sum_ng, 1) : max_ng) *
                          kRadStride);
  const size_t o_W = take(sizeof(double2) * (size_t)depth * max_ng);
  const size_t o_X = take(sizeof(double2) * (size_t)depth * max_ng);
  size_t max_group = 0;
  for (auto &g : groups) {
    size_t b = 0;
    for (int k = g.first; k < g.second; ++k) b += kslice[k];
    max_group = std::max(max_group, b);
  }
  const size_t o_sl = take(max_group);
  const size_t o_exp = take(sizeof(int) * 3 * (size_t)std::max<long long>(sum_ng, 1));
  const size_t o_tl = take(sizeof(int2) * std::max<size_t>(n_tl, 1));
  std::vector<size_t> o_leg(leg ? n_k : 0);
  for (int k = 0; k < (leg ? n_k : 0); ++k)
    if (n_g[k] > 0) o_leg[k] = take(legendre_ws_bytes(ctx, n_g[k], plans[k]));
  const size_t n_tab = (size_t)2 * n_k * nseg;  // problems over all groups and segments
  const size_t o_prob = take(sizeof(GemmProblem) * n_tab);
  const size_t o_map = take(sizeof(CUtensorMap) * 2 * n_tab);
  const size_t total = o;
  if (ctx->ws_batch.bytes < total) {
    if (ctx->batch_exec) cudaGraphExecDestroy(ctx->batch_exec);
    ctx->batch_exec = nullptr;
    ctx->batch_key.clear();
    if (ctx->ws_batch.ptr) cudaFree(ctx->ws_batch.ptr);
    ctx->ws_batch.ptr = nullptr;
    ctx->ws_batch.bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->ws_batch.ptr, total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_err(ctx, e, "cudaMalloc(batched workspace)");
    }
    ctx->ws_batch.bytes = total;
  }
  char *ws = (char *)ctx->ws_batch.ptr;
  double *d_kv = (double *)(ws + o_kv);
  double2 *F = (double2 *)(ws + o_F), *W = (double2 *)(ws + o_W), *X = (double2 *)(ws + o_X);
  int *d_exp = (int *)(ws + o_exp);
  int2 *d_tl = (int2 *)(ws + o_tl);
  GemmProblem *d_prob = (GemmProblem *)(ws + o_prob);
  CUtensorMap *d_map = (CUtensorMap *)(ws + o_map);
  // ---- per k-point offsets
  std::vector<long long> kv_off(n_k + 1, 0), tl_off(n_k + 1, 0);
  for (int k = 0; k < n_k; ++k) {
    kv_off[k + 1] = kv_off[k] + n_g[k];
    tl_off[k + 1] = tl_off[k] + (long long)tl[k].size();
  }
  auto slice_base = [&](int k, int g) {
    size_t b = 0;
    for (int j = groups[g].first; j < k; ++j) b += kslice[j];
    return (__nv_bfloat16 *)(ws + o_sl + b);
  };
  // ---- uploads (outside any capture): k vectors, tile lists, problem/map tables
  for (int k = 0; k < n_k; ++k)
    if (n_g[k] > 0)
      HSG_CUDA(ctx, cudaMemcpyAsync(d_kv + 3 * kv_off[k], kvec[k], sizeof(double) * 3 * n_g[k],
                                    cudaMemcpyHostToDevice, s));
  std::vector<int2> tl_all;
  tl_all.reserve(n_tl);
  for (int k = 0; k < n_k; ++k) tl_all.insert(tl_all.end(), tl[k].begin(), tl[k].end());
  if (n_tl) HSG_CUDA(ctx, cudaMemcpyAsync(d_tl, tl_all.data(), sizeof(int2) * n_tl, cudaMemcpyHostToDevice, s));
  std::vector<GemmProblem> hprob(n_tab);
  std::vector<CUtensorMap> hmap(2 * n_tab);
  std::vector<long long> launch_tiles;  // per (group, segment)
  std::vector<size_t> launch_first;     // first problem index per (group, segment)
  std::vector<int> launch_nprob;
  size_t pi = 0;
  for (size_t gi = 0; gi < groups.size(); ++gi)
    for (int sg = 0; sg < nseg; ++sg) {
      const int kb0 = sg * seg_kb, seg = std::min(seg_kb, nkb_all - kb0);
      launch_first.push_back(pi);
      long long tiles = 0;
      int np = 0;
      for (int k = groups[gi].first; k < groups[gi].second; ++k) {
        if (n_g[k] <= 0) continue;
        const long long plane = (long long)n_g[k] * ldk;
        __nv_bfloat16 *Wsl = slice_base(k, (int)gi), *Xsl = Wsl + 3 * units * plane, *Ysl = Xsl + 3 * units * plane;
        unsigned char *store = (unsigned char *)slice_base(k, (int)gi) + (kslice[k] - kstore[k]);
        int *eW = d_exp + 3 * kv_off[k], *eX = eW + n_g[k], *eY = eX + n_g[k];
        GemmProblem pr2[2];
        CUtensorMap ma[2], mb[2];
        const long long nt_k = (long long)tl[k].size();
        const bool ok =
            crt ? crt_problems(pr2, ma, mb, n_g[k], ldk, kb0, seg, nkb_all, false, uplo, Wsl, Xsl, Ysl, eW, eX, eY,
                               (double2 *)H[k], leg ? nullptr : (double2 *)S[k], ld[k], d_tl + tl_off[k], nt_k,
                               tiles, 0, kslots[k], store, pl.nmod, pl.bits, gram)
                : hs_problems(pr2, ma, mb, n_g[k], ldk, kb0, seg, false, uplo, Wsl, Xsl, Ysl, eW, eX, eY,
                              (double2 *)H[k], leg ? nullptr : (double2 *)S[k], ld[k], d_tl + tl_off[k], nt_k, tiles,
                              slices, gram);
        if (!ok) return set_err(ctx, HSGEN_ECUDA, "batched: cuTensorMapEncodeTiled failed");
        const int np_k = leg ? 1 : 2;  // H (and S) of this k-point
        for (int j = 0; j < np_k; ++j) {
          hprob[pi] = pr2[j];
          hmap[2 * pi] = ma[j];
          hmap[2 * pi + 1] = mb[j];
          ++pi;
          ++np;
        }
        tiles += np_k * nt_k;
      }
      launch_tiles.push_back(tiles);
      launch_nprob.push_back(np);
    }
  if (pi) {
    HSG_CUDA(ctx, cudaMemcpyAsync(d_prob, hprob.data(), sizeof(GemmProblem) * pi, cudaMemcpyHostToDevice, s));
    HSG_CUDA(ctx, cudaMemcpyAsync(d_map, hmap.data(), sizeof(CUtensorMap) * 2 * pi, cudaMemcpyHostToDevice, s));
  }
  // ---- the kernel sequence, captured once
  for (int k = 0; k < (leg ? n_k : 0); ++k)
    if (n_g[k] > 0) {
      hsgen_status st = legendre_upload(ctx, n_g[k], plans[k], ws + o_leg[k], s);
      if (st != HSGEN_OK) return st;
    }
  std::vector<long long> key = {(long long)(uintptr_t)ws, (long long)slices, (long long)pl.scheme, (long long)pl.nmod,
                                (long long)uplo, (long long)n_k,
                                (long long)ctx->kseg_blocks, (long long)ctx->tile_band, (long long)leg};
  for (int k = 0; k < n_k; ++k) {
    key.push_back(n_g[k]);
    key.push_back(ld[k]);
    if (leg)  // the captured launches carry each k-point's table extents
      for (int j = 0; j < 3; ++j) key.push_back(plans[k].span[j]);
    key.push_back((long long)(uintptr_t)H[k]);
    key.push_back((long long)(uintptr_t)S[k]);
  }
  if (!(ctx->batch_exec && ctx->batch_key == key)) {
    if (ctx->batch_exec) cudaGraphExecDestroy(ctx->batch_exec);
    ctx->batch_exec = nullptr;
    ctx->batch_key.clear();
    // Captured on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph then runs on the caller's.
    if (!ctx->capture_stream)
      HSG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    const cudaStream_t caller = s;
    s = ctx->capture_stream;
    HSG_CUDA(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    hsgen_status st = HSGEN_OK;
    ctx->launches = 0;
    auto body = [&]() -> hsgen_status {
      for (size_t gi = 0; gi < groups.size(); ++gi) {
        for (int k = groups[gi].first; k < groups[gi].second; ++k) {
          const int ng = n_g[k];
          if (ng <= 0) continue;
          const double *kd = d_kv + 3 * kv_off[k];
          const long long plane = (long long)ng * ldk;
          __nv_bfloat16 *Wsl = slice_base(k, (int)gi), *Xsl = Wsl + 3 * units * plane,
                        *Ysl = Xsl + 3 * units * plane;
          int *eW = d_exp + 3 * kv_off[k], *eX = eW + ng, *eY = eX + ng;
          double2 *Fk = leg ? F + (size_t)nt * kv_off[k] * kRadStride : F;
          HSG_LAUNCH(ctx, launch_radial(ng, kd, nt, ctx->d_radial, Fk, s));
          for (int t = 0; t < nt; ++t) {
            const int n = (int)ctx->atoms_of_type[t].size();
            if (!n) continue;
            HSG_LAUNCH(ctx, launch_coefficients(ctx->types[t].lc, ng, kd, Fk + (size_t)t * ng * kRadStride,
                                                ctx->d_atoms_by_type + ctx->atoms_by_type_start[t], n, ctx->d_pos,
                                                ctx->d_rot, ctx->d_off, 0, ctx->types[t].dpad, W, depth, s));
          }
          // W's slices for X = T W; in the moduli form they sit in X's residue planes, written after
          __nv_bfloat16 *Wfx = crt ? Xsl : Wsl;
          HSG_LAUNCH(ctx, launch_slice(W, depth, depth, nullptr, slices, 3, Wfx, ldk, plane, eW, ng, s));
          hsgen_status st2 = tapply_split(ctx, ng, 0, na, Wfx, ldk, eW, X, depth, slices, s);
          if (st2 != HSGEN_OK) return st2;
          if (crt) {
            HSG_LAUNCH(ctx, launch_residue(X, depth, depth, nullptr, pl.bits, cc, 3, Xsl, ldk, plane, eX, ng, s));
            if (!leg)
              HSG_LAUNCH(ctx, launch_residue_w_uw(W, depth, depth, ctx->d_urow, pl.bits, cc, Wsl, eW, Ysl, eY, ldk,
                                                  plane, ng, s));
            else if (!gram)
              HSG_LAUNCH(ctx, launch_residue(W, depth, depth, nullptr, pl.bits, cc, 3, Wsl, ldk, plane, eW, ng, s));
          } else {
            HSG_LAUNCH(ctx, launch_slice(X, depth, depth, nullptr, slices, 3, Xsl, ldk, plane, eX, ng, s));
            if (!leg)
              HSG_LAUNCH(ctx, launch_slice(W, depth, depth, ctx->d_urow, slices, 2, Ysl, ldk, plane, eY, ng, s));
          }
        }
        for (int sg = 0; sg < nseg; ++sg) {
          const size_t li = gi * nseg + sg;
          if (!launch_nprob[li]) continue;
          GemmParams P;
          std::memset(&P, 0, sizeof(P));
          P.gprob = d_prob + launch_first[li];
          P.gmap = d_map + 2 * launch_first[li];
          P.nprob = launch_nprob[li];
          P.ntiles = launch_tiles[li];
          P.s = slices;
          P.status = ctx->d_status;
          P.timeout_ns = (unsigned long long)ctx->opt.wait_timeout_ns;
          if (crt) {
            P.crt = cc;
            P.crt_order = ctx->crt_order;
            P.l2_hint = ctx->l2_hint;
            P.recon_apart = ctx->crt_recon_apart;
            HSG_LAUNCH(ctx, launch_crt(P, ctx->crt_geom, s, sg == nseg - 1));
            if (P.recon_apart && sg == nseg - 1) ++ctx->launches;  // crt_reconstruct_kernel
          } else {
            HSG_LAUNCH(ctx, launch_gemm(P, s));
          }
        }
        // Legendre form: S, and H's spherical tail added after the contraction wrote H
        for (int k = groups[gi].first; k < groups[gi].second && leg; ++k) {
          if (n_g[k] <= 0) continue;
          hsgen_status st3 = legendre_launch(ctx, n_g[k], d_kv + 3 * kv_off[k],
                                             F + (size_t)nt * kv_off[k] * kRadStride, plans[k], ws + o_leg[k],
                                             (double2 *)S[k], (double2 *)H[k], ld[k], s);
          if (st3 != HSGEN_OK) return st3;
        }
      }
      return HSGEN_OK;
    };
    st = body();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    s = caller;
    if (st != HSGEN_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaStreamEndCapture(batched)");
    e = cudaGraphInstantiate(&ctx->batch_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ctx->batch_exec = nullptr;
      return cuda_err(ctx, e, "cudaGraphInstantiate(batched)");
    }
    ctx->batch_key = key;
    ctx->stats.kernel_launches = ctx->launches;
    s = caller;
  }
  HSG_CUDA(ctx, cudaGraphLaunch(ctx->batch_exec, s));
  ctx->stats.slices = slices;
  ctx->stats.precision = HSGEN_SPLIT;
  ctx->stats.scheme = crt ? HSGEN_SCHEME_MODULI : HSGEN_SCHEME_SLICES;
  ctx->stats.moduli = pl.nmod;
  ctx->stats.bits = pl.bits;
  ctx->stats.products = crt ? pl.nmod : slices * (slices + 1) / 2;
  ctx->stats.atom_chunks = 1;
  ctx->phase_used[0] = 0;
  ctx->phase_used[1] = 0;
  ctx->phase_used[2] = 0;
  ctx->phase_used[3] = 0;
  ctx->stats.s_form = leg ? HSGEN_S_LEGENDRE : HSGEN_S_CONTRACTION;
  return split_post_status(ctx, s);
}

void split_release(hsgen_ctx *ctx) {
  for (auto &sp : ctx->types) {
    if (sp.d_Tsl) cudaFree(sp.d_Tsl);
    if (sp.d_Texp) cudaFree(sp.d_Texp);
    sp.d_Tsl = nullptr;
    sp.d_Texp = nullptr;
  }
  if (ctx->d_tiles) cudaFree(ctx->d_tiles);
  ctx->d_tiles = nullptr;
  ctx->tiles_n = -1;
  if (ctx->batch_exec) cudaGraphExecDestroy(ctx->batch_exec);
  ctx->batch_exec = nullptr;
  ctx->batch_key.clear();
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  ctx->capture_stream = nullptr;
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  ctx->copy_stream = nullptr;
  if (ctx->copy_ev) cudaEventDestroy(ctx->copy_ev);
  ctx->copy_ev = nullptr;
  if (ctx->status_ev) cudaEventDestroy(ctx->status_ev);
  ctx->status_ev = nullptr;
  ctx->status_pending = false;
  if (ctx->ws_batch.ptr) cudaFree(ctx->ws_batch.ptr);
  ctx->ws_batch.ptr = nullptr;
  ctx->ws_batch.bytes = 0;
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  ctx->d_status = nullptr;
  ctx->h_status = nullptr;
}

}  // namespace hsg
