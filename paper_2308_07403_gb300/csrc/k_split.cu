// k_split.cu -- the split-precision path: the big contractions of the inverse as exact BF16
// digit products on the tcgen05 tensor cores, with FP64 kept for the 64x64 diagonal leaves,
// the slicing, the recombination and the decode.
//
// Arithmetic (an Ozaki-style splitting, written from the published scheme of Ozaki, Ogita,
// Oishi and Rump, 2012, adapted to entrywise accuracy):
//   * Each operand is cut into chunks of KAPPA = 256 along K (64 when the graph runs in the
//     locality order, whose 64-node parts are compact).  Every (row, chunk) of A and
//     every (chunk, column) of B gets its own power of two 2^e with |x| 2^-e < 1/2, so a chunk
//     of small entries (far nodes, entries gamma^d) keeps its own scale.
//   * x 2^-e is written in s balanced base-128 digits d_p in [-64, 64] (round to nearest):
//         x = 2^e sum_p d_p 2^(-7 (p+1)) + r,   |r| <= 2^(e - 7 s - 1).
//     Every digit is an integer of at most 7 bits, exact in BF16.
//   * For a chunk, the digit products of equal weight g = p + q (p, q < s, p + q < s) are
//     summed by the tensor core into one FP32 accumulator in tensor memory: every product is
//     an integer of magnitude <= 2^12 and a group holds at most s of them per K entry, so a
//     chunk sum stays below KAPPA * s * 2^12 < 2^24 -- exact -- for s <= 15 with 256-wide
//     chunks and s <= 22 with 64-wide ones.
//   * The epilogue warps read each group sum, scale it by 2^(eA + eB - 7 (g + 2)) relative to a
//     per-entry reference exponent (the largest chunk scale eA + eB met so far; the accumulator
//     is rebased by an exact power of two when it grows), and add it into a float-float (two
//     FP32) accumulator; FP64 is touched once per output entry at the end.
// The operands of every product of the inverse are sign-definite, so the accumulated value is
// accurate relative to itself; the digit count s sets the precision.
//
// Kernel structure (one CTA per 128 x 128 output tile, 320 threads, 512 tensor-memory columns; with
// 256-wide chunks a cluster of two CTAs per 256 x 128 tile, tcgen05 cta_group::2, see Ring):
//   warp 0      TMA producer (one elected lane issues): digit tiles A_p[128 x 64] and B_q[128 x 64]
//               (a pair: each CTA its half of B, 64 x 64) into a 3-stage ring of two (pair, K step)
//               items per stage (a pair: 4 stages of two)
//   warp 1      TMEM allocator and MMA issuer (one elected lane issues): tcgen05.mma.kind::f16,
//               M=N=128 (a pair: M=256), K=16, 8 MMAs per wait; group accumulators
//               double-buffered in tensor memory (columns 0..255)
//   warps 2..9  epilogue: tcgen05.ld of each group sum, float-float accumulation with the low
//               words and each chunk's per-entry scale in tensor memory (columns 256..511),
//               final FP64 scale, the C update, a split-K partial, or the fused decode
// Tiles are launched longest K range first (triangular operands), and products of fewer tiles
// than SMs split K over several CTAs per tile (partials summed by ksplit_reduce_kernel).
// Every wait is bounded (about four seconds of %globaltimer); on expiry the CTA records
// RD_DEV_TIMEOUT, every role leaves its loop, and the tensor memory is freed.
//
// The inverse is organised recursively so that the FP64 work stays at the bottom (64 x 64 leaves,
// and FP64 products on small tiles for nodes of at most FP64_NODE rows, which are too small to
// fill the tensor cores):
//   factor(lo, hi):  factor the left half; U12 = L11^-1 A12; L21 = A21 U11^-1;
//                    A22 -= L21 U12; factor the right half; then the off-diagonal blocks of
//                    the inverses: L^-1_21 = -L22^-1 (L21 L11^-1), U^-1_12 = -U11^-1 (U12 U22^-1)
//   and finally Y = U^-1 L^-1 with the decode in the epilogue.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>

#include "rd_internal.cuh"

namespace {

constexpr int SIGMA = 7;          // bits per digit (balanced base 2^SIGMA)
constexpr int KAPPA_WIDE = 256;   // exponent / read-out chunk along K (natural order)
constexpr int KAPPA_NARROW = 64;  // the same with the locality order (compact 64-node parts)
constexpr int TM = 128, TN = 128, TK = 64;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr int TILE_BYTES = TM * TK * 2;            // one 128 x 64 BF16 tile: 16 KiB
constexpr int EXP_ZERO = -16384;                   // exponent of an all-zero chunk
constexpr int MAX_SLICES_WIDE = 15;    // group sums exact: 256 * 15 * 2^12 < 2^24
constexpr int MAX_SLICES_NARROW = 22;  // 64 * 22 * 2^12 < 2^24; group scale 2^(ACC_OFF - 7 (g + 2)) normal for g <= 21
constexpr int ACC_OFF = 64;            // the float-float accumulators hold an entry times 2^(ACC_OFF - reference)
constexpr int LEAF = RD_BF;                        // FP64 diagonal leaves (64)
constexpr unsigned long long WAIT_NS = 4000000000ull;
static_assert(SIGMA == RD_SPLIT_DIGIT_BITS && KAPPA_WIDE == RD_SCREEN_CHUNK && KAPPA_NARROW == RD_SCREEN_CHUNK_ORDERED,
              "range screen out of step with the digits");
static_assert(MAX_SLICES_WIDE == RD_SPLIT_MAX && MAX_SLICES_NARROW == RD_SPLIT_MAX_ORDERED, "digit limits");
static_assert((long long)KAPPA_WIDE * MAX_SLICES_WIDE * 4096 < (1 << 24) &&
                  (long long)KAPPA_NARROW * MAX_SLICES_NARROW * 4096 < (1 << 24),
              "group sums must stay exact in FP32");
static_assert(ACC_OFF - SIGMA * (MAX_SLICES_NARROW + 1) >= -126 && ACC_OFF - 2 * SIGMA + 24 + 17 < 127,
              "group scales normal, accumulators finite");

// instruction descriptor of tcgen05.mma.kind::f16: FP32 accumulator, BF16 A and B (both K-major),
// N = TN, and M = 128 (one CTA) or 256 (a CTA pair, 128 rows in each CTA's tensor memory)
constexpr uint32_t idesc(int m) {
  return (1u << 4)                        // D: FP32
         | (1u << 7)                      // A: BF16
         | (1u << 10)                     // B: BF16
         | ((uint32_t)(TN >> 3) << 17)    // N
         | ((uint32_t)(m >> 4) << 24);    // M
}

// Shared-memory layout of the two kernel variants.  One CTA per 128 x 128 tile (PAIR = false): a
// ring of 3 stages, each holding 2 items of (A, B) 16 KiB tiles.  A CTA pair per 256 x 128 tile
// (PAIR = true, tcgen05 cta_group::2): each CTA holds its own 128 rows of A (16 KiB) and half of
// the B tile (64 rows, 8 KiB) per item, so an item costs each CTA 24 KiB of L2 reads instead of
// 32 KiB and one MMA instruction does twice the work; the same 192 KiB then hold 2 stages of 4
// items.  Measured on the inverse product (256-wide chunks) with the issue loops run by whole warps:
// 2 items x 4 stages 7 % faster than 4 x 2 at n = 8192 (a stage's copies have three stages of MMAs
// to land in), 1 x 8 slower (a wait per 4 MMAs); for the one-CTA kernel with 64-wide chunks 2 x 3
// beats 3 x 2 and 1 x 6.  With 64-wide chunks, whose groups fill few items, the pair kernel is 2 %
// slower, so it runs for 256-wide chunks only.
// After the ring: the barriers (256 B), the chunk exponents of the tile's columns (2 x TN ints)
// and the per-entry reference exponents (TM x TN int16).
template <bool PAIR>
struct Ring {
  // (digit pair, K step) items per stage: each item is TK / 16 = 4 MMAs, and the MMA warp waits
  // once per stage
  static constexpr int ITEMS = 2;
  static constexpr int STAGES = PAIR ? 4 : 3;
  static constexpr int SLOTS = STAGES * ITEMS;
  static constexpr int A_BYTES = TILE_BYTES;
  static constexpr int B_BYTES = PAIR ? TILE_BYTES / 2 : TILE_BYTES;
  static constexpr int BAR_OFFSET = SLOTS * (A_BYTES + B_BYTES);
  static constexpr int ECOL_OFFSET = BAR_OFFSET + 256;
  static constexpr int REF_OFFSET = ECOL_OFFSET + 2 * TN * 4;
  static constexpr size_t SMEM = 1024 + REF_OFFSET + TM * TN * 2;
  static constexpr uint32_t IDESC = idesc(PAIR ? 2 * TM : TM);
};
static_assert((2 * Ring<true>::STAGES + 2 * 2 + 1) * 8 + 8 <= 256 && (2 * Ring<false>::STAGES + 2 * 2 + 1) * 8 + 8 <= 256,
              "barriers, tensor-memory slot and abort flag");
static_assert(Ring<false>::SMEM <= 232448 && Ring<true>::SMEM <= 232448, "shared memory of one CTA");
static_assert(Ring<true>::A_BYTES % 1024 == 0 && Ring<true>::B_BYTES % 1024 == 0, "128-byte swizzle atoms");

constexpr int16_t REF_NONE = -32768;                                    // no chunk with digits yet
// tensor memory: two accumulator buffers, the low words of the float-float accumulators, and the
// per-entry scale of the current chunk (one 32-bit column per tile column each)
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t TMEM_LO = 2 * TN;
constexpr uint32_t TMEM_SCALE = 3 * TN;

#ifdef RD_SPLIT_STATS
// Cycle counters of the split GEMM's roles (a build with RD_SPLIT_STATS only), summed over the
// launches that carry the fused decode (the inverse product Y = U^-1 L^-1), read by rd_split_stats:
//  0 MMA-warp cycles, 1 of them waiting for a free accumulator buffer, 2 waiting for a full operand
//  stage, 3 issuing (from a stage's arrival to its commit); 4 producer-warp cycles, 5 of them
//  waiting for a free stage; 6 epilogue cycles (warp 2 of each CTA), 7 of them waiting for a group
//  sum, 8 in the per-chunk renormalisation; 9 MMA warps counted, 10 epilogue warps counted,
//  11 digit groups, 12 MMA instructions.  (Pair leaders only for the MMA and producer warps.)
__device__ unsigned long long g_split_stats[16];
#endif

// ---- PTX wrappers -----------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// NOSLEEP: a zero suspend-time hint, for the MMA thread: every wait of the thread that issues the
// MMAs delays its next MMA (the tensor pipe's instruction queue is shallow), and a plain try_wait
// costs it more (measured: 56 % against 67 % of the tensor peak with one wait per 4 MMAs).
// CLUSTER: acquire at cluster scope, for barriers that the other CTA of a pair arrives on (its
// epilogue's release of an accumulator, its TMA copies, the pair's MMA commits).
template <bool NOSLEEP = false, bool CLUSTER = false>
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  if (CLUSTER && NOSLEEP)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  else if (CLUSTER)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  else if (NOSLEEP)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  return ok != 0;
}

// Wait for the phase of `parity` to complete; false when the CTA aborted or the deadline passed.
template <bool NOSLEEP = false, bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long deadline) {
  uint32_t spins = 0;
  while (!mbar_try_wait<NOSLEEP, CLUSTER>(bar, parity)) {
    if ((++spins & 1023u) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() > deadline) {
        *abort_flag = 1;
        return false;
      }
    }
  }
  return true;
}

// The same wait by every lane of a warp (each lane observes the phase itself, so whichever lane is
// elected to issue next has seen it); the outcome is the same in every lane.
template <bool NOSLEEP = false, bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                               unsigned long long deadline) {
  const bool ok = mbar_wait<NOSLEEP, CLUSTER>(bar, parity, abort_flag, deadline);
  return __all_sync(0xffffffffu, ok);
}

// ---- CTA pairs (a cluster of two CTAs sharing each MMA: tcgen05 cta_group::2) ------------------

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// the shared::cluster address of this CTA's shared-memory word `p` as seen in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_shared(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

// every thread of both CTAs (a full barrier across the cluster, with release/acquire ordering)
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// arrive on an mbarrier of either CTA of the pair (shared::cluster address)
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

// TMA tile loads (whole warp, the elected lane issues).  The pair form writes this CTA's shared memory
// and signals the pair leader's barrier (bar_cluster: a shared::cluster address, possibly in the
// peer CTA).
__device__ __forceinline__ void tma_load_2d_pair_w(uint32_t dst, const CUtensorMap* map, uint32_t bar_cluster, int x, int y) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n}\n"
      ::"r"(dst), "l"((uint64_t)map), "r"(bar_cluster), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d_w(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n}\n"
      ::"r"(dst), "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// SMEM matrix descriptor: K-major operand tile written by TMA with 128-byte swizzle
// (rows of 128 bytes, 8-row atoms of 1024 bytes stacked along M/N).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);     // start address
  d |= (uint64_t)(16u >> 4) << 16;             // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024u >> 4) << 32;           // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// The issuing instructions are executed by every lane of a converged warp, and the lane that
// elect.sync picks issues the one instruction: the addresses and descriptors are then values of a
// converged warp rather than of one divergent lane.
//
// umma_bf16_w: D (tensor memory) (+)= A B^T for one K = 16 step.  PAIR: M = 256 issued by the leader CTA of a
// pair; A's rows 0..127 come from the leader's shared memory and 128..255 from the peer's, B's rows
// (the N = 128 columns) 0..63 from the leader's and 64..127 from the peer's (same offsets in both),
// and each CTA's tensor memory receives its 128 rows.
template <bool PAIR>
__device__ __forceinline__ void umma_bf16_w(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  if (PAIR)
    asm volatile(
        "{\n .reg .pred e, p;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
        " @e tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(Ring<true>::IDESC), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred e, p;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(Ring<false>::IDESC), "r"(accumulate)
        : "memory");
}

// Arrive (once) on the barrier at shared address `bar` when every MMA issued so far has completed.
// PAIR: on the barrier at the same offset in each CTA of the pair named by `mask` (bit r = CTA rank r).
template <bool PAIR>
__device__ __forceinline__ void umma_commit_w(uint32_t bar, uint16_t mask = 3) {
  if (PAIR)
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n}\n" ::"r"(
            bar),
        "h"(mask)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx_w(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n @e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n}\n" ::"r"(
          bar),
      "r"(bytes)
      : "memory");
}

// tcgen05.ld of 8 columns without the wait; tmem_wait_ld(r) then waits for every prior load of this
// thread and ties r to the wait, so no use of r is scheduled before it
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}

// store 8 columns of this warp's 32 lanes, then wait for it (registers and columns are free
// to reuse after the call)
// 8 columns of this warp's lanes to tensor memory; the write completes at the next tmem_wait_st
// (each pass of the epilogue stores distinct columns, then waits once before they are read again)
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- slicing --------------------------------------------------------------------------------

__device__ __forceinline__ double view_load(const double* X, long long ld, int r, int c, int tri, int rows,
                                            int cols) {
  if (r >= rows || c >= cols) return 0.0;
  if (tri == RD_TRI_LOWER_UNIT) {
    if (r < c) return 0.0;
    if (r == c) return 1.0;
  } else if (tri == RD_TRI_UPPER) {
    if (r > c) return 0.0;
  }
  return X[(long long)r * ld + c];
}

// |x| as an integer that orders like the value (the bit pattern of a non-negative double)
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// exponent e of a chunk whose largest magnitude has the bit pattern mb: |mx| 2^-e in [1/4, 1/2)
// (ilogb(mx) + 2, from the bits: no FP64 instruction)
__device__ __forceinline__ int chunk_exponent_bits(unsigned long long mb) {
  if (mb == 0) return EXP_ZERO;
  const int ex = (int)(mb >> 52);
  if (ex != 0) return ex - 1023 + 2;
  return (63 - __clzll((long long)mb)) - 1074 + 2;  // subnormal: the leading mantissa bit
}

// F = round(|x| 2^(-e) 2^(7 s)) < 2^(7 s - 1) as F' 128^z: when the shift is a left shift,
// F = (m 2^(sh mod 7)) 128^z with z zero digits at the least significant end and F' < 2^59;
// otherwise F = round(m 2^sh) < 2^53 and z = 0 (m the 53-bit significand).
struct DigitSrc {
  uint64_t F;
  int z;
  bool neg;
};
__device__ __forceinline__ DigitSrc digit_src(double x, int e, int s) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  DigitSrc d;
  d.neg = (bits >> 63) != 0;
  d.F = 0;
  d.z = 0;
  int ex = (int)((bits >> 52) & 0x7FF);
  uint64_t m = bits & ((1ull << 52) - 1);
  if (ex == 0)
    ex = 1;  // subnormal: no implicit bit
  else
    m |= (1ull << 52);
  if (m != 0 && e != EXP_ZERO) {
    const int sh = ex - 1075 - e + SIGMA * s;
    if (sh >= 0) {
      d.z = sh / SIGMA;
      d.F = m << (sh - SIGMA * d.z);
    } else if (sh > -64) {
      const uint64_t half = 1ull << (-sh - 1);  // round half up
      d.F = (m + half) >> (-sh);                // m + half < 2^63
    }
  }
  return d;
}

// the next balanced base-128 digit (least significant first) of a DigitSrc; idx counts the
// digits taken so far
__device__ __forceinline__ int next_digit(DigitSrc& d, int idx) {
  if (idx < d.z) return 0;
  int v = (int)(uint32_t)(d.F & 127u);
  d.F >>= SIGMA;
  if (v >= 64) {
    v -= 128;
    d.F += 1;
  }
  return v;
}

// The balanced base-128 digits of x0 2^-e and x1 2^-e (|x| 2^-e < 1/2) for two adjacent K
// positions, most significant first: digit plane p at out[p * plane], the pair in one 4-byte
// store (out is 4-byte aligned).  Every digit is an integer in [-64, 64], exact in BF16.
__device__ __forceinline__ void write_digits2(double x0, double x1, int e, int s, __nv_bfloat16* out,
                                              long long plane) {
  DigitSrc a = digit_src(x0, e, s), b = digit_src(x1, e, s);
  for (int p = s - 1; p >= 1; --p) {
    const int da = next_digit(a, s - 1 - p), db = next_digit(b, s - 1 - p);
    *reinterpret_cast<__nv_bfloat162*>(out + (long long)p * plane) =
        __floats2bfloat162_rn((float)(a.neg ? -da : da), (float)(b.neg ? -db : db));
  }
  const int ta = (int)(uint32_t)a.F, tb = (int)(uint32_t)b.F;
  *reinterpret_cast<__nv_bfloat162*>(out) = __floats2bfloat162_rn((float)(a.neg ? -ta : ta), (float)(b.neg ? -tb : tb));
}

// A stacked batch (both slicing kernels): graph b = blockIdx.y (rows) or blockIdx.z (columns)
// reads its operand x_gs doubles further, writes its s_b = bg[b].s digit planes from plane b * s
// on (s is then the planes per graph) and its exponents e_gs ints further; s_b = 0 skips it.
struct SliceBatch {
  const rd_batch_graph* bg;  // nullptr: one graph
  long long x_gs, e_gs;
};

// Role A (row chunks contiguous in memory): one warp per (row, chunk), each lane taking pairs of
// adjacent K positions c0 + 2 lane + 64 t.  digits[p][row][k] (plane = rows_pad * k_pad),
// exps[chunk][row].
template <int KP>
__global__ void __launch_bounds__(256) slice_rows_kernel(const double* __restrict__ X, long long ld, int tri,
                                                         int rows, int cols, int rows_pad, int k_pad, int s,
                                                         __nv_bfloat16* __restrict__ dig, int* __restrict__ exps,
                                                         int* status, SliceBatch sb) {
  if (sb.bg) {
    const int b = blockIdx.y;
    X += (long long)b * sb.x_gs;
    dig += (long long)b * s * rows_pad * k_pad;
    exps += (long long)b * sb.e_gs;
    s = sb.bg[b].s;
    if (s == 0) return;
  }
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  const int nch = k_pad / KP;
  if (w >= (long long)rows_pad * nch) return;
  const int r = (int)(w / nch);
  const int c0 = (int)(w % nch) * KP;
  const long long plane = (long long)rows_pad * k_pad;
  double v[KP / 32];
  unsigned long long mb = 0;
#pragma unroll
  for (int t = 0; t < KP / 64; ++t) {
    const int c = c0 + 2 * lane + 64 * t;
    v[2 * t] = view_load(X, ld, r, c, tri, rows, cols);
    v[2 * t + 1] = view_load(X, ld, r, c + 1, tri, rows, cols);
    mb = max(mb, max(abs_bits(v[2 * t]), abs_bits(v[2 * t + 1])));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  const int e = chunk_exponent_bits(mb);
  if (lane == 0) exps[(long long)(c0 / KP) * rows_pad + r] = e;
#pragma unroll
  for (int t = 0; t < KP / 64; ++t)
    write_digits2(v[2 * t], v[2 * t + 1], e, s, dig + (long long)r * k_pad + c0 + 2 * lane + 64 * t, plane);
  (void)status;
}

// Role B (the operand is K x N row-major; digits are wanted K-major per column): a block of 256
// threads owns 16 columns of one chunk, stages the KP x 16 block through shared memory, and
// each warp slices 2 columns, each lane taking pairs of adjacent K positions.  digits[p][col][k],
// exps[chunk][col].
template <int KP>
__global__ void __launch_bounds__(256) slice_cols_kernel(const double* __restrict__ X, long long ld, int tri,
                                                         int krows, int cols, int cols_pad, int k_pad, int s,
                                                         __nv_bfloat16* __restrict__ dig, int* __restrict__ exps,
                                                         int* status, SliceBatch sb) {
  __shared__ double tile[KP][17];
  if (sb.bg) {
    const int b = blockIdx.z;
    X += (long long)b * sb.x_gs;
    dig += (long long)b * s * cols_pad * k_pad;
    exps += (long long)b * sb.e_gs;
    s = sb.bg[b].s;
    if (s == 0) return;
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * 16;
  const int c0 = blockIdx.y * KP;
  const long long plane = (long long)cols_pad * k_pad;
  for (int e = threadIdx.x; e < KP * 16; e += 256) {
    const int rr = e / 16, cc = e % 16;
    tile[rr][cc] = view_load(X, ld, c0 + rr, n0 + cc, tri, krows, cols);
  }
  __syncthreads();
#pragma unroll
  for (int cc = 0; cc < 2; ++cc) {
    const int col = warp * 2 + cc;
    double v[KP / 32];
    unsigned long long mb = 0;
#pragma unroll
    for (int t = 0; t < KP / 64; ++t) {
      v[2 * t] = tile[2 * lane + 64 * t][col];
      v[2 * t + 1] = tile[2 * lane + 1 + 64 * t][col];
      mb = max(mb, max(abs_bits(v[2 * t]), abs_bits(v[2 * t + 1])));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    const int e = chunk_exponent_bits(mb);
    const int n = n0 + col;
    if (lane == 0) exps[(long long)(c0 / KP) * cols_pad + n] = e;
#pragma unroll
    for (int t = 0; t < KP / 64; ++t)
      write_digits2(v[2 * t], v[2 * t + 1], e, s, dig + (long long)n * k_pad + c0 + 2 * lane + 64 * t, plane);
  }
  (void)status;
}

// ---- the split GEMM --------------------------------------------------------------------------

struct SplitArgs {
  const int* eA;     // [K_pad / KP][ma_pad]
  const int* eB;     // [K_pad / KP][nb_pad]
  int ma_pad, nb_pad;
  int M, N, K;       // M, N, K multiples of 64
  int s;
  int a_tri, b_tri;  // K-range skipping for triangular views
  double alpha, beta;
  double* C;
  long long ldc;
  int store_c;
  int c_rows, c_cols;  // bounds of the C store
  int32_t* D;        // fused decode (nullptr: off)
  long long ldd;
  int d_rows, d_cols;
  double log_gamma, tau;
  float inv_log2_gamma;  // 1 / log2(gamma) for the decode's FP32 fast path
  int* status;       // [0] first error, [1] detail
  // stores of C, D (and Y) go to row row_map[row] and column col_map[col] (nullptr: the identity):
  // the products of a graph in the locality order write back in the caller's node order
  const int32_t* row_map;
  const int32_t* col_map;
  // split K: ksplit CTAs per output tile, each over its share of the tile's chunks, writing the
  // unscaled FP64 partial sums to partial[ks][row][col] (ma_pad x nb_pad each); a reduction
  // kernel then applies alpha, beta, the bounds and the maps.  ksplit = 1: no partials.
  int ksplit;
  double* partial;
  // a stacked batch (nbatch > 1): the CTAs of graph b come after those of graphs 0..b-1; graph b
  // uses bg[b].s digits (0: skipped), its digit planes start at plane b * s_max of each operand's
  // buffer, its exponents ea_gs / eb_gs ints and its C c_gs doubles further; its D sits at
  // D + bg[b].off with leading dimension bg[b].n, and the C and D bounds are bg[b].n
  int nbatch;
  const rd_batch_graph* bg;
  int s_max;
  long long ea_gs, eb_gs, c_gs;
};

// Tile (row pair P of 256 rows, column J of 128) of CTA pair t, longest K range first, as the
// one-CTA order below: the inverse product (K from max(row, column) on) by increasing
// s = max(2P, J) (the row pair P = s / 2 for even s, then column J = s); a K range set by the
// column alone column-major (the last columns first for an upper-triangular B); by the row alone
// the last row pairs first for a lower-triangular A; otherwise row-major.
__device__ __forceinline__ void pair_tile(int t, int tp, int tn, int a_tri, int b_tri, int& P, int& J) {
  if (a_tri == RD_TRI_UPPER && b_tri == RD_TRI_LOWER_UNIT && tn == 2 * tp) {
    int rem = t;
    P = J = 0;
    for (int s = 0; s < tn; ++s) {
      if ((s & 1) == 0) {
        if (rem <= s) {  // row pair s / 2, columns 0..s
          P = s >> 1;
          J = rem;
          return;
        }
        rem -= s + 1;
        if (rem < (s >> 1)) {  // column s, row pairs 0 .. s/2 - 1
          P = rem;
          J = s;
          return;
        }
        rem -= s >> 1;
      } else {
        if (rem < ((s + 1) >> 1)) {  // column s, row pairs 0 .. (s - 1)/2
          P = rem;
          J = s;
          return;
        }
        rem -= (s + 1) >> 1;
      }
    }
    return;
  }
  if (a_tri == RD_TRI_FULL && b_tri != RD_TRI_FULL) {
    P = t % tp;
    J = t / tp;
    if (b_tri == RD_TRI_UPPER) J = tn - 1 - J;
    return;
  }
  P = t / tn;
  J = t % tn;
  if (a_tri == RD_TRI_LOWER_UNIT) P = tp - 1 - P;
}

// One CTA per 128 x 128 output tile (PAIR = false), or a cluster of two CTAs per 256 x 128 tile
// (PAIR = true: CTA rank r owns rows 128 r .. 128 r + 127 of the tile and half of the B tile; the
// leader, rank 0, issues the MMAs for both; every CTA runs its own producer and epilogue).
template <int KP, bool PAIR>
__global__ void __launch_bounds__(THREADS, 1)
    split_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const SplitArgs p) {
  using R = Ring<PAIR>;
  constexpr int STAGES = R::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + R::SLOTS * R::A_BYTES;
  uint64_t* full = (uint64_t*)(smem + R::BAR_OFFSET);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  int* ecol_s = (int*)(smem + R::ECOL_OFFSET);    // [2][TN]
  int16_t* ref_s = (int16_t*)(smem + R::REF_OFFSET);  // [TN][TM], column-major

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  const int tiles_n = (p.N + TN - 1) / TN, tiles_m = (p.M + TM - 1) / TM;
  unsigned unit = PAIR ? blockIdx.x / 2 : blockIdx.x;  // the CTA pair (or CTA) index
  // a stacked batch: the graph of this CTA, and its share of the launch
  int gb = 0;
  if (p.nbatch > 1) {
    const unsigned per_graph = (unsigned)(PAIR ? tiles_m / 2 : tiles_m) * (unsigned)tiles_n * (unsigned)p.ksplit;
    gb = (int)(unit / per_graph);
    unit %= per_graph;
  }
  const rd_batch_graph* bgr = p.nbatch > 1 ? p.bg + gb : nullptr;
  // a graph of a stacked batch without split work in this pass: nothing to do (both CTAs of a pair
  // belong to one graph, so a pair leaves together, before any barrier)
  if (bgr && bgr->s == 0) return;
  const int* eA = p.eA + (long long)gb * p.ea_gs;
  const int* eB = p.eB + (long long)gb * p.eb_gs;
  const int a_plane0 = gb * p.s_max, b_plane0 = gb * p.s_max;  // first digit plane of this graph
  const int ks_idx = (int)(unit % (unsigned)p.ksplit);
  const int tile = (int)(unit / (unsigned)p.ksplit);
  // Longest tiles first (the block scheduler starts CTAs in index order, so the last wave then
  // holds the short ones): with a triangular operand the K range of a tile depends on its row or
  // column (see kbeg / kend below).
  int m0, n0;  // the tile (of the pair: 256 rows) and this CTA's first row
  constexpr int ROWS = PAIR ? 2 * TM : TM;
  if (PAIR) {
    int P, J;
    pair_tile(tile, p.ma_pad / ROWS, p.nb_pad / TN, p.a_tri, p.b_tri, P, J);
    m0 = P * ROWS;
    n0 = J * TN;
  } else {
    int tr = tile / tiles_n, tc = tile % tiles_n;
    if (p.a_tri == RD_TRI_UPPER && p.b_tri == RD_TRI_LOWER_UNIT && tiles_m == tiles_n) {
      // K from max(row, col) on: shells of equal max(tr, tc), the outermost (shortest) last
      const int sh = (int)sqrtf((float)tile);
      const int shell = (sh + 1) * (sh + 1) <= tile ? sh + 1 : (sh * sh > tile ? sh - 1 : sh);
      const int o = tile - shell * shell;  // 0 .. 2 shell
      tr = o <= shell ? o : shell;
      tc = o <= shell ? shell : o - shell - 1;
    } else if (p.a_tri == RD_TRI_FULL && p.b_tri != RD_TRI_FULL) {
      // K depends on the tile column alone: column-major, so that a wave takes whole columns
      tr = tile % tiles_m;
      tc = tile / tiles_m;
      if (p.b_tri == RD_TRI_UPPER) tc = tiles_n - 1 - tc;  // K up to the column's end: the last columns first
    } else if (p.a_tri == RD_TRI_LOWER_UNIT) {
      tr = tiles_m - 1 - tr;  // K up to the tile row's end
    }
    m0 = tr * TM;
    n0 = tc * TN;
  }
  const int m_cta = m0 + (int)rank * TM;  // this CTA's rows of A and of the output
  // K range of the tile (of both CTAs of a pair: the union of their rows' ranges; the extra K steps
  // of one CTA's rows meet zeros of its triangular operand and add exact zeros)
  int kbeg = 0, kend = p.K;
  if (p.a_tri == RD_TRI_LOWER_UNIT) kend = min(kend, m0 + ROWS);
  if (p.a_tri == RD_TRI_UPPER) kbeg = max(kbeg, m0);
  if (p.b_tri == RD_TRI_LOWER_UNIT) kbeg = max(kbeg, n0);
  if (p.b_tri == RD_TRI_UPPER) kend = min(kend, n0 + TN);
  // With split K this CTA takes K steps [s_lo, s_hi) of the tile's range (a share of a chunk
  // keeps its group sums exact, and the chunk's scales are the same).  Chunks are aligned to
  // absolute multiples of KP; the first and last may be partial.
  if (p.ksplit > 1 && kbeg < kend) {
    const int steps = (kend - kbeg) / TK;
    const int s_lo = (int)(((long long)steps * ks_idx) / p.ksplit);
    const int s_hi = (int)(((long long)steps * (ks_idx + 1)) / p.ksplit);
    kend = kbeg + s_hi * TK;
    kbeg = kbeg + s_lo * TK;
  }
  const int cbeg = kbeg / KP;
  const int nchunks = (kbeg < kend) ? (kend + KP - 1) / KP - cbeg : 0;
  const int s = bgr ? bgr->s : p.s;  // (0: a graph of the batch that is not on the split path)

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], PAIR ? 2 * EPI_WARPS : EPI_WARPS);  // (a pair: both CTAs' epilogues)
    }
    mbar_init(drain, 1);
    // a CTA that timed out earlier leaves its mark in the status word: skip the work
    *abort_flag = (p.status && *(volatile int*)p.status == RD_DEV_TIMEOUT) ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // both CTAs of a pair allocate (the same columns of each CTA's tensor memory)
    if (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (PAIR) cluster_sync();  // the peer's barriers are initialised before any remote arrive
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const unsigned long long deadline = globaltimer() + WAIT_NS;
  const int nloop = *abort_flag ? 0 : nchunks;

  // The producer and the MMA issuer are whole warps whose every instruction sits between two
  // tensor-core instructions: one elected lane issues each copy, MMA and commit, and the loops keep
  // the per-item work to a few independent integer operations (no divisions; smem addresses,
  // descriptors and barrier addresses as a base plus compile-time offsets; items of a stage
  // unrolled).  The issuing warp runs its dependent scalar code at a few cycles per instruction,
  // sharing its SM sub-partition with two epilogue warps, and an M = 128, N = 128, K = 16 MMA takes 64.
  const uint32_t sA0 = smem_u32(sA), sB0 = smem_u32(sB);
  const uint32_t full0 = smem_u32(full), empty0 = smem_u32(empty);
  if (warp == 0) {
    {  // TMA producer, the whole warp (in each CTA of a pair: its own A rows and half of B)
      const uint32_t full_lead0 = PAIR ? mapa_shared(full, 0) : full0;  // the pair leader's full[0]
      const int b_col = n0 + (PAIR ? (int)rank * (TN / 2) : 0);
      const int a_row = PAIR ? m_cta : m0;
      int st = 0;
      uint32_t phase = 0;  // of the current pass over the stages
      bool ok = true;
#ifdef RD_SPLIT_STATS
      const unsigned long long pt0 = clock64();
      unsigned long long pwait = 0;
#endif
      for (int c = 0; c < nloop && ok; ++c) {
        const int kc0 = max(kbeg, (cbeg + c) * KP);
        const int ksteps = (min(kend, (cbeg + c + 1) * KP) - kc0) / TK;
        for (int g = 0; g < s && ok; ++g) {
          // the group's items (pair pa, K step ks) in order, R::ITEMS to a stage
          const int items = (g + 1) * ksteps;
          int pa = 0, ks = 0;
          int ya = (a_plane0 + 0) * p.ma_pad + a_row, yb = (b_plane0 + g) * p.nb_pad + b_col;
          for (int i0 = 0; i0 < items; i0 += R::ITEMS) {
#ifdef RD_SPLIT_STATS
            const unsigned long long pw0 = clock64();
#endif
            if (!mbar_wait_warp<false, PAIR>(&empty[st], phase ^ 1u, abort_flag, deadline)) {
              ok = false;
              break;
            }
#ifdef RD_SPLIT_STATS
            pwait += clock64() - pw0;
#endif
            const int cnt = min(R::ITEMS, items - i0);
            // the leader's barrier counts the bytes of both CTAs (a peer's copies may land first:
            // the transaction count goes negative until the leader's expect)
            if (leader) mbar_arrive_expect_tx_w(full0 + (uint32_t)(st * 8), cnt * (PAIR ? 2 : 1) * (R::A_BYTES + R::B_BYTES));
            const uint32_t bar = (PAIR ? full_lead0 : full0) + (uint32_t)(st * 8);
            const uint32_t da = sA0 + (uint32_t)(st * R::ITEMS * R::A_BYTES), db = sB0 + (uint32_t)(st * R::ITEMS * R::B_BYTES);
#pragma unroll
            for (int u = 0; u < R::ITEMS; ++u) {
              if (u < cnt) {
                const int ka = kc0 + ks * TK;
                if (PAIR) {
                  tma_load_2d_pair_w(da + u * R::A_BYTES, &tmA, bar, ka, ya);
                  tma_load_2d_pair_w(db + u * R::B_BYTES, &tmB, bar, ka, yb);
                } else {
                  tma_load_2d_w(da + u * R::A_BYTES, &tmA, bar, ka, ya);
                  tma_load_2d_w(db + u * R::B_BYTES, &tmB, bar, ka, yb);
                }
                if (++ks == ksteps) {  // next digit pair (pa + 1, g - pa - 1)
                  ks = 0;
                  ++pa;
                  ya += p.ma_pad;
                  yb -= p.nb_pad;
                }
              }
            }
            if (++st == STAGES) {
              st = 0;
              phase ^= 1u;
            }
          }
        }
      }
#ifdef RD_SPLIT_STATS
      if (p.D && leader && lane == 0) {
        atomicAdd(&g_split_stats[4], clock64() - pt0);
        atomicAdd(&g_split_stats[5], pwait);
      }
#endif
    }
  } else if (warp == 1) {
    if (leader) {  // MMA issuer, the whole warp (a pair's leader issues for both CTAs)
      // descriptors of slot 0 of A and B; a slot, a K = 16 step, adds its byte offset / 16 (the
      // start-address field holds shared-memory addresses below 256 KiB: no carry out of it)
      const uint64_t dA0 = sdesc_sw128(sA0), dB0 = sdesc_sw128(sB0);
      int st = 0, gi = 0;
      uint32_t phase = 0;
      bool ok = true;
#ifdef RD_SPLIT_STATS
      const unsigned long long mt0 = clock64();
      unsigned long long macc = 0, mfull = 0, missue = 0, mmas = 0;
#endif
      for (int c = 0; c < nloop && ok; ++c) {
        const int kc0 = max(kbeg, (cbeg + c) * KP);
        const int ksteps = (min(kend, (cbeg + c + 1) * KP) - kc0) / TK;
        for (int g = 0; g < s && ok; ++g, ++gi) {
          const int buf = gi & 1;
          const uint32_t use = (uint32_t)(gi >> 1);
#ifdef RD_SPLIT_STATS
          const unsigned long long ma0 = clock64();
#endif
          if (!mbar_wait_warp<true, PAIR>(&acc_empty[buf], (use + 1) & 1u, abort_flag, deadline)) {
            ok = false;
            break;
          }
#ifdef RD_SPLIT_STATS
          macc += clock64() - ma0;
#endif
          tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)(buf * TN);
          uint32_t acc = 0;
          const int items = (g + 1) * ksteps;
          for (int i0 = 0; i0 < items; i0 += R::ITEMS) {
#ifdef RD_SPLIT_STATS
            const unsigned long long mf0 = clock64();
#endif
            if (!mbar_wait_warp<true, PAIR>(&full[st], phase, abort_flag, deadline)) {
              ok = false;
              break;
            }
#ifdef RD_SPLIT_STATS
            const unsigned long long mi0 = clock64();
            mfull += mi0 - mf0;
#endif
            tc_fence_after();
            const int cnt = min(R::ITEMS, items - i0);
            const uint64_t da = dA0 + (uint64_t)((st * R::ITEMS * R::A_BYTES) >> 4);
            const uint64_t db = dB0 + (uint64_t)((st * R::ITEMS * R::B_BYTES) >> 4);
#pragma unroll
            for (int u = 0; u < R::ITEMS; ++u) {
              if (u < cnt) {
#pragma unroll
                for (int k16 = 0; k16 < TK / 16; ++k16) {
                  umma_bf16_w<PAIR>(dt, da + (uint64_t)((u * R::A_BYTES + k16 * 32) >> 4),
                                    db + (uint64_t)((u * R::B_BYTES + k16 * 32) >> 4), acc);
                  acc = 1;
                }
              }
            }
            umma_commit_w<PAIR>(empty0 + (uint32_t)(st * 8));  // (a pair: both CTAs' stage barriers)
#ifdef RD_SPLIT_STATS
            missue += clock64() - mi0;
            mmas += (unsigned long long)cnt * (TK / 16);
#endif
            if (++st == STAGES) {
              st = 0;
              phase ^= 1u;
            }
          }
          if (ok) umma_commit_w<PAIR>(smem_u32(&acc_full[buf]));
        }
      }
#ifdef RD_SPLIT_STATS
      if (p.D && lane == 0) {
        atomicAdd(&g_split_stats[0], clock64() - mt0);
        atomicAdd(&g_split_stats[1], macc);
        atomicAdd(&g_split_stats[2], mfull);
        atomicAdd(&g_split_stats[3], missue);
        atomicAdd(&g_split_stats[9], 1ull);
        atomicAdd(&g_split_stats[11], (unsigned long long)gi);
        atomicAdd(&g_split_stats[12], mmas);
      }
#endif
      // every MMA issued has completed before the tensor memory can be freed (bounded: a second)
      umma_commit_w<PAIR>(smem_u32(drain), 1);
      volatile int no_abort = 0;
      mbar_wait_warp<false, false>(drain, 0, &no_abort, globaltimer() + 1000000000ull);
    }
  } else {  // epilogue warps 2..9
    const int ew = warp - 2;
    const int quarter = warp & 3;      // tensor-memory lane quarter this warp may access
    const int half = ew >> 2;          // column half of the tile
    const int lrow = quarter * 32 + lane;
    const int row = m_cta + lrow;
    // float-float accumulators: high words in registers, low words in tensor memory, both relative
    // to a per-entry reference exponent (shared memory, int16) that follows the largest chunk scale
    // eA[c][row] + eB[c][col] met so far.  When a chunk's scale exceeds it, the accumulator is
    // rebased by that exact power of two, so every group term is at most 2^-14 of the reference,
    // and an entry far below the rest of its tile (a Y spanning hundreds of binades) keeps its own
    // scale.  A term more than 2^-126 below its entry's reference underflows: the entry is at least
    // its largest chunk's real contribution, which the chunk spread bounds far above that.  Each
    // chunk's scale relative to the reference, S = 2^(eA + eB - ref), is kept in tensor memory, so
    // a group term is G 2^(-7 (g + 2)) S.  Both words carry an extra 2^ACC_OFF, so that the group
    // scale stays a normal float up to 22 digits and an entry 2^-100 below its reference keeps
    // its low digits; the final FP64 scaling takes it off.
    float hi[64];
    int16_t* rf = ref_s + (half * 64) * TM + lrow;  // rf[j * TM]
    const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 64);  // this warp's lanes
    {
      uint32_t z[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) z[q] = 0u;
#pragma unroll
      for (int t = 0; t < 8; ++t) tmem_st8(tl + TMEM_LO + t * 8, z);
      tmem_wait_st();
    }
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      hi[j] = 0.f;
      rf[j * TM] = REF_NONE;
    }
    int gi = 0;
    bool ok = true;
#ifdef RD_SPLIT_STATS
    const unsigned long long et0 = clock64();
    unsigned long long ewait = 0, eren = 0;
#endif
    for (int c = 0; c < nloop; ++c) {  // every warp passes the barrier once per chunk
      const int kc = cbeg + c;
      const int cb = c & 1;
      if (ew < 4) {
        const int t = ew * 32 + lane;  // 0..127: one column each
        ecol_s[cb * TN + t] = eB[(long long)kc * p.nb_pad + n0 + t];
      }
      asm volatile("bar.sync 1, %0;" ::"r"(EPI_WARPS * 32) : "memory");
      if (!ok) continue;
      const int erow = eA[(long long)kc * p.ma_pad + row];
#ifdef RD_SPLIT_STATS
      const unsigned long long er0 = clock64();
#endif
      // renormalise the previous chunk's sums, rebase where this chunk's scale exceeds the
      // reference, and set this chunk's per-entry scale
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        uint32_t lr[8], sr[8];
        tmem_ld8_async(tl + TMEM_LO + t * 8, lr);
        tmem_wait_ld(lr);
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int j = t * 8 + jj;
          float l = __uint_as_float(lr[jj]);
          const float sum = hi[j] + l;
          l = l - (sum - hi[j]);
          hi[j] = sum;
          const int ec = ecol_s[cb * TN + half * 64 + j];
          const bool live = (erow != EXP_ZERO) && (ec != EXP_ZERO);
          const int sc = erow + ec;
          int r = rf[j * TM];
          if (live && sc > r) {
            const int d = r - sc;
            const float f = (d >= -126) ? __int_as_float((d + 127) << 23) : 0.f;
            hi[j] *= f;
            l *= f;
            r = sc;
            rf[j * TM] = (int16_t)sc;
          }
          const int d = sc - r;  // <= 0 for a live chunk
          sr[jj] = (live && d >= -126) ? (uint32_t)((d + 127) << 23) : 0u;
          lr[jj] = __float_as_uint(l);
        }
        tmem_st8(tl + TMEM_LO + t * 8, lr);
        tmem_st8(tl + TMEM_SCALE + t * 8, sr);
      }
      tmem_wait_st();
#ifdef RD_SPLIT_STATS
      eren += clock64() - er0;
#endif
      for (int g = 0; g < s; ++g, ++gi) {
        const int buf = gi & 1;
        const uint32_t use = (uint32_t)(gi >> 1);
#ifdef RD_SPLIT_STATS
        const unsigned long long ew0 = clock64();
#endif
        // warp-uniform outcome: the tensor-memory loads below are warp-wide
        if (!__all_sync(0xffffffffu, mbar_wait<false, PAIR>(&acc_full[buf], use & 1u, abort_flag, deadline))) {
          ok = false;
          break;
        }
#ifdef RD_SPLIT_STATS
        ewait += clock64() - ew0;
#endif
        tc_fence_after();
        const float cg = __int_as_float((127 + ACC_OFF - SIGMA * (g + 2)) << 23);  // 2^(ACC_OFF - 7 (g + 2))
#pragma unroll
        for (int t = 0; t < 8; ++t) {  // 8 columns at a time
          uint32_t gr[8], sr[8], lr[8];
          tmem_ld8_async(tl + (uint32_t)(buf * TN) + t * 8, gr);
          tmem_ld8_async(tl + TMEM_SCALE + t * 8, sr);
          tmem_ld8_async(tl + TMEM_LO + t * 8, lr);
          tmem_wait_ld(gr);
          tmem_wait_ld(sr);
          tmem_wait_ld(lr);
          if (t == 7) {  // all reads of the accumulator done: hand the buffer back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if (PAIR)
                mbar_arrive_cluster(mapa_shared(&acc_empty[buf], 0));  // the leader's MMA thread
              else
                mbar_arrive(&acc_empty[buf]);
            }
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = t * 8 + jj;
            const float term = (__uint_as_float(gr[jj]) * cg) * __uint_as_float(sr[jj]);
            const float sum = hi[j] + term;
            const float bp = sum - hi[j];
            const float err = (hi[j] - (sum - bp)) + (term - bp);
            hi[j] = sum;
            lr[jj] = __float_as_uint(__uint_as_float(lr[jj]) + err);
          }
          tmem_st8(tl + TMEM_LO + t * 8, lr);
        }
        tmem_wait_st();
      }
    }
#ifdef RD_SPLIT_STATS
    if (p.D && warp == 2 && lane == 0) {
      atomicAdd(&g_split_stats[6], clock64() - et0);
      atomicAdd(&g_split_stats[7], ewait);
      atomicAdd(&g_split_stats[8], eren);
      atomicAdd(&g_split_stats[10], 1ull);
    }
#endif
    // final values, 16 columns at a time (the tensor-memory loads are warp-wide: outside any
    // per-lane condition)
    const bool store = ok && !*abort_flag && s > 0;
    // this graph's stores (a stacked batch: its own C, D, bounds, gain and status)
    double* Cg = p.C ? p.C + (long long)gb * p.c_gs : nullptr;
    int32_t* Dg = (p.D && bgr) ? p.D + bgr->off : p.D;
    const long long ldd = bgr ? bgr->n : p.ldd;
    const int c_rows = bgr ? min(p.c_rows, bgr->n) : p.c_rows, c_cols = bgr ? min(p.c_cols, bgr->n) : p.c_cols;
    const int d_rows = bgr ? bgr->n : p.d_rows, d_cols = bgr ? bgr->n : p.d_cols;
    const double log_gamma = bgr ? bgr->log_gamma : p.log_gamma;
    const float inv_log2_gamma = bgr ? bgr->inv_log2_gamma : p.inv_log2_gamma;
    int* status_g = bgr ? const_cast<int*>(bgr->status) : p.status;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      uint32_t lr[8];
      tmem_ld8_async(tl + TMEM_LO + t * 8, lr);
      tmem_wait_ld(lr);
      if (!store) continue;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int j = t * 8 + jj;
        const int col = n0 + half * 64 + j;
        if (row >= p.M || col >= p.N) continue;
        double v = ldexp((double)hi[j] + (double)__uint_as_float(lr[jj]), (int)rf[j * TM] - ACC_OFF);
        if (p.partial) {  // split K: the unscaled partial sum
          p.partial[((long long)ks_idx * p.ma_pad + row) * p.nb_pad + col] = v;
          continue;
        }
        v = p.alpha * v;
        const long long orow = p.row_map ? p.row_map[row] : row;
        const long long ocol = p.col_map ? p.col_map[col] : col;
        if (Cg && row < c_rows && col < c_cols) {
          double* cp = Cg + orow * p.ldc + ocol;
          if (p.beta != 0.0) v = fma(p.beta, *cp, v);
          if (p.store_c) *cp = v;
        }
        if (Dg && row < d_rows && col < d_cols) {
          int32_t d;
          if (!isfinite(v)) {
            rd_set_status(status_g, RD_DEV_NONFINITE, (int)orow);
            d = RD_UNREACHABLE;
          } else {
            d = (row == col) ? 0 : rd_decode_entry_fast(v, inv_log2_gamma, log_gamma, p.tau);
          }
          Dg[orow * ldd + ocol] = d;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // a pair: neither CTA frees its tensor memory or leaves while the other's work (the leader's
  // MMAs into both, the peer's arrivals on the leader's barriers) may still touch it; every loop
  // above ends (bounded waits), so both CTAs arrive here
  if (PAIR) cluster_sync();
  if (*abort_flag && threadIdx.x == 0) rd_set_status(p.status, RD_DEV_TIMEOUT, blockIdx.x);
  // (the status word is only read at the start of a CTA: a stale value merely skips work)
  if (warp == 1) {
    tc_fence_after();
    if (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// Entrywise relative residual of sampled rows y of Y against the exact M: y^T M = e_g^T, i.e.
//   r_j = y_j - [j == g] - sum_{i : edge j -> i} X_ij y_i,   X = gamma A or gamma^W,
// relative to (|y^T| |M|)_j = |y_j| + sum |X_ij y_i| (the componentwise backward error).  Every product is FP64 here.  Because M is an
// M-matrix with Y >= 0, a small entrywise residual bounds the entrywise error of the row
// (error^T = r^T Y), and a wrong region of a row shows up where it meets the right part.
// The largest relative residual is OR-ed into res (bits of a non-negative double).
__global__ void row_residual_kernel(const double* __restrict__ rows, const int32_t* __restrict__ goals, int k,
                                    int n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ succ,
                                    const uint8_t* __restrict__ A, const float* __restrict__ W, double gamma,
                                    unsigned long long* __restrict__ res) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double worst = 0.0;
  if (t < (long long)k * n) {
    const int c = (int)(t / n), j = (int)(t % n);
    const double* y = rows + (long long)c * n;
    double acc = y[j] - (goals[c] == j ? 1.0 : 0.0);
    double scale = fabs(y[j]);  // componentwise: (|y^T| |M|)_j
    for (int q = ptr[j]; q < ptr[j + 1]; ++q) {
      const int i = succ[q];
      const double x = W ? pow(gamma, (double)W[(long long)i * n + j]) : gamma;
      const double term = x * y[i];
      acc -= term;
      scale += fabs(term);
    }
    (void)A;
    // an entry whose scale lies in FP64's subnormal range holds no digits to check (far entries
    // of a graph whose Y spans more than FP64's exponent range underflow on any path)
    worst = scale >= 0x1p-1022 ? fabs(acc) / scale : 0.0;
    if (!(worst <= 1.0)) worst = 1.0;
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0 && worst > 0.0) atomicMax(res, (unsigned long long)__double_as_longlong(worst));
}

// ---- host side ---------------------------------------------------------------------------------

// streaming multiprocessors of the current device (152 on GB300)
int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms <= 0) {
      cudaGetLastError();
      sms = 152;
    }
  }
  return sms;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

// 2D map over digit planes: inner dim k_pad (contiguous), outer dim s * rows_pad; boxes of TK x box_rows
cudaError_t make_map(CUtensorMap* m, const void* base, int k_pad, long long rows, int box_rows = TM) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)k_pad * 2};
  cuuint32_t box[2] = {TK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int round_up(int x, int a) { return (x + a - 1) / a * a; }

struct View {
  const double* p;
  long long ld;
  int rows, cols;
  int tri;
};

}  // namespace

struct rd_split_plan {
  int N = 0, s = 0, cap_s = 0;
  // the operand whose digits digB / eB hold when they may be reused: the final L^-1 of the current
  // factors (the inverse product, the self-check's and the goal solves' rows all multiply by it)
  bool b_cached = false;
  const double* b_p = nullptr;
  long long b_ld = 0;
  int b_rows = 0, b_cols = 0, b_tri = 0, b_cols_pad = 0, b_k_pad = 0, b_s = 0, b_kappa = 0;
  unsigned long long b_gen = 0;
  double* part = nullptr;  // split-K partial sums (grown on demand)
  size_t part_bytes = 0;
  __nv_bfloat16* digA = nullptr;
  __nv_bfloat16* digB = nullptr;
  int* eA = nullptr;
  int* eB = nullptr;
  int64_t bytes = 0;
  bool borrowed = false;  // digA, digB, eA, eB belong to a batch (rd_split_prepare_borrowed)
};

namespace {

// the batch part of a slicing launch: per-graph strides of the operand and of the exponents
// (exponent arrays hold k_pad / kappa chunks of rows_pad entries per graph)
SliceBatch slice_batch(const rd_ctx* h, const void* x, int rows_pad, int k_pad) {
  SliceBatch sb{};
  if (h->nbatch > 1) {
    sb.bg = h->dBatch;
    sb.x_gs = rd_batch_stride(h, x);
    sb.e_gs = (long long)(k_pad / h->kappa) * rows_pad;
  }
  return sb;
}

// Slice the A operand (rows x k) into digA/eA (chunks of h->kappa along k).
cudaError_t slice_a(rd_ctx* h, const View& v, int rows_pad, int k_pad, cudaStream_t st, rd_split_plan* P) {
  cudaError_t e = rd_prof_begin(h, st, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  const long long warps = (long long)rows_pad * (k_pad / h->kappa);
  const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
  const SliceBatch sb = slice_batch(h, v.p, rows_pad, k_pad);
  const dim3 grid(blocks, h->nbatch > 1 ? h->nbatch : 1);
  if (h->kappa == KAPPA_NARROW)
    slice_rows_kernel<KAPPA_NARROW><<<grid, 256, 0, st>>>(v.p, v.ld, v.tri, v.rows, v.cols, rows_pad, k_pad, P->s,
                                                          P->digA, P->eA, h->dStatus, sb);
  else
    slice_rows_kernel<KAPPA_WIDE><<<grid, 256, 0, st>>>(v.p, v.ld, v.tri, v.rows, v.cols, rows_pad, k_pad, P->s,
                                                        P->digA, P->eA, h->dStatus, sb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, st, RD_PROF_NONE, 0.0);
}

// Split-K reduction: C[map(row)][map(col)] = alpha sum_ks partial[ks][row][col] (+ beta C) over
// rows < c_rows, cols < c_cols, the partials summed in order of ks (deterministic; the partials of
// a sign-definite product share one sign, so the sum does not cancel).
__global__ void ksplit_reduce_kernel(const double* __restrict__ part, int ksplit, int ma_pad, int nb_pad, int rows,
                                     int cols, double alpha, double beta, double* C, long long ldc,
                                     const int32_t* __restrict__ row_map, const int32_t* __restrict__ col_map) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)rows * cols) return;
  const int r = (int)(t / cols), c = (int)(t % cols);
  double v = 0.0;
  for (int k = 0; k < ksplit; ++k) v += part[((long long)k * ma_pad + r) * nb_pad + c];
  v *= alpha;
  double* cp = C + (long long)(row_map ? row_map[r] : r) * ldc + (col_map ? col_map[c] : c);
  if (beta != 0.0) v = fma(beta, *cp, v);
  *cp = v;
}

// Slice the B operand (k x cols, row-major) into digB/eB (K-major per column).  With cacheable
// (B is the final L^-1 of the current factors), digits already sliced from the same view, digit
// count and chunk width for the same factorisation are reused.
cudaError_t slice_b(rd_ctx* h, const View& v, int cols_pad, int k_pad, cudaStream_t st, bool cacheable,
                    rd_split_plan* P) {
  if (cacheable && P->b_cached && P->b_p == v.p && P->b_ld == v.ld && P->b_rows == v.rows && P->b_cols == v.cols &&
      P->b_tri == v.tri && P->b_cols_pad == cols_pad && P->b_k_pad == k_pad && P->b_s == P->s &&
      P->b_kappa == h->kappa && P->b_gen == h->factor_gen)
    return cudaSuccess;
  P->b_cached = cacheable;
  P->b_p = v.p;
  P->b_ld = v.ld;
  P->b_rows = v.rows;
  P->b_cols = v.cols;
  P->b_tri = v.tri;
  P->b_cols_pad = cols_pad;
  P->b_k_pad = k_pad;
  P->b_s = P->s;
  P->b_kappa = h->kappa;
  P->b_gen = h->factor_gen;
  cudaError_t e = rd_prof_begin(h, st, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  const dim3 grid(cols_pad / 16, k_pad / h->kappa, h->nbatch > 1 ? h->nbatch : 1);
  const SliceBatch sb = slice_batch(h, v.p, cols_pad, k_pad);
  if (h->kappa == KAPPA_NARROW)
    slice_cols_kernel<KAPPA_NARROW><<<grid, 256, 0, st>>>(v.p, v.ld, v.tri, v.rows, v.cols, cols_pad, k_pad, P->s,
                                                          P->digB, P->eB, h->dStatus, sb);
  else
    slice_cols_kernel<KAPPA_WIDE><<<grid, 256, 0, st>>>(v.p, v.ld, v.tri, v.rows, v.cols, cols_pad, k_pad, P->s,
                                                        P->digB, P->eB, h->dStatus, sb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return rd_prof_end(h, st, RD_PROF_NONE, 0.0);
}

// ctas: one per 128 x 128 tile (times ksplit); a pair kernel runs them as clusters of two
template <int KP, bool PAIR>
cudaError_t launch_split(const CUtensorMap& ta, const CUtensorMap& tb, const SplitArgs& a, int ctas, cudaStream_t st) {
  static bool attr = false;
  const int smem = (int)Ring<PAIR>::SMEM;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(split_gemm_kernel<KP, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (!PAIR) {
    split_gemm_kernel<KP, false><<<ctas, THREADS, smem, st>>>(ta, tb, a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas, 1, 1);
  cfg.blockDim = dim3(THREADS, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, split_gemm_kernel<KP, true>, ta, tb, a);
}

// C (c_rows x c_cols, ldc) = alpha * A (M x K) * B (K x N) + beta * C; with D != nullptr the product is
// decoded into D (n x n) instead and Ystore (n x n, may be null) receives Y.  row_map / col_map send
// the stores to the caller's node order (see SplitArgs).  `flops` is the algorithmic count of one
// product; the profile counts the issued digit products.
cudaError_t split_gemm(rd_ctx* h, const View& A, const View& B, int M, int N, int K, double alpha, double beta,
                       double* C, long long ldc, int c_rows, int c_cols, int32_t* D, double* Ystore, double flops,
                       cudaStream_t st, const int32_t* row_map = nullptr, const int32_t* col_map = nullptr,
                       bool b_is_final_linv = false, rd_split_plan* plan = nullptr) {
  rd_split_plan* P = plan ? plan : h->split;  // (the side stream's products have a workspace of their own)
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if (M % 64 || N % 64 || K % 64) return cudaErrorInvalidValue;
  const int ma_pad = round_up(M, TM), nb_pad = round_up(N, TN), k_pad = round_up(K, h->kappa);  // k_pad <= N + 128
  cudaError_t e;
  if ((e = slice_a(h, A, ma_pad, k_pad, st, P)) != cudaSuccess) return e;
  if ((e = slice_b(h, B, nb_pad, k_pad, st, b_is_final_linv, P)) != cudaSuccess) return e;
  // CTA pairs (256 x 128 per cluster of two, half of each B tile per CTA) with 256-wide chunks when
  // the rows fill whole pairs, unless the handle asks for single CTAs
  const bool pair = h->split_pairs && h->kappa == KAPPA_WIDE && ma_pad % (2 * TM) == 0;
  const int nb = h->nbatch > 1 ? h->nbatch : 1;  // a stacked batch: the digit planes of every graph
  CUtensorMap ta, tb;
  if ((e = make_map(&ta, P->digA, k_pad, (long long)nb * P->s * ma_pad)) != cudaSuccess) return e;
  if ((e = make_map(&tb, P->digB, k_pad, (long long)nb * P->s * nb_pad, pair ? TN / 2 : TN)) != cudaSuccess) return e;
  SplitArgs a{};
  a.eA = P->eA;
  a.eB = P->eB;
  a.ma_pad = ma_pad;
  a.nb_pad = nb_pad;
  a.M = M;
  a.N = N;
  a.K = K;
  a.s = P->s;
  a.a_tri = A.tri;
  a.b_tri = B.tri;
  a.alpha = alpha;
  a.beta = beta;
  a.C = D ? Ystore : C;
  a.ldc = D ? (nb > 1 ? h->N : h->n) : ldc;  // (a stacked batch keeps Y in its N x N matrices)
  a.store_c = (a.C != nullptr);
  a.c_rows = D ? h->n : c_rows;
  a.c_cols = D ? h->n : c_cols;
  a.D = D;
  a.ldd = h->n;
  a.d_rows = D ? h->n : 0;
  a.d_cols = D ? h->n : 0;
  a.log_gamma = log(h->gamma);
  a.inv_log2_gamma = (float)(1.0 / log2(h->gamma));
  a.tau = h->tau;
  a.status = h->dStatus;
  a.row_map = row_map;
  a.col_map = col_map;
  a.nbatch = nb;
  a.bg = nb > 1 ? h->dBatch : nullptr;
  a.s_max = P->s;
  a.ea_gs = (long long)(k_pad / h->kappa) * ma_pad;
  a.eb_gs = (long long)(k_pad / h->kappa) * nb_pad;
  a.c_gs = rd_batch_stride(h, a.C);
  const int tiles = (ma_pad / TM) * (nb_pad / TN);
  // split K when the tiles leave SMs idle (products of a few tiles: the goal and self-check rows,
  // the middle of the recursion), up to two CTAs per SM and 8 per tile, at least one K step
  // (64) each; not with the fused decode
  int ksplit = 1;
  const int ksteps = K / TK, sms = num_sms();
  if (!D && a.store_c && tiles < sms && nb == 1) {  // (a batch has tiles enough)
    ksplit = (2 * sms) / tiles;
    if (ksplit > 8) ksplit = 8;
    if (ksplit > ksteps) ksplit = ksteps;
    if (ksplit < 1) ksplit = 1;
  }
  a.ksplit = ksplit;
  a.partial = nullptr;
  if (ksplit > 1) {
    const size_t need = (size_t)ksplit * ma_pad * nb_pad * sizeof(double);
    if (P->part_bytes < need) {
      if (P->part) {
        rd_dev_free(h, P->part);
        h->bytes -= (int64_t)P->part_bytes;
        P->bytes -= (int64_t)P->part_bytes;
        P->part = nullptr;
        P->part_bytes = 0;
      }
      if ((e = rd_dev_alloc(h, (void**)&P->part, need)) != cudaSuccess) return e;
      P->part_bytes = need;
      P->bytes += (int64_t)need;
      h->bytes += (int64_t)need;
    }
    a.partial = P->part;
  }
  if ((e = rd_prof_begin(h, st, RD_PROF_SPLIT)) != cudaSuccess) return e;
  const int ctas = tiles * ksplit * nb;
  if (pair)
    e = (h->kappa == KAPPA_NARROW) ? launch_split<KAPPA_NARROW, true>(ta, tb, a, ctas, st)
                                   : launch_split<KAPPA_WIDE, true>(ta, tb, a, ctas, st);
  else
    e = (h->kappa == KAPPA_NARROW) ? launch_split<KAPPA_NARROW, false>(ta, tb, a, ctas, st)
                                   : launch_split<KAPPA_WIDE, false>(ta, tb, a, ctas, st);
  if (e != cudaSuccess) return e;
  if ((e = rd_prof_end(h, st, RD_PROF_SPLIT, flops * nb * (double)P->s * (P->s + 1) / 2.0)) != cudaSuccess) return e;
  if (ksplit > 1) {
    if ((e = rd_prof_begin(h, st, RD_PROF_NONE)) != cudaSuccess) return e;
    const long long total = (long long)a.c_rows * a.c_cols;
    ksplit_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P->part, ksplit, ma_pad, nb_pad, a.c_rows,
                                                                          a.c_cols, alpha, beta, a.C, a.ldc, row_map,
                                                                          col_map);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = rd_prof_end(h, st, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

inline View full(const double* p, long long ld, int rows, int cols) { return View{p, ld, rows, cols, RD_TRI_FULL}; }
inline View tri(const double* p, long long ld, int n, int mode) { return View{p, ld, n, n, mode}; }

// Up to this node size the recursion's products run in FP64 with small tiles: 256^3 products are
// 4 tiles of 128 x 128, too few for the tensor cores even with split K, while an FP64 product on
// 16 x 16 tiles spreads over every SM.  At n = 8192 the 512^3 products of the 1024-row nodes took
// 167 us each in FP64; with split K over 64-wide K steps they fill the SMs on the tensor cores.
// (rd_ctx::fp64_node; 512 for one graph, smaller for a stacked batch, whose products have tiles enough)

rd_gemm_f64_args f64_args(const View& A, const View& B, int M, int N, int K, double alpha, double beta, double* C,
                          long long ldc) {
  rd_gemm_f64_args g{};
  g.A = A.p;
  g.lda = A.ld;
  g.a_tri = A.tri;
  g.B = B.p;
  g.ldb = B.ld;
  g.b_tri = B.tri;
  g.C = C;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.alpha = alpha;
  g.beta = beta;
  g.store_c = 1;
  g.c_rows = M;
  g.c_cols = N;
  return g;
}

cudaError_t product(rd_ctx* h, bool fp64, const View& A, const View& B, int M, int N, int K, double alpha,
                    double beta, double* C, long long ldc, double flops, cudaStream_t st) {
  if (!fp64) return split_gemm(h, A, B, M, N, K, alpha, beta, C, ldc, M, N, nullptr, nullptr, flops, st);
  rd_gemm_f64_args g{};
  g.A = A.p;
  g.lda = A.ld;
  g.a_tri = A.tri;
  g.B = B.p;
  g.ldb = B.ld;
  g.b_tri = B.tri;
  g.C = C;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.alpha = alpha;
  g.beta = beta;
  g.store_c = 1;
  g.c_rows = M;
  g.c_cols = N;
  return rd_gemm_f64(h, &g, 1, st, flops);
}

// the least node whose S_L runs on the side stream: smaller products are short, and so are the
// right halves they would overlap
constexpr int SIDE_MIN_NODE = 1024;

// elements of dSL: S_L and V of every depth at once (m1 m2 <= (m/2 + 63) m/2 each, down the right spine)
long long side_sl_elems(long long N) { return 2 * (N * N / 3 + 128 * N); }

// Recursive factorisation of the diagonal range [lo, hi) (see the header comment).  With the
// overlap on, a node's S_L = L21 L11^-1 (m2 x m1) and V = U11^-1 U12 (m1 x m2) are computed on the
// side stream into dSL + sl_off while the right half is factored (the right half's own go beyond
// them), and the U side's block becomes U^-1_12 = -V U22^-1: the same product reassociated, one
// product fewer after the right half.  Every product there is sign-definite (U11^-1 >= 0, U12 <= 0,
// U22^-1 >= 0), so the reassociation keeps each entry accurate relative to itself.
cudaError_t factor(rd_ctx* h, int lo, int hi, cudaStream_t st, long long sl_off = 0, int depth = 0) {
  const int m = hi - lo;
  if (m <= LEAF) return rd_lu_diag(h, lo, st);
  const bool f64 = m <= h->fp64_node;
  const int mid = lo + ((m / 2 + LEAF - 1) / LEAF) * LEAF;
  const int m1 = mid - lo, m2 = hi - mid;
  const long long N = h->N;
  double* LU = h->dLU;
  double* T = h->dT;
  cudaError_t e;
  if ((e = factor(h, lo, mid, st, sl_off, depth + 1)) != cudaSuccess) return e;
  double* A12 = LU + (long long)lo * N + mid;
  double* A21 = LU + (long long)mid * N + lo;
  double* A22 = LU + (long long)mid * N + mid;
  double* T11 = T + (long long)lo * N + lo;
  double* T22 = T + (long long)mid * N + mid;
  const double t1 = (double)m1 * (m1 + 1) / 2, t2 = (double)m2 * (m2 + 1) / 2;
  // U12 = L11^-1 A12 ; L21 = A21 U11^-1.  The split products slice their operands before they
  // write, so they run in place; the small-tile FP64 products do not own whole strips, so they
  // write to the scratch and the result is copied back.
  double* W0 = h->dS;  // free until the inverse products below
  if (f64) {
    // the two independent products of the pair in one launch (each fills only part of the GPU)
    double* W1 = h->dS + (long long)m1 * m2;
    const rd_gemm_f64_args pr[2] = {
        f64_args(tri(T11, N, m1, RD_TRI_LOWER_UNIT), full(A12, N, m1, m2), m1, m2, m1, 1.0, 0.0, W0, m2),
        f64_args(full(A21, N, m2, m1), tri(T11, N, m1, RD_TRI_UPPER), m2, m1, m1, 1.0, 0.0, W1, m1)};
    if ((e = rd_gemm_f64(h, pr, 2, st, 4.0 * t1 * m2)) != cudaSuccess) return e;
    if ((e = rd_copy_rows_out(h, W0, m2, m1, m2, A12, N, st)) != cudaSuccess) return e;
    if ((e = rd_copy_rows_out(h, W1, m1, m2, m1, A21, N, st)) != cudaSuccess) return e;
  } else {
    if ((e = product(h, false, tri(T11, N, m1, RD_TRI_LOWER_UNIT), full(A12, N, m1, m2), m1, m2, m1, 1.0, 0.0, A12,
                     N, 2.0 * t1 * m2, st)) != cudaSuccess)
      return e;
    if ((e = product(h, false, full(A21, N, m2, m1), tri(T11, N, m1, RD_TRI_UPPER), m2, m1, m1, 1.0, 0.0, A21, N,
                     2.0 * t1 * m2, st)) != cudaSuccess)
      return e;
  }
  // S_L = L21 L11^-1 and V = U11^-1 U12 need only the left half: on the side stream, while the right
  // half is factored (the right half writes none of A12, A21, T11; the side products have their own
  // digit workspace)
  const bool side = !f64 && m >= SIDE_MIN_NODE && h->side && h->split_side && depth < RD_SIDE_DEPTH &&
                    sl_off + 2LL * m1 * m2 <= side_sl_elems(N);
  double* SLs = side ? h->dSL + sl_off : nullptr;
  if (side) {
    const cudaEvent_t fork = h->side_ev[2 * depth], join = h->side_ev[2 * depth + 1];
    if ((e = cudaEventRecord(fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->side, fork, 0)) != cudaSuccess) return e;
    if ((e = split_gemm(h, full(A21, N, m2, m1), tri(T11, N, m1, RD_TRI_LOWER_UNIT), m2, m1, m1, 1.0, 0.0, SLs, m1, m2,
                        m1, nullptr, nullptr, 2.0 * t1 * m2, h->side, nullptr, nullptr, false, h->split_side)) !=
        cudaSuccess)
      return e;
    // V = U11^-1 U12 (the U side reassociated: U^-1_12 = -V U22^-1)
    if ((e = split_gemm(h, tri(T11, N, m1, RD_TRI_UPPER), full(A12, N, m1, m2), m1, m2, m1, 1.0, 0.0,
                        SLs + (long long)m1 * m2, m2, m1, m2, nullptr, nullptr, 2.0 * t1 * m2, h->side, nullptr,
                        nullptr, false, h->split_side)) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(join, h->side)) != cudaSuccess) return e;
  }
  // A22 -= L21 U12
  if ((e = product(h, f64, full(A21, N, m2, m1), full(A12, N, m1, m2), m2, m2, m1, -1.0, 1.0, A22, N,
                   2.0 * m2 * (double)m2 * m1, st)) != cudaSuccess)
    return e;
  if ((e = factor(h, mid, hi, st, side ? sl_off + 2LL * m1 * m2 : sl_off, depth + 1)) != cudaSuccess) return e;
  // L^-1_21 = -L22^-1 (L21 L11^-1) ; U^-1_12 = -U11^-1 (U12 U22^-1)
  double* SL = h->dS;                         // m2 x m1
  double* SU = h->dS + (long long)m1 * m2;    // m1 x m2
  if (f64) {  // the L and U chains side by side, two problems per launch
    const double fl = 2.0 * (m2 * t1 + m1 * t2);
    const rd_gemm_f64_args w[2] = {
        f64_args(full(A21, N, m2, m1), tri(T11, N, m1, RD_TRI_LOWER_UNIT), m2, m1, m1, 1.0, 0.0, SL, m1),
        f64_args(full(A12, N, m1, m2), tri(T22, N, m2, RD_TRI_UPPER), m1, m2, m2, 1.0, 0.0, SU, m2)};
    if ((e = rd_gemm_f64(h, w, 2, st, fl)) != cudaSuccess) return e;
    const rd_gemm_f64_args x[2] = {
        f64_args(tri(T22, N, m2, RD_TRI_LOWER_UNIT), full(SL, m1, m2, m1), m2, m1, m2, -1.0, 0.0,
                 T + (long long)mid * N + lo, N),
        f64_args(tri(T11, N, m1, RD_TRI_UPPER), full(SU, m2, m1, m2), m1, m2, m1, -1.0, 0.0, T + (long long)lo * N + mid,
                 N)};
    return rd_gemm_f64(h, x, 2, st, fl);
  }
  if (side) {  // S_L from the side stream
    if ((e = cudaStreamWaitEvent(st, h->side_ev[2 * depth + 1], 0)) != cudaSuccess) return e;
    SL = SLs;
  } else if ((e = product(h, f64, full(A21, N, m2, m1), tri(T11, N, m1, RD_TRI_LOWER_UNIT), m2, m1, m1, 1.0, 0.0, SL,
                          m1, 2.0 * t1 * m2, st)) != cudaSuccess) {
    return e;
  }
  if ((e = product(h, f64, tri(T22, N, m2, RD_TRI_LOWER_UNIT), full(SL, m1, m2, m1), m2, m1, m2, -1.0, 0.0,
                   T + (long long)mid * N + lo, N, 2.0 * t2 * m1, st)) != cudaSuccess)
    return e;
  if (side)  // U^-1_12 = -V U22^-1
    return product(h, f64, full(SLs + (long long)m1 * m2, m2, m1, m2), tri(T22, N, m2, RD_TRI_UPPER), m1, m2, m2, -1.0,
                   0.0, T + (long long)lo * N + mid, N, 2.0 * t2 * m1, st);
  if ((e = product(h, f64, full(A12, N, m1, m2), tri(T22, N, m2, RD_TRI_UPPER), m1, m2, m2, 1.0, 0.0, SU, m2,
                   2.0 * t2 * m1, st)) != cudaSuccess)
    return e;
  return product(h, f64, tri(T11, N, m1, RD_TRI_UPPER), full(SU, m2, m1, m2), m1, m2, m1, -1.0, 0.0,
                 T + (long long)lo * N + mid, N, 2.0 * t1 * m2, st);
}

// rows goals[c] of U^-1 (upper part of T, zero left of the diagonal) into R (64 x N); with the
// locality order, goal g sits at position pos[g]
__global__ void gather_uinv_rows_kernel(const double* __restrict__ T, long long N, const int32_t* __restrict__ goals,
                                        const int32_t* __restrict__ pos, int k, int n, int* status,
                                        double* __restrict__ R) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)RD_MAX_GOALS * N) return;
  const int c = (int)(t / N);
  const long long j = t % N;
  double v = 0.0;
  if (c < k) {
    const int32_t gc = goals[c];
    if (gc >= 0 && gc < n) {
      const long long g = pos ? pos[gc] : gc;
      if (j >= g) v = T[g * N + j];
    } else if (j == 0) {
      rd_goal_ok(gc, n, c, status);  // records the bad goal; its row stays zero
    }
  }
  R[t] = v;
}

}  // namespace

static void side_prepare(rd_ctx* h, int s);

rd_status rd_split_prepare(rd_ctx* h, int s) {
  const int smax = h->ordered ? MAX_SLICES_NARROW : MAX_SLICES_WIDE;
  if (s < 2 || s > smax) {
    h->err = h->ordered ? "split precision needs 2..22 digits in the locality order"
                        : "split precision needs 2..15 digits (0 = chosen by the library)";
    return RD_ERR_ARG;
  }
  if (!encode_fn()) {
    h->err = "cuTensorMapEncodeTiled is not available from the driver";
    return RD_ERR_UNSUPPORTED;
  }
  if (!h->split || h->split->N != h->N || h->split->cap_s < s) {
    rd_split_release(h);
    rd_split_plan* P = new rd_split_plan();
    h->split = P;
    P->N = h->N;
    P->cap_s = s;  // digit planes sized for this count; a later escalation reallocates
    // rows x K padded to whole chunks, for each graph of a stacked batch
    const size_t NK = (size_t)(h->nbatch > 1 ? h->nbatch : 1) * h->N * ((size_t)h->N + KAPPA_WIDE);
    const size_t dig = (size_t)s * NK * sizeof(__nv_bfloat16);
    const size_t ex = (NK / KAPPA_NARROW + 64) * sizeof(int);  // exponents of the narrowest chunks (every graph)
    cudaError_t e = cudaSuccess;
    auto get = [&](void** ptr, size_t bytes) {
      if (e == cudaSuccess) e = rd_dev_alloc(h, ptr, bytes);
      if (e == cudaSuccess) P->bytes += (int64_t)bytes;
    };
    get((void**)&P->digA, dig);
    get((void**)&P->digB, dig);
    get((void**)&P->eA, ex);
    get((void**)&P->eB, ex);
    if (e != cudaSuccess) {
      rd_split_release(h);
      h->err = std::string("split workspace: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? RD_ERR_OOM : RD_ERR_CUDA;
    }
    h->bytes += P->bytes;
  }
  h->split->s = s;
  h->slices = s;
  side_prepare(h, s);
  return RD_OK;
}

void rd_split_workspace(int N, int nbatch, int s, size_t* dig_bytes, size_t* exp_bytes) {
  const size_t NK = (size_t)(nbatch > 1 ? nbatch : 1) * N * ((size_t)N + KAPPA_WIDE);
  *dig_bytes = (size_t)s * NK * sizeof(__nv_bfloat16);
  *exp_bytes = (NK / KAPPA_NARROW + 64) * sizeof(int);
}

rd_status rd_split_prepare_borrowed(rd_ctx* h, int s, void* digA, void* digB, int* eA, int* eB) {
  if (s < 2 || s > MAX_SLICES_WIDE) return RD_ERR_ARG;
  if (!encode_fn()) {
    h->err = "cuTensorMapEncodeTiled is not available from the driver";
    return RD_ERR_UNSUPPORTED;
  }
  rd_split_release(h);
  rd_split_plan* P = new rd_split_plan();
  P->N = h->N;
  P->s = P->cap_s = s;
  P->borrowed = true;
  P->digA = static_cast<__nv_bfloat16*>(digA);
  P->digB = static_cast<__nv_bfloat16*>(digB);
  P->eA = eA;
  P->eB = eB;
  h->split = P;
  h->slices = s;
  return RD_OK;
}

// The overlap's streams, events, S_L buffer and side workspace (work in flight on either stream
// finishes first).
static void side_release(rd_ctx* h) {
  if (h->prio) cudaStreamSynchronize(h->prio);
  if (h->side) cudaStreamSynchronize(h->side);
  if (rd_split_plan* Q = h->split_side) {
    void* ptrs[] = {Q->digA, Q->digB, Q->eA, Q->eB, Q->part};
    for (void* q : ptrs)
      if (q) rd_dev_free(h, q);
    h->bytes -= (h->bytes >= Q->bytes) ? Q->bytes : 0;
    delete Q;
    h->split_side = nullptr;
  }
  if (h->dSL) {
    rd_dev_free(h, h->dSL);
    const int64_t b = (int64_t)side_sl_elems(h->N) * (int64_t)sizeof(double);
    h->bytes -= (h->bytes >= b) ? b : 0;
    h->dSL = nullptr;
  }
  for (cudaEvent_t& ev : h->side_ev)
    if (ev) cudaEventDestroy(ev), ev = nullptr;
  for (cudaEvent_t& ev : h->prio_ev)
    if (ev) cudaEventDestroy(ev), ev = nullptr;
  if (h->side) cudaStreamDestroy(h->side), h->side = nullptr;
  if (h->prio) cudaStreamDestroy(h->prio), h->prio = nullptr;
}

// The overlap's resources for s digits (one graph, N >= RD_SIDE_MIN_N); without them (any failure)
// the recursion runs on one stream, as for every other handle.
static void side_prepare(rd_ctx* h, int s) {
  if (!h->split_overlap || h->nbatch > 1 || h->N < RD_SIDE_MIN_N) return;
  if (h->split_side && h->split_side->cap_s >= s) {
    h->split_side->s = s;
    return;
  }
  side_release(h);
  cudaError_t e = cudaSuccess;
  int least = 0, greatest = 0;
  e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->prio, cudaStreamNonBlocking, greatest);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, least);
  for (cudaEvent_t& ev : h->side_ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  for (cudaEvent_t& ev : h->prio_ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  // the side products' operands: at most N/2 + 63 rows and columns (the recursion's first split)
  rd_split_plan* Q = nullptr;
  if (e == cudaSuccess) {
    Q = new rd_split_plan();
    h->split_side = Q;
    Q->N = h->N;
    Q->s = Q->cap_s = s;
    const size_t half = (size_t)h->N / 2 + 2 * TM;
    const size_t NK = half * (half + KAPPA_WIDE);
    const size_t dig = (size_t)s * NK * sizeof(__nv_bfloat16);
    const size_t ex = (NK / KAPPA_NARROW + 64) * sizeof(int);
    auto get = [&](void** ptr, size_t bytes) {
      if (e == cudaSuccess) e = rd_dev_alloc(h, ptr, bytes);
      if (e == cudaSuccess) Q->bytes += (int64_t)bytes;
    };
    get((void**)&Q->digA, dig);
    get((void**)&Q->digB, dig);
    get((void**)&Q->eA, ex);
    get((void**)&Q->eB, ex);
    if (e == cudaSuccess) h->bytes += Q->bytes;
  }
  if (e == cudaSuccess) {
    const size_t b = (size_t)side_sl_elems(h->N) * sizeof(double);
    e = rd_dev_alloc(h, (void**)&h->dSL, b);
    if (e == cudaSuccess) h->bytes += (int64_t)b;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();  // (not sticky: the handle goes on without the overlap)
    side_release(h);
  }
}

void rd_split_release(rd_ctx* h) {
  side_release(h);
  rd_split_plan* P = h->split;
  if (!P) return;
  if (P->borrowed) P->digA = P->digB = nullptr, P->eA = P->eB = nullptr;
  void* ptrs[] = {P->digA, P->digB, P->eA, P->eB, P->part};
  for (void* q : ptrs)
    if (q) rd_dev_free(h, q);
  h->bytes -= (h->bytes >= P->bytes) ? P->bytes : 0;
  delete P;
  h->split = nullptr;
}

// LU and both triangular inverses are produced together by the recursion.  With the overlap on,
// the recursion runs on the handle's high-priority stream (forked from s and joined back to it),
// so that its kernels take SMs before the side stream's S_L products.
cudaError_t rd_lu_split(rd_ctx* h, cudaStream_t s) {
  if (!h->prio) return factor(h, 0, h->N, s);
  cudaError_t e;
  if ((e = cudaEventRecord(h->prio_ev[0], s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(h->prio, h->prio_ev[0], 0)) != cudaSuccess) return e;
  if ((e = factor(h, 0, h->N, h->prio)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(h->prio_ev[1], h->prio)) != cudaSuccess) return e;
  return cudaStreamWaitEvent(s, h->prio_ev[1], 0);
}


cudaError_t rd_trmm_decode_split(rd_ctx* h, int32_t* D, double* Y, cudaStream_t s) {
  const int N = h->N;
  const double Nd = (double)N;
  const int32_t* map = h->ordered ? h->dOrd : nullptr;  // D and Y back in the caller's node order
  return split_gemm(h, tri(h->dT, N, N, RD_TRI_UPPER), tri(h->dT, N, N, RD_TRI_LOWER_UNIT), N, N, N, 1.0, 0.0,
                    nullptr, 0, 0, 0, D, Y, 2.0 * Nd * (Nd + 1) * (2 * Nd + 1) / 6.0, s, map, map, true);
}

// Self-check of the split result: 64 rows of Y spread over the graph, computed like the goal
// rows (rows of U^-1 times L^-1, the same digit products as the inverse product), and their
// largest entrywise relative residual against M.  Synchronises; *worst receives it.
cudaError_t rd_split_row_check(rd_ctx* h, double* worst, cudaStream_t s) {
  *worst = 0.0;
  if (!h->dSucc) return cudaSuccess;  // no successor lists (more than 2^31 edges): not checked
  const int k = h->n < RD_MAX_GOALS ? h->n : RD_MAX_GOALS;
  int32_t goals[RD_MAX_GOALS];
  for (int c = 0; c < k; ++c) goals[c] = (int32_t)(((long long)c * h->n) / k + (h->n / k) / 2);
  // its own goal buffer: a goal solve has its caller's goals in dGoals while it factors
  cudaError_t e = cudaMemcpyAsync(h->dCheckGoals, goals, k * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  double* rows = h->dS;  // free after the factorisation (64 x n doubles)
  if ((e = rd_goal_split(h, h->dCheckGoals, k, rows, s)) != cudaSuccess) return e;
  if (!h->succ_ready) {
    if ((e = rd_build_succ(h, s)) != cudaSuccess) return e;
    h->succ_ready = 1;
  }
  unsigned long long* res = reinterpret_cast<unsigned long long*>(h->dRed);  // [0] reused after load
  if ((e = cudaMemsetAsync(res, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
  const long long total = (long long)k * h->n;
  if ((e = rd_prof_begin(h, s, RD_PROF_NONE)) != cudaSuccess) return e;
  row_residual_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(rows, h->dCheckGoals, k, h->n, h->dDeg + (h->n + 1),
                                                                       h->dSucc, h->dA, h->weighted ? h->dW : nullptr,
                                                                       h->gamma, res);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  unsigned long long bits = 0;
  if ((e = cudaMemcpyAsync(&bits, res, sizeof(bits), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  memcpy(worst, &bits, sizeof(double));
  return cudaSuccess;
}

// Goal rows from the resident inverses: Y[g, :] = U^-1[g, :] L^-1, all goals in one product
// (64 x N times the lower-unit view of T), written straight into out (k x n).
cudaError_t rd_goal_split(rd_ctx* h, const int32_t* dgoals, int k, double* out, cudaStream_t s) {
  const long long N = h->N;
  cudaError_t e = rd_prof_begin(h, s, RD_PROF_NONE);
  if (e != cudaSuccess) return e;
  const long long total = RD_MAX_GOALS * N;
  gather_uinv_rows_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
      h->dT, N, dgoals, h->ordered ? h->dPos : nullptr, k, h->n, h->dStatus, h->dR);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rd_prof_end(h, s, RD_PROF_NONE, 0.0)) != cudaSuccess) return e;
  const double Nd = (double)N;
  return split_gemm(h, full(h->dR, N, RD_MAX_GOALS, (int)N), tri(h->dT, N, (int)N, RD_TRI_LOWER_UNIT), RD_MAX_GOALS,
                    (int)N, (int)N, 1.0, 0.0, out, h->n, k, h->n, nullptr, nullptr, RD_MAX_GOALS * Nd * (Nd + 1),
                    s, nullptr, h->ordered ? h->dOrd : nullptr, true);
}

// Cycle counters of the split GEMM's roles (the decode products since the last reset); a library built
// without RD_SPLIT_STATS has none.
extern "C" rd_status rd_split_stats(uint64_t* out, int32_t n, int32_t reset) {
  if (!out || n < 1 || n > 16) {
    rd_record_error("rd_split_stats: out not NULL, 1 <= n <= 16");
    return RD_ERR_ARG;
  }
#ifdef RD_SPLIT_STATS
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(out, g_split_stats, sizeof(uint64_t) * (size_t)n);
  if (e == cudaSuccess && reset) {
    const unsigned long long z[16] = {0};
    e = cudaMemcpyToSymbol(g_split_stats, z, sizeof(z));
  }
  if (e != cudaSuccess) {
    rd_record_error(std::string("rd_split_stats: ") + cudaGetErrorString(e));
    return RD_ERR_CUDA;
  }
  return RD_OK;
#else
  rd_record_error("rd_split_stats: this library was built without RD_SPLIT_STATS (build(stats=True))");
  return RD_ERR_UNSUPPORTED;
#endif
}
