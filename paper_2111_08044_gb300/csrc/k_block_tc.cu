// Tensor-core block pass (sm_103a): S' = S U^T on tiles of 128 rows x 64
// complex amplitudes (a window of n = 6 sites), the matrix-unit form of the
// paper's fused-gate contraction (Sec. II, Eq. 2 on fused operators).
//
// Arithmetic.  The FP32 accumulator of tcgen05.mma truncates toward zero
// when it aligns products and when it adds to D, which biases a long
// evolution (measured: a dissipative drift of the energy density).  The
// full-magnitude part of the product is therefore accumulated exactly:
//   - each state row (64 complex = 128 reals) with 2^e_r >= max |x| is cut
//     into three digits, x = 2^(e_r-7) (s0 + s1/256 + s2/65536): s0 and s1
//     balanced 8-bit digits at the row's own units (|s| <= 128, rounded to
//     nearest), s2 the remainder rounded to nearest bf16 (|s2| <= 128; the
//     residual is below 2^-25 of 2^e_r, finer than FP32 rounding of the
//     row's largest entry);
//   - each entry of the fused unitary likewise, u = 2^-7 (u0 + u1/256 +
//     u2/65536), u0 an integer and u1, u2 with 8 significant bits (bf16
//     values; only u0 must be an integer for the exact level-0 sum), the
//     last digit chosen between its two neighbours so that the represented
//     matrix is as close to unitary as the digits allow (a nearest rounding
//     leaves a defect that changes the norm by the same amount every
//     period);
//   - the digits are held as exact bf16 values at their true scale, so the
//     s0 u0 products are integers below 2^14 in units of 2^(e_r-14), and
//     their sum over K = 64 (both complex parts) stays below 2^21 units:
//     the level-0 accumulator is EXACT; all other products (s0u1, s1u0,
//     s0u2, s1u1, s2u0) are at most 2^-8 of the total and go to a second
//     accumulator, whose truncation is 2^-8 smaller relative to the result
//     (kind::f16 with bf16 inputs, FP32 accumulators in TMEM);
//   - the epilogue adds the two with round-to-nearest FP32 arithmetic.
//
// Per CTA (one per SM, persistent over tiles), three warpgroups whose
// register shares are rebalanced with setmaxnreg (168 a thread at launch,
// 128 x (216 + 232 + 56) in total, 224 + 224 + 56 for passes that measure
// nothing):
//   warps 0-3   converters: thread = TMEM lane m, which holds tile row r(m)
//               (a per-pass invertible map over GF(2), chosen so that the
//               epilogue's staging stores spread over the banks); digits of
//               the row into TMEM (tcgen05.st) as the A operand, in two
//               K-halves so that the next tile's conversion overlaps the
//               current tile's MMAs.  Warp 0 also allocates TMEM (512 columns).
//   warps 4-7   epilogue: tcgen05.ld of the two accumulators, energy terms
//               (<X> of window sites in-row; the diagonal part on the natural
//               layout of the period's last pass), then the fused relabel:
//               each amplitude goes to its output place in a 64 KiB staging
//               tile kept in the output's own order under the 128-byte
//               swizzle (one XOR per amplitude, visiting the row in Gray-code
//               order), and one TMA tensor store writes the tile back.
//   warp 8      issues the 96 MMAs of each tile (M=128, N=64, K=16, A in
//               TMEM, B in shared memory), half by half, from one lane of
//               the converged warp elected once; each k-step's 24 MMAs are
//               one asm block (small code: the kernel is bound by its
//               instruction cache more than by its issue rate).
//   warp 9      one thread keeps the TMA producer going: the pass's six
//               64x64 bf16 digit matrices once, then four 128-row x 128-byte
//               boxes per tile (cp.async.bulk.tensor.5d, 128-byte swizzle)
//               into a ring of seven box slots; a slot is refilled as soon as
//               the converters hold its rows in registers.
//   warps 10-11 idle (they complete the third warpgroup for setmaxnreg).
// Every wait is an mbarrier try_wait loop bounded by a clock budget; on
// timeout the CTA raises *status, drains its own copies and MMAs, frees
// TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "sv_block.h"
#include "sv_device.cuh"

namespace fsv {

namespace {

using namespace dev;

constexpr int kN = 6;                 // window width
constexpr int kCols = 1 << kN;        // complex amplitudes per row
constexpr int kRows = 128;            // tile rows = MMA M = TMEM lanes
constexpr int kThreads = 384;         // three warpgroups; registers 216 / 232 / 56 a thread
constexpr uint32_t kTileBytes = kRows * kCols * 8;   // 64 KiB
constexpr uint32_t kBoxBytes = kRows * 128;           // 16 KiB (one 128-byte column box)
constexpr int kSlots = 7;                             // input ring: 1.75 tiles of boxes
constexpr uint32_t kMatBytes = kCols * kCols * 2;     // one 64 x 64 bf16 matrix
constexpr uint32_t kWBytes = 6 * kMatBytes;           // Ur, Ui in three digits: 48 KiB
constexpr uint32_t kOffOut = 0;                       // output staging tile
constexpr uint32_t kOffW = kOffOut + kTileBytes;
constexpr uint32_t kOffRing = kOffW + kWBytes;
constexpr uint32_t kOffMisc = kOffRing + kSlots * kBoxBytes;
constexpr uint32_t kMiscBytes = 1024;
constexpr uint32_t kSmemBytes = kOffMisc + kMiscBytes + 1024;  // + alignment slack
static_assert(kSlots <= 8, "barrier block holds at most 8 slots");
static_assert(kSmemBytes <= 227 * 1024, "dynamic shared memory per CTA");
// TMEM columns: A (bf16 pairs) in two K-halves of 96 columns: half h at
// 96 h holds the s0 / s1 / s2 digit planes of the real and imaginary parts
// for k in [32 h, 32 h + 32) at offsets 0, 16, 32 (real) and 48, 64, 80
// (imaginary).  Accumulators after it.
constexpr uint32_t kAHalf = 96;
constexpr uint32_t kColR0 = 0, kColR1 = 16, kColR2 = 32, kColI0 = 48, kColI1 = 64, kColI2 = 80;
constexpr uint32_t kColAcc = 192;  // L0re, L0im, Rre, Rim (64 each)
constexpr long long kTimeoutCycles = 4000000000ll;  // about 2 s at 2 GHz

// misc block layout (offsets from kOffMisc)
enum : uint32_t {
  kBarFull = 0,      // kSlots x 8 (at most 8 slots): box slot loaded
  kBarEmpty = 64,    // kSlots x 8: box slot read by the converters
  kBarW = 128,       // operand block loaded
  kBarAReady = 136,  // 2 x 8: A half h written
  kBarAFree = 152,   // 2 x 8: A half h consumed by the MMAs
  kBarDFull = 168,   // accumulators complete
  kBarDFree = 176,   // accumulators read out
  kBarMmaDone = 184,
  kTmemSlot = 192,
  kAbort = 196,
  kBarWFree = 200,   // chain group: the MMAs are done with the operand block
  kRed = 256,        // 4 x 2 doubles
  kDiagQ = 512,      // 64 floats (to 768): window-window bond part of the diagonal
  kGroupCoef = 768,  // chain group: cx[6], diag_f[5], diag_lin0[6] of the current chain
};

// A tensor map written by the host into global memory is read through the
// tensormap proxy: acquire it before its first use.
__device__ __forceinline__ void tensormap_acquire(const void* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                   reinterpret_cast<uint64_t>(map))
               : "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false on abort (raised here on timeout, or by another role).
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile uint32_t* abort,
                                         int* status) {
  // the common case first: the phase is already complete
  if (__builtin_expect(mbar_try_wait(bar, parity), 1)) return true;
  const long long t0 = clock64();
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 31) == 0) {
      if (*abort) return false;
      if (clock64() - t0 > kTimeoutCycles) {
        *abort = 1;
        atomicExch(status, 1);
        return false;
      }
    }
  }
  return true;
}

// All 128 epilogue threads (named barrier 1) agree: true only if every
// thread's ok is true.  Each thread arrives exactly once per call.
__device__ __forceinline__ bool epilogue_all_ok(bool ok) {
  uint32_t any_bad;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n"
      " bar.red.or.pred p, 1, 128, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(any_bad)
      : "r"((uint32_t)(!ok))
      : "memory");
  return any_bad == 0;
}
__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, uint32_t src, int c0, int c1,
                                             int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group"
      " [%0, {%2, %3, %4}], [%1];" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(src), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, uint32_t src, int c0, int c1,
                                             int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group"
      " [%0, {%2, %3, %4, %5}], [%1];" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(src), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}
__device__ __forceinline__ void tma_store_5d(const CUtensorMap* map, uint32_t src, int c0, int c1,
                                             int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group"
      " [%0, {%2, %3, %4, %5, %6}], [%1];" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(src), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}
// Byte offset of a staging-tile byte under the 128-byte swizzle: the
// 16-byte chunk index (bits 4-6) is XORed with the 128-byte line index
// modulo 8 (bits 7-9).  Linear over XOR.
__host__ __device__ constexpr uint32_t swz128(uint32_t b) { return b ^ (((b >> 7) & 7u) << 4); }
// index of the lowest set bit of g > 0 (the bit a Gray code flips at step g)
__host__ __device__ constexpr int low_bit(int g) {
  int k = 0;
  while (!((g >> k) & 1)) ++k;
  return k;
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle, core matrices of
// 8 rows x 16 bytes (8 bf16); LBO = 1024 B between core matrices along K,
// SBO = 128 B between 8-row groups along N.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  return d;
}

// Instruction descriptor: kind::f16 with D = F32, A = B = BF16, both
// K-major, N = 64, M = 128, optional negation of B.
__host__ __device__ constexpr uint32_t make_idesc(int negate_b) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)negate_b << 14) |
         ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

// Issued by one elected lane while the whole warp runs the issue loop: the
// operands are then warp-uniform and the MMAs go out at the tensor pipe's
// rate (an N = 64 MMA every 32 cycles, against about 50 for a lone lane).
// The 24 MMAs of one k-step (K = 16) into the four accumulators, issued by
// the lane that `leader` marks (one elect for the whole loop), in one block
// so that each operand is moved to the issue path once per k-step:
//   L0re += s0r Ur0 - s0i Ui0         L0im += s0r Ui0 + s0i Ur0   (exact)
//   Rre  += s0r Ur1 + s1r Ur0 + s0r Ur2 + s1r Ur1 + s2r Ur0
//         - (s0i Ui1 + s1i Ui0 + s0i Ui2 + s1i Ui1 + s2i Ui0)
//   Rim  += s0r Ui1 + s1r Ui0 + s0r Ui2 + s1r Ui1 + s2r Ui0
//         + s0i Ur1 + s1i Ur0 + s0i Ur2 + s1i Ur1 + s2i Ur0
// (A digit planes s* in TMEM; the B digit matrices U* by descriptor; idesc
// ip adds, in subtracts; `accumulate` = 0 starts each accumulator).
__device__ __forceinline__ void mma_kstep(uint32_t leader, uint32_t accumulate, uint32_t l0r,
                                          uint32_t l0i, uint32_t rr, uint32_t ri, uint32_t r0,
                                          uint32_t r1, uint32_t r2, uint32_t i0, uint32_t i1,
                                          uint32_t i2, uint64_t ur0, uint64_t ur1, uint64_t ur2,
                                          uint64_t ui0, uint64_t ui1, uint64_t ui2, uint32_t ip,
                                          uint32_t in) {
#define FSV_MMA(d, a, b, i, p) " @e tcgen05.mma.cta_group::1.kind::f16 [" d "], [" a "], " b ", " i ", " p ";\n"
  asm volatile(
      "{\n .reg .pred e, p, t;\n"
      " setp.ne.b32 e, %0, 0;\n setp.ne.b32 p, %1, 0;\n setp.ne.b32 t, %18, 0;\n"
      FSV_MMA("%2", "%6", "%12", "%18", "p") FSV_MMA("%2", "%9", "%15", "%19", "t")
      FSV_MMA("%3", "%6", "%15", "%18", "p") FSV_MMA("%3", "%9", "%12", "%18", "t")
      FSV_MMA("%4", "%6", "%13", "%18", "p") FSV_MMA("%4", "%7", "%12", "%18", "t")
      FSV_MMA("%4", "%6", "%14", "%18", "t") FSV_MMA("%4", "%7", "%13", "%18", "t")
      FSV_MMA("%4", "%8", "%12", "%18", "t") FSV_MMA("%4", "%9", "%16", "%19", "t")
      FSV_MMA("%4", "%10", "%15", "%19", "t") FSV_MMA("%4", "%9", "%17", "%19", "t")
      FSV_MMA("%4", "%10", "%16", "%19", "t") FSV_MMA("%4", "%11", "%15", "%19", "t")
      FSV_MMA("%5", "%6", "%16", "%18", "p") FSV_MMA("%5", "%7", "%15", "%18", "t")
      FSV_MMA("%5", "%6", "%17", "%18", "t") FSV_MMA("%5", "%7", "%16", "%18", "t")
      FSV_MMA("%5", "%8", "%15", "%18", "t") FSV_MMA("%5", "%9", "%13", "%18", "t")
      FSV_MMA("%5", "%10", "%12", "%18", "t") FSV_MMA("%5", "%9", "%14", "%18", "t")
      FSV_MMA("%5", "%10", "%13", "%18", "t") FSV_MMA("%5", "%11", "%12", "%18", "t")
      "}\n" ::"r"(leader), "r"(accumulate), "r"(l0r), "r"(l0i), "r"(rr), "r"(ri), "r"(r0),
      "r"(r1), "r"(r2), "r"(i0), "r"(i1), "r"(i2), "l"(ur0), "l"(ur1), "l"(ur2), "l"(ui0),
      "l"(ui1), "l"(ui2), "r"(ip), "r"(in)
      : "memory");
#undef FSV_MMA
}

// tcgen05.commit from the lane that `leader` marks
__device__ __forceinline__ void mma_commit(uint32_t leader, uint32_t bar) {
  asm volatile(
      "{\n .reg .pred e;\n setp.ne.b32 e, %0, 0;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%1];\n}\n" ::"r"(
          leader),
      "r"(bar)
      : "memory");
}

// Two FP32 values rounded to nearest bf16 (one conversion instruction),
// packed with `lo` in the low half.
__device__ __forceinline__ uint32_t cvt_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Largest of three FP32 values (one three-input max on sm_100 and later).
__device__ __forceinline__ float max3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Two values with at most 8 significant bits each, packed as bf16x2 with
// `lo` in the low half: their FP32 encodings end in 16 zero bits, so the
// bf16 values are the high halves (a byte permute, no rounding).
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// Packed FP32 pairs (two lanes per instruction on the FP32 pipe).
__device__ __forceinline__ uint64_t f2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_split(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// Rounding with the FP32 adder: for |v| < 2^(q-1), (v + M) - M with
// M = 1.5 * 2^q is v rounded to nearest (ties to even) at the unit
// 2^(q-23); both additions are exact apart from that one rounding.
__device__ __forceinline__ uint64_t round_at2(uint64_t v, uint64_t m) { return sub2(add2(v, m), m); }
// 1.5 * 2^q as a float, for -126 < q < 128
__device__ __forceinline__ float magic(int q) {
  return __uint_as_float(((uint32_t)(q + 127) << 23) | 0x400000u);
}

// Tile row held by TMEM lane m: XOR over the set bits i of m of rowvec[i].
__device__ __forceinline__ int tile_row(const PassArgs& pa, int m) {
  int r = 0;
#pragma unroll
  for (int i = 0; i < 7; ++i)
    if ((m >> i) & 1) r ^= pa.rowvec[i];
  return r;
}

// kX: the pass measures <X> of window sites; kDiag: it measures the
// diagonal part and the norm (the period's last pass).  A pass whose CTAs
// run many tiles takes the instance of its combination, whose epilogue is
// compiled (and register-allocated) for only the work it does; short passes
// (small chains, many of them at once in a batch) all take the generic
// instance (kGeneric, flags read at run time), so that SMs switching between
// their CTAs keep one kernel's code in the instruction cache.
//
// kGroup (with kGeneric): one launch over the tiles of a chain group.  Tile
// g of the group is tile g mod 2^nt_log2 of chain g / 2^nt_log2; a CTA takes
// a contiguous range of them, so it meets each chain once.  At a change of
// chain the producer reloads the operand block once the MMAs are done with
// the previous one (kBarWFree), and the epilogue writes the previous chain's
// partial sums and takes the new chain's coefficients and descriptors.
template <bool kGeneric, bool kX, bool kDiag, bool kGroup = false>
__global__ void __launch_bounds__(kThreads, 1)
    k_block_tc(const __grid_constant__ CUtensorMap tmap_in,
               const __grid_constant__ CUtensorMap tmap_out, PassArgs pa, int* status,
               const GroupChain* __restrict__ grp, int nt_log2) {
  static_assert(!kGroup || kGeneric, "a group pass takes the generic epilogue");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(smem);
  uint8_t* misc = smem + kOffMisc;
  const uint32_t mbase = sbase + kOffMisc;
  volatile uint32_t* abort = reinterpret_cast<volatile uint32_t*>(misc + kAbort);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = pa.a;
  const long long ntiles = pa.ntiles;
  // this CTA's tiles: strided over the pass, or (group) a contiguous range
  const long long my_first = kGroup ? (long long)blockIdx.x * ntiles / gridDim.x : 0;
  const long long my_tiles =
      kGroup ? ((long long)blockIdx.x + 1) * ntiles / gridDim.x - my_first
             : (blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0);
  // tile index within its chain, and the chain, of this CTA's tile i
  auto tile_of = [&](long long i) -> long long {
    return kGroup ? ((my_first + i) & ((1ll << nt_log2) - 1)) : blockIdx.x + i * gridDim.x;
  };
  auto chain_of = [&](long long i) -> int { return kGroup ? (int)((my_first + i) >> nt_log2) : 0; };
  // tile i starts a chain other than tile i - 1's
  auto new_chain = [&](long long i) -> bool {
    return kGroup && i > 0 && chain_of(i) != chain_of(i - 1);
  };

  if (threadIdx.x == 0) {
    for (int b = 0; b < kSlots; ++b) {
      mbar_init(mbase + kBarFull + 8 * b, 1);
      mbar_init(mbase + kBarEmpty + 8 * b, 128);
    }
    mbar_init(mbase + kBarW, 1);
    mbar_init(mbase + kBarAReady, 128);
    mbar_init(mbase + kBarAReady + 8, 128);
    mbar_init(mbase + kBarAFree, 1);
    mbar_init(mbase + kBarAFree + 8, 1);
    mbar_init(mbase + kBarDFull, 1);
    mbar_init(mbase + kBarDFree, 128);
    mbar_init(mbase + kBarMmaDone, 1);
    mbar_init(mbase + kBarWFree, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     mbase + kTmemSlot)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(misc + kTmemSlot);

  const int wg = warp >> 2;
  if (wg == 0) {
    // ------------------------------------------------------------ converters
    // register shares: 216 / 232 / 56 when the epilogue measures, else
    // 224 / 224 / 56 (both sum to the 168 x 3 a thread the CTA launched with)
    if constexpr (kGeneric || kX || kDiag)
      asm volatile("setmaxnreg.inc.sync.aligned.u32 216;" ::: "memory");
    else asm volatile("setmaxnreg.inc.sync.aligned.u32 224;" ::: "memory");
    const int r = tile_row(pa, warp * 32 + lane);  // the tile row of this TMEM lane
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    for (long long i = 0; i < my_tiles; ++i) {
      // box c of tile i is load number g = 4 i + c, in ring slot g mod kSlots
      const long long g0 = 4 * i;
      const int s0 = (int)(g0 % kSlots);
      auto slot = [s0](int c) { return s0 + c >= kSlots ? s0 + c - kSlots : s0 + c; };
      // the row (64 complex) into registers box by box as they land;
      // exponent 2^e >= max |x|
      float4 row[32];
      float m = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const long long g = g0 + c;
        if (ok) ok = wait_bar(mbase + kBarFull + 8 * slot(c), (uint32_t)((g / kSlots) & 1), abort,
                              status);
        if (__any_sync(0xffffffffu, !ok)) {  // the warp leaves together
          ok = false;
          break;
        }
#pragma unroll
        for (int q = 8 * c; q < 8 * c + 8; ++q) {
          row[q] = *reinterpret_cast<const float4*>(smem + kOffRing + slot(c) * kBoxBytes +
                                                    r * 128 + (((q & 7) ^ (r & 7)) << 4));
          m = max3(max3(m, fabsf(row[q].x), fabsf(row[q].y)), fabsf(row[q].z), fabsf(row[q].w));
        }
      }
      if (!ok) break;
      // Hand the four slots back to the producer.  The next TMA load into a
      // slot writes through the async proxy, so the generic-proxy reads
      // above are ordered before it by a proxy fence ahead of the release
      // (without it the copy could overwrite a slot still being read).
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
      for (int c = 0; c < 4; ++c) mbar_arrive(mbase + kBarEmpty + 8 * slot(c));
      // 2^e >= max |x| (m = f 2^e, f in [0.5, 1)); rows below 2^-100 are
      // cut at that unit (their digits stay normal bf16 numbers)
      int e = -100;
      if (m > 0x1p-100f) frexpf(m, &e);
      // digit units 2^(e-7), 2^(e-15); the last digit is the remainder in bf16
      const uint64_t M0 = f2(magic(e + 16), magic(e + 16)), M1 = f2(magic(e + 8), magic(e + 8));
      for (int h = 0; h < 2 && ok; ++h) {
        if (i >= 1)
          ok = wait_bar(mbase + kBarAFree + 8 * h, (uint32_t)((i - 1) & 1), abort, status);
        if (__any_sync(0xffffffffu, !ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int c = 2 * h + cc;  // 16-amplitude chunk, k in [16 c, 16 c + 16)
          uint32_t r0[8], r1[8], r2[8], i0[8], i1[8], i2[8];
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            const float4 v = row[8 * c + s];
            // amplitudes k = 16c + 2s and 16c + 2s + 1: (v.x, v.y), (v.z, v.w)
            const uint64_t p[2] = {f2(v.x, v.y), f2(v.z, v.w)};
            float d0[4], d1[4], d2[4];  // re k, im k, re k+1, im k+1
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              // the first two digits at most 128 of their unit (8 bits,
              // exact in bf16); the remainders are exact, and the second
              // remainder (at most 2^(e-16)) is rounded to bf16 below
              const uint64_t a0 = round_at2(p[t], M0);
              const uint64_t q1 = sub2(p[t], a0);
              const uint64_t a1 = round_at2(q1, M1);
              f2_split(a0, d0[2 * t], d0[2 * t + 1]);
              f2_split(a1, d1[2 * t], d1[2 * t + 1]);
              f2_split(sub2(q1, a1), d2[2 * t], d2[2 * t + 1]);
            }
            r0[s] = pack_bf16x2(d0[0], d0[2]);
            i0[s] = pack_bf16x2(d0[1], d0[3]);
            r1[s] = pack_bf16x2(d1[0], d1[2]);
            i1[s] = pack_bf16x2(d1[1], d1[3]);
            r2[s] = cvt_bf16x2(d2[0], d2[2]);
            i2[s] = cvt_bf16x2(d2[1], d2[3]);
          }
          const uint32_t hb = lane_base + kAHalf * h + 8 * cc;
          tmem_st8(hb + kColR0, r0);
          tmem_st8(hb + kColR1, r1);
          tmem_st8(hb + kColR2, r2);
          tmem_st8(hb + kColI0, i0);
          tmem_st8(hb + kColI1, i1);
          tmem_st8(hb + kColI2, i2);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        mbar_arrive(mbase + kBarAReady + 8 * h);
      }
      if (__any_sync(0xffffffffu, !ok)) break;
    }
  } else if (wg == 1) {
    // ------------------------------------------------------------ epilogue
    if constexpr (kGeneric || kX || kDiag)
      asm volatile("setmaxnreg.inc.sync.aligned.u32 232;" ::: "memory");
    else asm volatile("setmaxnreg.inc.sync.aligned.u32 224;" ::: "memory");
    const int q = warp - 4;
    const int r = tile_row(pa, q * 32 + lane);  // the tile row of this TMEM lane
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    const bool elected = q == 0 && lane == 0;  // issues the tile's TMA store
    // Output tile bits: row bit b of this tile goes to output bit sigma[6+b],
    // window bit j to sigma[j]; output bits 0-5 are the next window (the
    // contiguous 64 amplitudes), bits 6-12 the next rows.  The staging tile
    // holds amplitude y at byte swz128(8 y), so the place of this row's
    // element c is row_off ^ (XOR over set bits j of c of col_off[j]).
    // Output bit o sits at bit spos[o] of the staging tile (ssig = spos o
    // sigma), an order chosen per pass against bank conflicts of the stores.
    uint32_t yrow = 0, ystage = 0;
    for (int bq = 0; bq < 7; ++bq) {
      yrow |= ((uint32_t)(r >> bq) & 1u) << pa.sigma[kN + bq];
      ystage |= ((uint32_t)(r >> bq) & 1u) << pa.ssig[kN + bq];
    }
    const uint32_t row_off = swz128(8u * ystage);
    uint32_t col_off[kN];
#pragma unroll
    for (int j = 0; j < kN; ++j) col_off[j] = swz128(8u << pa.ssig[j]);
    const uint32_t out_base = sbase + kOffOut;
    // Diagonal part of the period's last pass, per amplitude (x its natural
    // index) h(x) = J sum_p z_p z_{p+1} + sum_p cz_p z_p, z = 1 - 2 x_p.
    // Within a row only the output bits fed by window bits change with c:
    // h(x_c) = h(x_0) + sum_j c_j lin_j + Q[c], where lin_j is the change of
    // flipping window bit j alone (its field and its bonds to the fixed
    // bits, window neighbours counted at 0) and Q[c] = 4 J sum over adjacent
    // window pairs of c_j c_k, a 64-entry table shared by all rows.
    float* diag_q = reinterpret_cast<float*>(misc + kDiagQ);
    const bool do_x = kGeneric ? pa.x_mask != 0 : kX;
    const bool do_diag = kGeneric ? pa.diag != 0 : kDiag;
    // the measured coefficients: the pass's, or (group) the current chain's
    float* gco = reinterpret_cast<float*>(misc + kGroupCoef);
    auto CX = [&](int j) -> float {
      if constexpr (kGroup) return gco[j];
      else return pa.cx[j];
    };
    auto DF = [&](int k) -> float {
      if constexpr (kGroup) return gco[6 + k];
      else return pa.diag_f[k];
    };
    auto LIN0 = [&](int j) -> float {
      if constexpr (kGroup) return gco[11 + j];
      else return pa.diag_lin0[j];
    };
    if (!kGroup && do_diag) {
      if (r < kCols) {
        // window bits j and k are sites lo + j and lo + k: adjacent when
        // |j - k| = 1
        float qv = 0.f;
        for (int j = 0; j + 1 < kN; ++j)
          if (((r >> j) & 1) && ((r >> (j + 1)) & 1)) qv += 4.f * (float)pa.ep.J;
        diag_q[r] = qv;
      }
      epilogue_sync();
    }
    const float sc = (float)renorm_scale(pa.ep.rn);
    const uint64_t sc2 = f2(sc, sc);
    // per-thread energy and norm over its tiles: compensated FP32 sums
    // (Kahan), so that no FP64 instruction runs per tile
    float es_s = 0.f, es_c = 0.f, ns_s = 0.f, ns_c = 0.f;
    // energy partials of this CTA into part[2 blockIdx.x + {0, 1}] (fixed order)
    auto flush = [&](double* part) {
      if (!part) return;
      double eacc = (double)es_s - (double)es_c, nacc = (double)ns_s - (double)ns_c;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
        nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
      }
      double* red = reinterpret_cast<double*>(misc + kRed);
      if (lane == 0) {
        red[2 * q] = eacc;
        red[2 * q + 1] = nacc;
      }
      epilogue_sync();
      if (q == 0 && lane == 0) {
        part[2 * blockIdx.x] = (red[0] + red[2]) + (red[4] + red[6]);
        part[2 * blockIdx.x + 1] = (red[1] + red[3]) + (red[5] + red[7]);
      }
    };
    int cur = -1;  // group: the chain whose coefficients are loaded
    const CUtensorMap* map_out = &tmap_out;
    for (long long i = 0; i < my_tiles; ++i) {
      if constexpr (kGroup) {
        const int c = chain_of(i);
        if (c != cur) {
          if (cur >= 0) {
            flush(grp[cur].partial);
            es_s = es_c = ns_s = ns_c = 0.f;
          }
          epilogue_sync();  // the previous chain's coefficients are no longer read
          const GroupChain& gc = grp[c];
          if (q == 0 && lane < 17)
            gco[lane] = lane < 6 ? gc.cx[lane] : (lane < 11 ? gc.diag_f[lane - 6] : gc.diag_lin0[lane - 11]);
          if (do_diag && r < kCols) {
            float qv = 0.f;
            for (int j = 0; j + 1 < kN; ++j)
              if (((r >> j) & 1) && ((r >> (j + 1)) & 1)) qv += 4.f * gc.diag_f[0];
            diag_q[r] = qv;
          }
          map_out = reinterpret_cast<const CUtensorMap*>(gc.map_out);
          if (elected) tensormap_acquire(map_out);
          epilogue_sync();
          cur = c;
        }
      }
      const bool ok = wait_bar(mbase + kBarDFull, (uint32_t)(i & 1), abort, status);
      if (!epilogue_all_ok(ok)) break;  // the four epilogue warps leave together
      tc_fence_after();
      float re[kCols], im[kCols];
      const uint32_t acc = lane_base + kColAcc;
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        uint32_t v0[16], v1[16], w0[16], w1[16];
        tmem_ld16(acc + 16 * c4, v0);        // L0 re
        tmem_ld16(acc + 128 + 16 * c4, v1);  // R re
        tmem_ld16(acc + 64 + 16 * c4, w0);   // L0 im
        tmem_ld16(acc + 192 + 16 * c4, w1);  // R im
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
          const uint64_t sre = mul2(add2(f2(__uint_as_float(v0[e]), __uint_as_float(v0[e + 1])),
                                         f2(__uint_as_float(v1[e]), __uint_as_float(v1[e + 1]))),
                                    sc2);
          const uint64_t sim = mul2(add2(f2(__uint_as_float(w0[e]), __uint_as_float(w0[e + 1])),
                                         f2(__uint_as_float(w1[e]), __uint_as_float(w1[e + 1]))),
                                    sc2);
          f2_split(sre, re[16 * c4 + e], re[16 * c4 + e + 1]);
          f2_split(sim, im[16 * c4 + e], im[16 * c4 + e + 1]);
        }
      }
      tc_fence_before();
      mbar_arrive(mbase + kBarDFree);  // the accumulators may be overwritten
      float es = 0.f, ns = 0.f;
      if (do_x) {
        // <X_j> part of the row: 2 sum over c with bit j clear of
        // re_c re_c' + im_c im_c', c' = c + 2^j, for the bits this pass
        // measures; for j >= 1 two neighbouring columns go through one
        // packed FMA
#pragma unroll
        for (int j = 0; j < kN; ++j) {
          if (!((pa.x_mask >> j) & 1)) continue;
          float sj;
          if (j == 0) {
            float t0 = 0.f, t1 = 0.f;
#pragma unroll
            for (int c = 0; c < kCols; c += 2) {
              t0 = fmaf(re[c], re[c + 1], t0);
              t1 = fmaf(im[c], im[c + 1], t1);
            }
            sj = t0 + t1;
          } else {
            uint64_t xacc = f2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < kCols; c += 2) {
              if ((c >> j) & 1) continue;
              const int c2 = c + (1 << j);
              xacc = fma2(f2(re[c], re[c + 1]), f2(re[c2], re[c2 + 1]), xacc);
              xacc = fma2(f2(im[c], im[c + 1]), f2(im[c2], im[c2 + 1]), xacc);
            }
            float lo, hi;
            f2_split(xacc, lo, hi);
            sj = lo + hi;
          }
          es += 2.f * CX(j) * sj;
        }
      }
      const long long t = tile_of(i);
      const uint32_t tlo = (uint32_t)(t & ((1ll << (a - kN)) - 1));
      const uint32_t thi = (uint32_t)(t >> (a - kN));
      if (do_diag) {
        // the diagonal part and the norm on the amplitudes' natural indices:
        // x0, the row's amplitude at c = 0, mapped from the output's layout
        const uint64_t tbase = ((uint64_t)tlo << kN) | ((uint64_t)thi << (a + 7));
        const uint64_t x0 = to_natural(
            tbase | (yrow & (kCols - 1)) | ((uint64_t)(yrow >> kN) << a), kN, pa.diag_lo);
        // FP32 coefficients rounded on the host (no FP64 work per tile)
        Diag<float> dg;
        dg.L = pa.L;
        dg.J = DF(0);
        dg.cz_bulk = DF(1);
        dg.cz_first = DF(2);
        dg.cz_last = DF(3);
        dg.czsum = DF(4);
        dg.zzmask = (1ull << (pa.L - 1)) - 1;
        dg.bulkmask = ((1ull << pa.L) - 1) & ~1ull & ~(1ull << (pa.L - 1));
        const float h0 = dg(x0);
        // lin_j = -2 (cz + J sum of the neighbours' z at c = 0): the field and
        // the window neighbours (bit 0 at c = 0) come precomputed per pass;
        // only the neighbours outside the window are read from x0
        float lin[kN];
#pragma unroll
        for (int j = 0; j < kN; ++j) {
          float nb = 0.f;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int ps = pa.diag_nb[j][k];
            if (ps >= 0) nb += ((x0 >> ps) & 1) ? -1.f : 1.f;
          }
          lin[j] = fmaf(-2.f * dg.J, nb, LIN0(j));
        }
        // h(x_c) = h0 + L(c) + Q[c] with L(c) = sum_j c_j lin_j.  The row is
        // taken in pairs (c, c + 1) = (2k, 2k + 1), k in Gray-code order, so
        // W = (L(2k), L(2k) + lin_0) changes by one lin per step; packed,
        // sum_c p_c h = h0 S + sum_k P_k . (W_k + Q_k), S = sum_c p_c.
        float w_lo = 0.f, w_hi = lin[0];
        uint64_t tot = f2(0.f, 0.f), acc = tot;
        const uint64_t* q2 = reinterpret_cast<const uint64_t*>(diag_q);
#pragma unroll
        for (int g = 0; g < kCols / 2; ++g) {
          const int k = g ^ (g >> 1);
          if (g > 0) {
            const int b = low_bit(g);  // pair bit b is window bit b + 1
            const float d = ((k >> b) & 1) ? lin[b + 1] : -lin[b + 1];
            w_lo += d;
            w_hi += d;
          }
          const uint64_t rr = f2(re[2 * k], re[2 * k + 1]), ii = f2(im[2 * k], im[2 * k + 1]);
          const uint64_t p = fma2(rr, rr, mul2(ii, ii));
          tot = add2(tot, p);
          acc = fma2(p, add2(f2(w_lo, w_hi), q2[k]), acc);
        }
        float t_lo, t_hi, a_lo, a_hi;
        f2_split(tot, t_lo, t_hi);
        f2_split(acc, a_lo, a_hi);
        const float S = t_lo + t_hi;
        ns += S;
        es += fmaf(h0, S, a_lo + a_hi);
      }
      {
        const float ye = es - es_c, te = es_s + ye;
        es_c = (te - es_s) - ye;
        es_s = te;
        const float yn = ns - ns_c, tn = ns_s + yn;
        ns_c = (tn - ns_s) - yn;
        ns_s = tn;
      }
      // the staging tile is free once the previous tile's store has read it
      if (elected) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      epilogue_sync();
      // Relabelled write of the row, visiting c in Gray-code order so that
      // one XOR moves the place from one element to the next; the 32 lanes
      // of a store differ in row bits only.
      uint32_t o = row_off;
#pragma unroll
      for (int g = 0; g < kCols; ++g) {
        const int c = g ^ (g >> 1);
        if (g > 0) o ^= col_off[low_bit(g)];
        asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(out_base + o), "f"(re[c]),
                     "f"(im[c])
                     : "memory");
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      epilogue_sync();
      if (elected) {
        if (pa.st_ndims == 3) {
          // the natural order: output bits 4-5, then the rows
          tma_store_3d(map_out, out_base, 0, (int)(tlo << 2), (int)(thi << 7));
        } else {
          // the tile-index bits go to the store view's dimensions that their
          // state bits continue
          auto coord = [&](int d) {
            return (d == pa.st_tlo_dim ? (int)(tlo << pa.st_tlo_shift) : 0) |
                   (d == pa.st_thi_dim ? (int)(thi << pa.st_thi_shift) : 0);
          };
          if (pa.st_ndims == 4)
            tma_store_4d(map_out, out_base, 0, coord(1), coord(2), coord(3));
          else
            tma_store_5d(map_out, out_base, 0, coord(1), coord(2), coord(3), coord(4));
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    // the CTA's stores complete before its shared memory is released
    if (elected) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if constexpr (kGroup) {
      if (cur >= 0) flush(grp[cur].partial);
    } else {
      flush(pa.partial);
    }
  } else {
    // ----------------------------------- MMA issue (warp 8), producer (warp 9)
    asm volatile("setmaxnreg.dec.sync.aligned.u32 56;" ::: "memory");
    const uint32_t w0 = sbase + kOffW;
    if (warp == 8) {
      // the whole warp runs this loop; the MMAs and commits issue from one lane
      const uint32_t tm = __shfl_sync(0xffffffffu, tmem, 0);
      const uint64_t dr0 = make_desc(w0), dr1 = make_desc(w0 + kMatBytes),
                     dr2 = make_desc(w0 + 2 * kMatBytes), di0 = make_desc(w0 + 3 * kMatBytes),
                     di1 = make_desc(w0 + 4 * kMatBytes), di2 = make_desc(w0 + 5 * kMatBytes);
      constexpr uint32_t ip = make_idesc(0), in = make_idesc(1);
      const uint32_t l0r = tm + kColAcc, l0i = l0r + 64, rr_ = l0r + 128, ri_ = l0r + 192;
      uint32_t leader;  // the lane that issues the MMAs
      asm volatile("{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n selp.u32 %0, 1, 0, e;\n}\n"
                   : "=r"(leader));
      bool ok = __all_sync(0xffffffffu, wait_bar(mbase + kBarW, 0, abort, status));
      int wload = 0;  // group: operand blocks loaded after the first
      for (long long i = 0; i < my_tiles && ok; ++i) {
        if (new_chain(i)) {
          // the new chain's operand block
          ++wload;
          ok = __all_sync(0xffffffffu,
                          wait_bar(mbase + kBarW, (uint32_t)(wload & 1), abort, status));
          if (!ok) break;
        }
#pragma unroll 1
        for (int h = 0; h < 2 && ok; ++h) {
          // half h of tile i once its A digits are written and, for the first
          // half, once the epilogue has read out tile i - 1
          ok = wait_bar(mbase + kBarAReady + 8 * h, (uint32_t)(i & 1), abort, status);
          if (ok && h == 0 && i >= 1)
            ok = wait_bar(mbase + kBarDFree, (uint32_t)((i - 1) & 1), abort, status);
          ok = __all_sync(0xffffffffu, ok);  // the warp stays converged
          if (!ok) break;
          tc_fence_after();
          const uint32_t ab = tm + kAHalf * h;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            // global k-step 2h + ks (K = 16): two core matrices along K
            const uint64_t ko = (uint64_t)((2 * (2 * h + ks) * 1024) >> 4);
            const uint32_t acc = (h > 0 || ks > 0) ? 1u : 0u;
            const uint32_t r0 = ab + kColR0 + 8 * ks, r1 = ab + kColR1 + 8 * ks,
                           r2 = ab + kColR2 + 8 * ks;
            const uint32_t i0 = ab + kColI0 + 8 * ks, i1 = ab + kColI1 + 8 * ks,
                           i2 = ab + kColI2 + 8 * ks;
            mma_kstep(leader, acc, l0r, l0i, rr_, ri_, r0, r1, r2, i0, i1, i2, dr0 + ko, dr1 + ko,
                      dr2 + ko, di0 + ko, di1 + ko, di2 + ko, ip, in);
          }
          mma_commit(leader, mbase + kBarAFree + 8 * h);  // this half of A may be refilled
        }
        if (ok) mma_commit(leader, mbase + kBarDFull);
        // the operand block may be replaced once this tile's MMAs are done
        if (ok && i + 1 < my_tiles && new_chain(i + 1)) mma_commit(leader, mbase + kBarWFree);
      }
      // all issued MMAs complete before TMEM is released
      mma_commit(leader, mbase + kBarMmaDone);
      const long long t0 = clock64();
      while (!mbar_try_wait(mbase + kBarMmaDone, 0) && clock64() - t0 < kTimeoutCycles) {
      }
    } else if (warp == 9 && lane == 0) {
      // load number g is box (g mod 4) of tile g / 4, into slot g mod kSlots
      const CUtensorMap* map_in = &tmap_in;
      auto load_box = [&](long long g) {
        const long long t = tile_of(g >> 2);
        const int tlo = (int)(t & ((1ll << (a - kN)) - 1));
        const int thi = (int)(t >> (a - kN));
        const int slot = (int)(g % kSlots);
        const uint32_t bar = mbase + kBarFull + 8 * slot;
        mbar_expect_tx(bar, kBoxBytes);
        tma_load_5d(sbase + kOffRing + slot * kBoxBytes, map_in, bar, 0, (int)(g & 3), tlo, 0,
                    thi);
      };
      auto load_w = [&](const void* src) {
        mbar_expect_tx(mbase + kBarW, kWBytes);
        const uint8_t* wsrc = static_cast<const uint8_t*>(src);
        for (int q = 0; q < 3; ++q)
          bulk_load(w0 + q * (kWBytes / 3), wsrc + q * (kWBytes / 3), kWBytes / 3,
                    mbase + kBarW);
      };
      if constexpr (kGroup) {
        map_in = reinterpret_cast<const CUtensorMap*>(grp[chain_of(0)].map_in);
        tensormap_acquire(map_in);
        load_w(grp[chain_of(0)].W);
      } else {
        load_w(pa.W);
      }
      int wload = 0;  // group: operand blocks loaded after the first
      const long long nloads = 4 * my_tiles;
      long long issued = 0;
      for (; issued < nloads; ++issued) {
        // a slot is reused once the converters have read its previous box
        if (issued >= kSlots &&
            !wait_bar(mbase + kBarEmpty + 8 * (int)(issued % kSlots),
                      (uint32_t)((issued / kSlots - 1) & 1), abort, status))
          break;
        if ((issued & 3) == 0 && new_chain(issued >> 2)) {
          // a new chain: its descriptors for the boxes from here on
          map_in = reinterpret_cast<const CUtensorMap*>(grp[chain_of(issued >> 2)].map_in);
          tensormap_acquire(map_in);
        }
        load_box(issued);
        if ((issued & 3) == 3 && new_chain(issued >> 2)) {
          // and its operand block, once the new chain's first tile is on its
          // way and the MMAs of the previous chain are done with the old one
          if (!wait_bar(mbase + kBarWFree, (uint32_t)(wload & 1), abort, status)) {
            ++issued;
            break;
          }
          load_w(grp[chain_of(issued >> 2)].W);
          ++wload;
        }
      }
      if (*abort) {
        // drain copies nobody will consume before the CTA exits
        for (long long g = issued - kSlots < 0 ? 0 : issued - kSlots; g < issued; ++g) {
          const long long t0 = clock64();
          while (!mbar_try_wait(mbase + kBarFull + 8 * (int)(g % kSlots),
                                (uint32_t)((g / kSlots) & 1)) &&
                 clock64() - t0 < kTimeoutCycles) {
          }
        }
        const long long t0 = clock64();
        while (!mbar_try_wait(mbase + kBarW, (uint32_t)(wload & 1)) &&
               clock64() - t0 < kTimeoutCycles) {
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ------------------------------------------------------------------ host

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

uint16_t bf16_of(double v, double scale) {
  // v has at most 8 significant bits and scale is a power of two: v * scale
  // is exact in float and in bf16 (the low 16 bits of the float are zero)
  float f = (float)(v * scale);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

}  // namespace

bool block_tc_supported(int L, int n) { return n == kN && L >= kN + 7; }

size_t block_tc_w_bytes(int n) { return n == kN ? kWBytes : 0; }

namespace {
// 8-byte slot (bank pair, 0..15) contributed by staging-tile bit p to a
// staging byte address under the 128-byte swizzle: amplitude bits 0-3 are
// slot bits 0-3, bits 4-6 are XORed into slot bits 1-3, and higher bits only
// select the 128-byte line.
int staging_slot_bit(int p) { return p < 4 ? 1 << p : (p < 7 ? 1 << (p - 3) : 0); }
// Rank over GF(2) of k bit vectors of at most 8 bits.
int gf2_rank(const int* v, int k) {
  int piv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int r = 0;
  for (int i = 0; i < k; ++i) {
    int x = v[i];
    for (int b = 7; b >= 0 && x; --b) {
      if (!((x >> b) & 1)) continue;
      if (!piv[b]) {
        piv[b] = x;
        ++r;
        break;
      }
      x ^= piv[b];
    }
  }
  return r;
}
}  // namespace

int block_tc_row_map(const int8_t* sigma, const int8_t* spos, uint8_t* rowvec) {
  // The 32 lanes of an epilogue warp are TMEM lanes 32q + t, and a 64-bit
  // shared store is served per half-warp (lanes 0-15, then 16-31).  With
  // rows r(m) = M m over GF(2) the staging slot of lane t's store is linear
  // in t, so each half takes 2^(4 - rank) wavefronts, where rank is that of
  // the slot images of M's first four columns (4 at best: one lane a slot).
  int v[7];
  for (int b = 0; b < 7; ++b) v[b] = staging_slot_bit(spos[sigma[kN + b]]);
  auto img = [&](int m) {
    int x = 0;
    for (int b = 0; b < 7; ++b)
      if ((m >> b) & 1) x ^= v[b];
    return x;
  };
  const int reach = std::min(4, gf2_rank(v, 7));
  int m[7] = {0, 0, 0, 0, 0, 0, 0};
  auto independent = [&](int cand, int k) {
    int t[8];
    for (int i = 0; i < k; ++i) t[i] = m[i];
    t[k] = cand;
    return gf2_rank(t, k + 1) == k + 1;
  };
  // the natural columns first, so that a pass without conflicts keeps them
  int order[127 + 4], no = 0;
  for (int c : {8, 16, 32, 64}) order[no++] = c;
  for (int c = 1; c < 128; ++c) order[no++] = c;
  // Columns 0-2 keep row bits 0-2 (plus any of rows 3-6): the 8 lanes of
  // each quarter of a converter LDS.128 then read 8 different 16-byte chunks
  // of the swizzled box.  Column 3 is free.
  int best = -1;
  int bm[4] = {1, 2, 4, 8};
  for (int h = 0; h < 4096 && best < reach; ++h) {
    m[0] = 1 | ((h & 15) << 3);
    m[1] = 2 | (((h >> 4) & 15) << 3);
    m[2] = 4 | ((h >> 8) << 3);
    for (int i = 0; i < no && best < reach; ++i) {
      if (!independent(order[i], 3)) continue;
      const int im[4] = {img(m[0]), img(m[1]), img(m[2]), img(order[i])};
      const int r = gf2_rank(im, 4);
      if (r > best) {
        best = r;
        bm[0] = m[0];
        bm[1] = m[1];
        bm[2] = m[2];
        bm[3] = order[i];
      }
    }
  }
  for (int i = 0; i < 4; ++i) m[i] = bm[i];
  for (int k = 4; k < 7; ++k) {
    int pick = 0;
    for (int i = 0; i < no && !pick; ++i)
      if (independent(order[i], k)) pick = order[i];
    m[k] = pick;
  }
  int im4[4];
  for (int i = 0; i < 4; ++i) im4[i] = img(m[i]);
  int low[3] = {m[0] & 7, m[1] & 7, m[2] & 7};
  if (gf2_rank(m, 7) != 7 || gf2_rank(low, 3) != 3 || gf2_rank(im4, 4) != best) {
    for (int i = 0; i < 7; ++i) m[i] = 1 << i;  // not reached; the natural map is always valid
    for (int i = 0; i < 4; ++i) im4[i] = img(m[i]);
    best = gf2_rank(im4, 4);
  }
  for (int i = 0; i < 7; ++i) rowvec[i] = (uint8_t)m[i];
  return 2 << (4 - best);
}

namespace {
// State bit of output tile bit o for a tile whose rows start at state bit a:
// bits 0-5 are the next window, bits 6-12 the rows.
int out_state_bit(int o, int a) { return o < kN ? o : a + o - kN; }

// The store view of a staging order: staging bits 0-3 are one 128-byte line
// (dimension 0), and staging bits 4-12 split into runs of output bits on
// consecutive state bits, one dimension each (output bit 6 always starts a
// run: the tile-index bits below the rows lie between bits 5 and 6).
// Returns the number of runs, with the first output bit and length of each.
int store_runs(const int8_t* spos, int a, int* first, int* len) {
  int inv[13];
  for (int o = 0; o < 13; ++o) inv[spos[o]] = o;
  int nr = 0;
  for (int p = 4; p < 13; ++p) {
    const int o = inv[p];
    if (p > 4 && o != kN && out_state_bit(o, a) == out_state_bit(inv[p - 1], a) + 1) {
      ++len[nr - 1];
    } else {
      if (nr == 9) return 99;
      first[nr] = o;
      len[nr++] = 1;
    }
  }
  return nr;
}

// Fills the store fields of pa from pa.spos; false if the view needs more
// than the five dimensions a tensor map has.
bool set_store_view(PassArgs& pa) {
  int first[9], len[9];
  const int nr = store_runs(pa.spos, pa.a, first, len);
  if (nr > 4) return false;
  // a three-dimensional view is stored with the natural order's coordinates
  if (nr == 2 && (first[0] != 4 || len[0] != 2)) return false;
  pa.st_ndims = (int8_t)(nr + 1);
  for (int k = 0; k < nr; ++k) {
    const int last = first[k] + len[k] - 1;
    if (last == kN - 1) {  // the tile bits below the rows continue this run
      pa.st_tlo_dim = (int8_t)(k + 1);
      pa.st_tlo_shift = (int8_t)len[k];
    }
    if (last == 12) {  // the tile bits above the rows
      pa.st_thi_dim = (int8_t)(k + 1);
      pa.st_thi_shift = (int8_t)len[k];
    }
  }
  for (int q = 0; q < 13; ++q) pa.ssig[q] = pa.spos[pa.sigma[q]];
  return true;
}

// Largest rank the row map can give the slot images of its first four
// columns (columns 0-2 hold row bits 0-2 plus any of rows 3-6): a quick
// bound used to rank staging orders before the row map is searched.
int row_map_reach(const int* v) {
  const int rv = std::min(4, gf2_rank(v, 7));
  int span[16];
  for (int c = 0; c < 16; ++c) {
    span[c] = 0;
    for (int b = 0; b < 4; ++b)
      if ((c >> b) & 1) span[c] ^= v[3 + b];
  }
  int k = 0;
  for (int i = 0; i < 16 && k < 3; ++i)
    for (int j = 0; j < 16 && k < 3; ++j)
      for (int l = 0; l < 16 && k < 3; ++l) {
        const int t[3] = {v[0] ^ span[i], v[1] ^ span[j], v[2] ^ span[l]};
        k = std::max(k, gf2_rank(t, 3));
      }
  return std::min(rv, k + 1);
}
}  // namespace

// Stores at 8 wavefronts cost less than the scattered writes of a
// reordered store view; at 16 the conflicts dominate the pass.
constexpr int kRestageWavefronts = 16;

int block_tc_layout(PassArgs& pa) {
  for (int o = 0; o < 13; ++o) pa.spos[o] = (int8_t)o;
  set_store_view(pa);  // the natural order: three dimensions
  const int wf = block_tc_row_map(pa.sigma, pa.spos, pa.rowvec);
  if (wf < kRestageWavefronts) return wf;
  // Output bits for staging bits 4-6 (slot bits 1-3), the others above them
  // in increasing order; the best reach with the fewest store dimensions.
  int best_reach = -1, best_runs = 99;
  int8_t best[13];
  for (int x = 4; x < 13; ++x)
    for (int y = 4; y < 13; ++y)
      for (int z = 4; z < 13; ++z) {
        if (x == y || x == z || y == z) continue;
        int8_t sp[13];
        for (int o = 0; o < 4; ++o) sp[o] = (int8_t)o;
        sp[x] = 4;
        sp[y] = 5;
        sp[z] = 6;
        int p = 7;
        for (int o = 4; o < 13; ++o)
          if (o != x && o != y && o != z) sp[o] = (int8_t)p++;
        int first[9], len[9];
        const int nr = store_runs(sp, pa.a, first, len);
        if (nr > 4) continue;
        int v[7];
        for (int b = 0; b < 7; ++b) v[b] = staging_slot_bit(sp[pa.sigma[kN + b]]);
        const int reach = row_map_reach(v);
        if (reach > best_reach || (reach == best_reach && nr < best_runs)) {
          best_reach = reach;
          best_runs = nr;
          std::memcpy(best, sp, sizeof(best));
        }
      }
  if (best_reach < 0) return wf;
  PassArgs t = pa;
  std::memcpy(t.spos, best, sizeof(best));
  const int wf2 = block_tc_row_map(t.sigma, t.spos, t.rowvec);
  if (wf2 >= wf || !set_store_view(t)) return wf;
  pa = t;
  return wf2;
}

void block_tc_pack_w(int n, const std::vector<cd>& U, std::vector<uint32_t>& out) {
  // six K-major 64 x 64 bf16 digit matrices Ur0, Ur1, Ur2, Ui0, Ui1, Ui2
  // holding u0/128, u1/32768, u2/2^23 with u = 2^-7 (u0 + u1/256 + u2/65536)
  // (u0 an integer, |u_t| <= 128; the digits chosen by round_unitary_digits
  // so that the represented matrix is as close to unitary as they allow),
  // in the core-matrix order of make_desc: element (row j, col k) at
  // halfword ((k/8)*8 + j/8)*64 + (j%8)*8 + k%8
  out.assign(kWBytes / 4, 0u);
  if (n != kN) return;
  std::vector<double> dg((size_t)6 * kCols * kCols);
  round_unitary_digits(kCols, U.data(), dg.data());
  std::vector<uint16_t> h(kWBytes / 2, 0);
  const size_t m = (size_t)kCols * kCols;
  for (int j = 0; j < kCols; ++j)
    for (int k = 0; k < kCols; ++k) {
      const size_t e = (size_t)j * kCols + k;
      const size_t w = (size_t)(((k >> 3) * 8 + (j >> 3)) * 64 + (j & 7) * 8 + (k & 7));
      for (int ri = 0; ri < 2; ++ri) {
        double scale = 1.0 / 128.0;  // digits at their true scale
        for (int q = 0; q < 3; ++q) {
          h[(size_t)(3 * ri + q) * m + w] = bf16_of(dg[3 * (2 * e + ri) + q], scale);
          scale /= 256.0;
        }
      }
    }
  std::memcpy(out.data(), h.data(), kWBytes);
}

int block_tc_store_view(const PassArgs& pa, uint64_t* dims, uint64_t* strides, uint32_t* box) {
  int first[9], len[9];
  const int a = pa.a, L = pa.L;
  const int nr = store_runs(pa.spos, a, first, len);
  if (nr > 4 || nr + 1 != pa.st_ndims) return -1;
  for (int d = 0; d < 5; ++d) {
    dims[d] = d == 0 ? 16 : 1;
    box[d] = d == 0 ? 16 : 1;
  }
  for (int d = 0; d < 4; ++d) strides[d] = 0;
  for (int k = 0; k < nr; ++k) {
    const int last = first[k] + len[k] - 1;
    int bits = len[k];
    if (last == kN - 1) bits += a - kN;
    if (last == 12) bits += L - a - 7;
    dims[k + 1] = (uint64_t)1 << bits;
    strides[k] = (uint64_t)8 << out_state_bit(first[k], a);
    box[k + 1] = 1u << len[k];
  }
  return nr + 1;
}

// Two descriptors per pass: the load view (tile rows as 128-row boxes of
// 128 bytes: window amplitudes 16 c .. 16 c + 15 of each row) and the store
// view of the staging order: amplitudes 0-15 of an output row, then one
// dimension per run of the staging order (natural order: output bits 4-5
// joined with the tile bits below the row bits, output row bits 6-12 joined
// with the tile bits above them).
int block_tc_make_map(const PassArgs& pa, void* psi, void* map_out) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return SV_ECUDA;
  const int a = pa.a, L = pa.L;
  alignas(64) CUtensorMap maps[2];
  cuuint64_t dims[5] = {32, 4, (cuuint64_t)1 << (a - kN), 128, (cuuint64_t)1 << (L - a - 7)};
  cuuint64_t strides[4] = {128, 512, (cuuint64_t)8 << a, (cuuint64_t)8 << (a + 7)};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  cuuint32_t box_in[5] = {32, 1, 1, 128, 1};
  CUresult rc = fn(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, psi, dims, strides, box_in,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (rc != CUDA_SUCCESS) return SV_ECUDA;
  // store view: 8-byte elements (one complex amplitude each)
  uint64_t odims[5], ostrides[4];
  uint32_t obox[5];
  const int rank = block_tc_store_view(pa, odims, ostrides, obox);
  if (rank < 0) return SV_EINVAL;
  rc = fn(&maps[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, rank, psi, odims, ostrides, obox, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (rc != CUDA_SUCCESS) return SV_ECUDA;
  std::memcpy(map_out, maps, sizeof(maps));  // the caller's buffer need not be aligned
  return SV_OK;
}

size_t block_tc_map_bytes() { return 2 * sizeof(CUtensorMap); }

cudaError_t block_tc_prepare() {
  const void* fns[6] = {(const void*)k_block_tc<true, false, false>,
                        (const void*)k_block_tc<false, false, false>,
                        (const void*)k_block_tc<false, true, false>,
                        (const void*)k_block_tc<false, false, true>,
                        (const void*)k_block_tc<false, true, true>,
                        (const void*)k_block_tc<true, false, false, true>};
  for (const void* f : fns) {
    const cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_block_tc(const PassArgs& pa, void* psi, const void* map, int* status,
                            int grid, cudaStream_t s) {
  PassArgs p = pa;
  p.psi = psi;
  alignas(64) CUtensorMap maps[2];
  std::memcpy(maps, map, sizeof(maps));
  constexpr long long kMinTilesSpecialised = 32;  // tiles per CTA
  const long long per_cta = (p.ntiles + grid - 1) / grid;
  const dim3 g(grid), b(kThreads);
  if (per_cta < kMinTilesSpecialised)
    k_block_tc<true, false, false><<<g, b, kSmemBytes, s>>>(maps[0], maps[1], p, status, nullptr, 0);
  else if (p.diag && p.x_mask)
    k_block_tc<false, true, true><<<g, b, kSmemBytes, s>>>(maps[0], maps[1], p, status, nullptr, 0);
  else if (p.diag)
    k_block_tc<false, false, true><<<g, b, kSmemBytes, s>>>(maps[0], maps[1], p, status, nullptr, 0);
  else if (p.x_mask)
    k_block_tc<false, true, false><<<g, b, kSmemBytes, s>>>(maps[0], maps[1], p, status, nullptr, 0);
  else
    k_block_tc<false, false, false><<<g, b, kSmemBytes, s>>>(maps[0], maps[1], p, status, nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_block_tc_group(const PassArgs& pa, const GroupChain* chains, int nt_log2,
                                  int* status, int grid, cudaStream_t s) {
  // the kernel's descriptor parameters are unused: each chain's come from
  // the group array
  alignas(64) CUtensorMap unused[2];
  std::memset(unused, 0, sizeof(unused));
  k_block_tc<true, false, false, true><<<grid, kThreads, kSmemBytes, s>>>(
      unused[0], unused[1], pa, status, chains, nt_log2);
  return cudaGetLastError();
}

}  // namespace fsv
