// Tensor-core block pass (sm_103a): S' = S U^T on tiles of 128 rows x 64
// complex amplitudes (a window of n = 6 sites), the matrix-unit form of the
// paper's fused-gate contraction (Sec. II, Eq. 2 on fused operators).
//
// Per CTA (one per SM, persistent over tiles):
//   warp 8      TMA producer: four 128-row x 128-byte boxes per tile
//               (cp.async.bulk.tensor.5d, 128-byte swizzle) into a
//               double-buffered stage, plus the pass's operand block W once.
//   warps 0-3   converters: thread = row = TMEM lane; split every real and
//               imaginary part x into TF32 hi = rna(x), lo = rna(x - hi) and
//               store four de-interleaved planes Sr_hi, Si_hi, Sr_lo, Si_lo
//               into TMEM (tcgen05.st), the A operand.
//   warp 9      allocates TMEM (512 columns) and issues the MMAs:
//               D_re = Sr Ur^T - Si Ui^T, D_im = Sr Ui^T + Si Ur^T, each
//               product as hi*hi + hi*lo + lo*hi (TF32 x3 split, FP32
//               accumulate), M=128 N=64 K=8 tcgen05.mma.kind::tf32 with A in
//               TMEM and B = [Ur|Ui]_[hi|lo] resident in shared memory
//               (K-major, no swizzle); D double-buffered in TMEM.
//   warps 4-7   epilogue: tcgen05.ld of D, energy terms (<X> on window
//               sites in-row, the diagonal part on the natural layout of the
//               period's last pass), the fused relabel (write each amplitude
//               at its place in the next window's layout) into the stage
//               buffer, then a TMA store of the tile.
// Every wait is an mbarrier try_wait loop bounded by a clock budget; on
// timeout the CTA raises *status, drains its own copies and MMAs, frees
// TMEM and exits.
#include <cuda.h>
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
constexpr int kThreads = 320;         // 10 warps
constexpr uint32_t kStageBytes = kRows * kCols * 8;  // 64 KiB
constexpr uint32_t kBoxBytes = kRows * 128;           // 16 KiB
constexpr uint32_t kMatBytes = kCols * kCols * 4;     // one 64 x 64 TF32 matrix
constexpr uint32_t kWBytes = 6 * kMatBytes;           // Ur, Ui in three parts: 96 KiB
constexpr uint32_t kOffW = 0;
constexpr uint32_t kOffStage = kWBytes;
constexpr uint32_t kOffMisc = kOffStage + 2 * kStageBytes;
constexpr uint32_t kSmemBytes = kOffMisc + 1024 + 1024;  // misc + alignment slack
// TMEM columns.  The A operand is two K-halves (k < 32, k >= 32) of 128
// columns each, so the next tile's conversion can fill one half while the
// MMAs read the other: half h = [128 h, 128 h + 128) holds Sr_hi, Si_hi,
// Sr_lo, Si_lo for its 32 k's at offsets 0, 32, 64, 96.
constexpr uint32_t kColSrHi = 0, kColSiHi = 32, kColSrLo = 64, kColSiLo = 96;
constexpr uint32_t kColD = 256;  // D buffer b at kColD + 128 b: re [0,64), im [64,128)
constexpr long long kTimeoutCycles = 4000000000ll;  // about 2 s at 2 GHz

// misc block layout (offsets from kOffMisc)
enum : uint32_t {
  kBarFull = 0,     // 2 x 8: stage b loaded
  kBarW = 16,       // operand block loaded
  kBarAReady = 24,  // 2 x 8: A half h written
  kBarAFree = 40,   // 2 x 8: A half h consumed by the MMAs
  kBarDFull = 56,   // 2 x 8: D buffer b complete
  kBarDFree = 72,   // 2 x 8: D buffer b read out
  kBarSFree = 88,   // 2 x 8: stage b stored out
  kBarMmaDone = 104,
  kTmemSlot = 112,
  kAbort = 116,
  kSigmaCol = 128,  // 64 x uint16
  kRed = 256,       // 4 x 2 doubles
};

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

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(bar)
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
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
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
// 8 rows x 16 bytes; LBO = 1024 B between core matrices along K, SBO = 128 B
// between 8-row groups along N.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version
  return d;
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major,
// N = 64, M = 128, optional negation of B.
__host__ __device__ constexpr uint32_t make_idesc(int negate_b) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)negate_b << 14) |
         ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
    k_block_tc(const __grid_constant__ CUtensorMap tmap, PassArgs pa, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t sbase = smem_u32(smem);
  uint8_t* misc = smem + kOffMisc;
  const uint32_t mbase = sbase + kOffMisc;
  volatile uint32_t* abort = reinterpret_cast<volatile uint32_t*>(misc + kAbort);
  uint16_t* sigma_col = reinterpret_cast<uint16_t*>(misc + kSigmaCol);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int a = pa.a;
  const long long ntiles = pa.ntiles;
  const long long my_tiles =
      blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (threadIdx.x == 0) {
    mbar_init(mbase + kBarFull, 1);
    mbar_init(mbase + kBarFull + 8, 1);
    mbar_init(mbase + kBarW, 1);
    mbar_init(mbase + kBarAReady, 128);
    mbar_init(mbase + kBarAReady + 8, 128);
    mbar_init(mbase + kBarAFree, 1);
    mbar_init(mbase + kBarAFree + 8, 1);
    mbar_init(mbase + kBarDFull, 1);
    mbar_init(mbase + kBarDFull + 8, 1);
    mbar_init(mbase + kBarDFree, 128);
    mbar_init(mbase + kBarDFree + 8, 128);
    mbar_init(mbase + kBarSFree, 1);
    mbar_init(mbase + kBarSFree + 8, 1);
    mbar_init(mbase + kBarMmaDone, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (threadIdx.x < kCols) {  // output-tile bits contributed by column bits
    uint32_t y = 0;
    for (int q = 0; q < kN; ++q) y |= ((threadIdx.x >> q) & 1u) << pa.sigma[q];
    sigma_col[threadIdx.x] = (uint16_t)y;
  }
  if (warp == 9) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     mbase + kTmemSlot)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(misc + kTmemSlot);

  if (warp == 8) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      mbar_expect_tx(mbase + kBarW, kWBytes);
      const uint8_t* wsrc = static_cast<const uint8_t*>(pa.W);
      for (int q = 0; q < 4; ++q)
        bulk_load(sbase + kOffW + q * (kWBytes / 4), wsrc + q * (kWBytes / 4), kWBytes / 4,
                  mbase + kBarW);
      long long issued = 0;
      for (long long i = 0; i < my_tiles; ++i) {
        const int b = (int)(i & 1);
        const uint32_t k = (uint32_t)(i >> 1);
        if (i >= 2 && !wait_bar(mbase + kBarSFree + 8 * b, (k - 1) & 1, abort, status)) break;
        const long long t = blockIdx.x + i * gridDim.x;
        const int tlo = (int)(t & ((1ll << (a - kN)) - 1));
        const int thi = (int)(t >> (a - kN));
        const uint32_t bar = mbase + kBarFull + 8 * b;
        mbar_expect_tx(bar, kStageBytes);
        for (int c = 0; c < 4; ++c)
          tma_load_5d(sbase + kOffStage + b * kStageBytes + c * kBoxBytes, &tmap, bar, 0, c, tlo,
                      0, thi);
        issued = i + 1;
      }
      // drain loads nobody will consume (abort path) before the CTA exits
      for (long long i = issued - 2 < 0 ? 0 : issued - 2; i < issued && *abort; ++i) {
        const int b = (int)(i & 1);
        const long long t0 = clock64();
        while (!mbar_try_wait(mbase + kBarFull + 8 * b, (uint32_t)((i >> 1) & 1)) &&
               clock64() - t0 < kTimeoutCycles) {
        }
      }
    }
  } else if (warp == 9) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      bool ok = wait_bar(mbase + kBarW, 0, abort, status);
      tc_fence_after();
      const uint32_t w0 = sbase + kOffW;
      // B operands: Ur and Ui in three TF32 parts each (hi, lo, lo2)
      const uint64_t d_urh = make_desc(w0), d_url = make_desc(w0 + kMatBytes),
                     d_url2 = make_desc(w0 + 2 * kMatBytes),
                     d_uih = make_desc(w0 + 3 * kMatBytes),
                     d_uil = make_desc(w0 + 4 * kMatBytes),
                     d_uil2 = make_desc(w0 + 5 * kMatBytes);
      constexpr uint32_t id_pos = make_idesc(0), id_neg = make_idesc(1);
      for (long long i = 0; ok && i < my_tiles; ++i) {
        const int b = (int)(i & 1);
        const uint32_t k = (uint32_t)(i >> 1);
        if (i >= 2 && !wait_bar(mbase + kBarDFree + 8 * b, (k - 1) & 1, abort, status)) break;
        const uint32_t dre = tmem + kColD + 128 * b, dim = dre + 64;
        bool half_ok = true;
        for (int h = 0; h < 2 && half_ok; ++h) {
          if (!wait_bar(mbase + kBarAReady + 8 * h, (uint32_t)(i & 1), abort, status)) {
            half_ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t abase = tmem + 128 * h;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            // global k-step 4h + ks: two core matrices (1024 B apart) along K
            const uint64_t kofs = (uint64_t)((2 * (4 * h + ks) * 1024) >> 4);
            const uint32_t acc = (h > 0 || ks > 0) ? 1u : 0u;
            const uint32_t srh = abase + kColSrHi + 8 * ks, sih = abase + kColSiHi + 8 * ks;
            const uint32_t srl = abase + kColSrLo + 8 * ks, sil = abase + kColSiLo + 8 * ks;
            // D_re = Sr Ur^T - Si Ui^T with S = hi + lo, U = hi + lo + lo2
            mma_tf32(dre, srh, d_urh + kofs, id_pos, acc);
            mma_tf32(dre, srh, d_url + kofs, id_pos, 1);
            mma_tf32(dre, srh, d_url2 + kofs, id_pos, 1);
            mma_tf32(dre, srl, d_urh + kofs, id_pos, 1);
            mma_tf32(dre, sih, d_uih + kofs, id_neg, 1);
            mma_tf32(dre, sih, d_uil + kofs, id_neg, 1);
            mma_tf32(dre, sih, d_uil2 + kofs, id_neg, 1);
            mma_tf32(dre, sil, d_uih + kofs, id_neg, 1);
            // D_im = Sr Ui^T + Si Ur^T
            mma_tf32(dim, srh, d_uih + kofs, id_pos, acc);
            mma_tf32(dim, srh, d_uil + kofs, id_pos, 1);
            mma_tf32(dim, srh, d_uil2 + kofs, id_pos, 1);
            mma_tf32(dim, srl, d_uih + kofs, id_pos, 1);
            mma_tf32(dim, sih, d_urh + kofs, id_pos, 1);
            mma_tf32(dim, sih, d_url + kofs, id_pos, 1);
            mma_tf32(dim, sih, d_url2 + kofs, id_pos, 1);
            mma_tf32(dim, sil, d_urh + kofs, id_pos, 1);
          }
          mma_commit(mbase + kBarAFree + 8 * h);  // this half of A may be refilled
        }
        if (!half_ok) break;
        mma_commit(mbase + kBarDFull + 8 * b);
      }
      // all issued MMAs complete before TMEM is released
      mma_commit(mbase + kBarMmaDone);
      const long long t0 = clock64();
      while (!mbar_try_wait(mbase + kBarMmaDone, 0) && clock64() - t0 < kTimeoutCycles) {
      }
    }
  } else if (warp < 4) {
    // ---------------------------------------------------------- converters
    const int r = warp * 32 + lane;  // tile row = TMEM lane
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (long long i = 0; i < my_tiles; ++i) {
      const int b = (int)(i & 1);
      const uint32_t k = (uint32_t)(i >> 1);
      bool ok = wait_bar(mbase + kBarFull + 8 * b, k & 1, abort, status);
      if (__any_sync(0xffffffffu, !ok)) break;  // the warp leaves together
      const uint8_t* stage = smem + kOffStage + b * kStageBytes;
      for (int h = 0; h < 2 && ok; ++h) {
        if (i >= 1)
          ok = wait_bar(mbase + kBarAFree + 8 * h, (uint32_t)((i - 1) & 1), abort, status);
        if (__any_sync(0xffffffffu, !ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll 1
        for (int cc = 0; cc < 2; ++cc) {
          const int c = 2 * h + cc;  // 16-amplitude chunk, k in [16 c, 16 c + 16)
          uint32_t rh[16], ih[16], rl[16], il[16];
          const uint8_t* rowp = stage + c * kBoxBytes + r * 128;
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            const float4 v = *reinterpret_cast<const float4*>(rowp + ((s ^ (r & 7)) << 4));
            const float xs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const uint32_t hr = tf32_rna(xs[2 * e]), hi_ = tf32_rna(xs[2 * e + 1]);
              rh[2 * s + e] = hr;
              ih[2 * s + e] = hi_;
              rl[2 * s + e] = tf32_rna(xs[2 * e] - __uint_as_float(hr));
              il[2 * s + e] = tf32_rna(xs[2 * e + 1] - __uint_as_float(hi_));
            }
          }
          const uint32_t hb = lane_base + 128 * h + 16 * cc;
          tmem_st16(hb + kColSrHi, rh);
          tmem_st16(hb + kColSiHi, ih);
          tmem_st16(hb + kColSrLo, rl);
          tmem_st16(hb + kColSiLo, il);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        mbar_arrive(mbase + kBarAReady + 8 * h);
      }
      if (!ok) break;
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp - 4;
    const int r = q * 32 + lane;  // tile row = TMEM lane
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t yrow = 0;  // output-tile bits contributed by this row's bits
    for (int bq = 0; bq < 7; ++bq) yrow |= ((uint32_t)(r >> bq) & 1u) << pa.sigma[kN + bq];
    Diag<float> dg;
    if (pa.diag) dg.init(pa.ep, pa.L);
    const float sc = (float)renorm_scale(pa.ep.rn);
    double eacc = 0.0, nacc = 0.0;
    for (long long i = 0; i < my_tiles; ++i) {
      const int b = (int)(i & 1);
      const uint32_t k = (uint32_t)(i >> 1);
      const bool ok = wait_bar(mbase + kBarDFull + 8 * b, k & 1, abort, status);
      if (!epilogue_all_ok(ok)) break;  // the four epilogue warps leave together
      tc_fence_after();
      float re[kCols], im[kCols];
      const uint32_t dcol = lane_base + kColD + 128 * b;
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        uint32_t vr[16], vi[16];
        tmem_ld16(dcol + 16 * c4, vr);
        tmem_ld16(dcol + 64 + 16 * c4, vi);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          re[16 * c4 + e] = __uint_as_float(vr[e]) * sc;
          im[16 * c4 + e] = __uint_as_float(vi[e]) * sc;
        }
      }
      tc_fence_before();
      mbar_arrive(mbase + kBarDFree + 8 * b);  // D[b] may be overwritten
      float es = 0.f, ns = 0.f;
      if (pa.x_mask) {
#pragma unroll
        for (int j = 0; j < kN; ++j) {
          if (!((pa.x_mask >> j) & 1)) continue;
          float sj = 0.f;
#pragma unroll
          for (int c = 0; c < kCols; ++c) sj += re[c] * re[c ^ (1 << j)] + im[c] * im[c ^ (1 << j)];
          es += pa.cx[j] * sj;
        }
      }
      const long long t = blockIdx.x + i * gridDim.x;
      const uint64_t tlo = (uint64_t)t & ((1ull << (a - kN)) - 1);
      const uint64_t thi = (uint64_t)t >> (a - kN);
      const uint64_t tbase = (tlo << kN) | (thi << (a + 7));
      uint8_t* stage = smem + kOffStage + b * kStageBytes;
#pragma unroll
      for (int c = 0; c < kCols; ++c) {
        const uint32_t yo = yrow | sigma_col[c];
        const uint32_t ro = yo >> kN, co = yo & (kCols - 1);
        uint8_t* dst = stage + (co >> 4) * kBoxBytes + ro * 128 +
                       ((((co & 15) >> 1) ^ (ro & 7)) << 4) + ((co & 1) << 3);
        *reinterpret_cast<float2*>(dst) = make_float2(re[c], im[c]);
        if (pa.diag) {
          const float p2 = re[c] * re[c] + im[c] * im[c];
          ns += p2;
          es += p2 * dg(tbase + ((uint64_t)ro << a) + co);
        }
      }
      eacc += (double)es;
      nacc += (double)ns;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (q == 0 && lane == 0) {
        for (int cc = 0; cc < 4; ++cc)
          tma_store_5d(&tmap, sbase + kOffStage + b * kStageBytes + cc * kBoxBytes, 0, cc,
                       (int)tlo, 0, (int)thi);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        mbar_arrive(mbase + kBarSFree + 8 * b);
      }
    }
    if (q == 0 && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    // energy partials of this CTA (fixed order)
    if (pa.partial) {
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
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (q == 0 && lane == 0) {
        pa.partial[2 * blockIdx.x] = (red[0] + red[2]) + (red[4] + red[6]);
        pa.partial[2 * blockIdx.x + 1] = (red[1] + red[3]) + (red[5] + red[7]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 9) {
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

uint32_t tf32_round_host(double x) {
  float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return u;  // inf / nan unchanged
  u += 0xFFFu + ((u >> 13) & 1u);                   // round to nearest even at bit 13
  return u & 0xFFFFE000u;
}

}  // namespace

bool block_tc_supported(int L, int n) { return n == kN && L >= kN + 7; }

size_t block_tc_w_bytes(int n) { return n == kN ? kWBytes : 0; }

void block_tc_pack_w(int n, const std::vector<cd>& U, std::vector<uint32_t>& out) {
  // six K-major 64 x 64 TF32 matrices Ur_hi, Ur_lo, Ur_lo2, Ui_hi, Ui_lo,
  // Ui_lo2 (x = hi + lo + lo2 to about 33 bits) in the core-matrix order of
  // make_desc: element (row j, col k) at word ((k/4)*8 + j/8)*32 + (j%8)*4 + k%4
  out.assign(kWBytes / 4, 0u);
  if (n != kN) return;
  const size_t m = (size_t)kCols * kCols;
  for (int j = 0; j < kCols; ++j)
    for (int k = 0; k < kCols; ++k) {
      const cd u = U[(size_t)j * kCols + k];
      const size_t w = (size_t)(((k >> 2) * 8 + (j >> 3)) * 32 + (j & 7) * 4 + (k & 3));
      const double parts[2] = {u.real(), u.imag()};
      for (int ri = 0; ri < 2; ++ri) {
        double rest = parts[ri];
        for (int q = 0; q < 3; ++q) {
          const uint32_t t = tf32_round_host(rest);
          float tf;
          std::memcpy(&tf, &t, 4);
          out[(size_t)(3 * ri + q) * m + w] = t;
          rest -= (double)tf;
        }
      }
    }
}

int block_tc_make_map(const PassArgs& pa, void* psi, void* map_out) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return SV_ECUDA;
  const int a = pa.a, L = pa.L;
  cuuint64_t dims[5] = {32, 4, (cuuint64_t)1 << (a - kN), 128, (cuuint64_t)1 << (L - a - 7)};
  cuuint64_t strides[4] = {128, 512, (cuuint64_t)8 << a, (cuuint64_t)8 << (a + 7)};
  cuuint32_t box[5] = {32, 1, 1, 128, 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult rc = fn(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, psi,
                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return rc == CUDA_SUCCESS ? SV_OK : SV_ECUDA;
}

size_t block_tc_map_bytes() { return sizeof(CUtensorMap); }

cudaError_t block_tc_prepare() {
  return cudaFuncSetAttribute(k_block_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSmemBytes);
}

cudaError_t launch_block_tc(const PassArgs& pa, const void* map, int* status, int grid,
                            cudaStream_t s) {
  const CUtensorMap& m = *static_cast<const CUtensorMap*>(map);
  k_block_tc<<<grid, kThreads, kSmemBytes, s>>>(m, pa, status);
  return cudaGetLastError();
}

}  // namespace fsv
