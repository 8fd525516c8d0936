// Multi-gate form: a cache-blocked pass that applies many of the period's
// two-qubit gates (Eq. 2, gate by gate) to a tile of the state held in
// shared memory, instead of one gate per pass over the state (the plain
// form) or one fused dense unitary per pass (the block forms).
//
// A tile is 2^13 amplitudes (64 KiB): state bits 0-3 (16 contiguous
// amplitudes, one 128-byte line) and the 9 state bits A..A+8 of the pass's
// window, A = max(lo, 4) (for lo < 4 the tile is the 13 lowest bits; for
// L <= 13 it is the whole state).  The state keeps the natural layout, so
// windows move freely between passes.  Every gate of the pass then acts on
// two adjacent tile bits; it is applied to the whole tile with the plain
// form's gate tables (FP32 table + its residual, residual products first)
// between block barriers.  The sites whose last gate of the period is in
// the pass have their <X> measured on the tile at the end of the pass; the
// period's last pass measures the diagonal part and the norm.
//
// Cost per amplitude and gate: 32 FP32 FMA (table and residual), against
// 16 bytes of HBM traffic per amplitude and pass: a pass of G gates is
// bound by the FP32 pipe once G exceeds about 3.
#include <cuda_runtime.h>

#include <cstdint>

#include "sv_device.cuh"
#include "sv_internal.h"
#include "sv_kernels.h"

namespace fsv {

namespace {

using namespace dev;

constexpr int kMgThreads = 256;
// resident CTAs per SM (64 KiB of shared memory each), from the occupancy
// query at set-up; the persistent grid is that many per SM, so no CTA waits
// for another to finish
int g_mg_ctas_per_sm = 2;

__global__ void __launch_bounds__(kMgThreads) k_multigate(float2* __restrict__ psi, MultiArgs ma) {
  extern __shared__ float2 tile[];
  const int tb = ma.tb, A = ma.A;
  const uint32_t N = 1u << tb;
  const uint64_t ntiles = 1ull << (ma.L - tb);
  const int lowbits = A - 4;  // tile-index bits below the window (state bits 4..A-1)
  const uint64_t lowmask = (1ull << lowbits) - 1;
  const float sc = (float)renorm_scale(ma.ep.rn);
  Diag<float> dg;
  if (ma.diag) dg.init(ma.ep, ma.L);
  const float2* gbase = gate_ptr(ma.gates, ma.stride, ma.counter);
  double eacc = 0.0, nacc = 0.0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t base = ((t & lowmask) << 4) | ((t >> lowbits) << (A + tb - 4));
    auto state_index = [&](uint32_t e) -> uint64_t {
      return base | (e & 15u) | ((uint64_t)(e >> 4) << A);
    };
    // load (two amplitudes a thread, consecutive in the state)
    for (uint32_t e = 2 * threadIdx.x; e < N; e += 2 * blockDim.x) {
      const float4 v = *reinterpret_cast<const float4*>(psi + state_index(e));
      tile[e] = make_float2(v.x * sc, v.y * sc);
      tile[e + 1] = make_float2(v.z * sc, v.w * sc);
    }
    __syncthreads();
    for (int k = 0; k < ma.ngates; ++k) {
      const int q = __ldg(&ma.gq[k]);
      const float2* gp = gbase + (size_t)__ldg(&ma.gidx[k]) * kGateEntries;
      float2 g[16], gl[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        g[i] = __ldg(&gp[i]);
        gl[i] = __ldg(&gp[16 + i]);
      }
      const uint32_t qmask = (1u << q) - 1;
      const uint32_t off[4] = {0, 2u << q, 1u << q, 3u << q};  // r = 2 b_q + b_{q+1}
      for (uint32_t gi = threadIdx.x; gi < (N >> 2); gi += blockDim.x) {
        const uint32_t b0 = (gi & qmask) | ((gi >> q) << (q + 2));
        float2 v[4], w[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = tile[b0 + off[r]];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          // residual products first, then the table's on top (see k_plain.cu)
          float2 acc = czero<float2>();
#pragma unroll
          for (int c = 0; c < 4; ++c) acc = cmac(acc, gl[4 * r + c], v[c]);
#pragma unroll
          for (int c = 0; c < 4; ++c) acc = cmac(acc, g[4 * r + c], v[c]);
          w[r] = acc;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) tile[b0 + off[r]] = w[r];
      }
      __syncthreads();
    }
    // measurement on the tile, then the write-back
    float es = 0.f, ns = 0.f;
    for (int j = 0; j < ma.nx; ++j) {
      const uint32_t m = 1u << ma.xq[j];
      float s = 0.f;
      for (uint32_t e = threadIdx.x; e < N; e += blockDim.x)
        if (!(e & m)) s += cdotre(tile[e], tile[e | m]);
      es += 2.f * ma.xc[j] * s;
    }
    for (uint32_t e = 2 * threadIdx.x; e < N; e += 2 * blockDim.x) {
      const float2 a = tile[e], b = tile[e + 1];
      if (ma.diag) {
        const uint64_t x = state_index(e);
        const float pa = cabs2(a), pb = cabs2(b);
        ns += pa + pb;
        es += pa * dg(x) + pb * dg(x + 1);
      }
      *reinterpret_cast<float4*>(psi + state_index(e)) = make_float4(a.x, a.y, b.x, b.y);
    }
    if (ma.ep.partial) {
      eacc += (double)es;
      nacc += (double)ns;
    }
    __syncthreads();  // the tile is rewritten by the next load
  }
  if (ma.ep.partial) block_store_pair(eacc, nacc, ma.ep.partial);
}

}  // namespace

int multigate_grid(int L, const LaunchCfg& cfg) {
  const int tb = L < kMgTileBits ? L : kMgTileBits;
  const uint64_t ntiles = 1ull << (L - tb);
  uint64_t grid = (uint64_t)cfg.num_sms * g_mg_ctas_per_sm;
  if (grid > ntiles) grid = ntiles;
  return (int)grid;
}

cudaError_t multigate_prepare() {
  const int smem = (int)(sizeof(float2) << kMgTileBits);
  cudaError_t e = cudaFuncSetAttribute(k_multigate, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_multigate, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multigate, kMgThreads, smem);
  if (e == cudaSuccess && per_sm > 0) g_mg_ctas_per_sm = per_sm;
  return e;
}

cudaError_t launch_multigate(const MultiArgs& ma, void* psi, const LaunchCfg& cfg,
                             cudaStream_t s) {
  const size_t smem = sizeof(float2) << ma.tb;
  k_multigate<<<multigate_grid(ma.L, cfg), kMgThreads, smem, s>>>(static_cast<float2*>(psi), ma);
  return cudaGetLastError();
}

}  // namespace fsv
