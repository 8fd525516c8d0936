// Batched evolution of many independent chains: the resident form.
//
// A chain of L <= 14 sites (at most 128 KiB of complex64 amplitudes) lives
// in one CTA's shared memory for a whole run of periods: the CTA loads it,
// applies every gate of every period in shared memory (the Eq. 2
// contraction per group of four amplitudes), measures the energy density
// and norm at the end of each period, and writes the state back once.  One
// launch runs all resident chains, one CTA each.
#include <cuda_runtime.h>

#include <cstdint>

#include "sv_batch.h"
#include "sv_device.cuh"

namespace fsv {

namespace {

using namespace dev;

constexpr int kThreads = 512;

__global__ void __launch_bounds__(kThreads, 1)
    k_chain_resident(const ResidentChain* __restrict__ chains, const long long* __restrict__ counter,
                     int periods, int ring_len) {
  extern __shared__ float2 sp[];
  const ResidentChain& ch = chains[blockIdx.x];
  const int L = ch.L;
  const uint32_t n = 1u << L;
  const long long p0 = *counter;
  // the chain's coefficients in FP32 once, so that the per-amplitude
  // measurement below runs no FP64 instruction
  __shared__ float s_cz[kResidentMaxL], s_cx[kResidentMaxL];
  if (threadIdx.x < (unsigned)L) {
    s_cz[threadIdx.x] = (float)ch.cz[threadIdx.x];
    s_cx[threadIdx.x] = (float)ch.cx[threadIdx.x];
  }
  const float Jf = (float)ch.J;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) sp[i] = ch.psi[i];
  __syncthreads();
  __shared__ double se[kThreads / 32], sn[kThreads / 32];
  for (int p = 0; p < periods; ++p) {
    for (int g = 0; g < ch.ngates; ++g) {
      const int b = ch.bonds[g];
      float2 G[16], Gl[16];  // gate and its FP32 rounding residual
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        G[k] = ch.gates[kGateEntries * g + k];
        Gl[k] = ch.gates[kGateEntries * g + 16 + k];
      }
      const uint32_t lowmask = (1u << b) - 1;
      // local index r = 2 b_b + b_{b+1}: offsets of r = 0..3
      const uint32_t o1 = 2u << b, o2 = 1u << b, o3 = 3u << b;
      for (uint32_t q = threadIdx.x; q < (n >> 2); q += blockDim.x) {
        const uint32_t x = (q & lowmask) | ((q >> b) << (b + 2));
        const float2 v0 = sp[x], v1 = sp[x + o1], v2 = sp[x + o2], v3 = sp[x + o3];
        float2 w[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          // residual products first, then the table's on top: a bare first
          // product with a fixed table entry would bias the norm downwards
          float2 a = czero<float2>();
          a = cmac(a, Gl[4 * r + 0], v0);
          a = cmac(a, Gl[4 * r + 1], v1);
          a = cmac(a, Gl[4 * r + 2], v2);
          a = cmac(a, Gl[4 * r + 3], v3);
          a = cmac(a, G[4 * r + 0], v0);
          a = cmac(a, G[4 * r + 1], v1);
          a = cmac(a, G[4 * r + 2], v2);
          a = cmac(a, G[4 * r + 3], v3);
          w[r] = a;
        }
        sp[x] = w[0];
        sp[x + o1] = w[1];
        sp[x + o2] = w[2];
        sp[x + o3] = w[3];
      }
      __syncthreads();
    }
    // <H0> and the norm of the period's final state (natural layout)
    // per-thread sums over its amplitudes, compensated (Kahan) in FP32
    float es = 0.f, ec = 0.f, ns = 0.f, nc = 0.f;
    for (uint32_t x = threadIdx.x; x < n; x += blockDim.x) {
      const float2 v = sp[x];
      const float pr = cabs2(v);
      float d = 0.f;
      for (int i = 0; i < L; ++i) {
        const float zi = ((x >> i) & 1) ? -1.f : 1.f;
        d += s_cz[i] * zi;
        if (i + 1 < L) d += Jf * zi * (((x >> (i + 1)) & 1) ? -1.f : 1.f);
      }
      float ex = 0.f;
      for (int i = 0; i < L; ++i)
        if (!((x >> i) & 1)) ex += 2.f * s_cx[i] * cdotre(v, sp[x | (1u << i)]);
      const float ye = (pr * d + ex) - ec, te = es + ye;
      ec = (te - es) - ye;
      es = te;
      const float yn = pr - nc, tn = ns + yn;
      nc = (tn - ns) - yn;
      ns = tn;
    }
    double e = (double)es - (double)ec, nn = (double)ns - (double)nc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      nn += __shfl_xor_sync(0xffffffffu, nn, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
      se[w] = e;
      sn[w] = nn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double te = 0.0, tn = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        te += se[k];
        tn += sn[k];
      }
      const long long slot = (p0 + p) % ring_len;
      ch.ring[2 * slot] = te / ((double)L * tn);
      ch.ring[2 * slot + 1] = tn;
    }
    __syncthreads();
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) ch.psi[i] = sp[i];
}

__global__ void k_advance(long long* counter, int periods) { *counter += periods; }

}  // namespace

size_t resident_smem_bytes(int L) { return sizeof(float2) << L; }

cudaError_t resident_prepare(int max_L) {
  return cudaFuncSetAttribute(k_chain_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)resident_smem_bytes(max_L));
}

cudaError_t launch_chain_resident(const ResidentChain* chains, int nchains, int max_L,
                                  long long* counter, int periods, int ring_len,
                                  cudaStream_t s) {
  if (nchains <= 0 || periods <= 0) return cudaSuccess;
  k_chain_resident<<<nchains, kThreads, resident_smem_bytes(max_L), s>>>(chains, counter,
                                                                        periods, ring_len);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_advance<<<1, 1, 0, s>>>(counter, periods);
  return cudaGetLastError();
}

}  // namespace fsv
