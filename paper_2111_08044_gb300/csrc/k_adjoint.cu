// Adjoint (reverse-mode) gradient of the final energy density with respect
// to per-period drive parameters: the state psi and the adjoint state
// lambda are walked back through the period's operations, each un-applied
// on both, while 2 Re <lambda| dO O^dagger |psi> is accumulated (the
// derivative of <psi_P|H0|psi_P>/L through operation O, evaluated after it).
// Reverse evolution by U^dagger is the echo construction of Sec. V; the
// energy observable is Eq. 7 divided by L.
//
// Kernels:
//   k_apply_h0      lambda = (H0 / L) psi, and per-block partials of
//                   Re <psi|lambda> (the energy density of a unit-norm psi);
//   k_adjoint_gate  one two-site operation on bond (b, b+1): accumulates
//                   Re <lambda|D|psi> (D = dO O^dagger), then psi <- O^dag psi
//                   and lambda <- O^dag lambda, in place;
//   k_grad_reduce   the partials of a range of passes, summed in a fixed
//                   order, times 2, into one gradient entry.
#include <cuda_runtime.h>

#include <cstdint>

#include "sv_device.cuh"
#include "sv_internal.h"
#include "sv_kernels.h"

namespace fsv {

namespace {

using namespace dev;

constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

// Deterministic block sum of v, written to out[blockIdx.x].
__device__ inline void block_store(double v, double* out) {
  __shared__ double sv[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sv[w] = v;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    v = l < nw ? sv[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) out[blockIdx.x] = v;
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_apply_h0(const typename CT<R>::C* __restrict__ psi,
                                                       typename CT<R>::C* __restrict__ lam,
                                                       int L, H0Coef h, double* partial) {
  using C = typename CT<R>::C;
  const uint64_t n = 1ull << L;
  const R inv_l = (R)(1.0 / L);
  double acc = 0.0;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const C v = psi[x];
    // diagonal part: J sum_b z_b z_{b+1} + sum_i cz_i z_i, z = 1 - 2 b_i
    R d = 0;
    for (int i = 0; i < L; ++i) {
      const R zi = ((x >> i) & 1) ? (R)-1 : (R)1;
      d += (R)h.cz[i] * zi;
      if (i + 1 < L) d += (R)h.J * zi * (((x >> (i + 1)) & 1) ? (R)-1 : (R)1);
    }
    C out;
    out.x = d * v.x;
    out.y = d * v.y;
    // transverse part: sum_i cx_i X_i flips bit i
    for (int i = 0; i < L; ++i) {
      const C u = psi[x ^ (1ull << i)];
      out.x += (R)h.cx[i] * u.x;
      out.y += (R)h.cx[i] * u.y;
    }
    out.x *= inv_l;
    out.y *= inv_l;
    lam[x] = out;
    acc += (double)cdotre(v, out);
  }
  block_store(acc, partial);
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_adjoint_gate(typename CT<R>::C* __restrict__ psi,
                                                           typename CT<R>::C* __restrict__ lam,
                                                           int L, int b,
                                                           const typename CT<R>::C* __restrict__ od,
                                                           const typename CT<R>::C* __restrict__ dd,
                                                           double* partial) {
  using C = typename CT<R>::C;
  // od: O^dagger, dd: D = dO O^dagger; both 4x4 row-major with the local
  // index r = 2 b_b + b_{b+1} (site b is the high bit)
  __shared__ C so[16], sd[16];
  if (threadIdx.x < 16) {
    so[threadIdx.x] = od[threadIdx.x];
    sd[threadIdx.x] = dd[threadIdx.x];
  }
  __syncthreads();
  const uint64_t ng = 1ull << (L - 2);
  const uint64_t lowmask = (1ull << b) - 1;
  const uint64_t off[4] = {0, 2ull << b, 1ull << b, 3ull << b};  // r = 0..3
  double acc = 0.0;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng;
       g += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x = (g & lowmask) | ((g >> b) << (b + 2));
    C v[4], w[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      v[r] = psi[x + off[r]];
      w[r] = lam[x + off[r]];
    }
    R t = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      C dv = czero<C>();
#pragma unroll
      for (int c = 0; c < 4; ++c) dv = cmac(dv, sd[4 * r + c], v[c]);
      t += cdotre(w[r], dv);
    }
    acc += (double)t;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      C pv = czero<C>(), pw = czero<C>();
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        pv = cmac(pv, so[4 * r + c], v[c]);
        pw = cmac(pw, so[4 * r + c], w[c]);
      }
      psi[x + off[r]] = pv;
      lam[x + off[r]] = pw;
    }
  }
  block_store(acc, partial);
}

// out[0] = 2 * sum of partials[0 .. n), in a fixed order.
__global__ void __launch_bounds__(kThreads) k_grad_reduce(const double* __restrict__ partials,
                                                          long long n, double* out) {
  double s = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) s += partials[k];
  __shared__ double sh[kThreads];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = 2.0 * sh[0];
}

// out[0] = sum of partials (no factor), for the energy density
__global__ void __launch_bounds__(kThreads) k_sum(const double* __restrict__ partials, long long n,
                                                  double* out) {
  double s = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) s += partials[k];
  __shared__ double sh[kThreads];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

}  // namespace

int adjoint_grid(const LaunchCfg& cfg) { return cfg.num_sms * kBlocksPerSM; }

cudaError_t launch_apply_h0(int precision, const void* psi, void* lam, int L, const H0Coef& h,
                            double* partial, const LaunchCfg& cfg, cudaStream_t s) {
  const int grid = adjoint_grid(cfg);
  if (precision == SV_C128)
    k_apply_h0<double><<<grid, kThreads, 0, s>>>(static_cast<const double2*>(psi),
                                                 static_cast<double2*>(lam), L, h, partial);
  else
    k_apply_h0<float><<<grid, kThreads, 0, s>>>(static_cast<const float2*>(psi),
                                                static_cast<float2*>(lam), L, h, partial);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_gate(int precision, void* psi, void* lam, int L, int bond,
                                const void* odag, const void* dmat, double* partial,
                                const LaunchCfg& cfg, cudaStream_t s) {
  const int grid = adjoint_grid(cfg);
  if (precision == SV_C128)
    k_adjoint_gate<double><<<grid, kThreads, 0, s>>>(
        static_cast<double2*>(psi), static_cast<double2*>(lam), L, bond,
        static_cast<const double2*>(odag), static_cast<const double2*>(dmat), partial);
  else
    k_adjoint_gate<float><<<grid, kThreads, 0, s>>>(
        static_cast<float2*>(psi), static_cast<float2*>(lam), L, bond,
        static_cast<const float2*>(odag), static_cast<const float2*>(dmat), partial);
  return cudaGetLastError();
}

cudaError_t launch_grad_reduce(const double* partials, long long n, double* out, int times_two,
                               cudaStream_t s) {
  if (times_two)
    k_grad_reduce<<<1, kThreads, 0, s>>>(partials, n, out);
  else
    k_sum<<<1, kThreads, 0, s>>>(partials, n, out);
  return cudaGetLastError();
}

}  // namespace fsv
