// Energy moments and product-state overlaps of the current state.
//
//   k_h0_moments       per-block partials of Re <psi|H0 psi>, |H0 psi|^2 and
//                      |psi|^2: the mean energy E and its spread sigma_E of
//                      Eq. 10 and Eq. 11, with <H0^2> = |H0 psi|^2.  Each
//                      amplitude of H0 psi = D psi + sum_i cx_i X_i psi is
//                      formed on the fly from psi_x and its L bit-flip
//                      neighbours, so no second state is held;
//   k_bond_moments     the same for a general two-site chain (arbitrary
//                      Hermitian bond terms), from the four amplitudes that
//                      share each bond's quad;
//   k_factor_state     writes a product of site-group factors (a product or
//                      dimer-product initial state) from FP64 tables;
//   k_product_overlap  per-block partials of <phi|psi> for a product state
//                      phi_x = lo[x mod 2^m] hi[x >> m] (FP64 factor tables):
//                      the overlap of an echo's return with its start
//                      (Sec. V).
// All of them address psi in the natural layout (site i = bit i), which the
// state holds between periods.
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

// Compensated (Kahan) running sum in the state's precision.
template <typename R>
struct KahanSum {
  R s = 0, c = 0;
  __device__ __forceinline__ void add(R v) {
    const R y = v - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Deterministic block sums of k doubles, written to out[k * blockIdx.x + j].
template <int K>
__device__ void block_store_k(double (&v)[K], double* out) {
  __shared__ double sh[K][32];
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int j = 0; j < K; ++j) sh[j][w] = v[j];
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      double t = l < nw ? sh[j][l] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (l == 0) out[K * blockIdx.x + j] = t;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_h0_moments(const typename CT<R>::C* __restrict__ psi,
                                                         int L, H0Coef h, double* partial) {
  using C = typename CT<R>::C;
  // the coefficients once in the state's precision (no FP64 work per
  // amplitude for complex64)
  __shared__ R s_cx[34], s_cz[34];
  if (threadIdx.x < (unsigned)L) {
    s_cx[threadIdx.x] = (R)h.cx[threadIdx.x];
    s_cz[threadIdx.x] = (R)h.cz[threadIdx.x];
  }
  const R J = (R)h.J;
  __syncthreads();
  const uint64_t n = 1ull << L;
  KahanSum<R> e1, e2, nn;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const C v = psi[x];
    // diagonal part: J sum_b z_b z_{b+1} + sum_i cz_i z_i, z = 1 - 2 b_i
    R d = 0;
    for (int i = 0; i < L; ++i) {
      const R zi = ((x >> i) & 1) ? (R)-1 : (R)1;
      d += s_cz[i] * zi;
      if (i + 1 < L) d += J * zi * (((x >> (i + 1)) & 1) ? (R)-1 : (R)1);
    }
    C hv;
    hv.x = d * v.x;
    hv.y = d * v.y;
    // transverse part: cx_i X_i takes the amplitude with bit i flipped
    for (int i = 0; i < L; ++i) {
      const C u = psi[x ^ (1ull << i)];
      hv.x += s_cx[i] * u.x;
      hv.y += s_cx[i] * u.y;
    }
    e1.add(v.x * hv.x + v.y * hv.y);
    e2.add(hv.x * hv.x + hv.y * hv.y);
    nn.add(v.x * v.x + v.y * v.y);
  }
  double out[3] = {e1.value(), e2.value(), nn.value()};
  block_store_k<3>(out, partial);
}

// The same moments for a general two-site chain, H0 = sum_b h_b with
// arbitrary Hermitian 4x4 bond terms (local index r = 2 b_b + b_{b+1}):
// (H0 psi)_x = sum_b sum_r' h_b[r_b(x), r'] psi_{x with bits (b, b+1) = r'}.
template <typename R>
__global__ void __launch_bounds__(kThreads)
    k_bond_moments(const typename CT<R>::C* __restrict__ psi, int L,
                   const typename CT<R>::C* __restrict__ hb, double* partial) {
  using C = typename CT<R>::C;
  __shared__ C s_h[33 * 16];
  for (int k = threadIdx.x; k < 16 * (L - 1); k += blockDim.x) s_h[k] = hb[k];
  __syncthreads();
  const uint64_t n = 1ull << L;
  KahanSum<R> e1, e2, nn;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const C v = psi[x];
    C hv;
    hv.x = 0;
    hv.y = 0;
    for (int b = 0; b < L - 1; ++b) {
      const uint64_t bi = 1ull << b, bj = 1ull << (b + 1);
      const int r = 2 * (int)((x >> b) & 1) + (int)((x >> (b + 1)) & 1);
      const uint64_t base = x & ~(bi | bj);
      const C* row = s_h + 16 * b + 4 * r;
#pragma unroll
      for (int rp = 0; rp < 4; ++rp) {
        const C u = psi[base | ((rp >> 1) ? bi : 0) | ((rp & 1) ? bj : 0)];
        const C m = row[rp];
        hv.x += m.x * u.x - m.y * u.y;
        hv.y += m.x * u.y + m.y * u.x;
      }
    }
    e1.add(v.x * hv.x + v.y * hv.y);
    e2.add(hv.x * hv.x + hv.y * hv.y);
    nn.add(v.x * v.x + v.y * v.y);
  }
  double out[3] = {e1.value(), e2.value(), nn.value()};
  block_store_k<3>(out, partial);
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
    k_product_overlap(const typename CT<R>::C* __restrict__ psi, int L, int m,
                      const double2* __restrict__ lo, const double2* __restrict__ hi,
                      double* partial) {
  using C = typename CT<R>::C;
  const uint64_t n = 1ull << L;
  const uint64_t mask = (1ull << m) - 1;
  double ar = 0.0, ai = 0.0;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const double2 a = lo[x & mask], b = hi[x >> m];
    const double pr = a.x * b.x - a.y * b.y, pi = a.x * b.y + a.y * b.x;
    const C v = psi[x];
    const double vr = (double)v.x, vi = (double)v.y;
    // conj(phi_x) psi_x
    ar += pr * vr + pi * vi;
    ai += pr * vi - pi * vr;
  }
  double out[2] = {ar, ai};
  block_store_k<2>(out, partial);
}

// psi_x = lo[x mod 2^m] hi[x >> m] in the state's precision: a product of
// site-group factors (single sites, or the pairs of a dimer product state)
// from FP64 tables.
template <typename R>
__global__ void __launch_bounds__(kThreads)
    k_factor_state(typename CT<R>::C* __restrict__ psi, int L, int m,
                   const double2* __restrict__ lo, const double2* __restrict__ hi) {
  using C = typename CT<R>::C;
  const uint64_t n = 1ull << L;
  const uint64_t mask = (1ull << m) - 1;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const double2 a = lo[x & mask], b = hi[x >> m];
    C v;
    v.x = (R)(a.x * b.x - a.y * b.y);
    v.y = (R)(a.x * b.y + a.y * b.x);
    psi[x] = v;
  }
}

}  // namespace

int moments_grid(const LaunchCfg& cfg) { return cfg.num_sms * kBlocksPerSM; }

cudaError_t launch_factor_state(int precision, void* psi, int L, int m, const void* lo,
                                const void* hi, const LaunchCfg& cfg, cudaStream_t s) {
  const int grid = moments_grid(cfg);
  const double2* l2 = static_cast<const double2*>(lo);
  const double2* h2 = static_cast<const double2*>(hi);
  if (precision == SV_C128)
    k_factor_state<double><<<grid, kThreads, 0, s>>>(static_cast<double2*>(psi), L, m, l2, h2);
  else
    k_factor_state<float><<<grid, kThreads, 0, s>>>(static_cast<float2*>(psi), L, m, l2, h2);
  return cudaGetLastError();
}

cudaError_t launch_h0_moments(int precision, const void* psi, int L, const H0Coef& h,
                              double* partial, const LaunchCfg& cfg, cudaStream_t s) {
  const int grid = moments_grid(cfg);
  if (precision == SV_C128)
    k_h0_moments<double><<<grid, kThreads, 0, s>>>(static_cast<const double2*>(psi), L, h,
                                                   partial);
  else
    k_h0_moments<float><<<grid, kThreads, 0, s>>>(static_cast<const float2*>(psi), L, h,
                                                  partial);
  return cudaGetLastError();
}

cudaError_t launch_bond_moments(int precision, const void* psi, int L, const void* hb,
                                double* partial, const LaunchCfg& cfg, cudaStream_t s) {
  const int grid = moments_grid(cfg);
  if (precision == SV_C128)
    k_bond_moments<double><<<grid, kThreads, 0, s>>>(static_cast<const double2*>(psi), L,
                                                     static_cast<const double2*>(hb), partial);
  else
    k_bond_moments<float><<<grid, kThreads, 0, s>>>(static_cast<const float2*>(psi), L,
                                                    static_cast<const float2*>(hb), partial);
  return cudaGetLastError();
}

cudaError_t launch_product_overlap(int precision, const void* psi, int L, int m,
                                   const void* lo, const void* hi, double* partial,
                                   const LaunchCfg& cfg, cudaStream_t s) {
  const int grid = moments_grid(cfg);
  const double2* l2 = static_cast<const double2*>(lo);
  const double2* h2 = static_cast<const double2*>(hi);
  if (precision == SV_C128)
    k_product_overlap<double><<<grid, kThreads, 0, s>>>(static_cast<const double2*>(psi), L, m,
                                                        l2, h2, partial);
  else
    k_product_overlap<float><<<grid, kThreads, 0, s>>>(static_cast<const float2*>(psi), L, m,
                                                       l2, h2, partial);
  return cudaGetLastError();
}

}  // namespace fsv
