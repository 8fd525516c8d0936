// Device helpers shared by the kernels: complex arithmetic, the diagonal
// part of H0 in the natural layout, and deterministic block reductions.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "sv_internal.h"
#include "sv_kernels.h"

namespace fsv {
namespace dev {

template <typename R>
struct CT;
template <>
struct CT<float> {
  using C = float2;
  using V = float4;
  static constexpr int NV = 2;  // amplitudes per vector
  static constexpr int LV = 1;  // log2(NV)
};
template <>
struct CT<double> {
  using C = double2;
  using V = double2;
  static constexpr int NV = 1;
  static constexpr int LV = 0;
};

// Double-float real (SV_DF64): the unevaluated sum hi + lo of two FP32
// numbers, |lo| <= ulp(hi) / 2, about 48 significant bits.  Built from the
// error-free transformations of Dekker (1971) and Knuth: two_sum (the exact
// rounding error of a + b), fast_two_sum (the same when |a| >= |b|) and
// two_prod (the exact error of a * b, one FMA).  All steps use the _rn
// intrinsics, so the compiler neither contracts nor reorders them.
struct df {
  float hi, lo;
  df() = default;
  __device__ __forceinline__ df(int v) : hi((float)v), lo(0.f) {}  // exact below 2^24
  __device__ __forceinline__ df(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit df(double v) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};
struct __align__(16) dfc {
  df x, y;
};

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
// a + b: the exact sum of the leading parts, the trailing parts added to its
// error, one renormalisation; absolute error about 2^-46 (|a| + |b|)
__device__ __forceinline__ df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
// error of the product hi parts plus the cross terms (lo * lo dropped)
__device__ __forceinline__ float prod_err(df a, df b, float p) {
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  return __fmaf_rn(a.lo, b.hi, e);
}
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  return fast_two_sum(p, prod_err(a, b, p));
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }
// acc + a b + c d with one renormalisation: both products' leading parts
// enter exact sums, every error term is collected in one FP32 number
__device__ __forceinline__ df dot2_acc(df acc, df a, df b, df c, df d) {
  const float p1 = __fmul_rn(a.hi, b.hi), p2 = __fmul_rn(c.hi, d.hi);
  const float e1 = prod_err(a, b, p1), e2 = prod_err(c, d, p2);
  const df s1 = two_sum(acc.hi, p1);
  const df s2 = two_sum(s1.hi, p2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(acc.lo, s1.lo), __fadd_rn(s2.lo, e1)), e2);
  return fast_two_sum(s2.hi, lo);
}

template <>
struct CT<df> {
  using C = dfc;
  using V = dfc;
  static constexpr int NV = 1;
  static constexpr int LV = 0;
};

__device__ __forceinline__ void unpack(const dfc& v, dfc a[1]) { a[0] = v; }
__device__ __forceinline__ dfc pack(const dfc a[1]) { return a[0]; }
__device__ __forceinline__ dfc cmac(dfc acc, dfc g, dfc v) {
  acc.x = dot2_acc(acc.x, g.x, v.x, -g.y, v.y);
  acc.y = dot2_acc(acc.y, g.x, v.y, g.y, v.x);
  return acc;
}
__device__ __forceinline__ dfc shfl_xor(dfc v, int m) {
  v.x.hi = __shfl_xor_sync(0xffffffffu, v.x.hi, m);
  v.x.lo = __shfl_xor_sync(0xffffffffu, v.x.lo, m);
  v.y.hi = __shfl_xor_sync(0xffffffffu, v.y.hi, m);
  v.y.lo = __shfl_xor_sync(0xffffffffu, v.y.lo, m);
  return v;
}

__device__ __forceinline__ void unpack(const float4& v, float2 a[2]) {
  a[0] = make_float2(v.x, v.y);
  a[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ float4 pack(const float2 a[2]) {
  return make_float4(a[0].x, a[0].y, a[1].x, a[1].y);
}
__device__ __forceinline__ void unpack(const double2& v, double2 a[1]) { a[0] = v; }
__device__ __forceinline__ double2 pack(const double2 a[1]) { return a[0]; }

__device__ __forceinline__ float2 cmac(float2 acc, float2 g, float2 v) {
  acc.x = fmaf(g.x, v.x, acc.x);
  acc.x = fmaf(-g.y, v.y, acc.x);
  acc.y = fmaf(g.x, v.y, acc.y);
  acc.y = fmaf(g.y, v.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 cmac(double2 acc, double2 g, double2 v) {
  acc.x = fma(g.x, v.x, acc.x);
  acc.x = fma(-g.y, v.y, acc.x);
  acc.y = fma(g.x, v.y, acc.y);
  acc.y = fma(g.y, v.x, acc.y);
  return acc;
}
template <typename C>
__device__ __forceinline__ C czero() {
  C z;
  z.x = 0;
  z.y = 0;
  return z;
}
// Re(conj(a) b)
template <typename C>
__device__ __forceinline__ auto cdotre(C a, C b) -> decltype(a.x) {
  return a.x * b.x + a.y * b.y;
}
template <typename C>
__device__ __forceinline__ auto cabs2(C a) -> decltype(a.x) {
  return a.x * a.x + a.y * a.y;
}

__device__ __forceinline__ float2 shfl_xor(float2 v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}
__device__ __forceinline__ double2 shfl_xor(double2 v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  return v;
}

// Diagonal part of H0 at basis state x (site i = bit i):
//   J sum_b s_b s_{b+1} + sum_i cz_i s_i,  s = 1 - 2 b.
template <typename R>
struct Diag {
  R J, cz_bulk, cz_first, cz_last, czsum;
  uint64_t zzmask, bulkmask;
  int L;
  __device__ void init(const EpiParams& ep, int L_) {
    L = L_;
    J = (R)ep.J;
    cz_bulk = (R)ep.cz_bulk;
    cz_first = (R)ep.cz_first;
    cz_last = (R)ep.cz_last;
    czsum = (R)(ep.cz_bulk * (L_ - 2) + ep.cz_first + ep.cz_last);
    zzmask = (1ull << (L_ - 1)) - 1;
    bulkmask = ((1ull << L_) - 1) & ~1ull & ~(1ull << (L_ - 1));
  }
  __device__ __forceinline__ R operator()(uint64_t x) const {
    int flips = __popcll((x ^ (x >> 1)) & zzmask);
    int nb = __popcll(x & bulkmask);
    // bit tests as selects: a 64-bit integer to float conversion is slow
    R up = cz_bulk * (R)nb + ((x & 1) ? cz_first : (R)0) + (((x >> (L - 1)) & 1) ? cz_last : (R)0);
    return J * (R)(L - 1 - 2 * flips) + czsum - (R)2 * up;
  }
};

// Natural index (site i at bit i) of index x in the block layout whose
// window of n sites starts at site lo: window sites at bits 0..n-1, sites
// below lo at bits n..n+lo-1, the others in place (lo = 0: natural).
__device__ __forceinline__ uint64_t to_natural(uint64_t x, int n, int lo) {
  if (lo == 0) return x;
  const uint64_t win = x & ((1ull << n) - 1);
  const uint64_t below = (x >> n) & ((1ull << lo) - 1);
  const uint64_t rest = x & ~((1ull << (n + lo)) - 1);
  return (win << lo) | below | rest;
}

// Deterministic block sum of (e, n) written to out[2*blockIdx.x + {0,1}].
__device__ inline void block_store_pair(double e, double n, double* out) {
  __shared__ double se[32], sn[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    se[w] = e;
    sn[w] = n;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    e = l < nw ? se[l] : 0.0;
    n = l < nw ? sn[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    if (l == 0) {
      out[2 * blockIdx.x] = e;
      out[2 * blockIdx.x + 1] = n;
    }
  }
}

// Scale factor of the folded renormalisation (1 when this pass does none).
__device__ __forceinline__ double renorm_scale(const Renorm& rn) {
  if (!rn.ring || rn.every <= 0) return 1.0;
  const long long c = *rn.counter;
  if (c <= 0 || c % rn.every != 0) return 1.0;
  const double n2 = rn.ring[2 * ((c - 1) % rn.ring_len) + 1];
  return n2 > 0.0 ? 1.0 / sqrt(n2) : 1.0;
}

template <typename C>
__device__ __forceinline__ const C* gate_ptr(const C* base, long long stride,
                                             const long long* counter) {
  return stride ? base + (*counter) * stride : base;
}


}  // namespace dev
}  // namespace fsv
