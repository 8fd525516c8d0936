// Plain form: one in-place pass over the state per two-qubit gate, the
// contraction of Eq. 2 of arXiv 2111.08044 done as a 4x4 complex matvec per
// group of four amplitudes, plus the product-state initialisation, the
// per-period energy / norm reduction and the renormalisation pass.
//
// Layout: amplitude x = sum_i b_i 2^i, interleaved (re, im).  A complex64
// thread works on float4 vectors (two consecutive amplitudes); a complex128
// thread on double2 vectors (one amplitude).  Within a warp, consecutive
// lanes hold consecutive vectors, so every load and store instruction moves
// a contiguous 512-byte span.
//
// Gates on low bonds (both bits inside the span one warp covers in four
// loads) pair amplitudes across lanes with warp shuffles; gates on higher
// bonds pair four separate contiguous spans in registers.
//
// Gate tables (complex64): each 4x4 gate is an FP32 table plus the FP32
// residual of its FP64 entries, so the applied gate is exact to about 2^-48.
// The residual products are accumulated first and the table's products on
// top of them (lo_first).  Started from zero instead, the first rounding of
// each output is that of a bare product g v with a fixed g: its error then
// depends on where |v| falls within its binade, so it correlates with the
// result, and for gates close to the identity it shrank the norm by about
// 1.3e-9 per gate application (an FP32 emulation of the kernel reproduces
// this).  The residual sum varies with v independently of that grid and
// takes the bias out.
//
// Energy terms are folded into the gate passes (no extra pass over the
// state): the pass that applies the last gate of the period on site j also
// measures <X_j> (the one-site reduced state is final once its last gate has
// run), and the last pass of the period measures the diagonal part
// J sum Z Z + sum cz Z and the norm.  Partial sums: FP32 within a thread's
// iteration, FP64 across iterations, threads and blocks, in a fixed order.
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

// ---------------------------------------------------------------- high bonds
// Bond (i, i+1) with i >= LV + 5: each work item is one vector per member
// r = 2 b_i + b_{i+1} of NV four-amplitude groups; consecutive items are
// consecutive vectors, so a warp's four loads are four 512-byte spans.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_gate_high(
    typename CT<R>::C* __restrict__ psi, int L, int i,
    const typename CT<R>::C* __restrict__ gate_base, long long stride,
    const long long* __restrict__ counter, EpiParams ep, int store) {
  using C = typename CT<R>::C;
  using V = typename CT<R>::V;
  constexpr int NV = CT<R>::NV, LV = CT<R>::LV;
  const C* gp = gate_ptr(gate_base, stride, counter);
  const R sc = (R)renorm_scale(ep.rn);
  // the gate as hi + lo parts (lo = 0 in FP64): the FP32 table's rounding
  // error is carried along instead of being applied every period
  C g[16], gl[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    g[k] = gp[k];
    g[k].x *= sc;
    g[k].y *= sc;
    gl[k] = gp[16 + k];
    gl[k].x *= sc;
    gl[k].y *= sc;
  }
  Diag<R> dg;
  if (ep.flags & EPI_DIAG) dg.init(ep, L);
  const R cxh = (R)ep.cx_hi, cxl = (R)ep.cx_lo;
  const int lowbits = i - LV;
  const uint64_t nitems = 1ull << (L - 2 - LV);
  const uint64_t lowmask = (1ull << lowbits) - 1;
  const uint64_t off[4] = {0, 2ull << i, 1ull << i, 3ull << i};  // r = 0..3
  V* pv = reinterpret_cast<V*>(psi);
  double eacc = 0.0, nacc = 0.0;
  const uint64_t S = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t q0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q0 < nitems;
       q0 += 2 * S) {
    V a[2][4];
    uint64_t xs[2];
    bool ok[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint64_t q = q0 + u * S;
      ok[u] = q < nitems;
      xs[u] = ((q & lowmask) << LV) | ((q >> lowbits) << (i + 2));
      if (ok[u]) {
#pragma unroll
        for (int r = 0; r < 4; ++r) a[u][r] = pv[(xs[u] + off[r]) >> LV];
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!ok[u]) continue;
      C v[4][NV], w[4][NV];
#pragma unroll
      for (int r = 0; r < 4; ++r) unpack(a[u][r], v[r]);
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          // residual products first, then the table's on top (lo_first)
          C acc = czero<C>();
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (kGateLo<R>) acc = cmac(acc, gl[4 * r + c], v[c][k]);
#pragma unroll
          for (int c = 0; c < 4; ++c) acc = cmac(acc, g[4 * r + c], v[c][k]);
          w[r][k] = acc;
        }
      if (store) {
#pragma unroll
        for (int r = 0; r < 4; ++r) pv[(xs[u] + off[r]) >> LV] = pack(w[r]);
      }
      if (ep.flags) {
        R es = 0, ns = 0;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          if (ep.flags & EPI_X_HI)
            es += cxh * (R)2 * (cdotre(w[0][k], w[2][k]) + cdotre(w[1][k], w[3][k]));
          if (ep.flags & EPI_X_LO)
            es += cxl * (R)2 * (cdotre(w[0][k], w[1][k]) + cdotre(w[2][k], w[3][k]));
          if (ep.flags & EPI_DIAG) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              R p = cabs2(w[r][k]);
              ns += p;
              es += p * dg(xs[u] + off[r] + k);
            }
          }
        }
        eacc += (double)es;
        nacc += (double)ns;
      }
    }
  }
  if (ep.flags) block_store_pair(eacc, nacc, ep.partial);
}

// ----------------------------------------------------------------- low bonds
// Bond (I, I+1) with I + 1 < LV + 7: a warp iteration covers 2^(LV+7)
// consecutive amplitudes as four register chunks (address bits LV+5, LV+6)
// of 32 lanes (bits LV..LV+4) of NV-amplitude vectors (bits 0..LV-1).
// Partners across lanes come from warp shuffles.
template <int LV, int B>
struct BitPos {
  // kind: 0 in-vector, 1 lane, 2 register chunk
  static constexpr int kind = B < LV ? 0 : (B < LV + 5 ? 1 : 2);
  static constexpr int km = kind == 0 ? (1 << B) : 0;
  static constexpr int lm = kind == 1 ? (1 << (B - LV)) : 0;
  static constexpr int cm = kind == 2 ? (1 << (B - LV - 5)) : 0;
};

template <typename R, int I>
struct LowMasks {
  static constexpr int LV = CT<R>::LV;
  using Hi = BitPos<LV, I>;      // site I   (r bit 1)
  using Lo = BitPos<LV, I + 1>;  // site I+1 (r bit 0)
  // flip pattern d (bit 1: flip b_I, bit 0: flip b_{I+1})
  static constexpr int km(int d) { return ((d & 2) ? Hi::km : 0) | ((d & 1) ? Lo::km : 0); }
  static constexpr int lm(int d) { return ((d & 2) ? Hi::lm : 0) | ((d & 1) ? Lo::lm : 0); }
  static constexpr int cm(int d) { return ((d & 2) ? Hi::cm : 0) | ((d & 1) ? Lo::cm : 0); }
};

template <typename R, int I>
__device__ __forceinline__ int local_r(int c, int lane, int k) {
  using M = LowMasks<R, I>;
  int bh = ((k & M::Hi::km) | (lane & M::Hi::lm) | (c & M::Hi::cm)) != 0;
  int bl = ((k & M::Lo::km) | (lane & M::Lo::lm) | (c & M::Lo::cm)) != 0;
  return 2 * bh + bl;
}

// P[c][k] = value at the address with the pattern-d bits flipped.
template <typename R, int I, int D>
__device__ __forceinline__ void fetch(const typename CT<R>::C (&a)[4][CT<R>::NV],
                                      typename CT<R>::C (&p)[4][CT<R>::NV]) {
  using M = LowMasks<R, I>;
  constexpr int km = M::km(D), lm = M::lm(D), cm = M::cm(D);
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < CT<R>::NV; ++k) {
      auto v = a[c ^ cm][k ^ km];
      p[c][k] = lm ? shfl_xor(v, lm) : v;
    }
}

template <typename R, int I>
__global__ void __launch_bounds__(kThreads) k_gate_low(
    typename CT<R>::C* __restrict__ psi, int L,
    const typename CT<R>::C* __restrict__ gate_base, long long stride,
    const long long* __restrict__ counter, EpiParams ep, int store) {
  using C = typename CT<R>::C;
  using V = typename CT<R>::V;
  constexpr int NV = CT<R>::NV, LV = CT<R>::LV;
  __shared__ C gs[kGateEntries];  // hi parts, then lo parts
  const C* gp = gate_ptr(gate_base, stride, counter);
  if (threadIdx.x < kGateEntries) {
    const R sc = (R)renorm_scale(ep.rn);
    C g = gp[threadIdx.x];
    g.x *= sc;
    g.y *= sc;
    gs[threadIdx.x] = g;
  }
  __syncthreads();
  Diag<R> dg;
  if (ep.flags & EPI_DIAG) dg.init(ep, L);
  const R cxh = (R)ep.cx_hi, cxl = (R)ep.cx_lo;
  const int lane = threadIdx.x & 31;
  const uint64_t nwi = 1ull << (L - (LV + 7));
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  V* pv = reinterpret_cast<V*>(psi);
  double eacc = 0.0, nacc = 0.0;
  int rs[4][NV];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int k = 0; k < NV; ++k) rs[c][k] = local_r<R, I>(c, lane, k);
  for (uint64_t wi = gw; wi < nwi; wi += nw) {
    const uint64_t vbase = (wi << (LV + 7)) >> LV;  // in vectors
    C a[4][NV];
#pragma unroll
    for (int c = 0; c < 4; ++c) unpack(pv[vbase + ((uint64_t)c << 5) + lane], a[c]);
    C p1[4][NV], p2[4][NV], p3[4][NV], w[4][NV];
    fetch<R, I, 1>(a, p1);
    fetch<R, I, 2>(a, p2);
    fetch<R, I, 3>(a, p3);
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int r = rs[c][k];
        // residual products first, then the table's on top (lo_first)
        C acc = czero<C>();
        if (kGateLo<R>) {
          acc = cmac(acc, gs[16 + 4 * r + r], a[c][k]);
          acc = cmac(acc, gs[16 + 4 * r + (r ^ 1)], p1[c][k]);
          acc = cmac(acc, gs[16 + 4 * r + (r ^ 2)], p2[c][k]);
          acc = cmac(acc, gs[16 + 4 * r + (r ^ 3)], p3[c][k]);
        }
        acc = cmac(acc, gs[4 * r + r], a[c][k]);
        acc = cmac(acc, gs[4 * r + (r ^ 1)], p1[c][k]);
        acc = cmac(acc, gs[4 * r + (r ^ 2)], p2[c][k]);
        acc = cmac(acc, gs[4 * r + (r ^ 3)], p3[c][k]);
        w[c][k] = acc;
      }
    if (store) {
#pragma unroll
      for (int c = 0; c < 4; ++c) pv[vbase + ((uint64_t)c << 5) + lane] = pack(w[c]);
    }
    if (ep.flags) {
      R es = 0, ns = 0;
      if (ep.flags & EPI_X_HI) {
        C q[4][NV];
        fetch<R, I, 2>(w, q);
        R s = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < NV; ++k) s += cdotre(w[c][k], q[c][k]);
        es += cxh * s;
      }
      if (ep.flags & EPI_X_LO) {
        C q[4][NV];
        fetch<R, I, 1>(w, q);
        R s = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < NV; ++k) s += cdotre(w[c][k], q[c][k]);
        es += cxl * s;
      }
      if (ep.flags & EPI_DIAG) {
        const uint64_t abase = wi << (LV + 7);
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < NV; ++k) {
            R pr = cabs2(w[c][k]);
            ns += pr;
            es += pr * dg(abase + ((uint64_t)c << (LV + 5)) + ((uint64_t)lane << LV) + k);
          }
      }
      eacc += (double)es;
      nacc += (double)ns;
    }
  }
  if (ep.flags) block_store_pair(eacc, nacc, ep.partial);
}

// --------------------------------------------------------------- tiny chains
// L < LV + 7: one thread per four-amplitude group.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_gate_small(
    typename CT<R>::C* __restrict__ psi, int L, int i,
    const typename CT<R>::C* __restrict__ gate_base, long long stride,
    const long long* __restrict__ counter, EpiParams ep, int store) {
  using C = typename CT<R>::C;
  const C* gp = gate_ptr(gate_base, stride, counter);
  const R sc = (R)renorm_scale(ep.rn);
  Diag<R> dg;
  if (ep.flags & EPI_DIAG) dg.init(ep, L);
  const R cxh = (R)ep.cx_hi, cxl = (R)ep.cx_lo;
  const uint64_t ngroups = 1ull << (L - 2);
  const uint64_t lowmask = (1ull << i) - 1;
  const uint64_t off[4] = {0, 2ull << i, 1ull << i, 3ull << i};
  double eacc = 0.0, nacc = 0.0;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ngroups;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x = (q & lowmask) | ((q >> i) << (i + 2));
    C v[4], w[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = psi[x + off[r]];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      // residual products first, then the table's on top (lo_first)
      C acc = czero<C>();
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (kGateLo<R>) acc = cmac(acc, gp[16 + 4 * r + c], v[c]);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = cmac(acc, gp[4 * r + c], v[c]);
      acc.x *= sc;
      acc.y *= sc;
      w[r] = acc;
    }
    if (store) {
#pragma unroll
      for (int r = 0; r < 4; ++r) psi[x + off[r]] = w[r];
    }
    if (ep.flags) {
      R es = 0, ns = 0;
      if (ep.flags & EPI_X_HI) es += cxh * (R)2 * (cdotre(w[0], w[2]) + cdotre(w[1], w[3]));
      if (ep.flags & EPI_X_LO) es += cxl * (R)2 * (cdotre(w[0], w[1]) + cdotre(w[2], w[3]));
      if (ep.flags & EPI_DIAG)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          R p = cabs2(w[r]);
          ns += p;
          es += p * dg(x + off[r]);
        }
      eacc += (double)es;
      nacc += (double)ns;
    }
  }
  if (ep.flags) block_store_pair(eacc, nacc, ep.partial);
}

// ------------------------------------------------------------- period reduce
__device__ void period_reduce_block(const double* __restrict__ partials, long long n, int L,
                                    double* __restrict__ ring, int ring_len, long long* counter,
                                    int advance) {
  __shared__ double se[256], sn[256];
  double e = 0.0, nn = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) {
    e += partials[2 * k];
    nn += partials[2 * k + 1];
  }
  se[threadIdx.x] = e;
  sn[threadIdx.x] = nn;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      se[threadIdx.x] += se[threadIdx.x + s];
      sn[threadIdx.x] += sn[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long c = *counter;
    const long long slot = c % ring_len;
    // energy density of the normalised state: <psi|H0|psi> / (L <psi|psi>)
    ring[2 * slot] = sn[0] > 0.0 ? se[0] / (L * sn[0]) : 0.0;
    ring[2 * slot + 1] = sn[0];
    if (advance) *counter = c + 1;
  }
}

__global__ void __launch_bounds__(256) k_period_reduce(const double* __restrict__ partials,
                                                       long long n, int L,
                                                       double* __restrict__ ring,
                                                       int ring_len, long long* counter,
                                                       int advance) {
  period_reduce_block(partials, n, L, ring, ring_len, counter, advance);
}

// the period reduce of many chains, one block each
__global__ void __launch_bounds__(256) k_period_reduce_many(const ReduceItem* __restrict__ items) {
  const ReduceItem it = items[blockIdx.x];
  period_reduce_block(it.partials, it.n, it.L, it.ring, it.ring_len, it.counter, 1);
}

// ------------------------------------------------------------ product state
// psi_x = prod_i s_i[b_i(x)] as (low-site factor) x (high-site factor): the
// low T sites come from a shared table; each warp owns chunks of 2^T
// consecutive amplitudes and forms the chunk's high-site factor with a
// shuffle butterfly (lane s holds the factor of high site s), so every
// amplitude costs one complex multiply and the pass runs at write bandwidth.
// Factors are formed in FP64 and rounded once to R.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_product_state(typename CT<R>::C* __restrict__ psi,
                                                            int L,
                                                            const double* __restrict__ sp) {
  using C = typename CT<R>::C;
  constexpr int T = 10;
  __shared__ C tab[1 << T];
  const int t = L < T ? L : T;
  for (int j = threadIdx.x; j < (1 << t); j += blockDim.x) {
    double re = 1.0, im = 0.0;
    for (int s = 0; s < t; ++s) {
      const int b = (j >> s) & 1;
      const double sr = sp[4 * s + 2 * b], si = sp[4 * s + 2 * b + 1];
      const double nr = re * sr - im * si;
      im = re * si + im * sr;
      re = nr;
    }
    C v;
    v.x = (R)re;
    v.y = (R)im;
    tab[j] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  const int nh = L - t;  // high sites, at most 24
  const uint64_t nchunks = 1ull << nh;
  const uint32_t csize = 1u << t;
  for (uint64_t ch = (uint64_t)blockIdx.x * warps + warp; ch < nchunks;
       ch += (uint64_t)gridDim.x * warps) {
    double fr = 1.0, fi = 0.0;
    if (lane < nh) {
      const int b = (int)((ch >> lane) & 1);
      fr = sp[4 * (t + lane) + 2 * b];
      fi = sp[4 * (t + lane) + 2 * b + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double gr = __shfl_xor_sync(0xffffffffu, fr, o);
      const double gi = __shfl_xor_sync(0xffffffffu, fi, o);
      const double nr = fr * gr - fi * gi;
      fi = fr * gi + fi * gr;
      fr = nr;
    }
    const R hr = (R)fr, hi = (R)fi;
    C* __restrict__ out = psi + ch * csize;
    for (uint32_t j = lane; j < csize; j += 32) {
      const C lo = tab[j];
      C v;
      v.x = hr * lo.x - hi * lo.y;
      v.y = hr * lo.y + hi * lo.x;
      out[j] = v;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_scale(typename CT<R>::C* __restrict__ psi,
                                                    int L, const double* __restrict__ ring,
                                                    int ring_len,
                                                    const long long* __restrict__ counter) {
  using C = typename CT<R>::C;
  const long long c = *counter;
  const long long slot = ((c - 1) % ring_len + ring_len) % ring_len;
  const double n2 = ring[2 * slot + 1];
  const R s = (R)(n2 > 0.0 ? 1.0 / sqrt(n2) : 1.0);
  const uint64_t n = 1ull << L;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    C v = psi[x];
    v.x *= s;
    v.y *= s;
    psi[x] = v;
  }
}

// Double-float amplitudes to and from complex128 (state read-out and
// write-in of SV_DF64; off the evolution path).  to_c128: hi + lo, exact in
// FP64.  from_c128: hi = the nearest float, lo = the nearest float to the
// remainder (relative error at most 2^-48).
__global__ void __launch_bounds__(kThreads) k_df_to_c128(const dfc* __restrict__ src,
                                                         double2* __restrict__ dst, uint64_t n) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const dfc v = src[x];
    dst[x] = make_double2((double)v.x, (double)v.y);
  }
}
__global__ void __launch_bounds__(kThreads) k_c128_to_df(const double2* __restrict__ src,
                                                         dfc* __restrict__ dst, uint64_t n) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const double2 v = src[x];
    dfc o;
    o.x = df(v.x);
    o.y = df(v.y);
    dst[x] = o;
  }
}

template <typename R>
int gate_grid(int L, int bond, const LaunchCfg& cfg) {
  constexpr int LV = CT<R>::LV;
  const int gmax = cfg.num_sms * kBlocksPerSM;
  uint64_t work;  // thread-sized work units
  if (L < LV + 7) {
    work = 1ull << (L - 2);
  } else if (bond + 1 < LV + 7 && bond < LV + 5) {
    work = (1ull << (L - (LV + 7))) * 32;  // warps x 32
  } else {
    work = ((1ull << (L - 2 - LV)) + 1) / 2;
  }
  uint64_t blocks = (work + kThreads - 1) / kThreads;
  if (blocks > (uint64_t)gmax) blocks = gmax;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

template <typename R>
cudaError_t launch_gate_t(void* psi_, int L, int bond, const void* gate_base,
                          long long stride, const long long* counter,
                          const EpiParams& ep, int store, const LaunchCfg& cfg,
                          cudaStream_t s) {
  using C = typename CT<R>::C;
  constexpr int LV = CT<R>::LV;
  C* psi = static_cast<C*>(psi_);
  const C* g = static_cast<const C*>(gate_base);
  const int grid = gate_grid<R>(L, bond, cfg);
  if (L < LV + 7) {
    k_gate_small<R><<<grid, kThreads, 0, s>>>(psi, L, bond, g, stride, counter, ep, store);
  } else if (bond < LV + 5) {
    switch (bond) {
#define FSV_LOW_CASE(I)                                                                 \
  case I:                                                                               \
    k_gate_low<R, I><<<grid, kThreads, 0, s>>>(psi, L, g, stride, counter, ep, store); \
    break;
      FSV_LOW_CASE(0)
      FSV_LOW_CASE(1)
      FSV_LOW_CASE(2)
      FSV_LOW_CASE(3)
      FSV_LOW_CASE(4)
      FSV_LOW_CASE(5)
#undef FSV_LOW_CASE
      default:
        return cudaErrorInvalidValue;
    }
  } else {
    k_gate_high<R><<<grid, kThreads, 0, s>>>(psi, L, bond, g, stride, counter, ep, store);
  }
  return cudaGetLastError();
}

}  // namespace

int plain_gate_grid(int L, int bond, int precision, const LaunchCfg& cfg) {
  if (precision == SV_C128) return gate_grid<double>(L, bond, cfg);
  if (precision == SV_DF64) return gate_grid<df>(L, bond, cfg);
  return gate_grid<float>(L, bond, cfg);
}

cudaError_t launch_plain_gate(int precision, void* psi, int L, int bond,
                              const void* gate_base, long long period_stride,
                              const long long* counter, const EpiParams& ep, int store,
                              const LaunchCfg& cfg, cudaStream_t s) {
  if (precision == SV_C128)
    return launch_gate_t<double>(psi, L, bond, gate_base, period_stride, counter, ep,
                                 store, cfg, s);
  if (precision == SV_DF64)
    return launch_gate_t<df>(psi, L, bond, gate_base, period_stride, counter, ep, store, cfg,
                             s);
  return launch_gate_t<float>(psi, L, bond, gate_base, period_stride, counter, ep, store,
                              cfg, s);
}

cudaError_t launch_period_reduce(const double* partials, long long n, int L, double* ring,
                                 int ring_len, long long* counter, int advance,
                                 cudaStream_t s) {
  k_period_reduce<<<1, 256, 0, s>>>(partials, n, L, ring, ring_len, counter, advance);
  return cudaGetLastError();
}

cudaError_t launch_period_reduce_many(const ReduceItem* items, int count, cudaStream_t s) {
  k_period_reduce_many<<<count, 256, 0, s>>>(items);
  return cudaGetLastError();
}

cudaError_t launch_product_state(int precision, void* psi, int L, const double* spinors,
                                 const LaunchCfg& cfg, cudaStream_t s) {
  const int grid = cfg.num_sms * kBlocksPerSM;
  if (precision == SV_C128)
    k_product_state<double><<<grid, kThreads, 0, s>>>(static_cast<double2*>(psi), L, spinors);
  else if (precision == SV_DF64)
    k_product_state<df><<<grid, kThreads, 0, s>>>(static_cast<dfc*>(psi), L, spinors);
  else
    k_product_state<float><<<grid, kThreads, 0, s>>>(static_cast<float2*>(psi), L, spinors);
  return cudaGetLastError();
}

cudaError_t launch_renormalize(int precision, void* psi, int L, const double* ring,
                               int ring_len, const long long* counter,
                               const LaunchCfg& cfg, cudaStream_t s) {
  const int grid = cfg.num_sms * kBlocksPerSM;
  if (precision == SV_C128)
    k_scale<double><<<grid, kThreads, 0, s>>>(static_cast<double2*>(psi), L, ring, ring_len,
                                              counter);
  else if (precision == SV_DF64)
    k_scale<df><<<grid, kThreads, 0, s>>>(static_cast<dfc*>(psi), L, ring, ring_len, counter);
  else
    k_scale<float><<<grid, kThreads, 0, s>>>(static_cast<float2*>(psi), L, ring, ring_len,
                                             counter);
  return cudaGetLastError();
}

cudaError_t launch_df_convert(const void* src, void* dst, uint64_t n, int to_c128,
                              const LaunchCfg& cfg, cudaStream_t s) {
  const int grid = cfg.num_sms * kBlocksPerSM;
  if (to_c128)
    k_df_to_c128<<<grid, kThreads, 0, s>>>(static_cast<const dfc*>(src),
                                           static_cast<double2*>(dst), n);
  else
    k_c128_to_df<<<grid, kThreads, 0, s>>>(static_cast<const double2*>(src),
                                           static_cast<dfc*>(dst), n);
  return cudaGetLastError();
}

}  // namespace fsv
