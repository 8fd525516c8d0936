// Launch interface of the device kernels (host side).  Not public.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace fsv {

// Renormalisation folded into the first pass of a period: when the period
// counter c > 0 is a multiple of `every`, the pass scales what it writes by
// 1/sqrt(norm of period c-1), read from the energy ring.
struct Renorm {
  const double* ring = nullptr;
  int ring_len = 0;
  const long long* counter = nullptr;
  int every = 0;
};

// Energy terms measured by a plain gate pass, in the layout of the state
// pass that applies the gate (site i = bit i).
struct EpiParams {
  int flags = 0;           // EPI_* (sv_internal.h)
  double cx_hi = 0.0;      // coefficient of <X_i>     (site i = bond)
  double cx_lo = 0.0;      // coefficient of <X_{i+1}>
  double J = 0.0;          // ZZ coupling of every bond
  double cz_bulk = 0.0;    // Z coefficient of an interior site
  double cz_first = 0.0;   // Z coefficient of site 0
  double cz_last = 0.0;    // Z coefficient of site L-1
  double* partial = nullptr;  // [gridDim.x][2] (energy, norm) of this launch
  Renorm rn;                  // set on the first pass of a period only
};

// A gate table entry: 16 complex of the gate (row-major, local index
// r = 2 b_bond + b_{bond+1}) followed by 16 complex of its rounding
// residual (zero for FP64 tables), so that FP32 passes apply the FP64 gate
// to within 2^-48 instead of its FP32 rounding.
constexpr int kGateEntries = 32;
template <typename R>
constexpr bool kGateLo = sizeof(R) == 4;

// Multi-gate pass (k_multigate.cu): a tile of 2^tb amplitudes, state bits
// 0-3 and A..A+tb-5, in shared memory; the pass's gates applied one after
// another on adjacent tile bits.
constexpr int kMgTileBits = 13;
constexpr int kMgWindow = kMgTileBits - 4;  // sites a pass's window spans (L > 13)
constexpr int kMgMaxX = 16;
struct MultiArgs {
  int L = 0, tb = 0, A = 4;
  int ngates = 0;
  const int* gidx = nullptr;      // device: the pass's gates (indices into the period's list)
  const int* gq = nullptr;        // device: tile bit of each gate's first site
  const float2* gates = nullptr;  // gate tables, kGateEntries complex per gate
  long long stride = 0;           // per-period table stride (0: one table)
  const long long* counter = nullptr;
  int nx = 0;                     // sites whose <X> this pass measures
  int xq[kMgMaxX] = {};           // their tile bits
  float xc[kMgMaxX] = {};         // their coefficients
  int diag = 0;                   // the period's last pass: diagonal part and norm
  EpiParams ep;                   // diagonal coefficients, renormalisation, partials
};

struct LaunchCfg {
  int num_sms = 148;
  // at least this many tiles per CTA in block passes (0: one wave over the
  // SMs); batches set it so that several chains' passes share the device
  int min_tiles_per_cta = 0;
};

// Grid (blocks of 256 threads) used by the plain gate pass for this L and
// bond; it is also the number of partial pairs the pass writes.
int plain_gate_grid(int L, int bond, int precision, const LaunchCfg& cfg);
// Multi-gate pass: grid (it is also the number of partial pairs a pass writes),
// shared-memory opt-in (at build time, outside any capture) and launch.
int multigate_grid(int L, const LaunchCfg& cfg);
cudaError_t multigate_prepare();
cudaError_t launch_multigate(const MultiArgs& ma, void* psi, const LaunchCfg& cfg,
                             cudaStream_t s);

// Apply one 4x4 gate on bond `bond` in place (store = 1) or only measure
// (store = 0).  gate: 16 complex (float2 for C64, double2 for C128) at
// gate_base + (*counter) * period_stride (period_stride 0: fixed gate).
cudaError_t launch_plain_gate(int precision, void* psi, int L, int bond,
                              const void* gate_base, long long period_stride,
                              const long long* counter, const EpiParams& ep,
                              int store, const LaunchCfg& cfg, cudaStream_t s);

// Sum `n` (energy, norm) partial pairs in a fixed order and record
// (energy / (L norm), norm) at ring[(*counter) % ring_len], then ++*counter
// (advance != 0).
// One chain's period reduce: its partial pairs, ring and period counter.
struct ReduceItem {
  const double* partials = nullptr;
  long long n = 0;
  double* ring = nullptr;
  long long* counter = nullptr;
  int L = 0;
  int ring_len = 0;
};
// The period reduce of `count` chains (items: device array), counters advanced.
cudaError_t launch_period_reduce_many(const ReduceItem* items, int count, cudaStream_t s);
cudaError_t launch_period_reduce(const double* partials, long long n, int L,
                                 double* ring, int ring_len, long long* counter,
                                 int advance, cudaStream_t s);

// psi_x = prod_i s_i[b_i(x)]; spinors: device, 4*L doubles (normalised).
cudaError_t launch_product_state(int precision, void* psi, int L,
                                 const double* spinors, const LaunchCfg& cfg,
                                 cudaStream_t s);

// psi *= 1/sqrt(norm2), norm2 read from ring[((*counter) - 1) % ring_len].
cudaError_t launch_renormalize(int precision, void* psi, int L, const double* ring,
                               int ring_len, const long long* counter,
                               const LaunchCfg& cfg, cudaStream_t s);
// SV_DF64 state <-> complex128 (n amplitudes; to_c128: src double-float,
// dst complex128; else the reverse)
cudaError_t launch_df_convert(const void* src, void* dst, uint64_t n, int to_c128,
                              const LaunchCfg& cfg, cudaStream_t s);

// Coefficients of H0 = J sum_b Z_b Z_{b+1} + sum_i cx[i] X_i + sum_i cz[i] Z_i
// (L <= 34), passed by value to the adjoint seed kernel.
struct H0Coef {
  double J = 0.0;
  double cx[34] = {};
  double cz[34] = {};
};

// Blocks of the adjoint kernels (also the number of partials each writes).
int adjoint_grid(const LaunchCfg& cfg);
// Energy moments (3 partials a block: Re <psi|H0 psi>, |H0 psi|^2, |psi|^2)
// and the overlap <phi|psi> with a product state phi_x = lo[x mod 2^m]
// hi[x >> m] (2 partials a block); moments_grid blocks each.
int moments_grid(const LaunchCfg& cfg);
cudaError_t launch_h0_moments(int precision, const void* psi, int L, const H0Coef& h,
                              double* partial, const LaunchCfg& cfg, cudaStream_t s);
// General two-site chain: hb = (L-1) x 16 complex bond terms on the device
// (float2 for C64, double2 for C128); same partials as launch_h0_moments.
cudaError_t launch_bond_moments(int precision, const void* psi, int L, const void* hb,
                                double* partial, const LaunchCfg& cfg, cudaStream_t s);
// psi_x = lo[x mod 2^m] hi[x >> m] (lo, hi: FP64 complex tables on the device).
cudaError_t launch_factor_state(int precision, void* psi, int L, int m, const void* lo,
                                const void* hi, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_product_overlap(int precision, const void* psi, int L, int m,
                                   const void* lo, const void* hi, double* partial,
                                   const LaunchCfg& cfg, cudaStream_t s);

// lambda = (H0 / L) psi; partial[block] = that block's share of
// Re <psi|lambda>.
cudaError_t launch_apply_h0(int precision, const void* psi, void* lam, int L, const H0Coef& h,
                            double* partial, const LaunchCfg& cfg, cudaStream_t s);

// One reverse step on bond (bond, bond+1): partial[block] = that block's
// share of Re <lambda|D|psi>, then psi <- odag psi, lambda <- odag lambda.
// odag, dmat: 16 complex (float2 for C64, double2 for C128) on the device.
cudaError_t launch_adjoint_gate(int precision, void* psi, void* lam, int L, int bond,
                                const void* odag, const void* dmat, double* partial,
                                const LaunchCfg& cfg, cudaStream_t s);

// out[0] = sum of partials[0..n) (times 2 when times_two), fixed order.
cudaError_t launch_grad_reduce(const double* partials, long long n, double* out, int times_two,
                               cudaStream_t s);

}  // namespace fsv
