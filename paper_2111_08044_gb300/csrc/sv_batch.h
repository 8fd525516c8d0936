// Batched evolution of many independent chains (internal).  Not public.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "sv_internal.h"
#include "sv_kernels.h"

namespace fsv {

// One chain of the resident form (L <= 14): state, its period's folded
// gates (float2, 16 per gate, local index r = 2 b_bond + b_{bond+1}), the
// bond of each gate, the observable's coefficients, and its energy ring of
// (E / (L n), n) pairs.
struct ResidentChain {
  float2* psi = nullptr;
  const float2* gates = nullptr;
  const int* bonds = nullptr;
  double* ring = nullptr;
  int L = 0;
  int ngates = 0;
  double J = 0.0;
  double cx[14] = {};
  double cz[14] = {};
};

constexpr int kResidentMaxL = 14;

size_t resident_smem_bytes(int L);
cudaError_t resident_prepare(int max_L);
// `periods` periods of every chain in chains[0 .. nchains): energies go to
// ring slot (counter + p) mod ring_len; then *counter += periods.
cudaError_t launch_chain_resident(const ResidentChain* chains, int nchains, int max_L,
                                  long long* counter, int periods, int ring_len,
                                  cudaStream_t s);

// FP32 copy of a 4x4 unitary, rounded with a one-ulp search that keeps it
// unitary to FP32 resolution (sv_api.cu).
void round_unitary4(const cd* m, float2* out);

}  // namespace fsv
