// Tensor-core block pass (tcgen05 + TMA): not yet enabled in this build.
#include "sv_block.h"

namespace fsv {

bool block_tc_supported(int L, int n) {
  (void)L;
  (void)n;
  return false;
}

size_t block_tc_w_bytes(int n) {
  (void)n;
  return 0;
}

void block_tc_pack_w(int n, const std::vector<cd>& U, std::vector<uint32_t>& out) {
  (void)n;
  (void)U;
  out.clear();
}

cudaError_t launch_block_tc(const PassArgs& pa, void* psi, int grid, cudaStream_t s) {
  (void)pa;
  (void)psi;
  (void)grid;
  (void)s;
  return cudaErrorNotSupported;
}

}  // namespace fsv
