// Block form: fused n-site unitaries applied one pass per block, with the
// qubit relabelling folded into each pass's write.  Not public.
//
// State layout during a period.  While the window [lo, lo+n) is active,
// site s sits at bit position
//     s - lo   for lo <= s < lo + n   (the window on the lowest n bits),
//     n + s    for s < lo,
//     s        for s >= lo + n,
// so a window at lo = 0 is the natural layout (site i = bit i).  Moving the
// window from lo to lo' changes only positions 0..n-1 and the |lo'-lo|
// positions starting at n + min(lo, lo'); a pass therefore reads a tile of
// 2^(n+R) amplitudes (n window bits plus R <= 7 contiguous row bits starting
// at position a that cover the moved positions), multiplies each row of 2^n
// amplitudes by the fused unitary, and writes the tile back permuted into
// the next window's layout.  Every tile is read and written by one CTA, so
// the pass is in place.  Each period starts and ends in the natural layout.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "sv_internal.h"
#include "sv_kernels.h"

namespace fsv {

struct PassArgs {
  int L = 0, n = 0, R = 0, a = 0;
  int lo = 0;
  long long ntiles = 0;
  uint32_t x_mask = 0;       // window-local bits whose <X> this pass measures
  float cx[8] = {};          // coefficient per window-local bit
  int diag = 0;              // measure diagonal part + norm (output is natural layout)
  float diag_f[5] = {};      // J, cz bulk / first / last, sum of cz: ep's FP64 values in FP32
  // diagonal pass, window bit j (output site s_j): lin0[j] = -2 (cz(s_j) + J
  // * number of neighbours of s_j that are window sites, whose bit is 0 at
  // c = 0); nb[j][k]: the other neighbours' sites (-1: none)
  float diag_lin0[8] = {};
  int8_t diag_nb[8][2] = {};
  int diag_lo = 0;           // window position of the output's layout (0: natural)
  int8_t sigma[16] = {};     // output tile bit of input tile bit q
  // tensor-core pass: TMEM lane m holds tile row XOR over set bits i of m
  // of rowvec[i] (an invertible map, chosen against staging bank conflicts)
  uint8_t rowvec[7] = {1, 2, 4, 8, 16, 32, 64};
  // staging order: output tile bit o sits at bit spos[o] of the staging tile
  // (bits 0-3 fixed: one 128-byte line of the store); the store view's
  // tile-index coordinates go to dims st_tlo_dim / st_thi_dim (0: none),
  // shifted by those dims' box bits; st_ndims = 3 for the natural order
  int8_t spos[13] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12};
  int8_t ssig[13] = {};  // spos[sigma[k]]: staging bit of window / row bit k
  int8_t st_ndims = 3, st_tlo_dim = 1, st_tlo_shift = 2, st_thi_dim = 2, st_thi_shift = 7;
  const float2* U = nullptr; // fused unitary, FP32, row-major 2^n x 2^n
  // per output row j: FP32 residual of its largest entry and that entry's
  // column (re, im, column, 0); the CUDA-core pass starts row j's sum there
  const float4* Ulead = nullptr;
  const void* W = nullptr;   // tensor-core operand block of this pass
  void* psi = nullptr;       // state (set at launch)
  double* partial = nullptr; // per-CTA (energy, norm) pairs or nullptr
  int slot = -1;             // partials slot (host bookkeeping)
  EpiParams ep;              // diagonal coefficients
};

// Per chain and pass of a chain group (chains whose plans share every
// structural field: same L, windows, relabels and staging; they differ in
// operands and measured coefficients).  The group's tensor-core pass runs
// all chains' tiles in one launch.
struct alignas(64) GroupChain {
  unsigned char map_in[128];   // TMA descriptors (CUtensorMap) for this
  unsigned char map_out[128];  // chain's state
  const void* W = nullptr;     // the chain's operand block of this pass
  double* partial = nullptr;   // the chain's (energy, norm) pairs, or null
  float cx[8] = {};
  float diag_f[5] = {};
  float diag_lin0[8] = {};
};
static_assert(sizeof(GroupChain) % 64 == 0, "descriptors stay 64-byte aligned in an array");

struct BlockPlan {
  int L = 0, n = 0, R = 0, split = 0;
  int start = 0;  // window of the period's first pass; the layout between periods
  // launch sequences (indices into args): a period, the last period of an
  // evolution (its last pass writes the natural layout), and the relabel
  // steps from the natural layout to the start that begin an evolution
  std::vector<int> seq_cyc, seq_exit, seq_entry;
  // relabel steps from the period layout back to the natural one (identity)
  std::vector<int> seq_leave;
  bool tensor_cores = false;
  std::vector<BlockPass> passes;
  std::vector<PassArgs> args;
  float2* d_U = nullptr;
  float4* d_Ulead = nullptr;
  void* d_W = nullptr;
  size_t w_bytes_per_pass = 0;
  double* d_partials = nullptr;
  int nslots = 0;
  int maxb = 0;
  int grid = 0;
  LaunchCfg cfg;
  // tensor-core pass: one TMA descriptor per pass for the attached state
  std::vector<uint8_t> maps;   // passes x block_tc_map_bytes()
  void* maps_psi = nullptr;    // state pointer the descriptors were built for
  int* d_status = nullptr;     // raised by a pass whose bounded wait gave up
};

// Tile of the pass moving the window from lo to lo_next: its row bits start
// at position *a_out, and input tile bit q (window bits 0..n-1, then R row
// bits) goes to output tile bit sigma[q].  Empty on success, else the reason.
std::string block_tile_layout(int L, int n, int R, int lo, int lo_next, int* a_out,
                              int8_t* sigma);
int block_build(int L, const std::vector<Gate2>& gates, const Observable& obs, int n,
                int split, const LaunchCfg& cfg, bool cyclic, BlockPlan** out,
                std::string* msg);
void block_info(const BlockPlan* bp, int* passes, int* launches);
// Fold the periodic renormalisation into the period's first pass.
void block_set_renorm(BlockPlan* bp, const Renorm& rn);
size_t block_upload_bytes(const BlockPlan* bp);
// The relabel steps that begin an evolution (none when the start is 0).
cudaError_t block_enqueue_entry(BlockPlan* bp, void* psi, cudaStream_t s);
// The relabel steps from the period layout back to the natural one.
cudaError_t block_enqueue_leave(BlockPlan* bp, void* psi, cudaStream_t s);
// One period; `last`: the evolution's last period, which hands back the
// natural layout.
cudaError_t block_enqueue_period(BlockPlan* bp, void* psi, long long* counter, double* ring,
                                 int ring_len, cudaStream_t s, bool last);
// As block_enqueue_period with ev[k] recorded before pass k and
// ev[passes + 1] after the final reduce.
cudaError_t block_enqueue_period_events(BlockPlan* bp, void* psi, long long* counter,
                                        double* ring, int ring_len, cudaStream_t s,
                                        cudaEvent_t* ev, bool last);
void block_free(BlockPlan* bp);

// Chain groups: tensor-core chains whose plans share every structural field
// (same L, windows, relabels, staging orders and measured passes) run each
// pass of all chains as one launch, and their period reduces as one.
struct GroupMember {
  BlockPlan* plan = nullptr;
  void* psi = nullptr;           // the chain's state
  long long* counter = nullptr;  // its period counter and energy ring
  double* ring = nullptr;
};
struct BlockGroup;
bool block_same_structure(const BlockPlan* a, const BlockPlan* b);
// Descriptors, operands and coefficients of every chain and pass, and the
// group's own partial sums ([chains][slots][grid] pairs, zeroed: only CTAs
// that meet a chain write its pairs).
int block_group_build(const std::vector<GroupMember>& members, int ring_len,
                      const LaunchCfg& cfg, cudaStream_t s, BlockGroup** out, std::string* msg);
// Window of the group's periods (0: the natural layout, no entry steps).
int block_group_start(const BlockGroup* g);
// Chains in the group.
size_t block_group_size(const BlockGroup* g);
cudaError_t block_group_enqueue_entry(BlockGroup* g, cudaStream_t s);
cudaError_t block_group_enqueue_period(BlockGroup* g, cudaStream_t s, bool last);
void block_group_free(BlockGroup* g);

// Nonzero if a tensor-core pass reported a timed-out wait (synchronises s).
int block_status(BlockPlan* bp, cudaStream_t s);

// CUDA-core FP32 pass (any n, R); tensor-core pass (n = 6, R = 7).
cudaError_t launch_block_simt(const PassArgs& pa, void* psi, int grid, cudaStream_t s);
cudaError_t launch_block_tc(const PassArgs& pa, void* psi, const void* map, int* status,
                            int grid, cudaStream_t s);
// One tensor-core pass over the tiles of a chain group: pa is the pass's
// structure with ntiles = chains x 2^nt_log2; chains: device array, one per
// chain.  CTA b takes the contiguous tiles [b T / grid, (b + 1) T / grid).
cudaError_t launch_block_tc_group(const PassArgs& pa, const GroupChain* chains, int nt_log2,
                                  int* status, int grid, cudaStream_t s);
bool block_tc_supported(int L, int n);
cudaError_t block_tc_prepare();
size_t block_tc_map_bytes();
int block_tc_make_map(const PassArgs& pa, void* psi, void* map_out);
// Bytes of the tensor-core operand block of one pass, and its host layout.
size_t block_tc_w_bytes(int n);
// Row map of a tensor-core pass (n = 6, R = 7) for its relabel sigma: keeps
// the converters' 128-byte-swizzled row reads conflict-free and spreads each
// epilogue warp's staging stores over as many banks as sigma allows.
// Returns the staging wavefronts per warp store (2 is conflict-free) for the
// staging order spos.
int block_tc_row_map(const int8_t* sigma, const int8_t* spos, uint8_t* rowvec);
// Row map and staging order of a tensor-core pass: the natural staging
// order unless it leaves a store at 16 wavefronts, in which case the
// output bits placed at staging bits 4-6 (those the 128-byte swizzle folds
// into the bank bits) are chosen against the conflicts, with the store view
// rebuilt from the runs of consecutive state bits.  Fills rowvec, spos and
// st_*; returns the staging wavefronts per warp store.
int block_tc_layout(PassArgs& pa);
// The store view of a tensor-core pass (after block_tc_layout): dimension 0
// is 16 amplitudes, then one dimension per run of the staging order; dims,
// byte strides of dimensions 1.. and box extents.  Returns the rank (3-5),
// -1 if the staging order needs more dimensions than a tensor map has.
int block_tc_store_view(const PassArgs& pa, uint64_t* dims, uint64_t* strides, uint32_t* box);
void block_tc_pack_w(int n, const std::vector<cd>& U, std::vector<uint32_t>& out);

// Representable copies of a dim x dim unitary, as close to unitary as the
// format allows (host_round.cpp): each real entry takes one of the two
// values bracketing it, chosen by a coordinate descent on
// ||Ur^H Ur - I||_F^2 + tr(Ur^H Ur - I)^2 from nearest rounding.
//   FP32 entries (CUDA-core pass).  With lead != NULL, each row j's largest
//   entry is stored to nearest and applied together with its FP32 residual
//   lead[j] = (re, im, column, 0), so it counts as exact in the descent:
void round_unitary_fp32(int dim, const cd* U, float2* out, float4* lead);
//   tensor-core digits u = 2^-7 (u0 + u1/256 + u2/65536), u0 an integer and
//   u1, u2 with 8 significant bits (u2 the chosen one): digits[3 (2 e + p) + t]
//   is digit t of entry e's real (p = 0) or imaginary (p = 1) part.
void round_unitary_digits(int dim, const cd* U, double* digits);
// Run job(0..count-1) on up to 16 host threads.
void round_passes_parallel(int count, const std::function<void(int)>& job);

}  // namespace fsv
