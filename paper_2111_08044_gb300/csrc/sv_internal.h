// Internal declarations shared by the host builders, the C ABI and the
// kernel launchers.  Not part of the public interface.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/floquet_sv.h"

namespace fsv {

using cd = std::complex<double>;

// Epilogue flags of a plain gate pass: which energy terms it measures once
// its gate is applied (the gate is the last one of the period on that site,
// or the last gate of the period).
enum : int { EPI_X_HI = 1, EPI_X_LO = 2, EPI_DIAG = 4 };

}  // namespace fsv

struct sv_ctx;

namespace fsv {

// Batch-executor hooks into a context (sv_api.cu).
// A run of `periods` periods captured as one graph template (the caller
// destroys it): for a block plan whose periods start off site 0, the
// relabel into the period layout, the periods, and the last period's
// hand-back to the natural layout.
int ctx_capture_run(sv_ctx* ctx, int64_t periods, cudaGraph_t* out);
// Account for periods run through such graphs on the host mirror.
void ctx_advance(sv_ctx* ctx, int64_t periods);
// Block passes of later builds keep at least `tiles` tiles per CTA.
void ctx_set_min_tiles(sv_ctx* ctx, int tiles);
// Whether later block builds may start their periods off site 0 (the batch
// replays captured periods back to back and needs the natural layout).
void ctx_set_cyclic(sv_ctx* ctx, bool cyclic);
// (energy density, norm) of periods c0 .. c0+count-1 from the energy ring.
int ctx_read_energies(sv_ctx* ctx, int64_t c0, int64_t count, double* e, double* n);
// Periods the energy ring holds.
int ctx_ring_len();
struct BlockPlan;
// The tensor-core block plan of a context and the device objects its
// periods update (state, period counter, energy ring); SV_ESTATE when the
// context has no such plan.
int ctx_block_member(sv_ctx* ctx, BlockPlan** plan, void** psi, long long** counter,
                     double** ring);

struct Gate2 {
  int bond = 0;      // acts on sites (bond, bond + 1)
  cd m[16];          // row-major, local index r = 2 b_bond + b_{bond+1}
  int epi = 0;       // EPI_* flags
};

// Coefficients of the observable H0 = sum_b h_b written as
//   H0 = sum_i cx[i] X_i + sum_i cz[i] Z_i + J sum_b Z_b Z_{b+1}.
struct Observable {
  int L = 0;
  double J = 0.0;
  std::vector<double> cx, cz;
  // general two-site chain: H0 = sum_b h[b] (16 complex each); the Ising
  // fields above are then unused
  bool general = false;
  std::vector<cd> h;
};

// a1: bond Hamiltonian h_b (4x4, r = 2 b_i + b_{i+1}) of the driven chain
// at field hx (the per-period drive may differ from the observable's).
void bond_hamiltonian(int L, int b, double J, double hx, double hz, double ew,
                      cd h[16]);
// exp(-i tau h) of a 4x4 Hermitian matrix in FP64 (real-symmetric Jacobi
// diagonalisation of its 8x8 real embedding).
void expm_herm4(const cd h[16], double tau, cd g[16]);
// Frechet derivative of exp(-i tau h) in direction dh (Daleckii-Krein
// divided differences in the eigenbasis).
void expm_herm4_frechet(const cd h[16], const cd dh[16], double tau, cd g[16],
                        cd d[16]);
// kick exp(-i theta X)
void kick_matrix(double theta, cd r[4]);

// One operation of the adjoint sweep: a two-site operator O on bond
// (bond, bond+1), with O^dagger and D = (dO/dalpha) O^dagger for the
// parameter alpha it depends on (kind 0: the kick angle theta_p, kind 1:
// the drive field hx_p).
struct AdjOp {
  int bond = 0;
  int kind = 0;
  cd odag[16];
  cd d[16];
};
// The operations of one period in the reverse of their order of
// application: the kick (on site pairs (0,1), (2,3), ..., and site L-1
// alone for odd L), then the gate layers from last to first.
std::vector<AdjOp> adjoint_period_ops(int L, const sv_floquet_params &p, double theta,
                                      double hx);
// a1 + a2: the period's gates in application order with the kick folded
// into the last gate on each site and epilogue flags set.
std::vector<Gate2> period_gates(int L, const sv_floquet_params &p, double theta,
                                double hx);
Observable observable(int L, const sv_floquet_params &p);
// Share of the on-site fields (h_x, h_z) that site i carries in H0 = sum_b h_b:
// 1/2 from each bond it belongs to, edge_field_weight from an open end's
// single bond.  Allocates nothing.
double site_field_share(int L, int i, double ew);
bool params_valid(int L, const sv_floquet_params &p, std::string *why);

// Checkpoint files (host_checkpoint.cpp): header and payload checksum.
constexpr size_t kCkptHeaderBytes = 48;
struct CkptHeader {
  int L = 0;
  int precision = 0;
  int64_t period = 0;
  uint64_t payload_bytes = 0;
  uint64_t payload_sum = 0;
};
uint64_t ckpt_sum_begin();
// FNV-1a over little-endian 64-bit words (bytes: a multiple of 8).
uint64_t ckpt_sum_update(uint64_t h, const void* data, size_t bytes);
void ckpt_encode_header(const CkptHeader& h, unsigned char out[kCkptHeaderBytes]);
// Magic, header checksum and field ranges; false if any fails.
bool ckpt_decode_header(const unsigned char in[kCkptHeaderBytes], CkptHeader* h);

// a3: fusion of one period into n-site block passes (host, FP64).
struct BlockPass {
  int lo = 0;                 // window = sites lo .. lo+n-1, local bit j = site lo+j
  int n = 0;
  std::vector<int> gates;     // indices into the period's gate list, in order
  std::vector<cd> U;          // 2^n x 2^n, row-major
  std::vector<int> x_sites;   // sites whose <X> this pass measures
  bool diag = false;          // this pass measures the diagonal terms and norm
};
// The multi-gate form's passes: each applies, gate by gate, every pending
// gate of the period inside its window of w sites (the natural layout is
// kept, so windows move freely); x_sites and diag as for BlockPass.
struct MultiPass {
  int lo = 0;
  std::vector<int> gates;     // indices into the period's gate list, in order
  std::vector<int> x_sites;
  bool diag = false;
};
std::vector<MultiPass> multigate_plan(int L, const std::vector<Gate2> &gates, int w);

// cyclic: the period may start (and end) at the window s <= 7 that needs the
// fewest passes instead of at site 0 (passes[0].lo is the start).
std::vector<BlockPass> fusion_plan(int L, const std::vector<Gate2> &gates, int n,
                                   bool cyclic = false);

}  // namespace fsv
