// Block form: host construction of the pass descriptors and the CUDA-core
// FP32 block pass.  The CUDA-core pass applies any window width n <= 7 and
// any tile height; it serves chains too short for 128-row tensor-core tiles
// and is the reference form the tensor-core pass is checked against.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "sv_block.h"
#include "sv_device.cuh"

namespace fsv {

namespace {

using namespace dev;

constexpr int kSimtThreads = 512;

// position of site s while the window starts at lo (see sv_block.h)
int pos_of(int L, int n, int lo, int s) {
  (void)L;
  if (s >= lo && s < lo + n) return s - lo;
  if (s < lo) return n + s;
  return s;
}

// site held at position p while the window starts at lo
int site_at(int L, int n, int lo, int p) {
  (void)L;
  if (p < n) return lo + p;
  if (p < n + lo) return p - n;
  return p;
}

template <int N>
__global__ void __launch_bounds__(kSimtThreads) k_block_simt(float2* __restrict__ psi,
                                                             PassArgs pa) {
  constexpr int D = 1 << N;
  constexpr int DP = D + 1;  // padded row stride (bank spread)
  constexpr int CH = D < 16 ? D : 16;
  extern __shared__ float2 tile[];
  const int R = pa.R, rows = 1 << R, a = pa.a, L = pa.L;
  const int nel = rows * D;
  const int nitems = rows * (D / CH);
  const int nbits = N + R;
  Diag<float> dg;
  if (pa.diag) dg.init(pa.ep, L);
  const float sc = (float)renorm_scale(pa.ep.rn);
  double eacc = 0.0, nacc = 0.0;
  for (long long t = blockIdx.x; t < pa.ntiles; t += gridDim.x) {
    const uint64_t tlo = (uint64_t)t & ((1ull << (a - N)) - 1);
    const uint64_t thi = (uint64_t)t >> (a - N);
    const uint64_t base = (tlo << N) | (thi << (a + R));
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      const int r = e >> N, c = e & (D - 1);
      tile[r * DP + c] = psi[base + ((uint64_t)r << a) + c];
    }
    __syncthreads();
    float2 acc[2][CH];
    int rr[2], cb[2];
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int item = threadIdx.x + it * blockDim.x;
      rr[it] = item % rows;
      cb[it] = item / rows;
      // each output starts from its row's largest entry's FP32 residual
      // times that entry's amplitude: a sum started from a bare product
      // with a fixed entry rounds with an error that correlates with the
      // result (for passes of few gates, with one dominant entry per row,
      // it biased the norm by 1e-8 per period); the residual term varies
      // independently of that rounding grid and takes the bias out
#pragma unroll
      for (int j = 0; j < CH; ++j) acc[it][j] = make_float2(0.f, 0.f);
      if (item < nitems) {
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const float4 ld = __ldg(&pa.Ulead[cb[it] * CH + j]);
          acc[it][j] = cmac(acc[it][j], make_float2(ld.x, ld.y), tile[rr[it] * DP + (int)ld.z]);
        }
        for (int k = 0; k < D; ++k) {
          const float2 v = tile[rr[it] * DP + k];
#pragma unroll
          for (int j = 0; j < CH; ++j)
            acc[it][j] = cmac(acc[it][j], __ldg(&pa.U[(cb[it] * CH + j) * D + k]), v);
        }
      }
    }
    __syncthreads();
    // write the result at its place in the next window's layout
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int item = threadIdx.x + it * blockDim.x;
      if (item >= nitems) continue;
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int y = (rr[it] << N) | (cb[it] * CH + j);
        int yo = 0;
        for (int q = 0; q < nbits; ++q) yo |= ((y >> q) & 1) << pa.sigma[q];
        tile[(yo >> N) * DP + (yo & (D - 1))] = make_float2(acc[it][j].x * sc, acc[it][j].y * sc);
      }
    }
    __syncthreads();
    float es = 0.f, ns = 0.f;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      const int r = e >> N, c = e & (D - 1);
      const float2 v = tile[r * DP + c];
      const uint64_t x = base + ((uint64_t)r << a) + c;
      psi[x] = v;
      if (pa.x_mask) {
        for (int j = 0; j < N; ++j)
          if ((pa.x_mask >> j) & 1) {
            const int yf = e ^ (1 << pa.sigma[j]);
            es += pa.cx[j] * cdotre(v, tile[(yf >> N) * DP + (yf & (D - 1))]);
          }
      }
      if (pa.diag) {
        const float p = cabs2(v);
        ns += p;
        es += p * dg(to_natural(x, N, pa.diag_lo));
      }
    }
    eacc += (double)es;
    nacc += (double)ns;
    __syncthreads();
  }
  if (pa.partial) block_store_pair(eacc, nacc, pa.partial);
}

template <int N>
cudaError_t prepare_simt_n() {
  return cudaFuncSetAttribute(k_block_simt<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(float2) * 128 * ((1 << N) + 1)));
}

template <int N>
cudaError_t launch_simt_n(const PassArgs& pa, void* psi, int grid, cudaStream_t s) {
  const size_t smem = sizeof(float2) * ((size_t)1 << pa.R) * ((1 << N) + 1);
  k_block_simt<N><<<grid, kSimtThreads, smem, s>>>(static_cast<float2*>(psi), pa);
  return cudaGetLastError();
}

// Opt the CUDA-core pass for width n into its shared-memory size (called at
// build time, outside any stream capture).
cudaError_t prepare_simt(int n) {
  switch (n) {
    case 2: return prepare_simt_n<2>();
    case 3: return prepare_simt_n<3>();
    case 4: return prepare_simt_n<4>();
    case 5: return prepare_simt_n<5>();
    case 6: return prepare_simt_n<6>();
    case 7: return prepare_simt_n<7>();
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_block_simt(const PassArgs& pa, void* psi, int grid, cudaStream_t s) {
  switch (pa.n) {
    case 2: return launch_simt_n<2>(pa, psi, grid, s);
    case 3: return launch_simt_n<3>(pa, psi, grid, s);
    case 4: return launch_simt_n<4>(pa, psi, grid, s);
    case 5: return launch_simt_n<5>(pa, psi, grid, s);
    case 6: return launch_simt_n<6>(pa, psi, grid, s);
    case 7: return launch_simt_n<7>(pa, psi, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

// a pass's relabel moves the window by at most its 7 row bits
constexpr int kMaxShiftRows = 7;

std::string block_tile_layout(int L, int n, int R, int lo, int lo_next, int* a_out,
                              int8_t* sigma) {
  const int lo_min = std::min(lo, lo_next);
  const int delta = std::abs(lo_next - lo);
  if (delta > R) return "window moves by more than the tile's row bits";
  const int a = (R == L - n) ? n : std::max(n, std::min(n + lo_min, L - R));
  if (!(a <= n + lo_min && n + lo_min + delta <= a + R)) return "row bits miss moved sites";
  for (int q = 0; q < n + R; ++q) {
    const int p = q < n ? q : a + q - n;
    const int s = site_at(L, n, lo, p);
    const int po = pos_of(L, n, lo_next, s);
    int qo;
    if (po < n) qo = po;
    else if (po >= a && po < a + R) qo = po - a + n;
    else return "site leaves the tile";
    sigma[q] = (int8_t)qo;
  }
  for (int p = 0; p < L; ++p) {
    const bool in_tile = p < n || (p >= a && p < a + R);
    if (!in_tile && site_at(L, n, lo, p) != site_at(L, n, lo_next, p))
      return "layout change outside the tile";
  }
  *a_out = a;
  return std::string();
}

int block_build(int L, const std::vector<Gate2>& gates, const Observable& obs, int n,
                int split, const LaunchCfg& cfg, bool cyclic, BlockPlan** out,
                std::string* msg) {
  *out = nullptr;
  if (split != SV_SPLIT_BF16X3 && split != SV_SPLIT_FP32) {
    *msg = "unknown split";
    return SV_EINVAL;
  }
  BlockPlan* bp = new BlockPlan();
  bp->L = L;
  bp->n = n;
  bp->R = std::min(7, L - n);
  bp->split = split;
  bp->cfg = cfg;
  bp->passes = fusion_plan(L, gates, n, cyclic);
  const int P = (int)bp->passes.size();
  bp->start = bp->passes[0].lo;
  const int R = bp->R;
  bp->tensor_cores = split == SV_SPLIT_BF16X3 && block_tc_supported(L, n);
  const long long ntiles = 1ll << (L - n - R);
  const int per_sm = bp->tensor_cores ? 1 : 2;
  long long grid = std::min<long long>(ntiles, (long long)cfg.num_sms * per_sm);
  if (cfg.min_tiles_per_cta > 0) grid = std::min<long long>(grid, ntiles / cfg.min_tiles_per_cta);
  bp->grid = (int)std::max<long long>(1, grid);
  bp->maxb = bp->grid;
  auto fail = [&](const std::string& m) {
    *msg = m;
    block_free(bp);
    return SV_EINVAL;
  };
  // The launches: the period's P passes, each writing the next pass's layout
  // (the last one the start's); when the start is not site 0, the last
  // period of an evolution ends with a variant of the last pass that writes
  // toward the natural layout (plus relabel steps if it is more than 7 sites
  // away), and an evolution begins with relabel steps from the natural
  // layout to the start.  A relabel step applies the identity.
  struct Op {
    int src;  // pass whose unitary and measurements it applies, -1: identity
    int lo, lo_next;
  };
  std::vector<Op> ops;
  for (int k = 0; k < P; ++k) ops.push_back({k, bp->passes[k].lo, bp->passes[(k + 1) % P].lo});
  auto step = [](int from, int to) {
    return from + std::max(-kMaxShiftRows, std::min(kMaxShiftRows, to - from));
  };
  for (int k = 0; k < P; ++k) bp->seq_cyc.push_back(k);
  if (bp->start == 0) {
    bp->seq_exit = bp->seq_cyc;
  } else {
    for (int k = 0; k + 1 < P; ++k) bp->seq_exit.push_back(k);
    int lo = bp->passes[P - 1].lo, nx = step(lo, 0);
    bp->seq_exit.push_back((int)ops.size());
    ops.push_back({P - 1, lo, nx});
    while (nx != 0) {
      lo = nx;
      nx = step(lo, 0);
      bp->seq_exit.push_back((int)ops.size());
      ops.push_back({-1, lo, nx});
    }
    lo = 0;
    while (lo != bp->start) {
      nx = step(lo, bp->start);
      bp->seq_entry.push_back((int)ops.size());
      ops.push_back({-1, lo, nx});
      lo = nx;
    }
    lo = bp->start;
    while (lo != 0) {  // from the period layout back to the natural one
      nx = step(lo, 0);
      bp->seq_leave.push_back((int)ops.size());
      ops.push_back({-1, lo, nx});
      lo = nx;
    }
  }
  const BlockPass identity_pass = [&]() {
    BlockPass ip;
    ip.n = n;
    ip.U.assign((size_t)1 << (2 * n), cd(0.0, 0.0));
    for (size_t e = 0; e < ((size_t)1 << n); ++e) ip.U[e * ((size_t)1 << n) + e] = 1.0;
    return ip;
  }();
  std::vector<int> slot_of(P, -1);
  int slot = 0;
  for (size_t k = 0; k < ops.size(); ++k) {
    const BlockPass& ps = ops[k].src >= 0 ? bp->passes[ops[k].src] : identity_pass;
    const int lo = ops[k].lo;
    const int lo_next = ops[k].lo_next;
    PassArgs pa;
    pa.L = L;
    pa.n = n;
    pa.R = R;
    pa.lo = lo;
    pa.ntiles = ntiles;
    const std::string why = block_tile_layout(L, n, R, lo, lo_next, &pa.a, pa.sigma);
    if (!why.empty()) return fail(why);
    if (bp->tensor_cores) block_tc_layout(pa);
    for (int s : obs.general ? std::vector<int>() : ps.x_sites) {
      const int j = s - lo;
      if (j < 0 || j >= n) return fail("measured site outside window");
      pa.x_mask |= 1u << j;
      pa.cx[j] = (float)obs.cx[s];
    }
    pa.diag = ps.diag && !obs.general ? 1 : 0;
    if (pa.diag) {
      pa.diag_lo = lo_next;  // the output's layout (natural order: window at 0)
      pa.ep.flags = EPI_DIAG;
      pa.ep.J = obs.J;
      pa.ep.cz_first = obs.cz[0];
      pa.ep.cz_last = obs.cz[L - 1];
      pa.ep.cz_bulk = L >= 3 ? obs.cz[1] : 0.0;
      pa.diag_f[0] = (float)pa.ep.J;
      pa.diag_f[1] = (float)pa.ep.cz_bulk;
      pa.diag_f[2] = (float)pa.ep.cz_first;
      pa.diag_f[3] = (float)pa.ep.cz_last;
      pa.diag_f[4] = (float)(pa.ep.cz_bulk * (L - 2) + pa.ep.cz_first + pa.ep.cz_last);
      // per window bit: its site (window bit j is site lo + j in every
      // layout), its field, and which of its neighbours lie outside the window
      int site[8];
      for (int j = 0; j < n; ++j) site[j] = lo + j;
      for (int j = 0; j < n; ++j) {
        const int g = site[j];
        const double czg = g == 0 ? pa.ep.cz_first : (g == L - 1 ? pa.ep.cz_last : pa.ep.cz_bulk);
        int inside = 0;
        for (int k = 0; k < 2; ++k) {
          const int nb = k == 0 ? g - 1 : g + 1;
          pa.diag_nb[j][k] = -1;
          if (nb < 0 || nb >= L) continue;
          bool in_window = false;
          for (int jj = 0; jj < n; ++jj) in_window = in_window || site[jj] == nb;
          if (in_window) ++inside;
          else pa.diag_nb[j][k] = (int8_t)nb;
        }
        pa.diag_lin0[j] = (float)(-2.0 * (czg + pa.ep.J * inside));
      }
    }
    if (pa.x_mask || pa.diag) {
      // the exit variant of the last pass fills that pass's partials slot
      if (ops[k].src >= 0 && slot_of[ops[k].src] >= 0) pa.slot = slot_of[ops[k].src];
      else pa.slot = slot++;
      if (ops[k].src >= 0) slot_of[ops[k].src] = pa.slot;
    }
    bp->args.push_back(pa);
  }
  const int NA = (int)bp->args.size();
  bp->nslots = slot;
  // device buffers
  const size_t dim = (size_t)1 << n;
  // the operands of the P passes and of the identity (index P), rounded
  // close to unitary (host_round.cpp); every launch takes its source's copy
  const int NU = P + 1;
  std::vector<float2> uu(bp->tensor_cores ? 0 : (size_t)NU * dim * dim);
  std::vector<float4> ul(bp->tensor_cores ? 0 : (size_t)NU * dim);
  std::vector<std::vector<uint32_t>> uw(bp->tensor_cores ? NU : 0);
  round_passes_parallel(NU, [&](int k) {
    const std::vector<cd>& U = k < P ? bp->passes[k].U : identity_pass.U;
    if (bp->tensor_cores) block_tc_pack_w(n, U, uw[k]);
    else round_unitary_fp32((int)dim, U.data(), &uu[k * dim * dim], &ul[k * dim]);
  });
  std::vector<float2> hu(bp->tensor_cores ? 0 : (size_t)NA * dim * dim);
  std::vector<float4> hl(bp->tensor_cores ? 0 : (size_t)NA * dim);
  std::vector<std::vector<uint32_t>> hw(bp->tensor_cores ? NA : 0);
  for (int k = 0; k < NA; ++k) {
    const int from = ops[k].src >= 0 ? ops[k].src : P;
    if (bp->tensor_cores) {
      hw[k] = uw[from];
    } else {
      std::copy(uu.begin() + from * dim * dim, uu.begin() + (from + 1) * dim * dim,
                hu.begin() + k * dim * dim);
      std::copy(ul.begin() + from * dim, ul.begin() + (from + 1) * dim, hl.begin() + k * dim);
    }
  }
  if (!bp->tensor_cores &&
      (cudaMalloc(&bp->d_U, sizeof(float2) * hu.size()) != cudaSuccess ||
       cudaMemcpy(bp->d_U, hu.data(), sizeof(float2) * hu.size(), cudaMemcpyHostToDevice) !=
           cudaSuccess ||
       cudaMalloc(&bp->d_Ulead, sizeof(float4) * hl.size()) != cudaSuccess ||
       cudaMemcpy(bp->d_Ulead, hl.data(), sizeof(float4) * hl.size(), cudaMemcpyHostToDevice) !=
           cudaSuccess)) {
    cudaGetLastError();
    *msg = "unitary upload failed";
    block_free(bp);
    return SV_ENOMEM;
  }
  if (bp->tensor_cores) {
    bp->w_bytes_per_pass = block_tc_w_bytes(n);
    std::vector<uint32_t> all;
    for (int k = 0; k < NA; ++k) all.insert(all.end(), hw[k].begin(), hw[k].end());
    if (cudaMalloc(&bp->d_W, all.size() * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemcpy(bp->d_W, all.data(), all.size() * sizeof(uint32_t),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      *msg = "operand upload failed";
      block_free(bp);
      return SV_ENOMEM;
    }
  }
  const size_t pbytes = sizeof(double) * 2 * std::max(1, bp->nslots) * (size_t)bp->maxb;
  if (cudaMalloc(&bp->d_partials, pbytes) != cudaSuccess ||
      cudaMemset(bp->d_partials, 0, pbytes) != cudaSuccess) {
    cudaGetLastError();
    *msg = "partials allocation failed";
    block_free(bp);
    return SV_ENOMEM;
  }
  for (int k = 0; k < NA; ++k) {
    PassArgs& pa = bp->args[k];
    if (bp->d_U) {
      pa.U = bp->d_U + (size_t)k * dim * dim;
      pa.Ulead = bp->d_Ulead + (size_t)k * dim;
    }
    if (bp->d_W)
      pa.W = static_cast<const char*>(bp->d_W) + (size_t)k * bp->w_bytes_per_pass;
    if (pa.slot >= 0) pa.partial = bp->d_partials + 2 * (size_t)pa.slot * bp->maxb;
  }
  if (bp->tensor_cores) {
    if (block_tc_prepare() != cudaSuccess || cudaMalloc(&bp->d_status, sizeof(int)) != cudaSuccess ||
        cudaMemset(bp->d_status, 0, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      *msg = "tensor-core pass set-up failed";
      block_free(bp);
      return SV_ECUDA;
    }
  }
  if (prepare_simt(n) != cudaSuccess) {
    cudaGetLastError();
    *msg = "shared-memory opt-in failed";
    block_free(bp);
    return SV_ECUDA;
  }
  *out = bp;
  return SV_OK;
}

void block_set_renorm(BlockPlan* bp, const Renorm& rn) {
  if (!bp->args.empty()) bp->args[0].ep.rn = rn;
}

void block_info(const BlockPlan* bp, int* passes, int* launches) {
  if (passes) *passes = (int)bp->passes.size();
  if (launches) *launches = (int)bp->passes.size() + 1;
}

size_t block_upload_bytes(const BlockPlan* bp) {
  const size_t P = bp->args.size();
  const size_t dim = (size_t)1 << bp->n;
  const size_t u = bp->tensor_cores ? 0 : sizeof(float2) * dim * dim + sizeof(float4) * dim;
  return P * (u + bp->w_bytes_per_pass);
}

namespace {

// TMA descriptors embed the state address: (re)build them for psi.
cudaError_t ensure_maps(BlockPlan* bp, void* psi) {
  if (!bp->tensor_cores || bp->maps_psi == psi) return cudaSuccess;
  const size_t mb = block_tc_map_bytes();
  bp->maps.assign(mb * bp->args.size(), 0);
  for (size_t k = 0; k < bp->args.size(); ++k)
    if (block_tc_make_map(bp->args[k], psi, bp->maps.data() + k * mb) != SV_OK)
      return cudaErrorInvalidValue;
  bp->maps_psi = psi;
  return cudaSuccess;
}

cudaError_t launch_pass(BlockPlan* bp, size_t k, void* psi, cudaStream_t s) {
  if (bp->tensor_cores)
    return launch_block_tc(bp->args[k], psi, bp->maps.data() + k * block_tc_map_bytes(),
                           bp->d_status, bp->grid, s);
  return launch_block_simt(bp->args[k], psi, bp->grid, s);
}

}  // namespace

int block_status(BlockPlan* bp, cudaStream_t s) {
  if (!bp || !bp->d_status) return 0;
  int h = 0;
  if (cudaMemcpyAsync(&h, bp->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -1;
  return h;
}

cudaError_t block_enqueue_entry(BlockPlan* bp, void* psi, cudaStream_t s) {
  cudaError_t e = ensure_maps(bp, psi);
  if (e != cudaSuccess) return e;
  for (int k : bp->seq_entry) {
    e = launch_pass(bp, k, psi, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t block_enqueue_leave(BlockPlan* bp, void* psi, cudaStream_t s) {
  cudaError_t e = ensure_maps(bp, psi);
  if (e != cudaSuccess) return e;
  for (int k : bp->seq_leave) {
    e = launch_pass(bp, k, psi, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t block_enqueue_period(BlockPlan* bp, void* psi, long long* counter, double* ring,
                                 int ring_len, cudaStream_t s, bool last) {
  cudaError_t e = ensure_maps(bp, psi);
  if (e != cudaSuccess) return e;
  for (int k : last ? bp->seq_exit : bp->seq_cyc) {
    e = launch_pass(bp, k, psi, s);
    if (e != cudaSuccess) return e;
  }
  return launch_period_reduce(bp->d_partials, (long long)bp->nslots * bp->maxb, bp->L, ring,
                              ring_len, counter, 1, s);
}

cudaError_t block_enqueue_period_events(BlockPlan* bp, void* psi, long long* counter,
                                        double* ring, int ring_len, cudaStream_t s,
                                        cudaEvent_t* ev, bool last) {
  cudaError_t e = ensure_maps(bp, psi);
  if (e != cudaSuccess) return e;
  // events around the period's P passes (the exit variant's relabel steps,
  // if any, fall inside the last pass's interval) and the reduce
  const std::vector<int>& seq = last ? bp->seq_exit : bp->seq_cyc;
  const size_t P = bp->seq_cyc.size();
  for (size_t k = 0; k < seq.size(); ++k) {
    if (k < P) {
      e = cudaEventRecord(ev[k], s);
      if (e != cudaSuccess) return e;
    }
    e = launch_pass(bp, (size_t)seq[k], psi, s);
    if (e != cudaSuccess) return e;
  }
  e = cudaEventRecord(ev[P], s);
  if (e != cudaSuccess) return e;
  e = launch_period_reduce(bp->d_partials, (long long)bp->nslots * bp->maxb, bp->L, ring,
                           ring_len, counter, 1, s);
  if (e != cudaSuccess) return e;
  return cudaEventRecord(ev[P + 1], s);
}

// ------------------------------------------------------------ chain groups

struct BlockGroup {
  std::vector<GroupMember> m;
  std::vector<PassArgs> ops;        // structure of each pass, ntiles over the group
  GroupChain* d_chains = nullptr;   // [passes][chains]
  ReduceItem* d_reduce = nullptr;   // [chains]
  double* d_part = nullptr;         // [chains][measuring slots][grid] (energy, norm) pairs
  int nt_log2 = 0;
  int grid = 0;
};

namespace {
template <typename T, size_t N>
bool same_array(const T (&x)[N], const T (&y)[N]) {
  return std::memcmp(x, y, sizeof(x)) == 0;
}
bool same_pass(const PassArgs& x, const PassArgs& y) {
  return x.L == y.L && x.n == y.n && x.R == y.R && x.a == y.a && x.lo == y.lo &&
         x.ntiles == y.ntiles && x.x_mask == y.x_mask && x.diag == y.diag &&
         x.diag_lo == y.diag_lo && same_array(x.diag_nb, y.diag_nb) &&
         same_array(x.sigma, y.sigma) && same_array(x.rowvec, y.rowvec) &&
         same_array(x.spos, y.spos) && same_array(x.ssig, y.ssig) && x.st_ndims == y.st_ndims &&
         x.st_tlo_dim == y.st_tlo_dim && x.st_tlo_shift == y.st_tlo_shift &&
         x.st_thi_dim == y.st_thi_dim && x.st_thi_shift == y.st_thi_shift &&
         x.slot == y.slot && (x.partial == nullptr) == (y.partial == nullptr);
}
bool renorm_active(const PassArgs& pa) { return pa.ep.rn.ring && pa.ep.rn.every > 0; }
}  // namespace

bool block_same_structure(const BlockPlan* a, const BlockPlan* b) {
  if (!a || !b || !a->tensor_cores || !b->tensor_cores) return false;
  if (a->L != b->L || a->n != b->n || a->start != b->start || a->nslots != b->nslots ||
      a->args.size() != b->args.size() || a->seq_cyc != b->seq_cyc ||
      a->seq_exit != b->seq_exit || a->seq_entry != b->seq_entry || a->seq_leave != b->seq_leave)
    return false;
  for (size_t k = 0; k < a->args.size(); ++k)
    if (!same_pass(a->args[k], b->args[k])) return false;
  return true;
}

int block_group_build(const std::vector<GroupMember>& mem, int ring_len, const LaunchCfg& cfg,
                      cudaStream_t s, BlockGroup** out, std::string* msg) {
  *out = nullptr;
  if (mem.empty()) return SV_EINVAL;
  const BlockPlan* ref = mem[0].plan;
  for (const GroupMember& x : mem) {
    if (!block_same_structure(ref, x.plan)) {
      *msg = "the chains' plans differ";
      return SV_EINVAL;
    }
    for (const PassArgs& pa : x.plan->args)
      if (renorm_active(pa)) {
        *msg = "a group does not fold renormalisation";
        return SV_EUNSUPPORTED;
      }
  }
  const long long nt = ref->args[0].ntiles;
  int lg = 0;
  while ((1ll << lg) < nt) ++lg;
  for (const PassArgs& pa : ref->args)
    if (pa.ntiles != nt || (1ll << lg) != nt) {
      *msg = "tile counts differ between passes";
      return SV_EINVAL;
    }
  const size_t C = mem.size(), K = ref->args.size();
  BlockGroup* g = new BlockGroup();
  g->m = mem;
  g->nt_log2 = lg;
  // one CTA per SM, each with at least kGroupMinTiles tiles (a small group
  // then leaves SMs to the others instead of paying a CTA's set-up per tile)
  constexpr long long kGroupMinTiles = 4;
  g->grid = (int)std::max<long long>(
      1, std::min<long long>(cfg.num_sms, nt * (long long)C / kGroupMinTiles));
  g->ops = ref->args;
  for (PassArgs& pa : g->ops) {
    pa.ntiles = nt * (long long)C;
    pa.W = nullptr;        // per chain
    pa.partial = nullptr;  // per chain
  }
  // partial sums: the chains' own buffers hold one pair per CTA of their
  // own launches; a group launch has its own grid, so the group keeps a
  // buffer of [chains][slots][grid] pairs (zero where a CTA meets no tile
  // of the chain)
  const int S = std::max(1, ref->nslots), G = g->grid;
  const size_t part_pairs = C * (size_t)S * G;
  std::vector<GroupChain> hc(K * C);
  std::vector<uint8_t> maps(block_tc_map_bytes());
  cudaError_t e = cudaMalloc(&g->d_part, sizeof(double) * 2 * part_pairs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    block_group_free(g);
    *msg = "group partials allocation";
    return SV_ENOMEM;
  }
  for (size_t k = 0; k < K; ++k)
    for (size_t c = 0; c < C; ++c) {
      const PassArgs& pa = mem[c].plan->args[k];
      GroupChain& gc = hc[k * C + c];
      if (block_tc_make_map(pa, mem[c].psi, maps.data()) != SV_OK) {
        block_group_free(g);
        *msg = "tensor map";
        return SV_ECUDA;
      }
      std::memcpy(gc.map_in, maps.data(), sizeof(gc.map_in));
      std::memcpy(gc.map_out, maps.data() + sizeof(gc.map_in), sizeof(gc.map_out));
      gc.W = pa.W;
      gc.partial = pa.slot >= 0 ? g->d_part + 2 * ((c * S + pa.slot) * (size_t)G) : nullptr;
      std::memcpy(gc.cx, pa.cx, sizeof(gc.cx));
      std::memcpy(gc.diag_f, pa.diag_f, sizeof(gc.diag_f));
      std::memcpy(gc.diag_lin0, pa.diag_lin0, sizeof(gc.diag_lin0));
    }
  std::vector<ReduceItem> red(C);
  for (size_t c = 0; c < C; ++c) {
    const BlockPlan* bp = mem[c].plan;
    red[c].partials = g->d_part + 2 * (c * (size_t)S * G);
    red[c].n = (long long)S * G;
    red[c].ring = mem[c].ring;
    red[c].counter = mem[c].counter;
    red[c].L = bp->L;
    red[c].ring_len = ring_len;
  }
  e = cudaMalloc(&g->d_chains, sizeof(GroupChain) * hc.size());
  if (e == cudaSuccess) e = cudaMalloc(&g->d_reduce, sizeof(ReduceItem) * C);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_part, 0, sizeof(double) * 2 * part_pairs, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_chains, hc.data(), sizeof(GroupChain) * hc.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->d_reduce, red.data(), sizeof(ReduceItem) * C, cudaMemcpyHostToDevice,
                        s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host arrays are freed below
  if (e != cudaSuccess) {
    cudaGetLastError();
    block_group_free(g);
    *msg = "group upload";
    return SV_ECUDA;
  }
  *out = g;
  return SV_OK;
}

int block_group_start(const BlockGroup* g) { return g->m[0].plan->start; }

size_t block_group_size(const BlockGroup* g) { return g->m.size(); }

namespace {
cudaError_t group_pass(BlockGroup* g, int k, cudaStream_t s) {
  return launch_block_tc_group(g->ops[k], g->d_chains + (size_t)k * g->m.size(), g->nt_log2,
                               g->m[0].plan->d_status, g->grid, s);
}
}  // namespace

cudaError_t block_group_enqueue_entry(BlockGroup* g, cudaStream_t s) {
  for (int k : g->m[0].plan->seq_entry) {
    cudaError_t e = group_pass(g, k, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t block_group_enqueue_period(BlockGroup* g, cudaStream_t s, bool last) {
  const BlockPlan* ref = g->m[0].plan;
  for (int k : last ? ref->seq_exit : ref->seq_cyc) {
    cudaError_t e = group_pass(g, k, s);
    if (e != cudaSuccess) return e;
  }
  return launch_period_reduce_many(g->d_reduce, (int)g->m.size(), s);
}

void block_group_free(BlockGroup* g) {
  if (!g) return;
  cudaFree(g->d_chains);
  cudaFree(g->d_reduce);
  cudaFree(g->d_part);
  delete g;
}

void block_free(BlockPlan* bp) {
  if (!bp) return;
  cudaFree(bp->d_U);
  cudaFree(bp->d_Ulead);
  cudaFree(bp->d_W);
  cudaFree(bp->d_partials);
  cudaFree(bp->d_status);
  delete bp;
}

}  // namespace fsv
