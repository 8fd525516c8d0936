// C ABI of the batched evolution (include/floquet_sv.h, "batch" section):
// many independent chains on one device, each in its own slice of one
// caller-owned buffer.
//
// Every chain gets a context (sv_ctx) on its slice for initialisation and,
// for the plain, block and multi-gate forms, for its evolution graph.  Chains of at most
// 14 sites may instead run the resident form (k_batch.cu): one launch
// advances all of them, each in one CTA's shared memory.  An evolution is
// one CUDA graph per run of M periods: the resident launch; one branch per
// group of tensor-core chains whose plans share their structure (same L),
// each pass of all its chains one launch over all their tiles and each
// period's reduces one launch; and, for every other chain, its run of M
// periods captured from its context.  A block plan whose periods start off
// site 0 relabels into its period layout at the start of the run and hands
// back the natural layout at its end.
//
// The autotuner (form SV_BATCH_AUTO) times every form that fits a distinct
// L, run together for four periods through the same kind of graph (the
// CUDA-core block form at widths n = 5, 6 and 7, the tensor-core block form
// as a group, the plain, multi-gate and resident forms), and keeps the
// fastest (most chain-periods per second) for all chains of that L.  The resident form is
// timed on all chains of that L (one CTA each, so its rate grows with their
// number); the others, which fill the device with one chain, on up to eight.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "sv_batch.h"
#include "sv_block.h"

struct sv_batch {
  int device = 0;
  int n = 0;
  cudaStream_t stream = nullptr;      // caller's stream
  cudaStream_t cap_stream = nullptr;  // capture of the resident launch
  char* base = nullptr;
  std::vector<int> L;
  std::vector<size_t> off;
  std::vector<int> form;
  std::vector<int> width;      // block forms: window width n
  std::vector<sv_floquet_params> params;
  std::vector<const double*> spinors;  // caller's arrays, valid during create only
  std::vector<sv_ctx*> ctx;
  // resident chains
  std::vector<int> res;
  fsv::ResidentChain* d_res = nullptr;
  float2* d_rgates = nullptr;
  int* d_rbonds = nullptr;
  double* d_rring = nullptr;
  long long* d_rcount = nullptr;
  int res_maxL = 0;
  // graphs of one period and of M periods of every chain
  cudaGraphExec_t g1 = nullptr, gm = nullptr;
  std::vector<fsv::BlockGroup*> groups;  // chain groups the two graphs launch
  int M = 16;
  int64_t counter = 0;
  std::string err;
};

namespace {

constexpr size_t kAlign = 256;
// CUDA-core block passes of a batch share the device with other chains'
// passes: each CTA keeps a run of at least this many tiles.
constexpr int kDefaultTileRun = 8;
constexpr int kSimtWidths[3] = {5, 6, 7};
constexpr int kDefaultWidth = 6;

int bfail(sv_batch* b, int code, const char* fmt, ...) {
  if (b) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    b->err = buf;
  }
  return code;
}

#define BCUDA(call, what)                                                        \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) return bfail(b, SV_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

bool form_fits(int form, int L) {
  switch (form) {
    case SV_BATCH_PLAIN: return true;
    case SV_BATCH_BLOCK_SIMT: return L >= 6;
    case SV_BATCH_BLOCK_TC: return L >= 13;
    case SV_BATCH_RESIDENT: return L <= fsv::kResidentMaxL;
    case SV_BATCH_MULTIGATE: return true;
    default: return false;
  }
}

// The resident chains' device tables: descriptors, gates, bonds, energy
// rings and the shared period counter.
struct ResidentSet {
  fsv::ResidentChain* d_res = nullptr;
  float2* d_gates = nullptr;
  int* d_bonds = nullptr;
  double* d_ring = nullptr;
  long long* d_count = nullptr;
  int max_L = 0;
  int count = 0;
  void release() {
    cudaFree(d_res);
    cudaFree(d_gates);
    cudaFree(d_bonds);
    cudaFree(d_ring);
    cudaFree(d_count);
    *this = ResidentSet();
  }
};

int build_resident(sv_batch* b, const std::vector<int>& chains, ResidentSet* rs) {
  *rs = ResidentSet();
  if (chains.empty()) return SV_OK;
  const int ring = fsv::ctx_ring_len();
  std::vector<fsv::ResidentChain> hd(chains.size());
  std::vector<float2> gates;
  std::vector<int> bonds;
  std::vector<size_t> goff(chains.size());
  for (size_t k = 0; k < chains.size(); ++k) {
    const int c = chains[k];
    const sv_floquet_params& p = b->params[c];
    auto pg = fsv::period_gates(b->L[c], p, p.theta, p.hx);
    goff[k] = bonds.size();
    for (auto& g : pg) {
      float2 m[fsv::kGateEntries];
      fsv::round_unitary4(g.m, m);
      for (int e = 0; e < 16; ++e)
        m[16 + e] = make_float2((float)(g.m[e].real() - (double)m[e].x),
                                (float)(g.m[e].imag() - (double)m[e].y));
      gates.insert(gates.end(), m, m + fsv::kGateEntries);
      bonds.push_back(g.bond);
    }
    fsv::Observable o = fsv::observable(b->L[c], p);
    fsv::ResidentChain& r = hd[k];
    r.L = b->L[c];
    r.ngates = (int)pg.size();
    r.J = o.J;
    for (int i = 0; i < r.L; ++i) {
      r.cx[i] = o.cx[i];
      r.cz[i] = o.cz[i];
    }
    rs->max_L = std::max(rs->max_L, r.L);
  }
  rs->count = (int)chains.size();
  if (cudaMalloc(&rs->d_res, sizeof(fsv::ResidentChain) * hd.size()) != cudaSuccess ||
      cudaMalloc(&rs->d_gates, sizeof(float2) * gates.size()) != cudaSuccess ||
      cudaMalloc(&rs->d_bonds, sizeof(int) * bonds.size()) != cudaSuccess ||
      cudaMalloc(&rs->d_ring, sizeof(double) * 2 * ring * hd.size()) != cudaSuccess ||
      cudaMalloc(&rs->d_count, sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    rs->release();
    return bfail(b, SV_ENOMEM, "resident tables");
  }
  for (size_t k = 0; k < chains.size(); ++k) {
    fsv::ResidentChain& r = hd[k];
    r.psi = reinterpret_cast<float2*>(b->base + b->off[chains[k]]);
    r.gates = rs->d_gates + fsv::kGateEntries * goff[k];
    r.bonds = rs->d_bonds + goff[k];
    r.ring = rs->d_ring + 2 * (size_t)ring * k;
  }
  BCUDA(cudaMemcpyAsync(rs->d_res, hd.data(), sizeof(fsv::ResidentChain) * hd.size(),
                        cudaMemcpyHostToDevice, b->stream),
        "upload resident descriptors");
  BCUDA(cudaMemcpyAsync(rs->d_gates, gates.data(), sizeof(float2) * gates.size(),
                        cudaMemcpyHostToDevice, b->stream),
        "upload resident gates");
  BCUDA(cudaMemcpyAsync(rs->d_bonds, bonds.data(), sizeof(int) * bonds.size(),
                        cudaMemcpyHostToDevice, b->stream),
        "upload resident bonds");
  BCUDA(cudaMemsetAsync(rs->d_count, 0, sizeof(long long), b->stream), "reset counter");
  BCUDA(fsv::resident_prepare(rs->max_L), "resident attributes");
  BCUDA(cudaStreamSynchronize(b->stream), "synchronize");
  return SV_OK;
}

// Build the period evolution of chain c in its context for a graph form
// (block forms: window width n; CUDA-core passes keep kDefaultTileRun tiles
// per CTA at least).
int build_graph_form(sv_batch* b, int c, int form, int n) {
  fsv::ctx_set_min_tiles(b->ctx[c], kDefaultTileRun);
  sv_floquet_params p = b->params[c];
  p.theta_p = nullptr;
  p.hx_p = nullptr;
  p.n_period_params = 0;
  p.renorm_every = 0;
  if (form == SV_BATCH_PLAIN) {
    p.mode = SV_MODE_PLAIN;
  } else if (form == SV_BATCH_MULTIGATE) {
    p.mode = SV_MODE_MULTIGATE;
  } else {
    p.mode = SV_MODE_BLOCK;
    p.block_n = form == SV_BATCH_BLOCK_TC ? 6 : n;
    p.split = form == SV_BATCH_BLOCK_TC ? SV_SPLIT_BF16X3 : SV_SPLIT_FP32;
  }
  int rc = sv_build_floquet(b->ctx[c], &p);
  if (rc) return bfail(b, rc, "chain %d build: %s", c, sv_last_error(b->ctx[c]));
  return SV_OK;
}

// Tensor-core chains grouped by plan structure (an existing group of the
// same structure is reused); the other chains are returned in `rest`.
int make_groups(sv_batch* b, const std::vector<int>& chains, std::vector<int>* rest,
                std::vector<fsv::BlockGroup*>* groups) {
  std::vector<std::vector<fsv::GroupMember>> parts;
  for (int c : chains) {
    fsv::GroupMember m;
    if (fsv::ctx_block_member(b->ctx[c], &m.plan, &m.psi, &m.counter, &m.ring) != SV_OK) {
      rest->push_back(c);
      continue;
    }
    bool placed = false;
    for (auto& p : parts)
      if (fsv::block_same_structure(p[0].plan, m.plan)) {
        p.push_back(m);
        placed = true;
        break;
      }
    if (!placed) parts.push_back({m});
  }
  for (auto& p : parts) {
    fsv::BlockGroup* g = nullptr;
    std::string msg;
    int rc = fsv::block_group_build(p, fsv::ctx_ring_len(), p[0].plan->cfg, b->stream, &g, &msg);
    if (rc) return bfail(b, rc, "chain group: %s", msg.c_str());
    groups->push_back(g);
  }
  return SV_OK;
}

void free_groups(std::vector<fsv::BlockGroup*>* groups) {
  for (fsv::BlockGroup* g : *groups) fsv::block_group_free(g);
  groups->clear();
}

// One graph advancing `periods` periods of the given graph-form chains and
// of the resident set (if any).  Tensor-core chains run in groups, built on
// the first call (groups empty) and reused by later ones; the caller frees
// them after the graphs.
int make_graph(sv_batch* b, const std::vector<int>& chains, const ResidentSet* rs, int periods,
               cudaGraphExec_t* out, std::vector<fsv::BlockGroup*>* groups) {
  *out = nullptr;
  cudaGraph_t g = nullptr;
  BCUDA(cudaGraphCreate(&g, 0), "graph create");
  auto fail_g = [&](int rc) {
    cudaGraphDestroy(g);
    return rc;
  };
  if (rs && rs->count > 0) {
    cudaGraph_t rg = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t le = fsv::launch_chain_resident(rs->d_res, rs->count, rs->max_L, rs->d_count,
                                                  periods, fsv::ctx_ring_len(), b->cap_stream);
      e = cudaStreamEndCapture(b->cap_stream, &rg);
      if (le != cudaSuccess) e = le;
    }
    if (e != cudaSuccess) {
      if (rg) cudaGraphDestroy(rg);
      return fail_g(bfail(b, SV_ECUDA, "resident capture: %s", cudaGetErrorString(e)));
    }
    cudaGraphNode_t node;
    e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, rg);
    cudaGraphDestroy(rg);
    if (e != cudaSuccess)
      return fail_g(bfail(b, SV_ECUDA, "resident node: %s", cudaGetErrorString(e)));
  }
  std::vector<int> rest;
  if (groups->empty()) {
    int rc = make_groups(b, chains, &rest, groups);
    if (rc) return fail_g(rc);
  } else {
    // the groups were built for these chains by an earlier call
    size_t grouped = 0;
    for (int c : chains) {
      fsv::GroupMember m;
      if (fsv::ctx_block_member(b->ctx[c], &m.plan, &m.psi, &m.counter, &m.ring) != SV_OK)
        rest.push_back(c);
      else
        ++grouped;
    }
    size_t members = 0;
    for (fsv::BlockGroup* grp : *groups) members += fsv::block_group_size(grp);
    if (members != grouped)
      return fail_g(bfail(b, SV_ESTATE, "chain groups built for another set of chains"));
  }
  for (fsv::BlockGroup* grp : *groups) {
    cudaGraph_t pg = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed);
    cudaError_t le = cudaSuccess;
    if (e == cudaSuccess) {
      if (periods > 0 && fsv::block_group_start(grp) != 0)
        le = fsv::block_group_enqueue_entry(grp, b->cap_stream);
      for (int k = 0; k < periods && le == cudaSuccess; ++k)
        le = fsv::block_group_enqueue_period(grp, b->cap_stream, k + 1 == periods);
      e = cudaStreamEndCapture(b->cap_stream, &pg);
      if (le != cudaSuccess) e = le;
    }
    if (e != cudaSuccess) {
      if (pg) cudaGraphDestroy(pg);
      return fail_g(bfail(b, SV_ECUDA, "group capture: %s", cudaGetErrorString(e)));
    }
    cudaGraphNode_t node;
    e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, pg);
    cudaGraphDestroy(pg);
    if (e != cudaSuccess)
      return fail_g(bfail(b, SV_ECUDA, "group node: %s", cudaGetErrorString(e)));
  }
  for (int c : rest) {
    cudaGraph_t pg = nullptr;
    int rc = fsv::ctx_capture_run(b->ctx[c], periods, &pg);
    if (rc) return fail_g(bfail(b, rc, "chain %d capture: %s", c, sv_last_error(b->ctx[c])));
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, pg);
    cudaGraphDestroy(pg);
    if (e != cudaSuccess)
      return fail_g(bfail(b, SV_ECUDA, "chain node: %s", cudaGetErrorString(e)));
  }
  cudaError_t e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return bfail(b, SV_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  return SV_OK;
}

int reinit(sv_batch* b, int c) {
  int rc = sv_init(b->ctx[c], b->L[c], b->spinors[c]);
  if (rc) return bfail(b, rc, "chain %d init: %s", c, sv_last_error(b->ctx[c]));
  return SV_OK;
}

// Chain-periods per second of the chains `sample` run together, chain
// sample[i] in form forms[i] (the CUDA-core block form at width n).  The
// trial moves the states; they are initialised again after it.
int time_forms(sv_batch* b, const std::vector<int>& sample, const std::vector<int>& forms, int n,
               double* rate) {
  *rate = 0.0;
  constexpr int kPeriods = 4;
  ResidentSet rs;
  std::vector<int> graph_chains, res_chains;
  int rc = SV_OK;
  for (size_t i = 0; i < sample.size() && rc == SV_OK; ++i) {
    if (forms[i] == SV_BATCH_RESIDENT) {
      res_chains.push_back(sample[i]);
    } else {
      rc = build_graph_form(b, sample[i], forms[i], n);
      graph_chains.push_back(sample[i]);
    }
  }
  if (rc == SV_OK) rc = build_resident(b, res_chains, &rs);
  cudaGraphExec_t ge = nullptr;
  std::vector<fsv::BlockGroup*> groups;
  if (rc == SV_OK) rc = make_graph(b, graph_chains, &rs, kPeriods, &ge, &groups);
  if (rc == SV_OK) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
              cudaGraphLaunch(ge, b->stream) == cudaSuccess &&  // warm-up
              cudaEventRecord(e0, b->stream) == cudaSuccess &&
              cudaGraphLaunch(ge, b->stream) == cudaSuccess &&
              cudaEventRecord(e1, b->stream) == cudaSuccess &&
              cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f)
      *rate = (double)sample.size() * kPeriods / (ms * 1e-3);
    if (!ok) rc = bfail(b, SV_ECUDA, "autotune run: %s", cudaGetErrorString(cudaGetLastError()));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  if (ge) cudaGraphExecDestroy(ge);
  free_groups(&groups);
  rs.release();
  for (int c : sample) {
    int r2 = reinit(b, c);
    if (rc == SV_OK) rc = r2;
  }
  return rc;
}

int time_form(sv_batch* b, const std::vector<int>& sample, int form, int n, double* rate) {
  return time_forms(b, sample, std::vector<int>(sample.size(), form), n, rate);
}

int autotune(sv_batch* b) {
  std::map<int, std::vector<int>> byL;
  for (int c = 0; c < b->n; ++c) byL[b->L[c]].push_back(c);
  for (auto& kv : byL) {
    const int L = kv.first;
    std::vector<int> sample(kv.second.begin(),
                            kv.second.begin() + std::min<size_t>(8, kv.second.size()));
    int best = SV_BATCH_PLAIN, best_n = 0;
    double best_rate = -1.0;
    for (int f : {SV_BATCH_RESIDENT, SV_BATCH_BLOCK_TC, SV_BATCH_BLOCK_SIMT, SV_BATCH_PLAIN,
                  SV_BATCH_MULTIGATE}) {
      if (!form_fits(f, L)) continue;
      for (int n : kSimtWidths) {
        // widths for the CUDA-core form
        if (f != SV_BATCH_BLOCK_SIMT && n != kDefaultWidth) continue;
        if (f == SV_BATCH_BLOCK_SIMT && n > L) continue;
        // a resident chain uses one CTA, so its form scales with the chain
        // count up to the SM count: it is timed on every chain of this L;
        // the other forms fill the device with one chain's passes (the
        // tensor-core form as one group of the sample)
        double rate = 0.0;
        int rc = time_form(b, f == SV_BATCH_RESIDENT ? kv.second : sample, f, n, &rate);
        if (rc) return rc;
        if (rate > best_rate) {
          best_rate = rate;
          best = f;
          best_n = f == SV_BATCH_BLOCK_TC ? 6 : (f == SV_BATCH_BLOCK_SIMT ? n : 0);
        }
      }
    }
    for (int c : kv.second) {
      b->form[c] = best;
      b->width[c] = best_n;
    }
  }
  return SV_OK;
}

int setup(sv_batch* b) {
  std::vector<int> graph_chains;
  for (int c = 0; c < b->n; ++c) {
    if (b->form[c] == SV_BATCH_RESIDENT) {
      b->res.push_back(c);
    } else {
      int rc = build_graph_form(b, c, b->form[c],
                                b->width[c] > 0 ? b->width[c] : kDefaultWidth);
      if (rc) return rc;
    }
  }
  ResidentSet rs;
  int rc = build_resident(b, b->res, &rs);
  if (rc) return rc;
  b->d_res = rs.d_res;
  b->d_rgates = rs.d_gates;
  b->d_rbonds = rs.d_bonds;
  b->d_rring = rs.d_ring;
  b->d_rcount = rs.d_count;
  b->res_maxL = rs.max_L;
  return SV_OK;
}

ResidentSet resident_view(const sv_batch* b) {
  ResidentSet rs;
  rs.d_res = b->d_res;
  rs.d_gates = b->d_rgates;
  rs.d_bonds = b->d_rbonds;
  rs.d_ring = b->d_rring;
  rs.d_count = b->d_rcount;
  rs.max_L = b->res_maxL;
  rs.count = (int)b->res.size();
  return rs;
}

void destroy(sv_batch* b) {
  if (!b) return;
  if (b->g1) cudaGraphExecDestroy(b->g1);
  if (b->gm) cudaGraphExecDestroy(b->gm);
  free_groups(&b->groups);
  ResidentSet rs = resident_view(b);
  rs.release();
  for (sv_ctx* c : b->ctx)
    if (c) sv_destroy(c);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

}  // namespace

extern "C" {

size_t sv_batch_state_bytes(int n_chains, const int* L) {
  if (n_chains <= 0 || !L) return 0;
  size_t total = 0;
  for (int c = 0; c < n_chains; ++c) {
    if (L[c] < 2 || L[c] > 34) return 0;
    total = (total + kAlign - 1) / kAlign * kAlign;
    total += sizeof(float2) << L[c];
  }
  return total;
}

int sv_batch_create(sv_batch** out, int device, int n_chains, const int* L,
                    const sv_floquet_params* params, const double* product_states,
                    void* state_dev, size_t bytes, int form, void* cuda_stream) {
  if (!out) return SV_EINVAL;
  *out = nullptr;
  if (n_chains <= 0 || !L || !params || !product_states || !state_dev) return SV_EINVAL;
  if (form < SV_BATCH_AUTO || form > SV_BATCH_MULTIGATE) return SV_EINVAL;
  const size_t need = sv_batch_state_bytes(n_chains, L);
  if (need == 0 || bytes < need) return SV_EINVAL;
  if (reinterpret_cast<uintptr_t>(state_dev) % kAlign != 0) return SV_EINVAL;
  for (int c = 0; c < n_chains; ++c) {
    if (!fsv::params_valid(L[c], params[c], nullptr)) return SV_EINVAL;
    if (params[c].n_period_params != 0) return SV_EINVAL;
    if (params[c].h_bonds || params[c].inverse) return SV_EUNSUPPORTED;
  }
  sv_batch* b = new (std::nothrow) sv_batch();
  if (!b) return SV_ENOMEM;
  b->device = device;
  b->n = n_chains;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->base = static_cast<char*>(state_dev);
  b->L.assign(L, L + n_chains);
  b->params.assign(params, params + n_chains);
  b->ctx.assign(n_chains, nullptr);
  size_t off = 0, sp = 0;
  for (int c = 0; c < n_chains; ++c) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    b->off.push_back(off);
    off += sizeof(float2) << L[c];
    b->spinors.push_back(product_states + sp);
    sp += 4 * (size_t)L[c];
  }
  int prev = -1;
  cudaGetDevice(&prev);
  int rc = SV_OK;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    rc = SV_ECUDA;
  }
  for (int c = 0; c < n_chains && rc == SV_OK; ++c) {
    rc = sv_create(&b->ctx[c], device, SV_C64, cuda_stream);
    if (rc == SV_OK) rc = sv_attach_state(b->ctx[c], b->base + b->off[c], sizeof(float2) << L[c]);
    if (rc == SV_OK) rc = reinit(b, c);
  }
  if (rc == SV_OK) {
    b->form.assign(n_chains, SV_BATCH_PLAIN);
    b->width.assign(n_chains, 0);
    if (form == SV_BATCH_AUTO) {
      rc = autotune(b);
    } else {
      for (int c = 0; c < n_chains; ++c) {
        b->form[c] = form_fits(form, L[c]) ? form : SV_BATCH_PLAIN;
        if (b->form[c] == SV_BATCH_BLOCK_TC || b->form[c] == SV_BATCH_BLOCK_SIMT)
          b->width[c] = kDefaultWidth;
      }
    }
  }
  if (rc == SV_OK) rc = setup(b);
  b->spinors.clear();
  if (prev >= 0) cudaSetDevice(prev);
  if (rc != SV_OK) {
    destroy(b);
    return rc;
  }
  *out = b;
  return SV_OK;
}

int sv_batch_evolve(sv_batch* b, int64_t periods, double* energy_out, double* norm_out) {
  if (!b) return SV_EINVAL;
  if (periods < 0) return bfail(b, SV_EINVAL, "periods must be >= 0");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev};
  std::vector<int> graph_chains;
  for (int c = 0; c < b->n; ++c)
    if (b->form[c] != SV_BATCH_RESIDENT) graph_chains.push_back(c);
  ResidentSet rs = resident_view(b);
  if (!b->g1) {
    int rc = make_graph(b, graph_chains, &rs, 1, &b->g1, &b->groups);
    if (rc) return rc;
  }
  if (!b->gm && periods >= b->M) {
    int rc = make_graph(b, graph_chains, &rs, b->M, &b->gm, &b->groups);
    if (rc) return rc;
  }
  const int ring = fsv::ctx_ring_len();
  int64_t done = 0;
  std::vector<double> rbuf;
  while (done < periods) {
    const int64_t chunk = std::min<int64_t>(periods - done, ring);
    int64_t k = 0;
    for (; b->gm && k + b->M <= chunk; k += b->M)
      BCUDA(cudaGraphLaunch(b->gm, b->stream), "graph launch");
    for (; k < chunk; ++k) BCUDA(cudaGraphLaunch(b->g1, b->stream), "graph launch");
    for (int c : graph_chains) {
      double* e = energy_out ? energy_out + (size_t)c * periods + done : nullptr;
      double* n = norm_out ? norm_out + (size_t)c * periods + done : nullptr;
      if (e || n) {
        int rc = fsv::ctx_read_energies(b->ctx[c], b->counter, chunk, e, n);
        if (rc) return bfail(b, rc, "chain %d: %s", c, sv_last_error(b->ctx[c]));
      }
      fsv::ctx_advance(b->ctx[c], chunk);
    }
    if (!b->res.empty() && (energy_out || norm_out)) {
      rbuf.resize(2 * (size_t)ring * b->res.size());
      BCUDA(cudaMemcpyAsync(rbuf.data(), b->d_rring, sizeof(double) * rbuf.size(),
                            cudaMemcpyDeviceToHost, b->stream),
            "resident ring readback");
      BCUDA(cudaStreamSynchronize(b->stream), "synchronize");
      for (size_t r = 0; r < b->res.size(); ++r) {
        const int c = b->res[r];
        for (int64_t q = 0; q < chunk; ++q) {
          const int64_t slot = (b->counter + q) % ring;
          const double* src = rbuf.data() + 2 * ((size_t)ring * r + slot);
          if (energy_out) energy_out[(size_t)c * periods + done + q] = src[0];
          if (norm_out) norm_out[(size_t)c * periods + done + q] = src[1];
        }
      }
    }
    b->counter += chunk;
    done += chunk;
  }
  BCUDA(cudaStreamSynchronize(b->stream), "synchronize");
  return SV_OK;
}

int sv_batch_forms(const sv_batch* b, int* form_out) {
  if (!b || !form_out) return SV_EINVAL;
  for (int c = 0; c < b->n; ++c) form_out[c] = b->form[c];
  return SV_OK;
}

int sv_batch_widths(const sv_batch* b, int* n_out) {
  if (!b || !n_out) return SV_EINVAL;
  for (int c = 0; c < b->n; ++c) n_out[c] = b->width[c];
  return SV_OK;
}

const char* sv_batch_last_error(const sv_batch* b) { return b ? b->err.c_str() : ""; }

void sv_batch_destroy(sv_batch* b) { destroy(b); }

}  // extern "C"
