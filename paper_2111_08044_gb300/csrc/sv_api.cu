// C ABI of the simulator (include/floquet_sv.h): context, state attachment,
// period construction, evolution under a captured CUDA graph, energy
// readback.  All device work goes to the caller's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <limits>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "sv_batch.h"
#include "sv_block.h"
#include "sv_internal.h"
#include "sv_kernels.h"

using fsv::cd;

namespace {
constexpr int kRing = 1024;  // energy ring (periods between host readbacks)
}

struct sv_ctx {
  int device = 0;
  int precision = SV_C64;
  cudaStream_t stream = nullptr;      // caller's stream
  cudaStream_t cap_stream = nullptr;  // internal stream used only for capture
  fsv::LaunchCfg cfg;

  void* state = nullptr;
  size_t state_bytes = 0;
  int L = 0;
  bool inited = false;
  bool built = false;
  int64_t counter = 0;  // host mirror of the device period counter

  sv_floquet_params params{};
  std::vector<double> theta_p, hx_p;
  int64_t n_period_params = 0;
  std::vector<fsv::Gate2> gates;  // period 0 (the layout of every period)
  fsv::Observable obs;

  // device buffers owned by the library
  void* d_gates = nullptr;  // [n_tables][n_gates][16] complex
  size_t d_gates_bytes = 0;
  void* d_ident = nullptr;  // identity 4x4 (measurement passes)
  double* d_spinors = nullptr;
  double* d_part_evolve = nullptr;
  double* d_part_meas = nullptr;
  int part_slots_evolve = 0, part_slots_meas = 0;
  int maxb = 0;
  double* d_ring = nullptr;
  double* d_meas = nullptr;
  long long* d_counter = nullptr;
  fsv::BlockPlan* block = nullptr;  // block-mode plan and buffers
  std::vector<fsv::MultiArgs> mg;   // multi-gate passes of a period
  int* d_mg = nullptr;              // their gate indices and tile bits

  cudaGraphExec_t graph = nullptr;       // one period
  cudaGraphExec_t graph_exit = nullptr;  // an evolution's last period (block plans
                                         // whose periods start off site 0)
  bool cyclic = true;  // block plans may start their periods off site 0
  // Between evolve calls the state is in the natural layout unless the
  // caller asked to keep the period layout (sv_set_layout_policy); then
  // in_period_layout says whether it currently is in the plan's start layout.
  bool keep_layout = false;
  bool in_period_layout = false;

  int launches_per_period = 0;
  int passes_per_period = 0;
  size_t build_bytes = 0;
  std::string err;
};

namespace {

int fail(sv_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int cuda_fail(sv_ctx* c, cudaError_t e, const char* what) {
  return fail(c, SV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SV_CUDA(call, what)                         \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

size_t amp_bytes(int precision) { return precision == SV_C64 ? 8 : 16; }

void drop_graph(sv_ctx* ctx) {
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  if (ctx->graph_exit) {
    cudaGraphExecDestroy(ctx->graph_exit);
    ctx->graph_exit = nullptr;
  }
}

// Block plans whose periods start at a window off site 0 keep the state in
// that window's layout between periods: an evolution begins with relabel
// steps into it and its last period hands back the natural layout.
bool off_natural(const sv_ctx* ctx) {
  return ctx->params.mode == SV_MODE_BLOCK && ctx->block && ctx->block->start != 0;
}

void free_build(sv_ctx* ctx) {
  drop_graph(ctx);
  cudaFree(ctx->d_gates);
  ctx->d_gates = nullptr;
  ctx->d_gates_bytes = 0;
  cudaFree(ctx->d_part_evolve);
  ctx->d_part_evolve = nullptr;
  cudaFree(ctx->d_mg);
  ctx->d_mg = nullptr;
  ctx->mg.clear();
  if (ctx->block) {
    fsv::block_free(ctx->block);
    ctx->block = nullptr;
  }
  ctx->built = false;
}

fsv::EpiParams epi_for(const sv_ctx* ctx, int flags, int bond, double* partial) {
  fsv::EpiParams ep;
  ep.flags = flags;
  const fsv::Observable& o = ctx->obs;
  if (flags & fsv::EPI_X_HI) ep.cx_hi = o.cx[bond];
  if (flags & fsv::EPI_X_LO) ep.cx_lo = o.cx[bond + 1];
  if (flags & fsv::EPI_DIAG) {
    ep.J = o.J;
    ep.cz_first = o.cz[0];
    ep.cz_last = o.cz[o.L - 1];
    ep.cz_bulk = o.L >= 3 ? o.cz[1] : 0.0;
  }
  ep.partial = partial;
  return ep;
}

fsv::Renorm renorm_of(const sv_ctx* ctx) {
  fsv::Renorm rn;
  if (ctx->params.renorm_every > 0) {
    rn.ring = ctx->d_ring;
    rn.ring_len = kRing;
    rn.counter = ctx->d_counter;
    rn.every = ctx->params.renorm_every;
  }
  return rn;
}

// Enqueue one multi-gate period on stream s; ev (nullable) as for the
// profiled plain period, one event before each pass.
int enqueue_multigate_period(sv_ctx* ctx, cudaStream_t s, cudaEvent_t* ev) {
  const size_t P = ctx->mg.size();
  for (size_t k = 0; k < P; ++k) {
    fsv::MultiArgs ma = ctx->mg[k];
    if (k == 0) ma.ep.rn = renorm_of(ctx);
    if (ev) SV_CUDA(cudaEventRecord(ev[k], s), "event record");
    SV_CUDA(fsv::launch_multigate(ma, ctx->state, ctx->cfg, s), "multi-gate launch");
  }
  if (ev) SV_CUDA(cudaEventRecord(ev[P], s), "event record");
  SV_CUDA(fsv::launch_period_reduce(ctx->d_part_evolve,
                                    (long long)ctx->part_slots_evolve * ctx->maxb, ctx->L,
                                    ctx->d_ring, kRing, ctx->d_counter, 1, s),
          "period reduce launch");
  if (ev) SV_CUDA(cudaEventRecord(ev[P + 1], s), "event record");
  return SV_OK;
}

// Enqueue one plain-mode period on stream s.
int enqueue_plain_period(sv_ctx* ctx, cudaStream_t s) {
  if (ctx->params.mode == SV_MODE_MULTIGATE) return enqueue_multigate_period(ctx, s, nullptr);
  const int ng = (int)ctx->gates.size();
  const size_t cbytes = amp_bytes(ctx->precision);
  const long long stride = ctx->n_period_params > 0 ? (long long)ng * fsv::kGateEntries : 0;
  int slot = 0;
  for (int g = 0; g < ng; ++g) {
    const fsv::Gate2& gt = ctx->gates[g];
    double* part = gt.epi ? ctx->d_part_evolve + (size_t)slot * ctx->maxb * 2 : nullptr;
    if (gt.epi) ++slot;
    fsv::EpiParams ep = epi_for(ctx, gt.epi, gt.bond, part);
    if (g == 0) ep.rn = renorm_of(ctx);
    const char* gb = static_cast<const char*>(ctx->d_gates) + (size_t)g * fsv::kGateEntries * cbytes;
    SV_CUDA(fsv::launch_plain_gate(ctx->precision, ctx->state, ctx->L, gt.bond, gb, stride,
                                   ctx->d_counter, ep, 1, ctx->cfg, s),
            "plain gate launch");
  }
  SV_CUDA(fsv::launch_period_reduce(ctx->d_part_evolve,
                                    (long long)ctx->part_slots_evolve * ctx->maxb, ctx->L,
                                    ctx->d_ring, kRing, ctx->d_counter, 1, s),
          "period reduce launch");
  return SV_OK;
}

int enqueue_period(sv_ctx* ctx, cudaStream_t s, bool last = false) {
  if (ctx->params.mode == SV_MODE_BLOCK) {
    cudaError_t e = fsv::block_enqueue_period(ctx->block, ctx->state, ctx->d_counter,
                                              ctx->d_ring, kRing, s, last);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "block period launch");
    return SV_OK;
  }
  return enqueue_plain_period(ctx, s);
}

int capture_period(sv_ctx* ctx, bool last, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  SV_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed),
          "begin capture");
  int rc = enqueue_period(ctx, ctx->cap_stream, last);
  cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
  if (rc != SV_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return cuda_fail(ctx, e, "graph instantiate");
  }
  return SV_OK;
}

int ensure_graph(sv_ctx* ctx) {
  if (!ctx->graph) {
    int rc = capture_period(ctx, false, &ctx->graph);
    if (rc) return rc;
  }
  if (off_natural(ctx) && !ctx->graph_exit) return capture_period(ctx, true, &ctx->graph_exit);
  return SV_OK;
}

// Launch `count` periods; the state enters the period layout first if it is
// not there, and `last` (the call's last periods) hands back the natural
// layout unless the caller keeps the period layout between calls.
int launch_periods(sv_ctx* ctx, int64_t count, bool last) {
  const bool off = off_natural(ctx);
  if (count <= 0) return SV_OK;
  if (off && !ctx->in_period_layout) {
    cudaError_t e = fsv::block_enqueue_entry(ctx->block, ctx->state, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "relabel launch");
    ctx->in_period_layout = true;
  }
  for (int64_t k = 0; k < count; ++k) {
    const bool exit = off && last && !ctx->keep_layout && k + 1 == count;
    SV_CUDA(cudaGraphLaunch(exit ? ctx->graph_exit : ctx->graph, ctx->stream), "graph launch");
    if (exit) ctx->in_period_layout = false;
    ++ctx->counter;
  }
  return SV_OK;
}

// Bring a state kept in the period layout back to the natural layout.
int ensure_natural(sv_ctx* ctx) {
  if (!ctx->in_period_layout) return SV_OK;
  DeviceGuard dg(ctx->device);
  if (ctx->block) {
    cudaError_t e = fsv::block_enqueue_leave(ctx->block, ctx->state, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "relabel launch");
  }
  ctx->in_period_layout = false;
  return SV_OK;
}

int read_ring(sv_ctx* ctx, int64_t c0, int64_t count, double* e_out, double* n_out);

}  // namespace

// Hooks for the batch executor (sv_batch.cu); not part of the C ABI.
namespace fsv {

int ctx_capture_run(sv_ctx* ctx, int64_t periods, cudaGraph_t* out) {
  *out = nullptr;
  if (!ctx || !ctx->built) return SV_ESTATE;
  DeviceGuard dg(ctx->device);
  SV_CUDA(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed),
          "begin capture");
  int rc = SV_OK;
  if (off_natural(ctx) && periods > 0) {
    cudaError_t e = fsv::block_enqueue_entry(ctx->block, ctx->state, ctx->cap_stream);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "relabel launch");
  }
  for (int64_t k = 0; k < periods && rc == SV_OK; ++k)
    rc = enqueue_period(ctx, ctx->cap_stream, k + 1 == periods);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
  if (rc != SV_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
  *out = g;
  return SV_OK;
}

void ctx_advance(sv_ctx* ctx, int64_t periods) { ctx->counter += periods; }

void ctx_set_min_tiles(sv_ctx* ctx, int tiles) { ctx->cfg.min_tiles_per_cta = tiles; }

void ctx_set_cyclic(sv_ctx* ctx, bool cyclic) { ctx->cyclic = cyclic; }

int ctx_read_energies(sv_ctx* ctx, int64_t c0, int64_t count, double* e, double* n) {
  return read_ring(ctx, c0, count, e, n);
}

int ctx_ring_len() { return kRing; }

int ctx_block_member(sv_ctx* ctx, BlockPlan** plan, void** psi, long long** counter,
                     double** ring) {
  if (!ctx || !ctx->built || ctx->params.mode != SV_MODE_BLOCK || !ctx->block ||
      !ctx->block->tensor_cores)
    return SV_ESTATE;
  *plan = ctx->block;
  *psi = ctx->state;
  *counter = ctx->d_counter;
  *ring = ctx->d_ring;
  return SV_OK;
}

namespace {
double unitarity_defect(const double* re, const double* im) {
  double d = 0.0, tr = 0.0;
  for (int k = 0; k < 4; ++k)
    for (int l = 0; l < 4; ++l) {
      double sr = 0.0, si = 0.0;  // (M^dagger M)_{kl} = sum_i conj(M_ik) M_il
      for (int i = 0; i < 4; ++i) {
        sr += re[4 * i + k] * re[4 * i + l] + im[4 * i + k] * im[4 * i + l];
        si += re[4 * i + k] * im[4 * i + l] - im[4 * i + k] * re[4 * i + l];
      }
      if (k == l) {
        sr -= 1.0;
        tr += sr;
      }
      d += sr * sr + si * si;
    }
  return d + tr * tr;
}
}  // namespace

void round_unitary4(const cd* m, float2* out) {
  float f[32];
  double re[16], im[16];
  for (int k = 0; k < 16; ++k) {
    f[2 * k] = (float)m[k].real();
    f[2 * k + 1] = (float)m[k].imag();
  }
  auto load = [&]() {
    for (int k = 0; k < 16; ++k) {
      re[k] = f[2 * k];
      im[k] = f[2 * k + 1];
    }
  };
  load();
  double best = unitarity_defect(re, im);
  for (int sweep = 0; sweep < 20; ++sweep) {
    bool moved = false;
    for (int e = 0; e < 32; ++e) {
      const float orig = f[e];
      for (int dir = -1; dir <= 1; dir += 2) {
        f[e] = std::nextafter(orig, dir > 0 ? INFINITY : -INFINITY);
        load();
        const double d = unitarity_defect(re, im);
        if (d < best) {
          best = d;
          moved = true;
          break;
        }
        f[e] = orig;
      }
    }
    if (!moved) break;
  }
  for (int k = 0; k < 16; ++k) out[k] = make_float2(f[2 * k], f[2 * k + 1]);
}

}  // namespace fsv

namespace {

int check_ready(sv_ctx* ctx, bool need_built) {
  if (!ctx) return SV_EINVAL;
  if (!ctx->state) return fail(ctx, SV_ESTATE, "no state buffer attached");
  if (!ctx->inited) return fail(ctx, SV_ESTATE, "sv_init has not been called");
  if (need_built && !ctx->built) return fail(ctx, SV_ESTATE, "sv_build_floquet has not been called");
  return SV_OK;
}

// Read-only measurement of <H0> and the norm of the current state.
int measure(sv_ctx* ctx, double* e_out, double* n_out) {
  const int L = ctx->L;
  struct Item {
    int bond, flags;
  };
  std::vector<Item> items;
  for (int b = 0; b + 1 < L; b += 2)
    items.push_back({b, fsv::EPI_X_HI | fsv::EPI_X_LO | (b == 0 ? fsv::EPI_DIAG : 0)});
  if (L % 2 == 1) items.push_back({L - 2, fsv::EPI_X_LO});
  SV_CUDA(cudaMemsetAsync(ctx->d_part_meas, 0,
                          sizeof(double) * 2 * ctx->maxb * ctx->part_slots_meas, ctx->stream),
          "memset partials");
  for (size_t k = 0; k < items.size(); ++k) {
    fsv::EpiParams ep = epi_for(ctx, items[k].flags, items[k].bond,
                                ctx->d_part_meas + k * ctx->maxb * 2);
    SV_CUDA(fsv::launch_plain_gate(ctx->precision, ctx->state, L, items[k].bond,
                                   ctx->d_ident, 0, ctx->d_counter, ep, 0, ctx->cfg,
                                   ctx->stream),
            "measurement launch");
  }
  SV_CUDA(fsv::launch_period_reduce(ctx->d_part_meas, (long long)items.size() * ctx->maxb, L,
                                    ctx->d_meas, 1, ctx->d_counter, 0, ctx->stream),
          "measurement reduce");
  double h[2];
  SV_CUDA(cudaMemcpyAsync(h, ctx->d_meas, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream),
          "copy energy");
  SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
  if (e_out) *e_out = h[0];
  if (n_out) *n_out = h[1];
  return SV_OK;
}

// Copy ring slots of periods c0 .. c0+count-1 (count <= kRing) to the host.
int read_ring(sv_ctx* ctx, int64_t c0, int64_t count, double* e_out, double* n_out) {
  std::vector<double> buf(2 * (size_t)count);
  const int64_t s0 = c0 % kRing;
  const int64_t first = std::min<int64_t>(count, kRing - s0);
  SV_CUDA(cudaMemcpyAsync(buf.data(), ctx->d_ring + 2 * s0, sizeof(double) * 2 * first,
                          cudaMemcpyDeviceToHost, ctx->stream),
          "copy ring");
  if (first < count)
    SV_CUDA(cudaMemcpyAsync(buf.data() + 2 * first, ctx->d_ring,
                            sizeof(double) * 2 * (count - first), cudaMemcpyDeviceToHost,
                            ctx->stream),
            "copy ring");
  SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
  // a general two-site chain is not measured per period
  const double nan = std::numeric_limits<double>::quiet_NaN();
  for (int64_t k = 0; k < count; ++k) {
    if (e_out) e_out[k] = ctx->obs.general ? nan : buf[2 * k];
    if (n_out) n_out[k] = ctx->obs.general ? nan : buf[2 * k + 1];
  }
  if (ctx->block && fsv::block_status(ctx->block, ctx->stream) != 0)
    return fail(ctx, SV_ETIMEOUT, "a tensor-core block pass gave up a bounded wait");
  return SV_OK;
}

// E = <H0>, sigma_E and <psi|psi> of the current state (Ising or general
// two-site chain), partials summed on the host in a fixed order.
int energy_moments(sv_ctx* ctx, double* energy, double* sigma_e, double* norm2) {
  const int grid = fsv::moments_grid(ctx->cfg);
  const bool c128 = ctx->precision == SV_C128;
  const size_t nh = ctx->obs.general ? ctx->obs.h.size() : 0;
  const size_t hb_bytes = nh * (c128 ? sizeof(double2) : sizeof(float2));
  char* d_buf = nullptr;
  SV_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d_buf), hb_bytes + sizeof(double) * 3 * grid,
                          ctx->stream),
          "moments scratch");
  double* d_part = reinterpret_cast<double*>(d_buf + hb_bytes);
  std::vector<double> part((size_t)3 * grid);
  std::vector<double2> h64;
  std::vector<float2> h32;
  cudaError_t e = cudaSuccess;
  if (ctx->obs.general) {
    for (const fsv::cd& v : ctx->obs.h) {
      h64.push_back(make_double2(v.real(), v.imag()));
      h32.push_back(make_float2((float)v.real(), (float)v.imag()));
    }
    e = cudaMemcpyAsync(d_buf, c128 ? (const void*)h64.data() : (const void*)h32.data(), hb_bytes,
                        cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = fsv::launch_bond_moments(ctx->precision, ctx->state, ctx->L, d_buf, d_part, ctx->cfg,
                                   ctx->stream);
  } else {
    fsv::H0Coef h;
    h.J = ctx->obs.J;
    for (int i = 0; i < ctx->L; ++i) {
      h.cx[i] = ctx->obs.cx[i];
      h.cz[i] = ctx->obs.cz[i];
    }
    e = fsv::launch_h0_moments(ctx->precision, ctx->state, ctx->L, h, d_part, ctx->cfg,
                               ctx->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * part.size(),
                        cudaMemcpyDeviceToHost, ctx->stream);
  // the host buffers must outlive the copies above
  const cudaError_t es = cudaStreamSynchronize(ctx->stream);
  cudaFreeAsync(d_buf, ctx->stream);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "energy moments");
  double s1 = 0.0, s2 = 0.0, sn = 0.0;  // fixed order
  for (int b = 0; b < grid; ++b) {
    s1 += part[3 * b];
    s2 += part[3 * b + 1];
    sn += part[3 * b + 2];
  }
  if (!(sn > 0.0)) return fail(ctx, SV_ESTATE, "the state has zero norm");
  const double E = s1 / sn, var = s2 / sn - E * E;
  if (energy) *energy = E;
  if (sigma_e) *sigma_e = std::sqrt(std::max(var, 0.0));
  if (norm2) *norm2 = sn;
  return SV_OK;
}

// FP64 tables of a product of site-group factors (group = 1: spinors, L x 4
// doubles; group = 2: pair states, L/2 x 8 doubles with local index
// r = 2 b_{2k} + b_{2k+1}), each factor normalised: lo over the low m sites,
// hi over the rest.
int factor_tables(sv_ctx* ctx, int L, int group, const double* factors, int* m_out,
                  std::vector<double>* lo, std::vector<double>* hi) {
  const int ng = L / group, width = 1 << group;
  std::vector<std::complex<double>> f((size_t)ng * width);
  for (int g = 0; g < ng; ++g) {
    double n2 = 0.0;
    for (int r = 0; r < width; ++r) {
      f[(size_t)g * width + r] = {factors[2 * (g * width + r)], factors[2 * (g * width + r) + 1]};
      n2 += std::norm(f[(size_t)g * width + r]);
    }
    if (!(n2 > 0.0) || !std::isfinite(n2))
      return fail(ctx, SV_EINVAL, "factor %d has zero or non-finite norm", g);
    for (int r = 0; r < width; ++r) f[(size_t)g * width + r] /= std::sqrt(n2);
  }
  const int m = std::min(L, 12) / group * group;
  auto table = [&](int first, int count, std::vector<double>* t) {
    t->assign(2ull << count, 0.0);
    for (uint64_t x = 0; x < (1ull << count); ++x) {
      std::complex<double> v = 1.0;
      for (int s = 0; s < count; s += group) {
        int r = 0;  // the group's local index, its lowest site the high bit
        for (int k = 0; k < group; ++k) r = 2 * r + (int)((x >> (s + k)) & 1);
        v *= f[(size_t)((first + s) / group) * width + r];
      }
      (*t)[2 * x] = v.real();
      (*t)[2 * x + 1] = v.imag();
    }
  };
  table(0, m, lo);
  table(m, L - m, hi);
  *m_out = m;
  return SV_OK;
}

// <phi|psi> for the product of site-group factors phi (see factor_tables).
int product_overlap(sv_ctx* ctx, int group, const double* factors, double* overlap_re,
                    double* overlap_im) {
  const int L = ctx->L;
  std::vector<double> lo, hi;
  int m = 0;
  int rc = factor_tables(ctx, L, group, factors, &m, &lo, &hi);
  if (rc) return rc;
  DeviceGuard dg(ctx->device);
  const int grid = fsv::moments_grid(ctx->cfg);
  const size_t lo_b = sizeof(double) * lo.size(), hi_b = sizeof(double) * hi.size();
  char* d_buf = nullptr;
  SV_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d_buf), lo_b + hi_b + sizeof(double) * 2 * grid,
                          ctx->stream),
          "overlap scratch");
  double* d_part = reinterpret_cast<double*>(d_buf + lo_b + hi_b);
  std::vector<double> part((size_t)2 * grid);
  cudaError_t e = cudaMemcpyAsync(d_buf, lo.data(), lo_b, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_buf + lo_b, hi.data(), hi_b, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = fsv::launch_product_overlap(ctx->precision, ctx->state, L, m, d_buf, d_buf + lo_b,
                                    d_part, ctx->cfg, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * part.size(),
                        cudaMemcpyDeviceToHost, ctx->stream);
  // the host tables must outlive the copies above
  const cudaError_t es = cudaStreamSynchronize(ctx->stream);
  cudaFreeAsync(d_buf, ctx->stream);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "product overlap");
  double re = 0.0, im = 0.0;  // fixed order
  for (int b = 0; b < grid; ++b) {
    re += part[2 * b];
    im += part[2 * b + 1];
  }
  if (overlap_re) *overlap_re = re;
  if (overlap_im) *overlap_im = im;
  return SV_OK;
}

// One period with an event recorded before each launch and after the last.
int enqueue_period_profiled(sv_ctx* ctx, cudaStream_t s, cudaEvent_t* ev, bool last) {
  if (ctx->params.mode == SV_MODE_BLOCK) {
    cudaError_t e = fsv::block_enqueue_period_events(ctx->block, ctx->state, ctx->d_counter,
                                                     ctx->d_ring, kRing, s, ev, last);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "block period launch");
    return SV_OK;
  }
  if (ctx->params.mode == SV_MODE_MULTIGATE) return enqueue_multigate_period(ctx, s, ev);
  const int ng = (int)ctx->gates.size();
  const size_t cbytes = amp_bytes(ctx->precision);
  const long long stride = ctx->n_period_params > 0 ? (long long)ng * fsv::kGateEntries : 0;
  int slot = 0;
  for (int g = 0; g < ng; ++g) {
    const fsv::Gate2& gt = ctx->gates[g];
    double* part = gt.epi ? ctx->d_part_evolve + (size_t)slot * ctx->maxb * 2 : nullptr;
    if (gt.epi) ++slot;
    fsv::EpiParams ep = epi_for(ctx, gt.epi, gt.bond, part);
    if (g == 0) ep.rn = renorm_of(ctx);
    const char* gb = static_cast<const char*>(ctx->d_gates) + (size_t)g * fsv::kGateEntries * cbytes;
    SV_CUDA(cudaEventRecord(ev[g], s), "event record");
    SV_CUDA(fsv::launch_plain_gate(ctx->precision, ctx->state, ctx->L, gt.bond, gb, stride,
                                   ctx->d_counter, ep, 1, ctx->cfg, s),
            "plain gate launch");
  }
  SV_CUDA(cudaEventRecord(ev[ng], s), "event record");
  SV_CUDA(fsv::launch_period_reduce(ctx->d_part_evolve,
                                    (long long)ctx->part_slots_evolve * ctx->maxb, ctx->L,
                                    ctx->d_ring, kRing, ctx->d_counter, 1, s),
          "period reduce launch");
  SV_CUDA(cudaEventRecord(ev[ng + 1], s), "event record");
  return SV_OK;
}

// Defect of D = M^dagger M - I (4x4, FP64): |D|_F^2 + tr(D)^2.  The trace
// term is the mean norm change per application on a maximally mixed pair.

// FP32 copy of a 4x4 unitary: nearest rounding, then a coordinate descent
// over one-ulp moves of each entry that lowers the distance of the FP32
// matrix from unitarity (a plain rounding leaves a defect whose sign repeats
// every time the gate is applied, so the norm would drift steadily).

// The multi-gate passes of a period: per pass its gates' indices and tile
// bits (one device array for all passes), the sites whose <X> it measures,
// and the diagonal part on the period's last pass.
int build_multigate(sv_ctx* ctx, const std::vector<fsv::MultiPass>& plan) {
  const int L = ctx->L;
  const int tb = L < fsv::kMgTileBits ? L : fsv::kMgTileBits;
  std::vector<int> idx;
  std::vector<size_t> at;
  for (const auto& mp : plan) {
    at.push_back(idx.size());
    for (int g : mp.gates) idx.push_back(g);
    const int A = L <= fsv::kMgTileBits ? 4 : std::max(mp.lo, 4);
    for (int g : mp.gates) {
      const int b = ctx->gates[g].bond;
      idx.push_back(b < 4 ? b : b - A + 4);
    }
  }
  if (!idx.empty()) {
    if (cudaMalloc(&ctx->d_mg, sizeof(int) * idx.size()) != cudaSuccess) {
      cudaGetLastError();
      ctx->d_mg = nullptr;
      return fail(ctx, SV_ENOMEM, "multi-gate plan allocation failed");
    }
    SV_CUDA(cudaMemcpy(ctx->d_mg, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice),
            "upload multi-gate plan");
  }
  SV_CUDA(fsv::multigate_prepare(), "multi-gate shared-memory opt-in");
  const int ng = (int)ctx->gates.size();
  int slot = 0;
  for (size_t k = 0; k < plan.size(); ++k) {
    const fsv::MultiPass& mp = plan[k];
    fsv::MultiArgs ma;
    ma.L = L;
    ma.tb = tb;
    ma.A = L <= fsv::kMgTileBits ? 4 : std::max(mp.lo, 4);
    ma.ngates = (int)mp.gates.size();
    ma.gidx = ctx->d_mg + at[k];
    ma.gq = ctx->d_mg + at[k] + mp.gates.size();
    ma.gates = static_cast<const float2*>(ctx->d_gates);
    ma.stride = ctx->n_period_params > 0 ? (long long)ng * fsv::kGateEntries : 0;
    ma.counter = ctx->d_counter;
    const bool measures = !ctx->obs.general && (!mp.x_sites.empty() || mp.diag);
    if (measures) {
      for (int site : mp.x_sites) {
        if (ma.nx >= fsv::kMgMaxX) return fail(ctx, SV_EINVAL, "too many measured sites");
        ma.xq[ma.nx] = site < 4 ? site : site - ma.A + 4;
        ma.xc[ma.nx] = (float)ctx->obs.cx[site];
        ++ma.nx;
      }
      ma.diag = mp.diag ? 1 : 0;
      ma.ep = epi_for(ctx, mp.diag ? fsv::EPI_DIAG : 0, 0,
                      ctx->d_part_evolve + (size_t)slot * ctx->maxb * 2);
      ++slot;
    }
    ctx->mg.push_back(ma);
  }
  ctx->passes_per_period = (int)plan.size();
  ctx->launches_per_period = (int)plan.size() + 1;
  ctx->build_bytes = ctx->d_gates_bytes + sizeof(int) * idx.size();
  return SV_OK;
}

void upload_gates(const std::vector<fsv::Gate2>& gates, std::vector<float2>& out, size_t at) {
  for (size_t g = 0; g < gates.size(); ++g) {
    float2* e = &out[at + fsv::kGateEntries * g];
    fsv::round_unitary4(gates[g].m, e);
    for (int k = 0; k < 16; ++k)
      e[16 + k] = make_float2((float)(gates[g].m[k].real() - (double)e[k].x),
                              (float)(gates[g].m[k].imag() - (double)e[k].y));
  }
}

// double-float entries (re hi, re lo, im hi, im lo): hi the nearest float,
// lo the nearest float to the remainder; zero residual entries
float2 split_df(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}
void upload_gates(const std::vector<fsv::Gate2>& gates, std::vector<float4>& out, size_t at) {
  for (size_t g = 0; g < gates.size(); ++g)
    for (int k = 0; k < 16; ++k) {
      const float2 re = split_df(gates[g].m[k].real()), im = split_df(gates[g].m[k].imag());
      out[at + fsv::kGateEntries * g + k] = make_float4(re.x, re.y, im.x, im.y);
      out[at + fsv::kGateEntries * g + 16 + k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

void upload_gates(const std::vector<fsv::Gate2>& gates, std::vector<double2>& out, size_t at) {
  for (size_t g = 0; g < gates.size(); ++g)
    for (int k = 0; k < 16; ++k) {
      out[at + fsv::kGateEntries * g + k] =
          make_double2(gates[g].m[k].real(), gates[g].m[k].imag());
      out[at + fsv::kGateEntries * g + 16 + k] = make_double2(0.0, 0.0);
    }
}

// The gate tables of every period-parameter set, in the context's entry type.
template <typename E>
int upload_tables(sv_ctx* ctx, const sv_floquet_params& p, int64_t ntab, int ng) {
  std::vector<E> tab((size_t)ntab * ng * fsv::kGateEntries);
  for (int64_t k = 0; k < ntab; ++k) {
    auto gk = k == 0 ? ctx->gates : fsv::period_gates(ctx->L, p, ctx->theta_p[k], ctx->hx_p[k]);
    upload_gates(gk, tab, (size_t)k * ng * fsv::kGateEntries);
  }
  SV_CUDA(cudaMemcpyAsync(ctx->d_gates, tab.data(), ctx->d_gates_bytes, cudaMemcpyHostToDevice,
                          ctx->stream),
          "upload gates");
  SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
  return SV_OK;
}

// SV_DF64 state read-out (to_host) or write-in as complex128 amplitudes,
// through a device buffer of at most 64 MiB converted chunk by chunk.
int df_transfer(sv_ctx* ctx, void* host, bool to_host) {
  const uint64_t n = 1ull << ctx->L;
  const uint64_t chunk = std::min<uint64_t>(n, (64ull << 20) / 16);
  void* d_tmp = nullptr;
  SV_CUDA(cudaMallocAsync(&d_tmp, chunk * 16, ctx->stream), "conversion buffer");
  cudaError_t e = cudaSuccess;
  char* h = static_cast<char*>(host);
  char* st = static_cast<char*>(ctx->state);
  for (uint64_t at = 0; at < n && e == cudaSuccess; at += chunk) {
    const uint64_t m = std::min(chunk, n - at);
    if (to_host) {
      e = fsv::launch_df_convert(st + 16 * at, d_tmp, m, 1, ctx->cfg, ctx->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h + 16 * at, d_tmp, 16 * m, cudaMemcpyDefault, ctx->stream);
    } else {
      e = cudaMemcpyAsync(d_tmp, h + 16 * at, 16 * m, cudaMemcpyDefault, ctx->stream);
      if (e == cudaSuccess)
        e = fsv::launch_df_convert(d_tmp, st + 16 * at, m, 0, ctx->cfg, ctx->stream);
    }
    // the host chunk and the buffer are reused by the next iteration
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  cudaFreeAsync(d_tmp, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "double-float state transfer");
  return SV_OK;
}

// Calls that have no double-float kernels.
int no_df(sv_ctx* ctx, const char* what) {
  return fail(ctx, SV_EUNSUPPORTED, "%s needs SV_C64 or SV_C128", what);
}

}  // namespace

extern "C" {

int sv_version(void) { return 2; }

int sv_create(sv_ctx** out, int device, int precision, void* cuda_stream) {
  if (!out) return SV_EINVAL;
  *out = nullptr;
  if (precision != SV_C64 && precision != SV_C128 && precision != SV_DF64) return SV_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SV_ECUDA;
  }
  sv_ctx* ctx = new (std::nothrow) sv_ctx();
  if (!ctx) return SV_ENOMEM;
  ctx->device = device;
  ctx->precision = precision;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard dg(device);
  if (!dg.ok) {
    delete ctx;
    return SV_ECUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return SV_ECUDA;
  }
  ctx->cfg.num_sms = prop.multiProcessorCount;
  ctx->maxb = ctx->cfg.num_sms * 4;
  ctx->part_slots_meas = 18;  // ceil(34 / 2) + 1 measurement passes at most
  bool ok = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaMalloc(&ctx->d_spinors, sizeof(double) * 4 * 40) == cudaSuccess;
  ok = ok && cudaMalloc(&ctx->d_ring, sizeof(double) * 2 * kRing) == cudaSuccess;
  ok = ok && cudaMalloc(&ctx->d_meas, sizeof(double) * 2) == cudaSuccess;
  ok = ok && cudaMalloc(&ctx->d_counter, sizeof(long long)) == cudaSuccess;
  ok = ok && cudaMalloc(&ctx->d_ident, 16 * fsv::kGateEntries) == cudaSuccess;
  ok = ok && cudaMalloc(&ctx->d_part_meas, sizeof(double) * 2 * ctx->maxb *
                                               ctx->part_slots_meas) == cudaSuccess;
  if (ok) {
    if (precision == SV_C128) {
      double2 id[fsv::kGateEntries] = {};  // identity, zero residual
      for (int k = 0; k < 4; ++k) id[5 * k].x = 1.0;
      ok = cudaMemcpy(ctx->d_ident, id, sizeof(id), cudaMemcpyHostToDevice) == cudaSuccess;
    } else if (precision == SV_DF64) {
      float4 id[fsv::kGateEntries] = {};  // (re hi, re lo, im hi, im lo)
      for (int k = 0; k < 4; ++k) id[5 * k].x = 1.0f;
      ok = cudaMemcpy(ctx->d_ident, id, sizeof(id), cudaMemcpyHostToDevice) == cudaSuccess;
    } else {
      float2 id[fsv::kGateEntries] = {};
      for (int k = 0; k < 4; ++k) id[5 * k].x = 1.0f;
      ok = cudaMemcpy(ctx->d_ident, id, sizeof(id), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    ok = ok && cudaMemset(ctx->d_counter, 0, sizeof(long long)) == cudaSuccess;
    ok = ok && cudaMemset(ctx->d_ring, 0, sizeof(double) * 2 * kRing) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    sv_destroy(ctx);
    return SV_ENOMEM;
  }
  *out = ctx;
  return SV_OK;
}

int sv_attach_state(sv_ctx* ctx, void* dev_ptr, size_t bytes) {
  if (ctx) ctx->in_period_layout = false;  // the state is (re)written in the natural layout
  if (!ctx) return SV_EINVAL;
  if (!dev_ptr) return fail(ctx, SV_EINVAL, "null state pointer");
  if (reinterpret_cast<uintptr_t>(dev_ptr) % 256 != 0)
    return fail(ctx, SV_EINVAL, "state buffer must be 256-byte aligned");
  if (ctx->state != dev_ptr) drop_graph(ctx);
  ctx->state = dev_ptr;
  ctx->state_bytes = bytes;
  if (ctx->inited && bytes < (amp_bytes(ctx->precision) << ctx->L)) {
    ctx->inited = false;
  }
  return SV_OK;
}

int sv_init(sv_ctx* ctx, int L, const double* product_state) {
  if (ctx) ctx->in_period_layout = false;  // the state is (re)written in the natural layout
  if (!ctx) return SV_EINVAL;
  if (!ctx->state) return fail(ctx, SV_ESTATE, "no state buffer attached");
  const int lmax = ctx->precision == SV_C64 ? 34 : 33;
  if (L < 2 || L > lmax) return fail(ctx, SV_EINVAL, "L=%d out of range 2..%d", L, lmax);
  if (!product_state) return fail(ctx, SV_EINVAL, "null product_state");
  if (ctx->state_bytes < (amp_bytes(ctx->precision) << L))
    return fail(ctx, SV_EINVAL, "state buffer of %zu bytes is too small for L=%d",
                ctx->state_bytes, L);
  std::vector<double> sp(4 * (size_t)L);
  for (int i = 0; i < L; ++i) {
    const double* s = product_state + 4 * i;
    double n2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + s[3] * s[3];
    if (!(n2 > 0.0) || !std::isfinite(n2))
      return fail(ctx, SV_EINVAL, "site %d spinor has zero or non-finite norm", i);
    double inv = 1.0 / std::sqrt(n2);
    for (int k = 0; k < 4; ++k) sp[4 * i + k] = s[k] * inv;
  }
  DeviceGuard dg(ctx->device);
  if (L != ctx->L) free_build(ctx);
  SV_CUDA(cudaMemcpyAsync(ctx->d_spinors, sp.data(), sizeof(double) * sp.size(),
                          cudaMemcpyHostToDevice, ctx->stream),
          "upload spinors");
  SV_CUDA(fsv::launch_product_state(ctx->precision, ctx->state, L, ctx->d_spinors, ctx->cfg,
                                    ctx->stream),
          "product state launch");
  SV_CUDA(cudaMemsetAsync(ctx->d_counter, 0, sizeof(long long), ctx->stream), "reset counter");
  // the spinor buffer is read by the launch above before any later upload
  SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
  ctx->L = L;
  ctx->inited = true;
  ctx->counter = 0;
  return SV_OK;
}

int sv_build_floquet(sv_ctx* ctx, const sv_floquet_params* p) {
  if (!ctx) return SV_EINVAL;
  if (!p) return fail(ctx, SV_EINVAL, "null params");
  if (!ctx->inited) return fail(ctx, SV_ESTATE, "sv_init must come before sv_build_floquet");
  std::string why;
  if (!fsv::params_valid(ctx->L, *p, &why)) return fail(ctx, SV_EINVAL, "%s", why.c_str());
  if (p->mode == SV_MODE_BLOCK && p->n_period_params > 0)
    return fail(ctx, SV_EUNSUPPORTED, "per-period parameters need SV_MODE_PLAIN");
  if (p->mode == SV_MODE_BLOCK && ctx->precision != SV_C64)
    return fail(ctx, SV_EUNSUPPORTED, "block mode needs SV_C64");
  if (p->mode == SV_MODE_MULTIGATE && ctx->precision != SV_C64)
    return fail(ctx, SV_EUNSUPPORTED, "multi-gate mode needs SV_C64");
  DeviceGuard dg(ctx->device);
  {
    int rc = ensure_natural(ctx);  // the new plan starts from the natural layout
    if (rc) return rc;
  }
  free_build(ctx);
  ctx->params = *p;
  ctx->n_period_params = p->n_period_params;
  ctx->theta_p.clear();
  ctx->hx_p.clear();
  if (p->n_period_params > 0) {
    ctx->theta_p.assign(p->n_period_params, p->theta);
    ctx->hx_p.assign(p->n_period_params, p->hx);
    for (int64_t k = 0; k < p->n_period_params; ++k) {
      if (p->theta_p) ctx->theta_p[k] = p->theta_p[k];
      if (p->hx_p) ctx->hx_p[k] = p->hx_p[k];
      if (!std::isfinite(ctx->theta_p[k]) || !std::isfinite(ctx->hx_p[k]))
        return fail(ctx, SV_EINVAL, "non-finite per-period parameter at %lld", (long long)k);
    }
  }
  ctx->params.theta_p = nullptr;
  ctx->params.hx_p = nullptr;
  ctx->obs = fsv::observable(ctx->L, *p);
  const double th0 = p->n_period_params > 0 ? ctx->theta_p[0] : p->theta;
  const double hx0 = p->n_period_params > 0 ? ctx->hx_p[0] : p->hx;
  ctx->gates = fsv::period_gates(ctx->L, *p, th0, hx0);
  const int ng = (int)ctx->gates.size();
  if (p->mode == SV_MODE_BLOCK) {
    int n = p->block_n ? p->block_n : 6;
    if (n < 2 || n > 7) return fail(ctx, SV_EINVAL, "block_n must be in 2..7");
    if (n > ctx->L) n = ctx->L;
    std::string msg;
    int rc = fsv::block_build(ctx->L, ctx->gates, ctx->obs, n, p->split, ctx->cfg,
                              ctx->cyclic, &ctx->block, &msg);
    if (rc != SV_OK) return fail(ctx, rc, "block build: %s", msg.c_str());
    fsv::block_set_renorm(ctx->block, renorm_of(ctx));
    fsv::block_info(ctx->block, &ctx->passes_per_period, &ctx->launches_per_period);
    ctx->build_bytes = fsv::block_upload_bytes(ctx->block);
  } else {
    const int64_t ntab = p->n_period_params > 0 ? p->n_period_params : 1;
    const size_t cb = amp_bytes(ctx->precision);
    ctx->d_gates_bytes = (size_t)ntab * ng * fsv::kGateEntries * cb;
    if (cudaMalloc(&ctx->d_gates, ctx->d_gates_bytes) != cudaSuccess) {
      cudaGetLastError();
      ctx->d_gates = nullptr;
      return fail(ctx, SV_ENOMEM, "gate table allocation failed");
    }
    int slots = 0;
    std::vector<fsv::MultiPass> mplan;
    if (p->mode == SV_MODE_MULTIGATE) {
      const int w = ctx->L <= fsv::kMgTileBits ? ctx->L : fsv::kMgWindow;
      mplan = fsv::multigate_plan(ctx->L, ctx->gates, w);
      for (auto& mp : mplan)
        slots += !ctx->obs.general && (!mp.x_sites.empty() || mp.diag) ? 1 : 0;
    } else {
      for (auto& g : ctx->gates) slots += g.epi ? 1 : 0;
    }
    ctx->part_slots_evolve = slots;
    size_t pbytes = sizeof(double) * 2 * (size_t)ctx->maxb * slots;
    if (cudaMalloc(&ctx->d_part_evolve, pbytes) != cudaSuccess) {
      cudaGetLastError();
      ctx->d_part_evolve = nullptr;
      return fail(ctx, SV_ENOMEM, "partials allocation failed");
    }
    SV_CUDA(cudaMemsetAsync(ctx->d_part_evolve, 0, pbytes, ctx->stream), "memset partials");
    int urc = SV_OK;
    if (ctx->precision == SV_C128) urc = upload_tables<double2>(ctx, *p, ntab, ng);
    else if (ctx->precision == SV_DF64) urc = upload_tables<float4>(ctx, *p, ntab, ng);
    else urc = upload_tables<float2>(ctx, *p, ntab, ng);
    if (urc) return urc;
    ctx->passes_per_period = ng;
    ctx->launches_per_period = ng + 1;
    ctx->build_bytes = ctx->d_gates_bytes;
    if (p->mode == SV_MODE_MULTIGATE) {
      int rc = build_multigate(ctx, mplan);
      if (rc) return rc;
    }
  }
  ctx->built = true;
  return SV_OK;
}

int sv_evolve(sv_ctx* ctx, int64_t periods, double* energy_out, double* norm_out) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (periods < 0) return fail(ctx, SV_EINVAL, "periods must be >= 0");
  if (ctx->n_period_params > 0 && ctx->counter + periods > ctx->n_period_params)
    return fail(ctx, SV_EINVAL, "per-period parameters cover %lld periods, asked up to %lld",
                (long long)ctx->n_period_params, (long long)(ctx->counter + periods));
  DeviceGuard dg(ctx->device);
  rc = ensure_graph(ctx);
  if (rc) return rc;
  int64_t done = 0;
  while (done < periods) {
    const int64_t chunk = std::min<int64_t>(periods - done, kRing);
    const int64_t c0 = ctx->counter;
    rc = launch_periods(ctx, chunk, done + chunk == periods);
    if (rc) return rc;
    if (energy_out || norm_out) {
      rc = read_ring(ctx, c0, chunk, energy_out ? energy_out + done : nullptr,
                     norm_out ? norm_out + done : nullptr);
      if (rc) return rc;
    }
    done += chunk;
  }
  if (!energy_out && !norm_out) SV_CUDA(cudaGetLastError(), "evolve");
  return SV_OK;
}

int sv_evolve_profiled(sv_ctx* ctx, int64_t periods, double* energy_out, double* norm_out,
                       double* pass_ms) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  if (periods < 0) return fail(ctx, SV_EINVAL, "periods must be >= 0");
  if (periods > kRing) return fail(ctx, SV_EINVAL, "at most %d periods per profiled call", kRing);
  if (ctx->n_period_params > 0 && ctx->counter + periods > ctx->n_period_params)
    return fail(ctx, SV_EINVAL, "per-period parameters exhausted");
  DeviceGuard dg(ctx->device);
  const int nl = ctx->launches_per_period;
  std::vector<cudaEvent_t> ev(nl + 1, nullptr);
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (auto& x : ev)
        if (x) cudaEventDestroy(x);
      return fail(ctx, SV_ECUDA, "event create failed");
    }
  const int64_t c0 = ctx->counter;
  rc = SV_OK;
  if (periods > 0 && off_natural(ctx) && !ctx->in_period_layout) {
    cudaError_t e = fsv::block_enqueue_entry(ctx->block, ctx->state, ctx->stream);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "relabel launch");
    else ctx->in_period_layout = true;
  }
  for (int64_t p = 0; p < periods && rc == SV_OK; ++p) {
    const bool exit = p + 1 == periods && !ctx->keep_layout;
    rc = enqueue_period_profiled(ctx, ctx->stream, ev.data(), exit);
    if (rc == SV_OK && exit && off_natural(ctx)) ctx->in_period_layout = false;
    if (rc) break;
    ++ctx->counter;
    if (rc == SV_OK) {
      cudaError_t e = cudaEventSynchronize(ev[nl]);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "event synchronize");
    }
    for (int k = 0; k < nl && rc == SV_OK && pass_ms; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) == cudaSuccess) pass_ms[k] += ms;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  if (energy_out || norm_out) return read_ring(ctx, c0, periods, energy_out, norm_out);
  return SV_OK;
}

int sv_expect_energy(sv_ctx* ctx, double* energy_density, double* norm2) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  rc = ensure_natural(ctx);  // a state kept in the period layout
  if (rc) return rc;
  DeviceGuard dg(ctx->device);
  if (ctx->obs.general) {
    if (ctx->precision == SV_DF64) return no_df(ctx, "measuring a general chain");
    double E = 0.0;
    rc = energy_moments(ctx, &E, nullptr, norm2);
    if (rc == SV_OK && energy_density) *energy_density = E / ctx->L;
    return rc;
  }
  return measure(ctx, energy_density, norm2);
}

int sv_energy_moments(sv_ctx* ctx, double* energy, double* sigma_e, double* norm2) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  rc = ensure_natural(ctx);  // a state kept in the period layout
  if (rc) return rc;
  if (ctx->precision == SV_DF64) return no_df(ctx, "sv_energy_moments");
  DeviceGuard dg(ctx->device);
  return energy_moments(ctx, energy, sigma_e, norm2);
}

int sv_overlap_product(sv_ctx* ctx, const double* spinors, double* overlap_re,
                       double* overlap_im) {
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  rc = ensure_natural(ctx);  // a state kept in the period layout
  if (rc) return rc;
  if (!spinors) return fail(ctx, SV_EINVAL, "null spinors");
  if (ctx->precision == SV_DF64) return no_df(ctx, "sv_overlap_product");
  return product_overlap(ctx, 1, spinors, overlap_re, overlap_im);
}

int sv_overlap_pairs(sv_ctx* ctx, const double* pair_states, double* overlap_re,
                     double* overlap_im) {
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  rc = ensure_natural(ctx);  // a state kept in the period layout
  if (rc) return rc;
  if (!pair_states) return fail(ctx, SV_EINVAL, "null pair_states");
  if (ctx->L % 2) return fail(ctx, SV_EINVAL, "pair states need an even L");
  if (ctx->precision == SV_DF64) return no_df(ctx, "sv_overlap_pairs");
  return product_overlap(ctx, 2, pair_states, overlap_re, overlap_im);
}

int sv_init_pairs(sv_ctx* ctx, int L, const double* pair_states) {
  if (ctx) ctx->in_period_layout = false;  // the state is (re)written in the natural layout
  if (!ctx) return SV_EINVAL;
  if (!ctx->state) return fail(ctx, SV_ESTATE, "no state buffer attached");
  if (ctx->precision == SV_DF64) return no_df(ctx, "sv_init_pairs");
  const int lmax = ctx->precision == SV_C64 ? 34 : 33;
  if (L < 2 || L > lmax || L % 2)
    return fail(ctx, SV_EINVAL, "L=%d must be even and in 2..%d", L, lmax);
  if (!pair_states) return fail(ctx, SV_EINVAL, "null pair_states");
  if (ctx->state_bytes < (amp_bytes(ctx->precision) << L))
    return fail(ctx, SV_EINVAL, "state buffer of %zu bytes is too small for L=%d",
                ctx->state_bytes, L);
  std::vector<double> lo, hi;
  int m = 0;
  const int rt = factor_tables(ctx, L, 2, pair_states, &m, &lo, &hi);
  if (rt) return rt;
  DeviceGuard dg(ctx->device);
  if (L != ctx->L) free_build(ctx);
  const size_t lo_b = sizeof(double) * lo.size(), hi_b = sizeof(double) * hi.size();
  char* d_buf = nullptr;
  SV_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d_buf), lo_b + hi_b, ctx->stream),
          "pair tables");
  cudaError_t e = cudaMemcpyAsync(d_buf, lo.data(), lo_b, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_buf + lo_b, hi.data(), hi_b, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = fsv::launch_factor_state(ctx->precision, ctx->state, L, m, d_buf, d_buf + lo_b, ctx->cfg,
                                 ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(ctx->d_counter, 0, sizeof(long long), ctx->stream);
  // the host tables must outlive the copies above
  const cudaError_t es = cudaStreamSynchronize(ctx->stream);
  cudaFreeAsync(d_buf, ctx->stream);
  if (e == cudaSuccess) e = es;
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pair state");
  ctx->L = L;
  ctx->inited = true;
  ctx->counter = 0;
  return SV_OK;
}

int sv_renormalize(sv_ctx* ctx, double* norm2_before) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  rc = ensure_natural(ctx);  // a state kept in the period layout
  if (rc) return rc;
  DeviceGuard dg(ctx->device);
  double n2 = 0.0;
  rc = measure(ctx, nullptr, &n2);
  if (rc) return rc;
  // place the norm where the scale pass reads it (ring slot counter - 1)
  const int64_t slot = ((ctx->counter - 1) % kRing + kRing) % kRing;
  SV_CUDA(cudaMemcpyAsync(ctx->d_ring + 2 * slot + 1, &n2, sizeof(double),
                          cudaMemcpyHostToDevice, ctx->stream),
          "upload norm");
  SV_CUDA(fsv::launch_renormalize(ctx->precision, ctx->state, ctx->L, ctx->d_ring, kRing,
                                  ctx->d_counter, ctx->cfg, ctx->stream),
          "renormalize launch");
  SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
  if (norm2_before) *norm2_before = n2;
  return SV_OK;
}

int sv_adjoint(sv_ctx* ctx, int64_t periods, double* grad_theta, double* grad_hx,
               double* energy_density) {
  int rc = check_ready(ctx, true);
  if (rc) return rc;
  rc = ensure_natural(ctx);  // a state kept in the period layout
  if (rc) return rc;
  if (ctx->precision == SV_DF64) return no_df(ctx, "sv_adjoint");
  if (ctx->params.mode != SV_MODE_PLAIN)
    return fail(ctx, SV_EUNSUPPORTED, "the adjoint needs SV_MODE_PLAIN");
  if (ctx->n_period_params <= 0)
    return fail(ctx, SV_ESTATE, "the adjoint needs per-period parameters (n_period_params > 0)");
  if (periods < 1 || periods > ctx->n_period_params)
    return fail(ctx, SV_EINVAL, "periods=%lld outside 1..%lld (the per-period parameters)",
                (long long)periods, (long long)ctx->n_period_params);
  if (ctx->counter != 0)
    return fail(ctx, SV_ESTATE, "the adjoint starts at period 0 (counter is %lld)",
                (long long)ctx->counter);
  const int L = ctx->L;
  const int64_t P = periods;
  const bool c128 = ctx->precision == SV_C128;
  const size_t cb = amp_bytes(ctx->precision);
  DeviceGuard dg(ctx->device);
  // operation tables of every period, reverse order within a period
  std::vector<std::vector<fsv::AdjOp>> ops((size_t)P);
  for (int64_t k = 0; k < P; ++k)
    ops[k] = fsv::adjoint_period_ops(L, ctx->params, ctx->theta_p[k], ctx->hx_p[k]);
  const size_t nop = ops[0].size();
  const size_t tab_elems = (size_t)P * nop * 32;  // odag, d per operation
  std::vector<float2> tab32;
  std::vector<double2> tab64;
  if (c128)
    tab64.resize(tab_elems);
  else
    tab32.resize(tab_elems);
  for (int64_t k = 0; k < P; ++k)
    for (size_t o = 0; o < nop; ++o) {
      const fsv::AdjOp& op = ops[k][o];
      const size_t at = ((size_t)k * nop + o) * 32;
      if (c128) {
        for (int e = 0; e < 16; ++e) {
          tab64[at + e] = make_double2(op.odag[e].real(), op.odag[e].imag());
          tab64[at + 16 + e] = make_double2(op.d[e].real(), op.d[e].imag());
        }
      } else {
        fsv::round_unitary4(op.odag, &tab32[at]);
        for (int e = 0; e < 16; ++e)
          tab32[at + 16 + e] = make_float2((float)op.d[e].real(), (float)op.d[e].imag());
      }
    }
  const int grid = fsv::adjoint_grid(ctx->cfg);
  const size_t npart = nop * (size_t)grid;
  void* d_lam = nullptr;
  void* d_tab = nullptr;
  double* d_part = nullptr;
  double* d_grad = nullptr;
  auto release = [&]() {
    cudaFree(d_lam);
    cudaFree(d_tab);
    cudaFree(d_part);
    cudaFree(d_grad);
  };
  if (cudaMalloc(&d_lam, cb << L) != cudaSuccess ||
      cudaMalloc(&d_tab, tab_elems * (c128 ? sizeof(double2) : sizeof(float2))) != cudaSuccess ||
      cudaMalloc(&d_part, sizeof(double) * npart) != cudaSuccess ||
      cudaMalloc(&d_grad, sizeof(double) * (2 * (size_t)P + 1)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(ctx, SV_ENOMEM, "adjoint buffers (%zu bytes for lambda)", cb << L);
  }
  auto run = [&]() -> int {
    SV_CUDA(cudaMemcpyAsync(d_tab, c128 ? (const void*)tab64.data() : (const void*)tab32.data(),
                            tab_elems * (c128 ? sizeof(double2) : sizeof(float2)),
                            cudaMemcpyHostToDevice, ctx->stream),
            "upload adjoint tables");
    // forward to psi_P without storing states
    int r = sv_evolve(ctx, P, nullptr, nullptr);
    if (r) return r;
    // seed lambda = (H0 / L) psi_P; f = Re <psi_P|lambda>
    fsv::H0Coef h;
    h.J = ctx->obs.J;
    for (int i = 0; i < L; ++i) {
      h.cx[i] = ctx->obs.cx[i];
      h.cz[i] = ctx->obs.cz[i];
    }
    SV_CUDA(fsv::launch_apply_h0(ctx->precision, ctx->state, d_lam, L, h, d_part, ctx->cfg,
                                 ctx->stream),
            "adjoint seed launch");
    SV_CUDA(fsv::launch_grad_reduce(d_part, grid, d_grad + 2 * P, 0, ctx->stream),
            "energy reduce launch");
    // reverse sweep: each operation's partials in its own slice, then the
    // period's kick and drive slices summed in a fixed order
    const size_t eb = c128 ? sizeof(double2) : sizeof(float2);
    for (int64_t k = P - 1; k >= 0; --k) {
      size_t nkick = 0;
      for (size_t o = 0; o < nop; ++o) {
        const fsv::AdjOp& op = ops[k][o];
        if (op.kind == 0) ++nkick;
        const char* base = static_cast<const char*>(d_tab) + ((size_t)k * nop + o) * 32 * eb;
        SV_CUDA(fsv::launch_adjoint_gate(ctx->precision, ctx->state, d_lam, L, op.bond, base,
                                         base + 16 * eb, d_part + o * (size_t)grid, ctx->cfg,
                                         ctx->stream),
                "adjoint gate launch");
      }
      // the kick operations come first in each period's list
      SV_CUDA(fsv::launch_grad_reduce(d_part, (long long)(nkick * grid), d_grad + 2 * k, 1,
                                      ctx->stream),
              "gradient reduce launch");
      SV_CUDA(fsv::launch_grad_reduce(d_part + nkick * grid, (long long)((nop - nkick) * grid),
                                      d_grad + 2 * k + 1, 1, ctx->stream),
              "gradient reduce launch");
    }
    std::vector<double> hg(2 * (size_t)P + 1);
    SV_CUDA(cudaMemcpyAsync(hg.data(), d_grad, sizeof(double) * hg.size(),
                            cudaMemcpyDeviceToHost, ctx->stream),
            "gradient readback");
    SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
    for (int64_t k = 0; k < P; ++k) {
      if (grad_theta) grad_theta[k] = hg[2 * k];
      if (grad_hx) grad_hx[k] = hg[2 * k + 1];
    }
    if (energy_density) *energy_density = hg[2 * P];
    // psi is back at its starting point: so is the period counter
    SV_CUDA(cudaMemsetAsync(ctx->d_counter, 0, sizeof(long long), ctx->stream),
            "reset counter");
    SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
    ctx->counter = 0;
    return SV_OK;
  };
  rc = run();
  release();
  return rc;
}

int sv_get_state(sv_ctx* ctx, void* host_dst, size_t bytes) {
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  rc = ensure_natural(ctx);  // a state kept in the period layout
  if (rc) return rc;
  const size_t need = amp_bytes(ctx->precision) << ctx->L;
  if (!host_dst || bytes < need) return fail(ctx, SV_EINVAL, "host buffer too small");
  DeviceGuard dg(ctx->device);
  if (ctx->precision == SV_DF64) return df_transfer(ctx, host_dst, true);
  SV_CUDA(cudaMemcpyAsync(host_dst, ctx->state, need, cudaMemcpyDefault, ctx->stream),
          "copy state");
  SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
  return SV_OK;
}

namespace {
int record_norm(sv_ctx* ctx, int64_t period);
}  // namespace

int sv_set_state(sv_ctx* ctx, const void* host_src, size_t bytes, int64_t period) {
  if (ctx) ctx->in_period_layout = false;  // the state is (re)written in the natural layout
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  const size_t need = amp_bytes(ctx->precision) << ctx->L;
  if (!host_src || bytes < need) return fail(ctx, SV_EINVAL, "host buffer too small");
  if (period < 0) return fail(ctx, SV_EINVAL, "period must be >= 0");
  DeviceGuard dg(ctx->device);
  long long c = period;
  if (ctx->precision == SV_DF64) {
    rc = df_transfer(ctx, const_cast<void*>(host_src), false);
    if (rc) return rc;
  } else {
    SV_CUDA(cudaMemcpyAsync(ctx->state, host_src, need, cudaMemcpyHostToDevice, ctx->stream),
            "copy state");
  }
  SV_CUDA(cudaMemcpyAsync(ctx->d_counter, &c, sizeof(c), cudaMemcpyHostToDevice, ctx->stream),
          "set counter");
  SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
  ctx->counter = period;
  // the folded renormalisation of the next period reads the norm recorded
  // for period - 1: record the norm of the state just set
  return record_norm(ctx, period);
}

namespace {
// Host staging of checkpoint copies: pinned chunks of 64 MiB.
struct Pinned {
  void* p = nullptr;
  size_t bytes = 0;
  explicit Pinned(size_t b) {
    if (cudaMallocHost(&p, b) == cudaSuccess) bytes = b;
    else {
      cudaGetLastError();
      p = nullptr;
    }
  }
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};
constexpr size_t kCkptChunk = (size_t)64 << 20;

// Record the norm of the state just set as that of period - 1, for the
// folded renormalisation of the next period.
int record_norm(sv_ctx* ctx, int64_t period) {
  if (period <= 0 || !ctx->built) return SV_OK;
  double n2 = 1.0;
  int rc = measure(ctx, nullptr, &n2);
  if (rc) return rc;
  const int64_t slot = (period - 1) % kRing;
  SV_CUDA(cudaMemcpyAsync(ctx->d_ring + 2 * slot + 1, &n2, sizeof(double),
                          cudaMemcpyHostToDevice, ctx->stream),
          "record norm");
  SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
  return SV_OK;
}
}  // namespace

int sv_save(sv_ctx* ctx, const char* path) {
  int rc = check_ready(ctx, false);
  if (rc) return rc;
  rc = ensure_natural(ctx);  // a state kept in the period layout
  if (rc) return rc;
  if (!path) return fail(ctx, SV_EINVAL, "null path");
  DeviceGuard dg(ctx->device);
  fsv::CkptHeader h;
  h.L = ctx->L;
  h.precision = ctx->precision;
  h.period = ctx->counter;
  h.payload_bytes = amp_bytes(ctx->precision) << ctx->L;
  Pinned buf(std::min<size_t>(kCkptChunk, h.payload_bytes));
  if (!buf.p) return fail(ctx, SV_ENOMEM, "pinned staging buffer");
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ctx, SV_EINVAL, "cannot open %s for writing", path);
  unsigned char hb[fsv::kCkptHeaderBytes] = {};
  bool ok = std::fwrite(hb, 1, sizeof(hb), f) == sizeof(hb);  // rewritten at the end
  uint64_t sum = fsv::ckpt_sum_begin();
  const char* src = static_cast<const char*>(ctx->state);
  for (uint64_t off = 0; ok && off < h.payload_bytes; off += buf.bytes) {
    const size_t n = (size_t)std::min<uint64_t>(buf.bytes, h.payload_bytes - off);
    cudaError_t e = cudaMemcpyAsync(buf.p, src + off, n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      std::fclose(f);
      return cuda_fail(ctx, e, "copy state");
    }
    sum = fsv::ckpt_sum_update(sum, buf.p, n);
    ok = std::fwrite(buf.p, 1, n, f) == n;
  }
  h.payload_sum = sum;
  fsv::ckpt_encode_header(h, hb);
  ok = ok && std::fseek(f, 0, SEEK_SET) == 0 && std::fwrite(hb, 1, sizeof(hb), f) == sizeof(hb);
  ok = (std::fclose(f) == 0) && ok;
  return ok ? SV_OK : fail(ctx, SV_EINVAL, "write to %s failed", path);
}

int sv_load(sv_ctx* ctx, const char* path) {
  if (ctx) ctx->in_period_layout = false;  // the state is (re)written in the natural layout
  if (!ctx) return SV_EINVAL;
  if (!path) return fail(ctx, SV_EINVAL, "null path");
  if (!ctx->state) return fail(ctx, SV_ESTATE, "no state buffer attached");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, SV_EINVAL, "cannot open %s", path);
  unsigned char hb[fsv::kCkptHeaderBytes];
  fsv::CkptHeader h;
  if (std::fread(hb, 1, sizeof(hb), f) != sizeof(hb) || !fsv::ckpt_decode_header(hb, &h)) {
    std::fclose(f);
    return fail(ctx, SV_EINVAL, "%s is not a checkpoint (header)", path);
  }
  if (h.precision != ctx->precision) {
    std::fclose(f);
    return fail(ctx, SV_EINVAL, "checkpoint precision differs from the context's");
  }
  if (ctx->state_bytes < h.payload_bytes) {
    std::fclose(f);
    return fail(ctx, SV_EINVAL, "state buffer smaller than the checkpoint's %llu bytes",
                (unsigned long long)h.payload_bytes);
  }
  if (ctx->built && ctx->L != h.L) {
    std::fclose(f);
    return fail(ctx, SV_EINVAL, "checkpoint L = %d, built evolution L = %d", h.L, ctx->L);
  }
  DeviceGuard dg(ctx->device);
  Pinned buf(std::min<size_t>(kCkptChunk, h.payload_bytes));
  if (!buf.p) {
    std::fclose(f);
    return fail(ctx, SV_ENOMEM, "pinned staging buffer");
  }
  uint64_t sum = fsv::ckpt_sum_begin();
  char* dst = static_cast<char*>(ctx->state);
  bool ok = true;
  for (uint64_t off = 0; ok && off < h.payload_bytes; off += buf.bytes) {
    const size_t n = (size_t)std::min<uint64_t>(buf.bytes, h.payload_bytes - off);
    ok = std::fread(buf.p, 1, n, f) == n;
    if (!ok) break;
    sum = fsv::ckpt_sum_update(sum, buf.p, n);
    cudaError_t e = cudaMemcpyAsync(dst + off, buf.p, n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      std::fclose(f);
      return cuda_fail(ctx, e, "copy state");
    }
  }
  ok = ok && std::fgetc(f) == EOF;
  std::fclose(f);
  // the amplitudes are in place; the counter and the L only change on success
  if (!ok || sum != h.payload_sum)
    return fail(ctx, SV_EINVAL, "%s: payload truncated or checksum mismatch", path);
  ctx->L = h.L;
  ctx->inited = true;
  long long c = h.period;
  SV_CUDA(cudaMemcpyAsync(ctx->d_counter, &c, sizeof(c), cudaMemcpyHostToDevice, ctx->stream),
          "set counter");
  SV_CUDA(cudaStreamSynchronize(ctx->stream), "synchronize");
  ctx->counter = h.period;
  return record_norm(ctx, h.period);
}

int sv_set_layout_policy(sv_ctx* ctx, int keep_period_layout) {
  if (!ctx) return SV_EINVAL;
  if (keep_period_layout != 0 && keep_period_layout != 1)
    return fail(ctx, SV_EINVAL, "keep_period_layout must be 0 or 1");
  ctx->keep_layout = keep_period_layout != 0;
  return ctx->keep_layout ? SV_OK : ensure_natural(ctx);
}

int64_t sv_period_counter(const sv_ctx* ctx) { return ctx ? ctx->counter : -1; }

int sv_pass_info(const sv_ctx* ctx, int* passes_per_period, int* gates_per_period,
                 int* launches_per_period) {
  if (!ctx) return SV_EINVAL;
  if (!ctx->built) return SV_ESTATE;
  if (passes_per_period) *passes_per_period = ctx->passes_per_period;
  if (gates_per_period) *gates_per_period = (int)ctx->gates.size();
  if (launches_per_period) *launches_per_period = ctx->launches_per_period;
  return SV_OK;
}

int sv_form_info(const sv_ctx* ctx, int* tensor_cores, int* block_n) {
  if (!ctx) return SV_EINVAL;
  if (!ctx->built) return SV_ESTATE;
  const bool blk = ctx->params.mode == SV_MODE_BLOCK && ctx->block;
  if (tensor_cores) *tensor_cores = blk && ctx->block->tensor_cores ? 1 : 0;
  if (block_n) *block_n = blk ? ctx->block->n : 0;
  return SV_OK;
}

int sv_build_bytes(const sv_ctx* ctx, size_t* h2d_bytes) {
  if (!ctx) return SV_EINVAL;
  if (!ctx->built) return SV_ESTATE;
  if (h2d_bytes) *h2d_bytes = ctx->build_bytes;
  return SV_OK;
}

const char* sv_last_error(const sv_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void sv_destroy(sv_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard dg(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_build(ctx);
  cudaFree(ctx->d_ident);
  cudaFree(ctx->d_spinors);
  cudaFree(ctx->d_part_meas);
  cudaFree(ctx->d_ring);
  cudaFree(ctx->d_meas);
  cudaFree(ctx->d_counter);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

// ------------------------------------------------------------------- host

int sv_host_bond_gates(int L, const sv_floquet_params* p, double* gates_out,
                       double* kick_out) {
  if (!p) return SV_EINVAL;
  if (!fsv::params_valid(L, *p, nullptr)) return SV_EINVAL;
  const double tau = p->T / p->K;
  if (gates_out)
    for (int b = 0; b < L - 1; ++b) {
      cd h[16], g[16];
      fsv::bond_hamiltonian(L, b, p->J, p->hx, p->hz, p->edge_field_weight, h);
      fsv::expm_herm4(h, tau, g);
      for (int k = 0; k < 16; ++k) {
        gates_out[32 * b + 2 * k] = g[k].real();
        gates_out[32 * b + 2 * k + 1] = g[k].imag();
      }
    }
  if (kick_out) {
    cd r[4];
    fsv::kick_matrix(p->theta, r);
    for (int k = 0; k < 4; ++k) {
      kick_out[2 * k] = r[k].real();
      kick_out[2 * k + 1] = r[k].imag();
    }
  }
  return SV_OK;
}

int sv_host_period_gates(int L, const sv_floquet_params* p, int* n_gates, int* bonds_out,
                         double* mats_out) {
  if (!p || !n_gates) return SV_EINVAL;
  if (!fsv::params_valid(L, *p, nullptr)) return SV_EINVAL;
  auto gates = fsv::period_gates(L, *p, p->theta, p->hx);
  const int cap = *n_gates;
  *n_gates = (int)gates.size();
  if (!bonds_out && !mats_out) return SV_OK;
  if (cap < (int)gates.size()) return SV_EINVAL;
  for (size_t g = 0; g < gates.size(); ++g) {
    if (bonds_out) bonds_out[g] = gates[g].bond;
    if (mats_out)
      for (int k = 0; k < 16; ++k) {
        mats_out[32 * g + 2 * k] = gates[g].m[k].real();
        mats_out[32 * g + 2 * k + 1] = gates[g].m[k].imag();
      }
  }
  return SV_OK;
}

int sv_host_fusion_plan(int L, const sv_floquet_params* p, int n, int* n_passes,
                        int* window_lo, int* gate_count, double* unitaries_out) {
  if (!p || !n_passes) return SV_EINVAL;
  if (!fsv::params_valid(L, *p, nullptr)) return SV_EINVAL;
  if (n < 2 || n > 7 || n > L) return SV_EINVAL;
  auto gates = fsv::period_gates(L, *p, p->theta, p->hx);
  auto plan = fsv::fusion_plan(L, gates, n, true);
  const int cap = *n_passes;
  *n_passes = (int)plan.size();
  if (!window_lo && !gate_count && !unitaries_out) return SV_OK;
  if (cap < (int)plan.size()) return SV_EINVAL;
  const size_t dim = (size_t)1 << n;
  for (size_t k = 0; k < plan.size(); ++k) {
    if (window_lo) window_lo[k] = plan[k].lo;
    if (gate_count) gate_count[k] = (int)plan[k].gates.size();
    if (unitaries_out)
      for (size_t e = 0; e < dim * dim; ++e) {
        unitaries_out[k * 2 * dim * dim + 2 * e] = plan[k].U[e].real();
        unitaries_out[k * 2 * dim * dim + 2 * e + 1] = plan[k].U[e].imag();
      }
  }
  return SV_OK;
}

int sv_host_pass_operand(int L, const sv_floquet_params* p, int n, int pass, int split,
                         double* operand_out) {
  if (!p || !operand_out) return SV_EINVAL;
  if (!fsv::params_valid(L, *p, nullptr)) return SV_EINVAL;
  if (n < 2 || n > 7 || n > L) return SV_EINVAL;
  if (split != SV_SPLIT_BF16X3 && split != SV_SPLIT_FP32) return SV_EINVAL;
  if (split == SV_SPLIT_BF16X3 && n != 6) return SV_EINVAL;
  auto gates = fsv::period_gates(L, *p, p->theta, p->hx);
  auto plan = fsv::fusion_plan(L, gates, n, true);
  if (pass < 0 || pass >= (int)plan.size()) return SV_EINVAL;
  const size_t dim = (size_t)1 << n;
  const std::vector<fsv::cd>& U = plan[pass].U;
  if (split == SV_SPLIT_FP32) {
    std::vector<float2> f(dim * dim);
    std::vector<float4> lead(dim);
    fsv::round_unitary_fp32((int)dim, U.data(), f.data(), lead.data());
    for (size_t e = 0; e < dim * dim; ++e) {
      operand_out[2 * e] = f[e].x;
      operand_out[2 * e + 1] = f[e].y;
    }
    for (size_t j = 0; j < dim; ++j) {  // the leading entries with their residuals
      const size_t e = j * dim + (size_t)lead[j].z;
      operand_out[2 * e] += lead[j].x;
      operand_out[2 * e + 1] += lead[j].y;
    }
  } else {
    std::vector<double> d(6 * dim * dim);
    fsv::round_unitary_digits((int)dim, U.data(), d.data());
    for (size_t e = 0; e < 2 * dim * dim; ++e)
      operand_out[e] = (d[3 * e] + d[3 * e + 1] / 256.0 + d[3 * e + 2] / 65536.0) / 128.0;
  }
  return SV_OK;
}

int sv_host_block_layout(int L, const sv_floquet_params* p, int n, int* n_passes,
                         int* tile_a, int* sigma_out, unsigned char* rows_out,
                         int* store_wavefronts, int* x_sites_out,
                         unsigned char* staging_out) {
  if (!p || !n_passes) return SV_EINVAL;
  if (!fsv::params_valid(L, *p, nullptr)) return SV_EINVAL;
  if (n < 2 || n > 7 || n >= L) return SV_EINVAL;
  auto gates = fsv::period_gates(L, *p, p->theta, p->hx);
  auto plan = fsv::fusion_plan(L, gates, n, true);
  const int P = (int)plan.size();
  const int cap = *n_passes;
  *n_passes = P;
  if (!tile_a && !sigma_out && !rows_out && !store_wavefronts && !x_sites_out && !staging_out)
    return SV_OK;
  if (cap < P) return SV_EINVAL;
  const int R = std::min(7, L - n);
  const bool tc = n == 6 && R == 7;
  for (int k = 0; k < P; ++k) {
    int a = 0;
    int8_t sig[16] = {};
    if (!fsv::block_tile_layout(L, n, R, plan[k].lo, plan[(k + 1) % P].lo, &a, sig).empty())
      return SV_EINVAL;
    fsv::PassArgs pa;
    pa.L = L;
    pa.n = n;
    pa.R = R;
    pa.a = a;
    std::memcpy(pa.sigma, sig, sizeof(sig));
    const int wf = tc ? fsv::block_tc_layout(pa) : 0;
    const uint8_t* rows = pa.rowvec;
    if (staging_out)
      for (int q = 0; q < 13; ++q) staging_out[13 * k + q] = tc ? (unsigned char)pa.spos[q] : 0;
    if (tile_a) tile_a[k] = a;
    if (sigma_out)
      for (int q = 0; q < 13; ++q) sigma_out[13 * k + q] = q < n + R ? sig[q] : -1;
    if (rows_out)
      for (int i = 0; i < 7; ++i) rows_out[7 * k + i] = tc ? rows[i] : 0;
    if (store_wavefronts) store_wavefronts[k] = wf;
    if (x_sites_out) {
      int mask = 0;
      for (int site : plan[k].x_sites) mask |= 1 << (site - plan[k].lo);
      x_sites_out[k] = mask;
    }
  }
  return SV_OK;
}

int sv_host_store_view(int L, const sv_floquet_params* p, int n, int pass, int* rank,
                       unsigned long long* dims, unsigned long long* strides, unsigned* box,
                       int* coord) {
  if (!p || !rank || !dims || !strides || !box || !coord) return SV_EINVAL;
  if (!fsv::params_valid(L, *p, nullptr)) return SV_EINVAL;
  if (!fsv::block_tc_supported(L, n)) return SV_EINVAL;
  auto gates = fsv::period_gates(L, *p, p->theta, p->hx);
  auto plan = fsv::fusion_plan(L, gates, n, true);
  const int P = (int)plan.size();
  if (pass < 0 || pass >= P) return SV_EINVAL;
  fsv::PassArgs pa;
  pa.L = L;
  pa.n = n;
  pa.R = 7;
  if (!fsv::block_tile_layout(L, n, 7, plan[pass].lo, plan[(pass + 1) % P].lo, &pa.a, pa.sigma)
           .empty())
    return SV_EINVAL;
  fsv::block_tc_layout(pa);
  uint64_t d[5], st[4];
  uint32_t b[5];
  const int r = fsv::block_tc_store_view(pa, d, st, b);
  if (r < 0) return SV_EINVAL;
  *rank = r;
  for (int k = 0; k < 5; ++k) {
    dims[k] = d[k];
    box[k] = b[k];
  }
  for (int k = 0; k < 4; ++k) strides[k] = st[k];
  coord[0] = pa.st_tlo_dim;
  coord[1] = pa.st_tlo_shift;
  coord[2] = pa.st_thi_dim;
  coord[3] = pa.st_thi_shift;
  return SV_OK;
}

}  // extern "C"
