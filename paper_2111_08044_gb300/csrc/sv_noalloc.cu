// sv_energy_noalloc: the energy / norm measurement of a chain state for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a stream is being
// captured into a CUDA graph with a memory pool it does not own, processes
// whose device memory is fully handed to an outside allocator, or service
// loops that must not allocate after start-up.  This entry point takes the
// state and an output buffer from the caller and keeps its reduction scratch
// in a fixed device array of this file, allocated when the library is loaded
// on a device and held until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "sv_internal.h"
#include "sv_kernels.h"

namespace {

// One measurement pass per even bond plus one for the last site of an odd
// chain: at most 18 passes for L <= 34, each writing one (energy, norm) pair
// per block, with at most kMaxBlocks blocks per pass.
constexpr int kMaxPasses = 18;
constexpr int kMaxBlocks = 1024;
constexpr size_t kScratchDoubles = (size_t)2 * kMaxPasses * kMaxBlocks;  // 288 KiB

static __device__ __align__(256) double g_scratch[kScratchDoubles];
// identity gates with zero residual parts (kGateEntries complex each)
static __device__ __align__(256) float2 g_ident64[fsv::kGateEntries] = {
    {1.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {1.f, 0.f},
    {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {1.f, 0.f}, {0.f, 0.f},
    {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {1.f, 0.f}};
static __device__ __align__(256) double2 g_ident128[fsv::kGateEntries] = {
    {1.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {1.0, 0.0},
    {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {1.0, 0.0}, {0.0, 0.0},
    {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {1.0, 0.0}};
static __device__ long long g_counter = 0;  // read (never advanced) by the reduce

struct DeviceSymbols {
  bool ready = false;
  double* scratch = nullptr;
  void* ident64 = nullptr;
  void* ident128 = nullptr;
  long long* counter = nullptr;
  int num_sms = 0;
};

constexpr int kMaxDevices = 64;
DeviceSymbols g_dev[kMaxDevices];
std::mutex g_mu;

// Device addresses of this file's arrays on the current device.  In host
// code the array names are host-side stand-ins, not device addresses.
int setup_device(int dev, DeviceSymbols* out) {
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSymbols& d = g_dev[dev];
  if (!d.ready) {
    if (cudaGetSymbolAddress((void**)&d.scratch, g_scratch) != cudaSuccess ||
        cudaGetSymbolAddress(&d.ident64, g_ident64) != cudaSuccess ||
        cudaGetSymbolAddress(&d.ident128, g_ident128) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.counter, g_counter) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) !=
            cudaSuccess) {
      cudaGetLastError();
      d = DeviceSymbols();
      return SV_ECUDA;
    }
    d.ready = true;
  }
  *out = d;
  return SV_OK;
}

}  // namespace

extern "C" int sv_energy_noalloc(const void* psi_dev, int L, int precision,
                                 const sv_floquet_params* p, double* out_dev,
                                 void* cuda_stream) {
  if (!psi_dev || !out_dev || !p) return SV_EINVAL;
  if (precision != SV_C64 && precision != SV_C128) return SV_EINVAL;
  const int lmax = precision == SV_C128 ? 33 : 34;
  if (L < 2 || L > lmax) return SV_EINVAL;  // beyond the scratch's size
  if (!fsv::params_valid(L, *p, nullptr)) return SV_EINVAL;
  // a general two-site chain's observable is sum_b H_b, which these
  // Ising-form passes do not measure (sv_expect_energy sends such chains to
  // the general-bond kernel)
  if (p->h_bonds) return SV_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SV_ECUDA;
  }
  DeviceSymbols sym;
  int rc = setup_device(dev, &sym);
  if (rc != SV_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  fsv::LaunchCfg cfg;
  // the gate passes launch at most 4 blocks per SM; cap the SM count so that
  // every pass fits in its kMaxBlocks slice of the scratch
  cfg.num_sms = sym.num_sms < kMaxBlocks / 4 ? sym.num_sms : kMaxBlocks / 4;
  const void* ident = precision == SV_C128 ? sym.ident128 : sym.ident64;
  const double ew = p->edge_field_weight;
  int npass = 0;
  int bonds[kMaxPasses], flags[kMaxPasses];
  for (int b = 0; b + 1 < L; b += 2) {
    bonds[npass] = b;
    flags[npass++] = fsv::EPI_X_HI | fsv::EPI_X_LO | (b == 0 ? fsv::EPI_DIAG : 0);
  }
  if (L % 2 == 1) {
    bonds[npass] = L - 2;
    flags[npass++] = fsv::EPI_X_LO;
  }
  // every call starts from a zeroed scratch: the reduce sums whole slices
  if (cudaMemsetAsync(sym.scratch, 0, sizeof(double) * 2 * kMaxBlocks * npass, s) !=
      cudaSuccess) {
    cudaGetLastError();
    return SV_ECUDA;
  }
  for (int k = 0; k < npass; ++k) {
    fsv::EpiParams ep;
    ep.flags = flags[k];
    const int b = bonds[k];
    if (flags[k] & fsv::EPI_X_HI) ep.cx_hi = p->hx * fsv::site_field_share(L, b, ew);
    if (flags[k] & fsv::EPI_X_LO) ep.cx_lo = p->hx * fsv::site_field_share(L, b + 1, ew);
    if (flags[k] & fsv::EPI_DIAG) {
      ep.J = p->J;
      ep.cz_first = p->hz * fsv::site_field_share(L, 0, ew);
      ep.cz_last = p->hz * fsv::site_field_share(L, L - 1, ew);
      ep.cz_bulk = L >= 3 ? p->hz * fsv::site_field_share(L, 1, ew) : 0.0;
    }
    ep.partial = sym.scratch + (size_t)2 * kMaxBlocks * k;
    // each pass writes one (energy, norm) pair per block into its slice
    if (fsv::plain_gate_grid(L, b, precision, cfg) > kMaxBlocks) return SV_EINVAL;
    cudaError_t e = fsv::launch_plain_gate(precision, const_cast<void*>(psi_dev), L, b, ident,
                                           0, sym.counter, ep, /*store=*/0, cfg, s);
    if (e != cudaSuccess) return SV_ECUDA;
  }
  cudaError_t e = fsv::launch_period_reduce(sym.scratch, (long long)npass * kMaxBlocks, L,
                                            out_dev, 1, sym.counter, /*advance=*/0, s);
  return e == cudaSuccess ? SV_OK : SV_ECUDA;
}
