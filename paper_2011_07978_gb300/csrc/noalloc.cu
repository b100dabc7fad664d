// dlbchem_integrate_static: the cost-sorted queued integration for callers
// that cannot allocate device memory while they run.
//
// Who needs it: a flow solver that reserves all of its device memory when it
// starts (its own pool, a fixed budget per GPU) and must not call cudaMalloc
// inside its time loop, both because cudaMalloc can fail once the pool owns
// the device and because it synchronises the whole device.
// dlbchem_integrate grows its work list and sort buffers with cudaMalloc the
// first time it sees a larger field; this entry point instead takes that
// scratch from one fixed array compiled into the library.
//
// The array holds the queue counter, the work list, the sort keys, their
// ping-pong copies and the radix histograms for up to kStaticMaxCells cells
// (5.3 MB). It lives in this file's own module, which CUDA loads lazily: the
// module (and with it the array's device memory) is loaded on a device when
// its address is first looked up, and dlbchem_create does that on the
// context's device. From then on that device holds the array until the
// process exits. All calls share it: calls that overlap on the GPU (two
// streams, two threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/dlbchem.h"
#include "dlb_common.cuh"
#include "dlb_ctx.h"

namespace {

constexpr int64_t kStaticMaxCells = DLBCHEM_STATIC_MAX_CELLS;
constexpr int64_t kTiles = (kStaticMaxCells + 255) / 256;
constexpr size_t kOffCounter = 0;      // unsigned long long, cleared by every call
constexpr size_t kOffTotal = 8;        // int64 work-list length, written by every call
constexpr size_t kOffList = 256;
constexpr size_t kOffListAlt = kOffList + 4 * kStaticMaxCells;
constexpr size_t kOffKeys = kOffListAlt + 4 * kStaticMaxCells;
constexpr size_t kOffKeysAlt = kOffKeys + 4 * kStaticMaxCells;
constexpr size_t kOffHist = kOffKeysAlt + 4 * kStaticMaxCells;
constexpr size_t kScratchBytes = kOffHist + 256 * 4 * kTiles;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Device address of g_static_scratch per device ordinal. In host code the
// symbol name is only a host-side stand-in, so the address is fetched with
// cudaGetSymbolAddress, with the device current, once per device (from
// dlbchem_create; a device whose look-up failed there is tried again by the
// first static call on it).
std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_addr[kMaxDevices] = {};

cudaError_t scratch_for_device(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = ptr;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return cudaSuccess;
}

int fail(dlbchem_ctx* c, int code, const std::string& msg) {
  c->err = msg;
  return code;
}

}  // namespace

namespace dlb {
// Loads the scratch array's module on the current device (called by
// dlbchem_create with the context's device current).
cudaError_t static_scratch_prepare(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  unsigned char* base = nullptr;
  return scratch_for_device(dev, &base);
}
}  // namespace dlb

extern "C" int dlbchem_integrate_static(dlbchem_ctx* c, int64_t n, double dt, const double* T, const double* p,
                                        const double* Y, double* T_out, double* Y_out, int32_t* steps,
                                        int32_t* status, void* stream) {
  if (!c) return DLBCHEM_BAD_ARG;
  c->err.clear();
  if (n < 0) return fail(c, DLBCHEM_BAD_ARG, "ncells must be >= 0");
  if (n > kStaticMaxCells)
    return fail(c, DLBCHEM_BAD_ARG, "ncells exceeds DLBCHEM_STATIC_MAX_CELLS (262144) of dlbchem_integrate_static; "
                                    "split the field into batches or use dlbchem_integrate");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(c, DLBCHEM_BAD_ARG, "dt must be positive and finite");
  if (n == 0) return DLBCHEM_OK;
  if (!T || !p || !Y || !T_out || !Y_out) return fail(c, DLBCHEM_BAD_ARG, "NULL array pointer");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(c, DLBCHEM_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != c->device || dev < 0 || dev >= kMaxDevices)
    return fail(c, DLBCHEM_BAD_ARG, "the current device is not the context's device");
  unsigned char* base = nullptr;
  e = scratch_for_device(dev, &base);
  if (e != cudaSuccess) return fail(c, DLBCHEM_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  auto* counter = reinterpret_cast<unsigned long long*>(base + kOffCounter);
  auto* total = reinterpret_cast<int64_t*>(base + kOffTotal);
  auto* list = reinterpret_cast<int32_t*>(base + kOffList);
  auto* list_alt = reinterpret_cast<int32_t*>(base + kOffListAlt);
  auto* keys = reinterpret_cast<uint32_t*>(base + kOffKeys);
  auto* keys_alt = reinterpret_cast<uint32_t*>(base + kOffKeysAlt);
  auto* hist = reinterpret_cast<int32_t*>(base + kOffHist);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  // work list in index order with the cost keys, then longest first
  e = dlb::launch_init_list(n, steps, list, keys, total, s);
  if (e == cudaSuccess && steps) e = dlb::launch_sort(n, total, keys, list, keys_alt, list_alt, hist, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return fail(c, DLBCHEM_CUDA, std::string("scheduling kernels: ") + cudaGetErrorString(e));
  dlb::KernelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m = c->dm;
  a.P.rtol = c->opt.rtol; a.P.atol = c->opt.atol; a.P.hmin_frac = c->opt.hmin_frac; a.P.dt = dt;
  a.P.max_steps = c->opt.max_steps; a.P.isothermal = c->opt.isothermal; a.P.precision = c->opt.precision;
  a.L = c->L;
  a.n = n; a.T = T; a.p = p; a.Y = Y; a.Tout = T_out; a.Yout = Y_out; a.steps = steps; a.status = status;
  a.perm = list; a.nqueue = total; a.queue = 1; a.counter = counter; a.chunk = c->opt.chunk;
  a.m64 = c->opt.precision == 1 ? c->d_m64 : nullptr;   // allocated once, at creation
  // mixed precision: count the steps whose refinement fell back to the FP64
  // LU in the context's own counter (allocated at creation)
  if (c->opt.precision == 1) {
    a.fallbacks = c->d_counter + 2;
    e = cudaMemsetAsync(c->d_counter + 2, 0, 8, s);
    if (e != cudaSuccess) return fail(c, DLBCHEM_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  }
  int64_t grid = (n + c->teams - 1) / c->teams;
  if (grid > int64_t(c->num_sms) * c->blocks_per_sm) grid = int64_t(c->num_sms) * c->blocks_per_sm;
  e = dlb::launch_rosenbrock(c->wpc, unsigned(grid), 32 * c->wpc * c->teams, c->smem_bytes, s, a);
  if (e != cudaSuccess) return fail(c, DLBCHEM_CUDA, std::string("integrator launch: ") + cudaGetErrorString(e));
  // what dlbchem_last_stats reports for this call (nothing mapped, no work
  // list kept in the context, no timing)
  c->last_n = n;
  c->last_mapping = 0;
  c->last_listed = 0;
  c->timed_last = false;
  for (int i = 0; i < 10; ++i) c->stats[i] = 0;
  c->stats[0] = n; c->stats[2] = -1; c->stats[3] = 32 * c->wpc; c->stats[4] = c->teams;
  c->stats[5] = grid; c->stats[6] = c->smem_bytes; c->stats[7] = 1 + (steps ? 12 : 0) + 1;
  c->stats[9] = c->opt.precision;
  return DLBCHEM_OK;
}
