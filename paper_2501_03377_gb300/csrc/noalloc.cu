// tpcg_residual_norms_noalloc: FP64 residual of a candidate solution without a
// plan and without any device allocation.
//
// Who needs it: code that must not call cudaMalloc at the moment it checks a
// solution -- a time-stepping loop that cannot afford the implicit device
// synchronisation cudaMalloc/cudaFree may cause, a host application that
// gives this library a fixed device budget at start-up and owns every
// allocation after that, or code running where allocation is not permitted
// at all.  Everything else in this library allocates its scratch when a plan
// is created; this entry point instead keeps its scratch (the per-block
// partial sums of two reductions and their arrival counters) in one
// file-scope __device__ array.
//
// It is a variant of the residual evaluation of the PCG driver: the FP64
// 7-point stencil of eq. ourproblem with the same ghost values and a
// deterministic two-stage reduction, one grid point per thread with direct
// neighbour loads, and no residual vector is written.
#include <cmath>
#include <mutex>

#include "tpcg_dev.cuh"

namespace tpcg {
namespace {

constexpr int kNaMaxBlocks = 2048;  // reduction blocks the static scratch can hold

struct NoAllocScratch {
  double partials[kNaMaxBlocks * 2];  // per-block partial sums
  unsigned tickets[2];                // arrival counters of the two reductions (must start at 0)
  double mean;                        // mean of eta removed for singular operators
};

// Shared by every call on a device; holds the last call's contents.  Every GPU
// that loads the library keeps this array (about 33 KB) until the process exits.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
// Per device: the context the address was looked up in and the address.  A new primary context (after
// cudaDeviceReset) loads the module again and moves the array, so the address is looked up again
// whenever the current context is not the one it was taken in.
struct ScratchSlot {
  void* ctx = nullptr;
  NoAllocScratch* addr = nullptr;
};
ScratchSlot g_scratch_slot[kMaxDevices];
std::mutex g_scratch_mutex;

typedef int (*CtxGetCurrentFn)(void**);  // cuCtxGetCurrent (CUresult, CUcontext*)

// The driver's current context of this thread (looked up through the runtime: no driver library link).
void* current_context() {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(ptr);
    tried = true;
  }
  void* ctx = nullptr;
  if (fn && fn(&ctx) != 0) ctx = nullptr;
  return ctx;
}

// Device address of the static scratch for the current device, looked up with the device current the
// first time it is used in a context (cudaGetSymbolAddress allocates nothing).
int scratch_for_current_device(int dev, NoAllocScratch** out) {
  if (dev < 0 || dev >= kMaxDevices) return TPCG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchSlot& slot = g_scratch_slot[dev];
  void* ctx = current_context();
  if (!slot.addr || slot.ctx != ctx) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return TPCG_ERR_CUDA;
    }
    slot.addr = reinterpret_cast<NoAllocScratch*>(p);
    slot.ctx = ctx;
  }
  *out = slot.addr;
  return TPCG_OK;
}

__device__ __forceinline__ int na_ghost(int g, int n, int bc) {
  if (g >= 0 && g < n) return g;
  if (g == -1) return bc == kBcP ? n - 1 : ((bc == kBcN || bc == kBcND) ? 0 : -1);
  if (g == n) return bc == kBcP ? 0 : ((bc == kBcN || bc == kBcDN) ? n - 1 : -1);
  return -1;
}

__global__ void __launch_bounds__(256) k_na_eta_sum(long long N, const double* __restrict__ eta,
                                                    NoAllocScratch* s, int singular) {
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    acc[0] += __ldg(eta + i);
  grid_reduce<1>(acc, s->partials, &s->tickets[0], gridDim.x, blockIdx.x,
                 [s, N, singular](const double(&v)[1]) { s->mean = singular ? v[0] / (double)N : 0.0; });
}

// out[0] = ||eta_hat - L ups||_2, out[1] = ||eta_hat||_2, out[2] = removed mean.
__global__ void __launch_bounds__(256) k_na_residual(Geom g, const double* __restrict__ eta,
                                                     const double* __restrict__ ups, NoAllocScratch* s,
                                                     double* out) {
  const double mean = s->mean;
  const unsigned plane = (unsigned)g.nx * (unsigned)g.ny;  // N < 2^31: 32-bit index arithmetic
  const bool has_z = g.nz > 1;
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    const unsigned ui = (unsigned)i;
    const int k = (int)(ui / plane);
    const unsigned rem = ui - (unsigned)k * plane;
    const int y = (int)(rem / (unsigned)g.nx), x = (int)(rem - (unsigned)y * (unsigned)g.nx);
    const double c = __ldg(ups + i);
    auto at = [&](int xx, int yy, int kk) {
      return (xx < 0 || yy < 0 || kk < 0) ? 0.0 : __ldg(ups + (long long)kk * plane + (long long)yy * g.nx + xx);
    };
    const int xl = na_ghost(x - 1, g.nx, g.bc[0]), xr = na_ghost(x + 1, g.nx, g.bc[0]);
    const int yl = na_ghost(y - 1, g.ny, g.bc[1]), yr = na_ghost(y + 1, g.ny, g.bc[1]);
    double w = fma(2.0, c, -(at(xl, y, k) + at(xr, y, k))) * g.ih2[0] +
               fma(2.0, c, -(at(x, yl, k) + at(x, yr, k))) * g.ih2[1];
    if (has_z) {
      const int kl = na_ghost(k - 1, g.nz, g.bc[2]), kr = na_ghost(k + 1, g.nz, g.bc[2]);
      w = fma(fma(2.0, c, -(at(x, y, kl) + at(x, y, kr))), g.ih2[2], w);
    }
    const double e = __ldg(eta + i) - mean;
    const double r = e - w;
    acc[0] = fma(r, r, acc[0]);
    acc[1] = fma(e, e, acc[1]);
  }
  grid_reduce<2>(acc, s->partials, &s->tickets[1], gridDim.x, blockIdx.x, [s, out](const double(&v)[2]) {
    out[0] = sqrt(v[0]);
    out[1] = sqrt(v[1]);
    out[2] = s->mean;
  });
}

}  // namespace
}  // namespace tpcg

using namespace tpcg;

extern "C" int tpcg_residual_norms_noalloc(int nx, int ny, int nz, const int bc[3], const double h[3],
                                           const double* eta, const double* ups, double* out, void* stream) {
  if (!bc || !h || !eta || !ups || !out) return TPCG_ERR_INVALID_ARG;
  if (nx < 3 || ny < 3 || !(nz == 1 || nz >= 3)) return TPCG_ERR_INVALID_ARG;
  const int naxes = (nz == 1) ? 2 : 3;
  for (int m = 0; m < naxes; ++m) {
    if (bc[m] < 0 || bc[m] > 4) return TPCG_ERR_INVALID_ARG;
    if (!(h[m] > 0.0) || !std::isfinite(h[m])) return TPCG_ERR_INVALID_ARG;  // as tpcg_plan_create
  }
  const long long N = (long long)nx * ny * nz;
  if (N > 2147483647LL) return TPCG_ERR_UNSUPPORTED;  // beyond the supported grid size
  // an error left pending by the caller's own work is theirs: report it without consuming it
  if (cudaPeekAtLastError() != cudaSuccess) return TPCG_ERR_CUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TPCG_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return TPCG_ERR_CUDA;
  NoAllocScratch* s = nullptr;
  int rc = scratch_for_current_device(dev, &s);
  if (rc) return rc;
  Geom g{};
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  bool singular = true;
  for (int m = 0; m < 3; ++m) {
    g.bc[m] = (m < naxes) ? bc[m] : kBcN;
    g.ih2[m] = (m < naxes) ? 1.0 / (h[m] * h[m]) : 0.0;
    g.ih2f[m] = (float)g.ih2[m];
    g.nih2[m] = -g.ih2[m];
    if (m < naxes && !(bc[m] == kBcP || bc[m] == kBcN)) singular = false;
  }
  g.uniform = (g.ih2[0] == g.ih2[1]) && (naxes == 2 || g.ih2[2] == g.ih2[0]);
  g.N = N;
  const long long want = (N + 255) / 256;
  const int blocks = (int)std::min<long long>(std::min<long long>(want, (long long)sms * 8), kNaMaxBlocks);
  cudaStream_t st = (cudaStream_t)stream;
  // the arrival counters must start at zero; an aborted earlier call may have left them set
  if (cudaMemsetAsync(s->tickets, 0, sizeof(s->tickets), st) != cudaSuccess) return TPCG_ERR_CUDA;
  k_na_eta_sum<<<blocks, 256, 0, st>>>(N, eta, s, singular ? 1 : 0);
  if (cudaGetLastError() != cudaSuccess) return TPCG_ERR_CUDA;
  k_na_residual<<<blocks, 256, 0, st>>>(g, eta, ups, s, out);
  if (cudaGetLastError() != cudaSuccess) return TPCG_ERR_CUDA;
  return TPCG_OK;
}
