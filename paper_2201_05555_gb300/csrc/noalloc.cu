// Cloud-in-cell deposit for callers that cannot allocate device memory.
//
// Some callers own every byte of device memory through their own pool or a
// fixed memory plan decided at start-up, and may not call cudaMalloc (the
// allocation can fail mid-run or break the plan), nor afford the device-wide
// synchronisation that cudaFree implies.  vp_deposit_cic needs a context
// whose workspace is allocated with cudaMalloc; this variant allocates
// nothing.  Its only scratch, the int64 fixed-point charge counts, is a
// file-scope device array below, which every GPU that loads the library
// holds (1 MiB) until the process exits.
#include "vp_internal.cuh"

#include <atomic>
#include <cmath>

// p * Nx must not exceed this many counts (2^17 int64 = 1 MiB).
#define VP_NOALLOC_MAX_COUNTS 131072
#define VP_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned long long g_noalloc_counts[VP_NOALLOC_MAX_COUNTS];

namespace {
// Device address of g_noalloc_counts on each device, looked up once with
// that device current.  In host code the symbol name itself is only a
// host-side stand-in and must never be handed to a kernel.  The address is
// that of the device's primary context (the one the CUDA runtime uses); a
// caller that makes another context current with the driver API must not use
// this entry point.
std::atomic<unsigned long long*> g_counts_addr[VP_NOALLOC_MAX_DEVICES];
std::atomic<int> g_sms[VP_NOALLOC_MAX_DEVICES];

vp_status counts_address(int dev, unsigned long long** out, int* sms) {
  unsigned long long* p = g_counts_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_counts) != cudaSuccess || !addr) {
      (void)cudaGetLastError();
      return VP_ECUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      (void)cudaGetLastError();
      return VP_ECUDA;
    }
    g_sms[dev].store(n, std::memory_order_relaxed);
    p = static_cast<unsigned long long*>(addr);
    g_counts_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  *sms = g_sms[dev].load(std::memory_order_relaxed);
  return VP_OK;
}
}  // namespace

extern "C" vp_status vp_deposit_cic_noalloc(const vp_grid* grid, int64_t N, int32_t p,
                                            const double* X_dev, int64_t ldx, double* rho_dev,
                                            void* stream) {
  if (!grid || !X_dev || !rho_dev || ldx < N) return VP_EINVAL;
  // the grid checks of vp_deposit_cic: an infinite L or mp, or a non-finite
  // Mq or background, would give a silently wrong rho
  if (grid->Nx < 3 || grid->Nx > VP_MAX_NX || !(grid->L > 0.0) || !std::isfinite(grid->L) ||
      !(grid->mp > 0.0) || !std::isfinite(grid->mp) || !std::isfinite(grid->Mq) ||
      !std::isfinite(grid->background))
    return VP_EINVAL;
  if (N < 1 || N >= (int64_t(1) << 31) || p < 1 || p > 65535) return VP_EINVAL;
  if ((int64_t)p * grid->Nx > VP_NOALLOC_MAX_COUNTS) return VP_EUNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= VP_NOALLOC_MAX_DEVICES) {
    (void)cudaGetLastError();
    return VP_ECUDA;
  }
  unsigned long long* counts = nullptr;
  int sms = 0;
  vp_status s = counts_address(dev, &counts, &sms);
  if (s != VP_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // The array keeps whatever the previous call left: clear the part used now.
  if (cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * p * grid->Nx, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return VP_ECUDA;
  }
  const vpk::GridC g = vpk::make_gridc(*grid, N);
  if (vpk::deposit_samples_launch(g, N, p, X_dev, ldx, counts, sms, st) != cudaSuccess ||
      vpk::counts_to_rho_launch(g, p, counts, rho_dev, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return VP_ECUDA;
  }
  return VP_OK;
}

// ------------------------------------------------------------- self-test
// A bounded wait that runs out: one block waits on an mbarrier that no copy
// and no thread ever completes, `spins` polls per thread, then records
// VP_ETIMEDOUT in the context's status word and returns.  Nothing is in
// flight when it ends, so the context stays usable.
namespace {
__global__ void k_selftest_wait(int spins, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  mbar_wait(&bar, 0, status, spins);
}
}  // namespace

extern "C" vp_status vp_selftest_wait(vp_ctx* ctx, int32_t spins, void* stream) {
  if (!ctx || spins < 1 || spins > (1 << 22)) return VP_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_selftest_wait<<<1, 64, 0, st>>>(spins, ctx->d_status);
  return cudaGetLastError() == cudaSuccess ? VP_OK : VP_ECUDA;
}
