// Allocation-free variant of the FP64 mass/momentum reduction.
//
// Some callers cannot call cudaMalloc: code whose device memory all belongs
// to its own pool or framework allocator (cudaMalloc can synchronise the
// device and takes memory the pool has already claimed), or code running
// under a fixed device-memory budget.  lbm3_mass_noalloc serves them: it
// reduces a caller-owned population array into a caller-owned output and
// keeps its block partial sums in the file-scope array below instead of
// allocating.
//
// The array (kStaticPartials blocks x 5 doubles = 40 KiB) is part of the
// library image: every GPU that loads liblbm3 holds it until the process
// exits.  In host code its name is only a host-side stand-in, so its device
// address is looked up once per device with cudaGetSymbolAddress (on the
// first call made on that device, with that device current) and cached.

#include <mutex>

#include "../../include/lbm3.h"
#include "lbm3_internal.h"

namespace lbm3 {
namespace {

constexpr int kStaticPartials = 1024;           // blocks of the partial-sum pass
constexpr int kNodesPerBlock = 256 * 64;        // 256 threads x 64 nodes each
constexpr long long kStaticMaxNodes = static_cast<long long>(kStaticPartials) * kNodesPerBlock;  // 16,777,216
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_partial[kStaticPartials * 5];

std::mutex g_mu;
double* g_partial_ptr[kMaxDevices] = {};

// Device address of g_static_partial on the current device (looked up once).
cudaError_t static_partials(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_partial_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_partial);
    if (e != cudaSuccess) return e;
    g_partial_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partial_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace lbm3

extern "C" lbm3_status lbm3_mass_noalloc(const float* dev_f, int32_t nx, int32_t ny, void* cuda_stream,
                                         double* dev_out) {
  if (!dev_f || !dev_out || nx <= 0 || ny <= 0) return LBM3_EINVAL;
  const long long N = static_cast<long long>(nx) * ny;
  if (N > lbm3::kStaticMaxNodes) return LBM3_EINVAL;  // the static partial array is full
  double* partial = nullptr;
  if (lbm3::static_partials(&partial) != cudaSuccess) {
    cudaGetLastError();
    return LBM3_ECUDA;
  }
  const int blocks = static_cast<int>((N + lbm3::kNodesPerBlock - 1) / lbm3::kNodesPerBlock);
  // Each call writes partial[0 .. 5*blocks) before reading it back, so stale
  // contents from an earlier call are never used and nothing needs clearing.
  const cudaError_t e = lbm3::launch_reduce(dev_f, static_cast<int>(N), partial, blocks, dev_out,
                                            static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return LBM3_ECUDA;
  return LBM3_OK;
}
