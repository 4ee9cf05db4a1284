// afs_eval_fe_grad_noalloc: FE and gradient evaluation that allocates no
// device memory.
//
// afs_eval_fe_grad needs a buffer for the per-occurrence derivatives and
// allocates it on first use. Some callers cannot allocate at that point:
// cudaMalloc and cudaFree synchronise the device and take a driver-wide lock,
// which a latency-critical loop or a process whose other streams must keep
// running cannot afford, and some processes have all device memory reserved by
// another allocator (a framework's caching allocator, for example). For them
// this entry point keeps that buffer in a fixed file-scope device array.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/afsat.h"
#include "afsat_internal.h"

namespace {

// 16 MiB of device memory, held on every GPU that loads the library until the
// process exits. It holds (literal occurrences) x (restarts per chunk) floats;
// chunks of 32..256 restarts are used, so instances up to 131072 literal
// occurrences with derivative rows (those outside 3-literal constraints)
// fit.
constexpr long long kScratchBytes = 16LL << 20;
constexpr long long kScratchFloats = kScratchBytes / static_cast<long long>(sizeof(float));
static __device__ __align__(256) float g_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

// Device address of g_scratch on the current device. In host code the name
// g_scratch is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached. A device reset
// (cudaDeviceReset, or another component resetting the primary context)
// unloads the library's device module and makes the cached address stale:
// the entry point must not be used on a device after such a reset in the same
// process.
int scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return afs::set_error(AFS_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return afs::set_error(AFS_E_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_dev[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr)
      return afs::set_error(AFS_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_scratch_dev[dev] = p;
  }
  *out = static_cast<float*>(g_scratch_dev[dev]);
  return AFS_OK;
}

}  // namespace

extern "C" int afs_eval_fe_grad_noalloc(afs_handle* h, const float* x_dev, int32_t B, float* fe_dev,
                                        float* grad_dev, void* stream) {
  if (!h || !x_dev) return afs::set_error(AFS_E_ARG, "NULL argument");
  if (B <= 0) return afs::set_error(AFS_E_ARG, "B must be positive");
  float* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != AFS_OK) return rc;
  // Nothing in the buffer needs to start at zero: every derivative a gradient
  // sum reads is written by the FE kernels of the same column chunk first.
  return afs::eval_into_scratch(h, x_dev, afs::XT_F32, B, fe_dev, grad_dev, scratch, kScratchFloats,
                                static_cast<cudaStream_t>(stream));
}
