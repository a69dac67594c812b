// ffeq_equalize_noalloc: the equalizer for callers that cannot allocate device
// memory.
//
// ffeq_equalize needs a caller-provided workspace for the per-(subcarrier,
// cluster) Gram matrices and MRC outputs that pass from the contraction kernel
// to the solve kernel.  Some callers cannot provide one: a real-time receive
// chain must not call cudaMalloc on its per-slot path (the allocator's latency
// is unbounded and it can synchronize the device), and a plug-in running inside
// a host framework may own no device memory beyond the buffers it is handed.
// This entry point takes its workspace from a fixed array compiled into the
// library instead, so the caller passes only inputs and outputs.
//
// The array is a file-scope static __device__ object of kScratchBytes: every
// GPU that loads this library holds it until the process exits.  Host code
// cannot use the name `g_scratch` as a device pointer (on the host it names a
// stand-in object); its device address is fetched with cudaGetSymbolAddress
// once per device, with that device current, on the first call made on it.
#include <atomic>
#include <cstdint>
#include <mutex>

#include "ffeq.h"
#include "ffeq_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;   // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::atomic<void*> g_scratch_ptr[kMaxDevices];
std::mutex g_setup_mutex;

// Device address of g_scratch on the current device; nullptr on failure.
void* scratch_address(int dev) {
  void* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (p) return p;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  p = g_scratch_ptr[dev].load(std::memory_order_relaxed);
  if (p) return p;
  void* addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_scratch) != cudaSuccess || addr == nullptr) return nullptr;
  g_scratch_ptr[dev].store(addr, std::memory_order_release);
  return addr;
}

}  // namespace

extern "C" ffeq_status ffeq_equalize_noalloc(const ffeq_plan* plan, const void* H, const void* y, float N0,
                                             float Es, void* z, float* sigma2, float* llr, int* info,
                                             void* stream) {
  if (!plan) return FFEQ_ERR_INVALID_ARG;
  size_t need = 0;
  ffeq_status r = ffeq_workspace_size(plan, &need);
  if (r != FFEQ_OK) return r;
  if (need > kScratchBytes) return FFEQ_ERR_UNSUPPORTED;   // problem too large for the fixed array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FFEQ_ERR_CUDA;
  void* ws = scratch_address(dev);
  if (!ws) return FFEQ_ERR_CUDA;
  // Nothing in the array needs clearing: every workspace element the solve
  // kernel reads is written by the contraction kernel earlier in this call.
  return ffeq_equalize(plan, H, y, N0, Es, z, sigma2, llr, info, ws, kScratchBytes, stream);
}
