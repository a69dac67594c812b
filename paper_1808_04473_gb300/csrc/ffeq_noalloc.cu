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
// stand-in object); its device address is fetched with cudaGetSymbolAddress,
// with the device current, on the first call made in each CUDA context (the
// primary context of a device, a context created after cudaDeviceReset, or a
// context the caller made current through the driver API), and cached under
// that context's unique ID.
#include <cstdint>

#include "ffeq.h"
#include "ffeq_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;   // 64 MiB per device

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

ffeq::SymbolAddressCache g_scratch_cache;

}  // namespace

extern "C" ffeq_status ffeq_equalize_noalloc(const ffeq_plan* plan, const void* H, const void* y, float N0,
                                             float Es, void* z, float* sigma2, float* llr, int* info,
                                             void* stream) {
  if (!plan) return FFEQ_ERR_INVALID_ARG;
  size_t need = 0;
  ffeq_status r = ffeq_workspace_size(plan, &need);
  if (r != FFEQ_OK) return r;
  if (need > kScratchBytes) return FFEQ_ERR_UNSUPPORTED;   // problem too large for the fixed array
  cudaError_t e = cudaSuccess;
  void* ws = ffeq::cached_symbol_address(
      g_scratch_cache, [](void** out) { return cudaGetSymbolAddress(out, g_scratch); }, &e);
  if (!ws) return static_cast<ffeq_status>(ffeq::record_cuda_error(e));
  // Nothing in the array needs clearing: every workspace element the solve
  // kernel reads is written by the contraction kernel earlier in this call.
  return ffeq_equalize(plan, H, y, N0, Es, z, sigma2, llr, info, ws, kScratchBytes, stream);
}
