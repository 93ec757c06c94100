// Static device scratch for the allocation-free solve (mcrt_solve_qrad_noalloc).
//
// Some callers may not allocate device memory while they run: hosts that
// reserve the whole device memory budget up front (a DNS solver that owns the
// GPU between its own time steps, a serving process with a fixed memory plan)
// and treat any later cudaMalloc as an error or an unpredictable stall.  For
// them the FP32 solve can take its scratch -- the per-ray samples, the
// per-position step sums and the counters -- from this file-scope array instead
// of the context's cudaMalloc'ed buffers.  The array is part of the library's
// device image: every GPU that loads the library holds it until the process
// exits.
#include <mutex>

#include "mcrt_internal.h"

namespace mcrt {
namespace {

constexpr size_t kNoallocScratchBytes = size_t(64) << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_addr[64] = {};

}  // namespace

size_t noalloc_scratch_bytes() { return kNoallocScratchBytes; }

// Device address of the array on `device`, which must be the current device.
// Host code cannot use the symbol's name as an address, so the address is looked
// up once per device with cudaGetSymbolAddress and cached.
cudaError_t noalloc_scratch(int device, void **out) {
  *out = nullptr;
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[device]) {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[device] = ptr;
  }
  *out = g_noalloc_addr[device];
  return cudaSuccess;
}

}  // namespace mcrt
