// hofem_apply_static: the FP64 operator apply r = A u with its two (2D) or four (3D)
// intermediate arrays placed in a fixed, file-scope device array instead of plan
// workspace, for callers that must not allocate device memory at call time -- e.g.
// code running under a framework allocator that forbids raw cudaMalloc, or real-time
// loops that cannot afford cudaMalloc's device-wide synchronisation.  The paper has no
// counterpart to this entry point.
//
// The array holds kStaticScratchDoubles FP64 values (32 MiB).  Every GPU that loads the
// library keeps it resident until the process exits.  All calls share it: calls whose
// work overlaps on the GPU (e.g. on two streams) race on it, so callers serialise them.
// No part of it needs clearing: the first axis sweep writes every entry of the
// intermediates before the next sweep reads them.
#include <mutex>

#include "common.cuh"
#include "residual.cuh"

namespace hofem {

constexpr size_t kStaticScratchDoubles = (size_t)4 << 20;   // 4,194,304 doubles = 32 MiB

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
double* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of g_static_scratch on the current device.  Outside stream capture the
// address is looked up again on every call, so that a context torn down and re-created
// (cudaDeviceReset) never leaves a stale cached address; inside capture the address
// cached by the last uncaptured call on this device is used (set-up happens there).
cudaError_t static_scratch_address(cudaStream_t s, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (cap == cudaStreamCaptureStatusNone || !g_static_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

}  // namespace

size_t static_scratch_doubles() { return kStaticScratchDoubles; }

cudaError_t static_scratch_pointer(cudaStream_t s, double** out) { return static_scratch_address(s, out); }

}  // namespace hofem
