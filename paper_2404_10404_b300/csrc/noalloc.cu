// A statement-digest entry point that allocates nothing.
//
// sisu_statement_digest asks the CUDA allocator for its Merkle-tree level
// buffers on every call.  Some callers cannot allow that: a serving loop
// or framework that owns all device memory through its own pool (a
// driver allocation can synchronise the device and fragments the pool), or
// code that runs while the framework's allocator is locked.  This variant
// keeps its scratch in a fixed array in the library's device memory
// instead, and writes the digest to a device buffer the caller provides.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/sisu.h"
#include "internal.h"
#include "launch.cuh"

namespace sisu {

// Largest input the fixed scratch serves: 65,536 chunks of 1024 bytes.
constexpr size_t kNoAllocMaxLeaves = size_t(1) << 16;
constexpr size_t kNoAllocWords = 2 * 8 * kNoAllocMaxLeaves + 16 + 8;  // two tree levels + slack + digest

// The scratch: every GPU that loads the library holds these 4 MiB until the
// process exits.  All calls share it (see the header).
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

// The digest words (big-endian) as the 32 digest bytes, into the caller's buffer.
__global__ void k_digest_words_to_bytes(const uint32_t* words, uint8_t* out) {
  const int i = threadIdx.x;
  if (i < 32) out[i] = (uint8_t)(words[i >> 2] >> (24 - 8 * (i & 3)));
}

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256];  // device address of the scratch, per device ordinal
}  // namespace

}  // namespace sisu

using namespace sisu;

namespace {
// True when p is device memory (or managed memory) that this device's
// kernels may read and write.  cudaPointerGetAttributes allocates nothing;
// an ordinary host pointer comes back as unregistered memory.
bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // the error it set is not sticky: clear it
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int launch_fail(int rc, const char* what) {
  char msg[256];
  snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString((cudaError_t)rc));
  return report_error(SISU_ERR_CUDA, msg);
}
}  // namespace

extern "C" int sisu_statement_digest_noalloc(const uint8_t* data, size_t len, uint8_t* out, void* stream) {
  if (!out || (len && !data)) return report_error(SISU_ERR_INVALID_ARG, "NULL data or output");
  if (len > kNoAllocMaxLeaves * 1024)
    return report_error(SISU_ERR_TOO_LARGE,
                        "sisu_statement_digest_noalloc serves at most 67108864 bytes (64 MiB) of input; "
                        "use sisu_statement_digest for larger inputs");
  // both buffers must be device memory: a host address handed to the
  // kernels would fault the GPU
  if (!device_pointer(out)) return report_error(SISU_ERR_INVALID_ARG, "out is not device memory");
  if (len && !device_pointer(data)) return report_error(SISU_ERR_INVALID_ARG, "data is not device memory");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
    return report_error(SISU_ERR_CUDA, "no current CUDA device");
  void* base;
  {
    // first call on this device: look up the array's device address (the
    // host-side name of a __device__ array is not a device pointer)
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
        return report_error(SISU_ERR_CUDA, "cudaGetSymbolAddress of the fixed digest scratch failed");
      g_noalloc_ptr[dev] = p;
    }
    base = g_noalloc_ptr[dev];
  }
  uint32_t* scratch = (uint32_t*)base;
  uint32_t* words = scratch + (kNoAllocWords - 8);
  cudaStream_t st = (cudaStream_t)stream;
  // the tree levels overwrite the scratch before reading it: nothing needs
  // to start at zero
  int rc = launch_digest_bytes(data, len, scratch, words, st);
  if (rc != (int)cudaSuccess) return launch_fail(rc, "digest tree launch");
  k_digest_words_to_bytes<<<1, 32, 0, st>>>(words, out);
  rc = post_launch();
  if (rc != (int)cudaSuccess) return launch_fail(rc, "digest bytes launch");
  return SISU_OK;
}
