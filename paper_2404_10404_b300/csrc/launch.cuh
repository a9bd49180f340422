// Launch helpers shared by the kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "internal.h"

namespace sisu {

constexpr unsigned kSMs = 148;  // B300: 148 SMs on two dies

// grid size for n items, capped at per_sm blocks per SM (grid-stride loops)
inline unsigned grid_for(size_t n, unsigned bd, unsigned per_sm = 16) {
  size_t g = (n + bd - 1) / bd;
  size_t cap = (size_t)kSMs * per_sm;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

inline int post_launch() {
  launches_add(1);
  return (int)cudaGetLastError();
}

// Launch with programmatic stream serialization: the kernel's CTAs may be
// scheduled while its predecessor in the stream is finishing, which hides
// the launch gap between the short kernels of a proof.  Such a kernel must
// begin with pdl_wait().
template <typename... K, typename... A>
inline int launch_pdl_smem(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                           A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
  if (e != cudaSuccess) return (int)e;
  return post_launch();
}

template <typename... K, typename... A>
inline int launch_pdl(void (*kernel)(K...), dim3 grid, dim3 block, cudaStream_t st, A&&... args) {
  return launch_pdl_smem(kernel, grid, block, 0, st, std::forward<A>(args)...);
}

#ifdef __CUDACC__
// First statement of a kernel launched by launch_pdl: waits until the
// predecessor grid has completed and its writes are visible (a no-op without
// a programmatic predecessor).  No early trigger: the successor's CTAs are
// placed as this grid's CTAs exit, so they wait out only the last CTAs (a
// round's serial end) and never crowd a running grid (measured: triggering
// at kernel start made the medium step 2% slower, waiting only 0.4% faster
// than plain launches).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

}  // namespace sisu
