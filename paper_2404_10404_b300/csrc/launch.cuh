// Launch helpers shared by the kernel translation units.
#pragma once
#include <cuda_runtime.h>

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

}  // namespace sisu
