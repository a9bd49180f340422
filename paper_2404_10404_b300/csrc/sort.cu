// Ascending sort of canonical field elements: the prover's side of the
// pairwise-distinct check (Sec. 3.4.2, Algorithm 2), which hands the
// verifier the sorted permutation A* of the list A.
//
// Least-significant-digit radix sort on the 256-bit little-endian values,
// one byte a pass, skipping every byte on which all elements agree (found
// by one pass over the list first): validator indexes below 2^21 take three
// passes, uniform field elements all 32.  A pass is a per-CTA histogram of
// the byte over contiguous tiles (stored tile-major, so that both the
// histogram's writes and the scan's walks down a byte value's column are
// coalesced; the per-value totals added atomically), one exclusive scan of
// the counts in (byte value, tile) order by one CTA per byte value, and a
// stable scatter: each CTA walks its tile
// in chunks of 256, ranks equal bytes inside a warp with a match mask and
// across warps with per-warp counts in shared memory.  Stability across
// passes is what makes the byte-at-a-time order the full order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/sisu.h"
#include "fr.cuh"
#include "internal.h"
#include "launch.cuh"

namespace sisu {

constexpr int kSortBD = 256;
constexpr uint32_t kSortTilesPerSM = 8;
constexpr uint64_t kSortMinTile = 2048;
static_assert(kSortBD == 256, "one thread per byte value in the histogram and the scatter");

__device__ __forceinline__ uint32_t key_byte(const Fr& x, uint32_t d) { return (x.v[d >> 2] >> (8 * (d & 3))) & 0xffu; }

// bit d of *mask: some element's byte d differs from element 0's; bit 0 of
// *err: an element is not below r
__global__ void k_sort_varying(const uint32_t* __restrict__ a, uint64_t n, uint32_t* mask, uint32_t* err) {
  const Fr x0 = fr_load(a, 0);
  uint32_t m = 0, bad = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const Fr x = fr_load(a, i);
    if (!fr_lt_modulus(x)) bad = 1;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const uint32_t diff = x.v[w] ^ x0.v[w];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if ((diff >> (8 * b)) & 0xffu) m |= 1u << (4 * w + b);
    }
  }
  m = __reduce_or_sync(0xffffffffu, m);
  bad = __reduce_or_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (m) atomicOr(mask, m);
    if (bad) atomicOr(err, 1u);
  }
}

// cnt[c * 256 + v] = elements of tile c whose byte d is v; tot[v] += the
// tile's count (tot zero before the pass)
__global__ void __launch_bounds__(kSortBD) k_sort_hist(const uint32_t* __restrict__ a, uint64_t n, uint64_t tile,
                                                       uint32_t d, uint32_t* __restrict__ cnt,
                                                       uint32_t* __restrict__ tot) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t b = blockIdx.x * tile, e = min(n, b + tile);
  for (uint64_t i = b + threadIdx.x; i < e; i += kSortBD) atomicAdd(&h[key_byte(fr_load(a, i), d)], 1u);
  __syncthreads();
  cnt[(size_t)blockIdx.x * 256 + threadIdx.x] = h[threadIdx.x];
  if (h[threadIdx.x]) atomicAdd(&tot[threadIdx.x], h[threadIdx.x]);
}

// In-place exclusive scan of the G x 256 tile-major counts in (byte value,
// tile) order: CTA v (one per byte value, 256 threads) starts from the
// elements of smaller byte values (the totals tot[0..v-1]) and scans its
// value's column over the tiles, a few consecutive tiles a thread.  CTA 0
// also clears tot_next, the totals of the next pass.
__global__ void __launch_bounds__(256) k_sort_scan(uint32_t* __restrict__ c, uint32_t G,
                                                   const uint32_t* __restrict__ tot, uint32_t* __restrict__ tot_next) {
  __shared__ uint32_t wbase[8], wscan[8];
  const uint32_t v = blockIdx.x, lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t below = __reduce_add_sync(0xffffffffu, threadIdx.x < v ? tot[threadIdx.x] : 0u);
  if (lane == 0) wbase[warp] = below;
  const uint32_t per = (G + 255) / 256, t0 = min(G, threadIdx.x * per), t1 = min(G, t0 + per);
  uint32_t s = 0;
  for (uint32_t t = t0; t < t1; ++t) s += c[(size_t)t * 256 + v];
  uint32_t incl = s;  // inclusive scan of the thread sums: in the warp, then over the warps
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) wscan[warp] = incl;
  __syncthreads();
  uint32_t run = incl - s;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    run += wbase[w];
    if ((uint32_t)w < warp) run += wscan[w];
  }
  for (uint32_t t = t0; t < t1; ++t) {
    const uint32_t x = c[(size_t)t * 256 + v];
    c[(size_t)t * 256 + v] = run;
    run += x;
  }
  if (v == 0) tot_next[threadIdx.x] = 0;
}

// stable scatter of tile c by byte d to dst[off[c * 256 + v] + rank]
__global__ void __launch_bounds__(kSortBD) k_sort_scatter(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                                                          uint64_t n, uint64_t tile, uint32_t d,
                                                          const uint32_t* __restrict__ off) {
  constexpr int NW = kSortBD / 32;
  __shared__ uint32_t base[256];     // tile offset of byte value v plus the elements placed so far
  __shared__ uint32_t wcnt[NW][256];  // elements of byte value v in warp w of the current chunk
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  base[threadIdx.x] = off[(size_t)blockIdx.x * 256 + threadIdx.x];
  const uint64_t b = blockIdx.x * tile, e = min(n, b + tile);
  for (uint64_t c0 = b; c0 < e; c0 += kSortBD) {  // uniform over the block
#pragma unroll
    for (int w = 0; w < NW; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const uint64_t i = c0 + threadIdx.x;
    const bool in = i < e;
    Fr x = fr_zero();
    uint32_t v = 256u + lane;  // lanes past the end match no byte value and no other lane
    if (in) {
      x = fr_load(src, i);
      v = key_byte(x, d);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, v);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (in && rank == 0) wcnt[warp][v] = __popc(peers);
    __syncthreads();
    if (in) {
      uint32_t pos = base[v] + rank;
      for (int w = 0; w < warp; ++w) pos += wcnt[w][v];
      fr_store(dst, pos, x);
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) tot += wcnt[w][threadIdx.x];
    base[threadIdx.x] += tot;
  }
}

namespace {

int sort_err(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return report_error(SISU_ERR_CUDA, m.c_str());
}

#define SCK(call, what)                                \
  do {                                                 \
    cudaError_t e_ = (cudaError_t)(call);              \
    if (e_ != cudaSuccess) return sort_err(e_, what);  \
  } while (0)

struct SortBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  ~SortBuf() {
    if (p) cudaFreeAsync(p, st);
  }
};

}  // namespace
}  // namespace sisu

using namespace sisu;

extern "C" int sisu_sort_elements(const uint8_t* in, uint64_t n, int on_device, void* stream, uint8_t* out,
                                  uint32_t* passes) {
  if (passes) *passes = 0;
  if (n && (!in || !out)) return report_error(SISU_ERR_INVALID_ARG, "NULL element array");
  if (n >= (1ull << 32)) return report_error(SISU_ERR_TOO_LARGE, "at most 2^32 - 1 elements");
  if (on_device && n && ((((uintptr_t)in) | ((uintptr_t)out)) & 15))
    return report_error(SISU_ERR_INVALID_ARG, "device element arrays must be 16-byte aligned");
  if (on_device && n) {
    if (int rc = require_device(in, "in")) return rc;
    if (int rc = require_device(out, "out")) return rc;
  }
  if (n == 0) return SISU_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)n * 32;
  // tiles of at least kSortMinTile elements (fewer counts for the single-CTA
  // scan), at most kSortTilesPerSM per SM
  const uint32_t G = (uint32_t)std::max<uint64_t>(
      1, std::min<uint64_t>((n + kSortMinTile - 1) / kSortMinTile, (uint64_t)kSMs * kSortTilesPerSM));
  const uint64_t tile = (n + G - 1) / G;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  // two element buffers, the counts, the flag words
  SortBuf buf;
  buf.st = st;
  SCK(cudaMallocAsync(&buf.p, 2 * al(bytes) + al((size_t)256 * G * 4) + 256 + 2048, st), "cudaMallocAsync");
  uint8_t* p = (uint8_t*)buf.p;
  uint32_t* A = (uint32_t*)p;
  uint32_t* B = (uint32_t*)(p + al(bytes));
  uint32_t* cnt = (uint32_t*)(p + 2 * al(bytes));
  uint32_t* flags = (uint32_t*)(p + 2 * al(bytes) + al((size_t)256 * G * 4));
  uint32_t* tot = flags + 64;  // two sets of 256 per-value totals, by pass parity
  SCK(cudaMemcpyAsync(A, in, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st), "copy in");
  SCK(cudaMemsetAsync(flags, 0, 256 + 1024, st), "memset");  // the flags and the first pass's totals
  k_sort_varying<<<grid_for(n, kSortBD, 8), kSortBD, 0, st>>>(A, n, flags, flags + 1);
  int rc = post_launch();
  if (rc) return sort_err((cudaError_t)rc, "sort");
  uint32_t hflags[2];
  SCK(cudaMemcpyAsync(hflags, flags, 8, cudaMemcpyDeviceToHost, st), "copy out");
  SCK(cudaStreamSynchronize(st), "sort");
  if (hflags[1] & 1u) return report_error(SISU_ERR_NOT_CANONICAL, "an element is not below r");
  uint32_t np = 0;
  for (uint32_t d = 0; d < 32; ++d) {
    if (!((hflags[0] >> d) & 1u)) continue;  // every element has the same byte d
    uint32_t* tot_cur = tot + 256 * (np & 1u);
    uint32_t* tot_nxt = tot + 256 * ((np + 1u) & 1u);
    k_sort_hist<<<G, kSortBD, 0, st>>>(A, n, tile, d, cnt, tot_cur);
    rc = post_launch();
    if (!rc) {
      k_sort_scan<<<256, 256, 0, st>>>(cnt, G, tot_cur, tot_nxt);
      rc = post_launch();
    }
    if (!rc) {
      k_sort_scatter<<<G, kSortBD, 0, st>>>(A, B, n, tile, d, cnt);
      rc = post_launch();
    }
    if (rc) return sort_err((cudaError_t)rc, "sort");
    std::swap(A, B);
    ++np;
  }
  SCK(cudaMemcpyAsync(out, A, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st), "copy out");
  SCK(cudaStreamSynchronize(st), "sort");
  if (passes) *passes = np;
  return SISU_OK;
}
