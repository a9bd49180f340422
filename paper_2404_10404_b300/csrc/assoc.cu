// Associative hash (Sec. 3.4.1, Algorithm 1) and the pairwise-distinct
// check (Sec. 3.4.2, Algorithm 2) on the device.
//
// F(e): r = 0, then three times r = (r + e + 2^32 - 1)^3, in the BN254
// scalar field.  The hash of a list is the sum of F over it, so it does not
// depend on the order of the list and a list's hash continues from the hash
// of an earlier list by addition (the running value H_pre of Sec. 3.4.2).
// Algorithm 2 accepts a list A and a claimed sorted permutation A* when
// their hashes agree and A* is strictly ascending.
//
// Work layout: the elements of all segments (sub-lists hashed separately,
// the paper's M sub-circuits) form one array of 32-byte canonical values.
// The host cuts every segment into chunks of 8192 elements; a resident
// wave of CTAs takes the chunks in order from an atomic counter and sums F
// over each (threads stride the chunk, so a warp reads 1 KB contiguous per
// step), and a second launch adds each segment's chunk sums, one warp per
// segment.  F costs one fixed-multiplier product (e R from the canonical
// e), three Montgomery squares and three Montgomery products; the path is
// bound by the integer multiply-add pipe, not by HBM (32 bytes per element
// against about 1,450 multiply-adds).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/sisu.h"
#include "fr_wide.cuh"
#include "internal.h"
#include "launch.cuh"

namespace sisu {

constexpr int kAssocBD = 256;
constexpr uint64_t kAssocChunk = 8192;
constexpr uint32_t kAssocAdd = 4294967295u;  // 2^32 - 1, added every round of Algorithm 1

// device error word bits
constexpr uint32_t kAssocNotCanonical = 1u;

// R^3 mod p: a Montgomery product with it multiplies by R^2
SISU_FR_CONST(fr_r3, 0xb4bf0040u, 0x5e94d8e1u, 0x1cfbb6b8u, 0x2a489cbeu, 0xa19fcfedu, 0x893cc664u, 0x7fcc657cu,
              0x0cf8594bu)

// the CTA's constants: the fixed-multiplier coefficients of R^2 mod p (so
// that fr_mul_fixed(e, K) = e R, the Montgomery form of a canonical e) in
// shK[0..63], those of R^3 mod p (x -> x R^2) in shK[64..127], and
// (2^32 - 1) R
__device__ __forceinline__ void assoc_consts(uint32_t* shK, Fr* sh_c) {
  if (threadIdx.x < 8) fr_store(shK, threadIdx.x, fr_fixed_coeff(fr_r2(), (int)threadIdx.x));
  if (threadIdx.x >= 32 && threadIdx.x < 40) fr_store(shK, threadIdx.x - 24, fr_fixed_coeff(fr_r3(), (int)threadIdx.x - 32));
  if (threadIdx.x == 8) {
    Fr c = fr_zero();
    c.v[0] = kAssocAdd;
    *sh_c = fr_from_canonical(c);
  }
  __syncthreads();
}

__device__ __forceinline__ Fr fr_from_u64x4(uint64_t w0, uint64_t w1, uint64_t w2, uint64_t w3) {
  Fr x;
  const uint64_t w[4] = {w0, w1, w2, w3};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    x.v[2 * i] = (uint32_t)w[i];
    x.v[2 * i + 1] = (uint32_t)(w[i] >> 32);
  }
  return x;
}

// F(e) in Montgomery form for a canonical e below 2^32 (a validator index).
// With a = e + 2^32 - 1 < 2^33 the first round's cube a^3 < 2^99 and the
// second base t = a^3 + a < 2^100 are exact integers, and so is t^2 < 2^200
// (all below p): the first round needs no modular arithmetic, the second
// one Montgomery product, t^3 R = MontMul(t^2, t R^2) with t R^2 from the
// fixed-multiplier rows of t's four limbs (coefficients of R^3).  About 890
// multiply-adds where the general path takes 1,450.
__device__ __forceinline__ Fr assoc_F_small(uint32_t e, const uint32_t* K2, const uint32_t* K3) {
  const uint64_t a = (uint64_t)e + 0xffffffffull;  // < 2^33
  // a^2 = (s1:s0) < 2^66, a^3 = (c1:c0) < 2^99
  const uint64_t s0 = a * a, s1 = __umul64hi(a, a);
  const uint64_t c0 = s0 * a, c1 = __umul64hi(s0, a) + s1 * a;
  // t = a^3 + a < 2^100 = (t1:t0)
  const uint64_t t0 = c0 + a, t1 = c1 + (t0 < a ? 1u : 0u);
  // u = t^2 < 2^200 = (u3:u2:u1:u0)
  const uint64_t ll = t0 * t0, lh = __umul64hi(t0, t0);
  const uint64_t m0 = t0 * t1, m1 = __umul64hi(t0, t1);  // t0 t1, counted twice
  const uint64_t hh = t1 * t1, hh1 = __umul64hi(t1, t1);
  const uint64_t d0 = m0 << 1, d1 = (m1 << 1) | (m0 >> 63), d2 = m1 >> 63;
  const uint64_t u0 = ll;
  const uint64_t u1 = lh + d0;
  const uint64_t k1 = u1 < d0 ? 1u : 0u;
  const uint64_t x2 = hh + d1;
  const uint64_t k2a = x2 < d1 ? 1u : 0u;
  const uint64_t u2 = x2 + k1;
  const uint64_t k2b = u2 < k1 ? 1u : 0u;
  const uint64_t u3 = hh1 + d2 + k2a + k2b;
  const Fr tR2 = fr_mul_fixed_rows<4>(fr_from_u64x4(t0, t1, 0, 0), K3);  // t R^2
  const Fr r2 = fr_mul(fr_from_u64x4(u0, u1, u2, u3), tR2);            // t^3 R
  const Fr aR = fr_mul_fixed_rows<2>(fr_from_u64x4(a, 0, 0, 0), K2);     // a R
  const Fr t2 = fr_add(r2, aR);
  return fr_mul(fr_sqr(t2), t2);
}

// F(e) in Montgomery form for a canonical e; `small`: every lane of the warp
// holds a value below 2^32
__device__ __forceinline__ Fr assoc_F(const Fr& e, bool small, const uint32_t* K, const Fr& c) {
  if (small) return assoc_F_small(e.v[0], K, K + 64);
  const Fr a = fr_add(fr_mul_fixed(e, K), c);  // (e + 2^32 - 1) R
  Fr r = fr_mul(fr_sqr(a), a);
  Fr t = fr_add(r, a);
  r = fr_mul(fr_sqr(t), t);
  t = fr_add(r, a);
  return fr_mul(fr_sqr(t), t);
}

// x > y for canonical values (plain 256-bit integers)
__device__ __forceinline__ bool u256_gt(const Fr& x, const Fr& y) {
#pragma unroll
  for (int i = 7; i >= 0; --i)
    if (x.v[i] != y.v[i]) return x.v[i] > y.v[i];
  return false;
}

template <int NV>
__device__ __forceinline__ void assoc_block_sum(Fr (&v)[NV]) {
  __shared__ Fr red[NV][kAssocBD / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) v[t] = fr_warp_sum(v[t]);
  if (lane == 0)
#pragma unroll
    for (int t = 0; t < NV; ++t) red[t][warp] = v[t];
  __syncthreads();
  if (warp == 0)
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = fr_warp_sum(lane < kAssocBD / 32 ? red[t][lane] : fr_zero());
  __syncthreads();
}

// Sum of F over chunk k = elements [chunks[3k], chunks[3k+1]) of `a` into
// partials[stride k + off].  CTAs take chunks in order from the counter
// *next (zero at launch), so uneven segments leave no CTA with a whole
// chunk more than another.  A warp whose elements are all below 2^32 (the
// validator indexes of Sec. 3.4.2) converts them with the one-row product.
__global__ void __launch_bounds__(kAssocBD, 2) k_assoc_chunks(const uint32_t* __restrict__ a,
                                                          const uint64_t* __restrict__ chunks, uint32_t nchunks,
                                                          uint32_t* __restrict__ partials, uint32_t stride,
                                                          uint32_t off, uint32_t* next, uint32_t* flag) {
  __shared__ __align__(16) uint32_t shK[128];
  __shared__ Fr sh_c;
  __shared__ uint32_t sh_ch;
  assoc_consts(shK, &sh_c);
  const Fr c = sh_c;
  uint32_t err = 0;
  for (;;) {
    if (threadIdx.x == 0) sh_ch = atomicAdd(next, 1u);
    __syncthreads();
    const uint32_t ch = sh_ch;
    __syncthreads();  // every thread has read sh_ch before thread 0 takes the next chunk
    if (ch >= nchunks) break;
    const uint64_t b = chunks[3 * (size_t)ch], e = chunks[3 * (size_t)ch + 1];
    Fr acc = fr_zero();
    for (uint64_t i0 = b; i0 < e; i0 += kAssocBD) {  // uniform trip count over the block
      const uint64_t i = i0 + threadIdx.x;
      const bool in = i < e;
      Fr x = in ? fr_load(a, i) : fr_zero();
      if (!fr_lt_modulus(x)) {
        err |= kAssocNotCanonical;
        x = fr_zero();
      }
      const bool small = __all_sync(0xffffffffu, (x.v[1] | x.v[2] | x.v[3] | x.v[4] | x.v[5] | x.v[6] | x.v[7]) == 0);
      const Fr f = assoc_F(x, small, shK, c);
      if (in) acc = fr_add(acc, f);
    }
    Fr v[1] = {acc};
    assoc_block_sum<1>(v);
    if (threadIdx.x == 0) fr_store(partials, (size_t)stride * ch + off, v[0]);
  }
  if (err) atomicOr(flag, err);
}

// unordered[k] = 1 when some element i of chunk k, other than the first of
// its segment (chunks[3k+2]), is not above element i - 1 (as integers)
__global__ void __launch_bounds__(kAssocBD) k_order_chunks(const uint32_t* __restrict__ s,
                                                          const uint64_t* __restrict__ chunks, uint32_t nchunks,
                                                          uint32_t* __restrict__ unordered) {
  for (uint32_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const uint64_t b = chunks[3 * (size_t)ch], e = chunks[3 * (size_t)ch + 1], sb = chunks[3 * (size_t)ch + 2];
    bool bad = false;
    for (uint64_t i = b + threadIdx.x; i < e; i += kAssocBD)
      if (i > sb && !u256_gt(fr_load(s, i), fr_load(s, i - 1))) bad = true;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) unordered[ch] = bad ? 1u : 0u;
  }
}

// out[NV g + t] = canonical(h_pre[g] + sum of the chunk sums of segment g),
// one warp per (segment, value); h_pre canonical (null: 0)
__global__ void k_assoc_finish(const uint32_t* __restrict__ partials, const uint32_t* __restrict__ seg_chunk,
                               uint32_t nseg, int NV, const uint32_t* __restrict__ h_pre, uint32_t* __restrict__ out,
                               uint32_t* flag) {
  const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= nseg * (uint32_t)NV) return;
  const uint32_t g = wid / NV, t = wid - g * NV;
  Fr x = fr_zero();
  for (uint32_t k = seg_chunk[g] + lane; k < seg_chunk[g + 1]; k += 32)
    x = fr_add(x, fr_load(partials, (size_t)NV * k + t));
  x = fr_warp_sum(x);
  if (lane == 0) {
    if (h_pre) {
      const Fr h = fr_load(h_pre, g);
      if (!fr_lt_modulus(h)) atomicOr(flag, kAssocNotCanonical);
      x = fr_add(x, fr_from_canonical(h));
    }
    fr_store(out, wid, fr_to_canonical(x));
  }
}

namespace {

struct DevBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, st);
  }
};

int cuda_err(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return report_error(SISU_ERR_CUDA, m.c_str());
}

#define ACK(call, what)                                 \
  do {                                                  \
    cudaError_t e_ = (cudaError_t)(call);               \
    if (e_ != cudaSuccess) return cuda_err(e_, what);   \
  } while (0)

// Hash the segments of `a` (and, with `pair`, of `s`): out receives
// NV x nseg canonical values (segment-major); with `pair`, seg_unordered[g]
// = 1 when segment g of `s` is not strictly ascending.
// One run of the kernels over a list (and, for `pair`, its claimed sort),
// in three phases so that two runs can share the device without a host
// round trip between them: prepare (device buffers, the chunk table and, for
// host lists, the lists themselves copied in: copies from pageable memory
// wait for the stream, so both runs copy before either launches), launch,
// collect (results copied out, one stream synchronisation).
// pair: hash a and s (out: per segment 64 bytes, a's hash then s's) and
// check the order of s; otherwise hash a (out: 32 bytes a segment) and,
// with `order`, check the order of a.  seg_unordered (pair or order): per
// segment, whether two neighbours are not strictly ascending.
struct AssocJob {
  DevBuf buf;
  std::vector<uint32_t> seg_chunk;
  uint32_t nseg = 0, nchunks = 0;
  int NV = 1;
  bool pair = false, ord = false, pre = false;
  uint64_t n = 0;
  const uint8_t* da = nullptr;
  const uint8_t* ds = nullptr;
  uint64_t* d_chunks = nullptr;
  uint32_t *d_seg = nullptr, *d_part = nullptr, *d_pre = nullptr, *d_out = nullptr, *d_flag = nullptr;
};

int assoc_prepare(AssocJob& j, const uint8_t* a, const uint8_t* s, bool pair, bool order, const uint64_t* offsets,
                  uint32_t nseg, const uint8_t* h_pre, int on_device, cudaStream_t st) {
  j.NV = pair ? 2 : 1;
  j.pair = pair;
  j.ord = pair || order;
  j.pre = h_pre != nullptr;
  j.nseg = nseg;
  const uint64_t n = j.n = offsets[nseg];
  const int NV = j.NV;
  // chunks of 8192 elements (32 a thread), each inside one segment, taken
  // in order by the CTAs
  const uint64_t ch = kAssocChunk;
  std::vector<uint64_t> chunks;
  j.seg_chunk.assign(nseg + 1, 0);
  for (uint32_t g = 0; g < nseg; ++g) {
    j.seg_chunk[g] = (uint32_t)(chunks.size() / 3);
    for (uint64_t b = offsets[g]; b < offsets[g + 1]; b += ch) {
      chunks.push_back(b);
      chunks.push_back(std::min(offsets[g + 1], b + ch));
      chunks.push_back(offsets[g]);
    }
  }
  j.seg_chunk[nseg] = (uint32_t)(chunks.size() / 3);
  const uint32_t nchunks = j.nchunks = j.seg_chunk[nseg];
  // one device block: chunk table, segment table, partials, h_pre, out,
  // flag, then (host inputs) the elements
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t b_chunks = al(chunks.size() * 8 + 8), b_seg = al((nseg + 1) * 4), b_part = al((size_t)NV * nchunks * 32 + 32),
               b_pre = al((size_t)nseg * 32), b_out = al((size_t)NV * nseg * 32),
               b_flag = al(12 + (size_t)nchunks * 4);
  const size_t b_in = on_device ? 0 : al((size_t)n * 32) * (pair ? 2 : 1);
  j.buf.st = st;
  ACK(cudaMallocAsync(&j.buf.p, b_chunks + b_seg + b_part + b_pre + b_out + b_flag + b_in, st), "cudaMallocAsync");
  uint8_t* base = (uint8_t*)j.buf.p;
  j.d_chunks = (uint64_t*)base;
  j.d_seg = (uint32_t*)(base + b_chunks);
  j.d_part = (uint32_t*)(base + b_chunks + b_seg);
  j.d_pre = (uint32_t*)(base + b_chunks + b_seg + b_part);
  j.d_out = (uint32_t*)(base + b_chunks + b_seg + b_part + b_pre);
  j.d_flag = (uint32_t*)(base + b_chunks + b_seg + b_part + b_pre + b_out);
  uint8_t* d_in = base + b_chunks + b_seg + b_part + b_pre + b_out + b_flag;
  j.da = a;
  j.ds = s;
  if (!on_device && n) {
    ACK(cudaMemcpyAsync(d_in, a, (size_t)n * 32, cudaMemcpyHostToDevice, st), "copy in");
    j.da = d_in;
    if (pair) {
      ACK(cudaMemcpyAsync(d_in + al((size_t)n * 32), s, (size_t)n * 32, cudaMemcpyHostToDevice, st), "copy in");
      j.ds = d_in + al((size_t)n * 32);
    }
  }
  if (!chunks.empty())
    ACK(cudaMemcpyAsync(j.d_chunks, chunks.data(), chunks.size() * 8, cudaMemcpyHostToDevice, st), "copy in");
  ACK(cudaMemcpyAsync(j.d_seg, j.seg_chunk.data(), (nseg + 1) * 4, cudaMemcpyHostToDevice, st), "copy in");
  if (h_pre) ACK(cudaMemcpyAsync(j.d_pre, h_pre, (size_t)nseg * 32, cudaMemcpyHostToDevice, st), "copy in");
  ACK(cudaMemsetAsync(j.d_flag, 0, 12, st), "memset");
  return SISU_OK;
}

int assoc_launch(AssocJob& j, cudaStream_t st) {
  const uint32_t nchunks = j.nchunks;
  uint32_t* d_next = j.d_flag + 1;  // two chunk counters
  uint32_t* d_unord = j.d_flag + 3;
  if (nchunks) {
    static int occ = 0;
    if (occ == 0) {
      int k = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, k_assoc_chunks, kAssocBD, 0);
      occ = (e == cudaSuccess && k > 0) ? k : 1;
    }
    const unsigned grid = (unsigned)std::min<uint64_t>(nchunks, (uint64_t)kSMs * occ);
    const long prof = prof_begin(j.ord ? kProfAssocPair : kProfAssocHash, (double)j.n * j.NV, st);
    k_assoc_chunks<<<grid, kAssocBD, 0, st>>>((const uint32_t*)j.da, j.d_chunks, nchunks, j.d_part, j.NV, 0, d_next,
                                              j.d_flag);
    int rc = post_launch();
    if (!rc && j.pair) {
      k_assoc_chunks<<<grid, kAssocBD, 0, st>>>((const uint32_t*)j.ds, j.d_chunks, nchunks, j.d_part, j.NV, 1,
                                                d_next + 1, j.d_flag);
      rc = post_launch();
    }
    if (!rc && j.ord) {
      k_order_chunks<<<(unsigned)std::min<uint64_t>(nchunks, (uint64_t)kSMs * 8), kAssocBD, 0, st>>>(
          (const uint32_t*)(j.pair ? j.ds : j.da), j.d_chunks, nchunks, d_unord);
      rc = post_launch();
    }
    prof_end(prof, st);
    if (rc) return cuda_err((cudaError_t)rc, "associative hash");
  }
  const uint32_t warps = j.nseg * j.NV;
  k_assoc_finish<<<(warps * 32 + 255) / 256, 256, 0, st>>>(j.d_part, j.d_seg, j.nseg, j.NV, j.pre ? j.d_pre : nullptr,
                                                            j.d_out, j.d_flag);
  int rc = post_launch();
  if (rc) return cuda_err((cudaError_t)rc, "associative hash");
  return SISU_OK;
}

int assoc_collect(AssocJob& j, cudaStream_t st, uint8_t* out, uint32_t* host_flag, int* seg_unordered) {
  ACK(cudaMemcpyAsync(out, j.d_out, (size_t)j.NV * j.nseg * 32, cudaMemcpyDeviceToHost, st), "copy out");
  ACK(cudaMemcpyAsync(host_flag, j.d_flag, 4, cudaMemcpyDeviceToHost, st), "copy out");
  std::vector<uint32_t> unord(j.ord ? j.nchunks : 0);
  if (j.ord && j.nchunks)
    ACK(cudaMemcpyAsync(unord.data(), j.d_flag + 3, (size_t)j.nchunks * 4, cudaMemcpyDeviceToHost, st), "copy out");
  ACK(cudaStreamSynchronize(st), "associative hash");
  if (j.ord)
    for (uint32_t g = 0; g < j.nseg; ++g) {
      seg_unordered[g] = 0;
      for (uint32_t k = j.seg_chunk[g]; k < j.seg_chunk[g + 1]; ++k) seg_unordered[g] |= (int)unord[k];
    }
  return SISU_OK;
}

int assoc_run(const uint8_t* a, const uint8_t* s, bool pair, bool order, const uint64_t* offsets, uint32_t nseg,
              const uint8_t* h_pre, int on_device, cudaStream_t st, uint8_t* out, uint32_t* host_flag,
              int* seg_unordered) {
  AssocJob j;
  int rc = assoc_prepare(j, a, s, pair, order, offsets, nseg, h_pre, on_device, st);
  if (!rc) rc = assoc_launch(j, st);
  if (!rc) rc = assoc_collect(j, st, out, host_flag, seg_unordered);
  return rc;
}

// acc = (acc + y) mod r for canonical little-endian 256-bit values
void add_mod_r(uint64_t acc[4], const uint8_t* y) {
  static const uint64_t r[4] = {0x43e1f593f0000001ull, 0x2833e84879b97091ull, 0xb85045b68181585dull,
                                0x30644e72e131a029ull};
  uint64_t b[4];
  memcpy(b, y, 32);
  unsigned __int128 c = 0;
  for (int i = 0; i < 4; ++i) {
    c += (unsigned __int128)acc[i] + b[i];
    acc[i] = (uint64_t)c;
    c >>= 64;
  }
  bool ge = c != 0;  // a carry out of 2^256 exceeds r; else compare from the top
  if (!ge) {
    ge = true;
    for (int i = 3; i >= 0; --i)
      if (acc[i] != r[i]) {
        ge = acc[i] > r[i];
        break;
      }
  }
  if (ge) {
    unsigned __int128 bw = 0;
    for (int i = 0; i < 4; ++i) {
      const unsigned __int128 d = (unsigned __int128)acc[i] - r[i] - (uint64_t)bw;
      acc[i] = (uint64_t)d;
      bw = (d >> 64) ? 1 : 0;
    }
  }
}

int check_elems(const uint8_t* p, uint64_t n, int on_device) {
  if (n && !p) return report_error(SISU_ERR_INVALID_ARG, "NULL element array");
  if (on_device && n && ((uintptr_t)p & 15))
    return report_error(SISU_ERR_INVALID_ARG, "device element arrays must be 16-byte aligned");
  if (on_device && n) return require_device(p, "element array");
  return SISU_OK;
}

}  // namespace
}  // namespace sisu

using namespace sisu;

extern "C" int sisu_assoc_hash_segments(const uint8_t* elems, const uint64_t* offsets, uint32_t n_segments,
                                        const uint8_t* h_pre, int on_device, void* stream, uint8_t* out) {
  if (!offsets || !out || n_segments == 0) return report_error(SISU_ERR_INVALID_ARG, "NULL offsets/out or no segment");
  if (offsets[0] != 0) return report_error(SISU_ERR_INVALID_ARG, "offsets[0] must be 0");
  for (uint32_t g = 0; g < n_segments; ++g)
    if (offsets[g + 1] < offsets[g]) return report_error(SISU_ERR_INVALID_ARG, "offsets must not decrease");
  int rc = check_elems(elems, offsets[n_segments], on_device);
  if (rc) return rc;
  uint32_t flag = 0;
  rc = assoc_run(elems, nullptr, false, false, offsets, n_segments, h_pre, on_device, (cudaStream_t)stream, out,
                 &flag, nullptr);
  if (rc) return rc;
  if (flag & kAssocNotCanonical) return report_error(SISU_ERR_NOT_CANONICAL, "an element or h_pre is not below r");
  return SISU_OK;
}

extern "C" int sisu_assoc_hash(const uint8_t* elems, uint64_t n, const uint8_t* h_pre, int on_device, void* stream,
                               uint8_t* out) {
  const uint64_t offsets[2] = {0, n};
  return sisu_assoc_hash_segments(elems, offsets, 1, h_pre, on_device, stream, out);
}

extern "C" int sisu_pairwise_distinct_check_segments(const uint8_t* a, const uint8_t* a_sorted,
                                                     const uint64_t* offsets, uint32_t n_segments, int on_device,
                                                     void* stream, int* results, uint8_t* h_a, uint8_t* h_sorted) {
  if (!offsets || !results || n_segments == 0)
    return report_error(SISU_ERR_INVALID_ARG, "NULL offsets/results or no segment");
  if (offsets[0] != 0) return report_error(SISU_ERR_INVALID_ARG, "offsets[0] must be 0");
  for (uint32_t g = 0; g < n_segments; ++g)
    if (offsets[g + 1] < offsets[g]) return report_error(SISU_ERR_INVALID_ARG, "offsets must not decrease");
  int rc = check_elems(a, offsets[n_segments], on_device);
  if (!rc) rc = check_elems(a_sorted, offsets[n_segments], on_device);
  if (rc) return rc;
  std::vector<uint8_t> h((size_t)64 * n_segments);
  std::vector<int> unord(n_segments);
  uint32_t flag = 0;
  rc = assoc_run(a, a_sorted, true, false, offsets, n_segments, nullptr, on_device, (cudaStream_t)stream, h.data(),
                 &flag, unord.data());
  if (rc) return rc;
  if (flag & kAssocNotCanonical) return report_error(SISU_ERR_NOT_CANONICAL, "an element is not below r");
  for (uint32_t g = 0; g < n_segments; ++g) {
    const uint8_t* hg = h.data() + 64 * (size_t)g;
    if (h_a) memcpy(h_a + 32 * (size_t)g, hg, 32);
    if (h_sorted) memcpy(h_sorted + 32 * (size_t)g, hg + 32, 32);
    results[g] = (memcmp(hg, hg + 32, 32) == 0 && !unord[g]) ? 1 : 0;
  }
  return SISU_OK;
}

extern "C" int sisu_pairwise_distinct_check(const uint8_t* a, const uint8_t* a_sorted, uint64_t n, int on_device,
                                            void* stream, int* result, uint8_t* h_a, uint8_t* h_sorted) {
  const uint64_t offsets[2] = {0, n};
  return sisu_pairwise_distinct_check_segments(a, a_sorted, offsets, 1, on_device, stream, result, h_a, h_sorted);
}

extern "C" int sisu_assoc_epochs(const uint8_t* a, const uint8_t* a_sorted, const uint64_t* slot_offsets,
                                 uint32_t n_slots, uint32_t slots_per_epoch, int on_device, void* stream,
                                 uint8_t* slot_hashes, int* results, uint8_t* h_a, uint8_t* h_sorted) {
  if (!slot_offsets || !slot_hashes || !results || n_slots == 0)
    return report_error(SISU_ERR_INVALID_ARG, "NULL slot offsets/hashes/results or no slot");
  if (slots_per_epoch == 0 || n_slots % slots_per_epoch)
    return report_error(SISU_ERR_INVALID_ARG, "the slots must make whole epochs");
  if (slot_offsets[0] != 0) return report_error(SISU_ERR_INVALID_ARG, "offsets[0] must be 0");
  for (uint32_t g = 0; g < n_slots; ++g)
    if (slot_offsets[g + 1] < slot_offsets[g]) return report_error(SISU_ERR_INVALID_ARG, "offsets must not decrease");
  int rc = check_elems(a, slot_offsets[n_slots], on_device);
  if (!rc) rc = check_elems(a_sorted, slot_offsets[n_slots], on_device);
  if (rc) return rc;
  // Algorithm 1 on every slot of a, and the hash and the order of a_sorted
  // over every epoch: both runs prepared, then both launched, then both
  // collected
  const uint32_t ne = n_slots / slots_per_epoch;
  std::vector<uint64_t> eoff(ne + 1);
  for (uint32_t e = 0; e <= ne; ++e) eoff[e] = slot_offsets[(size_t)e * slots_per_epoch];
  std::vector<uint8_t> hs((size_t)32 * ne);
  std::vector<int> unord(ne);
  const cudaStream_t st = (cudaStream_t)stream;
  AssocJob ja, js;
  rc = assoc_prepare(ja, a, nullptr, false, false, slot_offsets, n_slots, nullptr, on_device, st);
  if (!rc) rc = assoc_prepare(js, a_sorted, nullptr, false, true, eoff.data(), ne, nullptr, on_device, st);
  if (!rc) rc = assoc_launch(ja, st);
  if (!rc) rc = assoc_launch(js, st);
  uint32_t flag_a = 0, flag_s = 0;
  if (!rc) rc = assoc_collect(ja, st, slot_hashes, &flag_a, nullptr);
  if (!rc) rc = assoc_collect(js, st, hs.data(), &flag_s, unord.data());
  if (rc) return rc;
  if ((flag_a | flag_s) & kAssocNotCanonical) return report_error(SISU_ERR_NOT_CANONICAL, "an element is not below r");
  // the hash of a over an epoch: the sum of its slots' hashes
  for (uint32_t e = 0; e < ne; ++e) {
    uint64_t acc[4] = {0, 0, 0, 0};
    for (uint32_t k = 0; k < slots_per_epoch; ++k) add_mod_r(acc, slot_hashes + 32 * ((size_t)e * slots_per_epoch + k));
    uint8_t ha[32];
    memcpy(ha, acc, 32);
    if (h_a) memcpy(h_a + 32 * (size_t)e, ha, 32);
    if (h_sorted) memcpy(h_sorted + 32 * (size_t)e, hs.data() + 32 * (size_t)e, 32);
    results[e] = (memcmp(ha, hs.data() + 32 * (size_t)e, 32) == 0 && !unord[e]) ? 1 : 0;
  }
  return SISU_OK;
}
