// Forward evaluation of the circuit and Merkle statement digests.
//
// Data layout in HBM: layer l's values are a copy-major table of
// 2^c x 2^s_l elements, element (b, g) at index b * 2^s_l + g, each element
// 32 bytes (8 limbs, Montgomery form) so that one element is two 128-bit
// accesses and a gathered element touches exactly one 32-byte sector.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "launch.cuh"
#include "sha256.cuh"

namespace sisu {

// ---------------------------------------------------------------------------
// inputs: canonical -> Montgomery, zero padding, canonicity check

// copies b0 .. b0 + nb - 1 of the input layer
__global__ void k_inputs_to_mont(const uint32_t* in, uint32_t* V, uint32_t b0, uint32_t nb, uint32_t s,
                                 uint32_t Creal, uint32_t wreal, uint32_t* err) {
  const size_t total = (size_t)nb << s;
  const uint32_t mask = (1u << s) - 1u;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
    const size_t idx = ((size_t)b0 << s) + k;
    uint32_t b = (uint32_t)(idx >> s), x = (uint32_t)(idx & mask);
    Fr v = fr_zero();
    if (b < Creal && x < wreal) {
      Fr raw = fr_load(in, (size_t)b * wreal + x);
      if (!fr_lt_modulus(raw)) {
        atomicOr(err, 1u);
        raw = fr_zero();
      }
      v = fr_from_canonical(raw);
    }
    fr_store(V, idx, v);
  }
}

int launch_inputs_to_mont(const uint32_t* in, uint32_t* V, uint32_t b0, uint32_t nb, uint32_t s, uint32_t Creal,
                          uint32_t wreal, uint32_t* err, void* stream) {
  size_t n = (size_t)nb << s;
  k_inputs_to_mont<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(in, V, b0, nb, s, Creal, wreal, err);
  return post_launch();
}

// Montgomery layer -> canonical, unpadded (n_copies x width)
__global__ void k_layer_to_canonical(const uint32_t* V, uint32_t* out, uint32_t s, uint32_t Creal, uint32_t wreal) {
  const size_t total = (size_t)Creal * wreal;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    size_t b = idx / wreal, x = idx % wreal;
    fr_store(out, idx, fr_to_canonical(fr_load(V, (b << s) + x)));
  }
}

int launch_layer_to_canonical(const uint32_t* V, uint32_t* out, uint32_t c, uint32_t s, uint32_t Creal,
                              uint32_t wreal, void* stream) {
  (void)c;
  size_t n = (size_t)Creal * wreal;
  k_layer_to_canonical<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(V, out, s, Creal, wreal);
  return post_launch();
}

// ---------------------------------------------------------------------------
// forward evaluation of one layer (Sec. 2.2): V_i(b, g) = op_g(V_{i+1}(b, in1 g), V_{i+1}(b, in2 g))
//
// Threads walk each copy's gates in the sorted order (mul gates, add gates,
// then the gates with no entry, whose value is 0), so a warp holds one kind
// of gate: with the wiring order nearly every warp mixed the two and all of
// it waited for the Montgomery products of its mul lanes.  The outputs go
// to each gate's own position (one 32-byte sector per element).  Layers
// where every gate has at most one entry only.

__global__ void k_eval_layer(const uint32_t* __restrict__ Vn, uint32_t* __restrict__ V,
                             const uint4* __restrict__ sg, uint32_t nmul, uint32_t ntot, uint32_t b0, uint32_t nb,
                             uint32_t s, uint32_t sn) {
  pdl_wait();
  const size_t total = (size_t)nb << s;
  const uint32_t mask = (1u << s) - 1u;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
    const size_t idx = ((size_t)b0 << s) + k;
    const uint32_t b = (uint32_t)(idx >> s), q = (uint32_t)(idx & mask);
    const uint4 gi = sg[q];
    Fr out = fr_zero();
    if (q < ntot) {
      const uint32_t* row = Vn + (((size_t)b << sn) << 3);
      const Fr x = fr_load(row, gi.x), y = fr_load(row, gi.y);
      out = q < nmul ? fr_mul(x, y) : fr_add(x, y);
    }
    fr_store(V, ((size_t)b << s) + gi.z, out);
  }
}

// A layer of accumulation gates (Sec. 3.4.3): gate g of copy b is the sum
// of its entries eo[offo[g] .. offo[g+1]) (0 when it has none).
__global__ void k_eval_layer_acc(const uint32_t* __restrict__ Vn, uint32_t* __restrict__ V,
                                 const uint32_t* __restrict__ offo, const uint2* __restrict__ eo, uint32_t b0,
                                 uint32_t nb, uint32_t s, uint32_t sn) {
  const size_t total = (size_t)nb << s;
  const uint32_t mask = (1u << s) - 1u;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
    const size_t idx = ((size_t)b0 << s) + k;
    const uint32_t b = (uint32_t)(idx >> s), g = (uint32_t)(idx & mask);
    const uint32_t* row = Vn + (((size_t)b << sn) << 3);
    Fr acc = fr_zero();
    for (uint32_t e = offo[g], ee = offo[g + 1]; e < ee; ++e) {
      const uint2 io = eo[e];
      const Fr x = fr_load(row, io.x & 0x3fffffffu), y = fr_load(row, io.y);
      acc = fr_add(acc, (io.x >> 30) ? fr_mul(x, y) : fr_add(x, y));
    }
    fr_store(V, idx, acc);
  }
}

// The same evaluation with each copy's row of layer i + 1 staged in shared
// memory (rows of at most kRowStageMax elements, 64 KiB): a CTA takes one
// copy at a time, copies the row in with 16-byte cp.async (a hardware wait,
// no spin) and gathers both inputs of every gate from shared memory instead
// of from scattered 32-byte sectors in L2/DRAM; several CTAs per SM keep
// loads of some copies in flight while others compute.
constexpr uint32_t kRowStageMax = 2048;
constexpr uint32_t kRowThreads = 256;

__global__ void __launch_bounds__(kRowThreads) k_eval_layer_row(const uint32_t* __restrict__ Vn,
                                                                uint32_t* __restrict__ V,
                                                                const uint4* __restrict__ sg, uint32_t nmul,
                                                                uint32_t ntot, uint32_t b0, uint32_t nb, uint32_t s,
                                                                uint32_t sn) {
  pdl_wait();
  extern __shared__ __align__(16) uint32_t row[];
  const uint32_t wn16 = 2u << sn, W = 1u << s;  // the row's 16-byte pieces, the layer's gates
  for (uint32_t bi = blockIdx.x; bi < nb; bi += gridDim.x) {
    const size_t b = (size_t)b0 + bi;
    const uint4* src = reinterpret_cast<const uint4*>(Vn + ((b << sn) << 3));
    for (uint32_t k = threadIdx.x; k < wn16; k += kRowThreads)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(row + 4 * k)),
                   "l"(src + k)
                   : "memory");
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < W; q += kRowThreads) {
      const uint4 gi = sg[q];
      Fr out = fr_zero();
      if (q < ntot) {
        const Fr x = fr_load(row, gi.x), y = fr_load(row, gi.y);
        out = q < nmul ? fr_mul(x, y) : fr_add(x, y);
      }
      fr_store(V, (b << s) + gi.z, out);
    }
    __syncthreads();  // the row is read before the next copy's lands
  }
}

int launch_eval_layer(const uint32_t* Vn, uint32_t* V, const DevLayer& L, uint32_t b0, uint32_t nb, uint32_t s,
                      uint32_t sn, void* stream) {
  size_t n = (size_t)nb << s;
  if (!L.offo && (1u << sn) <= kRowStageMax && nb >= kSMs) {
    static int per_sm[12] = {0};
    const size_t smem = (size_t)32 << sn;
    if (smem > 48 * 1024) {
      static bool attr = false;
      if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_eval_layer_row, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(32 * kRowStageMax));
        if (e != cudaSuccess) return (int)e;
        attr = true;
      }
    }
    int& ps = per_sm[sn];
    if (ps == 0) {
      int m = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_eval_layer_row, kRowThreads, smem) != cudaSuccess || m < 1)
        m = 1;
      ps = m;
    }
    const unsigned grid = (unsigned)std::min<size_t>(nb, (size_t)kSMs * ps);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = kRowThreads;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_eval_layer_row, Vn, V, L.sgate, L.nmul, L.ntot, b0, nb, s, sn);
    if (e != cudaSuccess) return (int)e;
    return post_launch();
  }
  if (L.offo)
    k_eval_layer_acc<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(Vn, V, L.offo, L.eo, b0, nb, s, sn);
  else
    return launch_pdl(k_eval_layer, grid_for(n, 256), 256, (cudaStream_t)stream, Vn, V, L.sgate, L.nmul, L.ntot, b0,
                      nb, s, sn);
  return post_launch();
}

// General circuits (Sec. 2.7): the virtual layer X_i of gate layer i, row
// by row: X_i[b][u] = V_{i+1}[b][u] for u < 2^sn, then the used gates of
// deeper layers (map[u - 2^sn] = {layer, gate}), zero up to 2^sx.
__global__ void k_gather_x(GatherLayers gl, uint32_t next, const uint2* __restrict__ map, uint32_t nmap,
                           uint32_t* __restrict__ X, uint32_t C, uint32_t sn, uint32_t sx) {
  const size_t total = (size_t)C << sx;
  const uint32_t wn = 1u << sn, mask = (1u << sx) - 1;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t b = idx >> sx;
    const uint32_t u = (uint32_t)(idx & mask);
    Fr v = fr_zero();
    if (u < wn) {
      v = fr_load(gl.V[next], (b << sn) + u);
    } else if (u - wn < nmap) {
      const uint2 m = map[u - wn];
      v = fr_load(gl.V[m.x], (b << gl.s[m.x]) + m.y);
    }
    fr_store(X, idx, v);
  }
}

int launch_gather_x(const GatherLayers& gl, uint32_t next, const uint2* map, uint32_t nmap, uint32_t* X, uint32_t C,
                    uint32_t sn, uint32_t sx, void* stream) {
  k_gather_x<<<grid_for((size_t)C << sx, 256), 256, 0, (cudaStream_t)stream>>>(gl, next, map, nmap, X, C, sn, sx);
  return post_launch();
}

// ---------------------------------------------------------------------------
// Merkle statement digest over 1024-byte chunks (32 field elements each):
//   leaf = H(chunk || 0x00), node = H(left || right || 0x01),
//   odd last node moved up, digest = H(root || u64le len || 0x03).

__device__ __forceinline__ void elem_words(const uint32_t* tab, size_t i, uint32_t* w) {
  Fr v = fr_to_canonical(fr_load(tab, i));
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = bswap32(v.v[k]);
}

// leaf L of a table of nelem elements: H(32 canonical elements || 0x00)
__device__ __forceinline__ void digest_leaf_table(const uint32_t* __restrict__ tab, size_t nelem, size_t L,
                                                  uint32_t* __restrict__ out) {
  const size_t first = L * 32;
  const uint32_t count = (uint32_t)min((size_t)32, nelem - first);
  uint32_t h[8], blk[16];
  sha256_init(h);
  uint32_t e = 0;
  for (; e + 1 < count; e += 2) {
    elem_words(tab, first + e, blk);
    elem_words(tab, first + e + 1, blk + 8);
    sha256_compress(h, blk);
  }
  const uint64_t bits = ((uint64_t)count * 32 + 1) * 8;
  if (e < count) {  // one element left: it, the tag and the length fit one block
    elem_words(tab, first + e, blk);
    blk[8] = 0x00800000u;
#pragma unroll
    for (int k = 9; k < 14; ++k) blk[k] = 0;
  } else {
    blk[0] = 0x00800000u;
#pragma unroll
    for (int k = 1; k < 14; ++k) blk[k] = 0;
  }
  blk[14] = (uint32_t)(bits >> 32);
  blk[15] = (uint32_t)bits;
  sha256_compress(h, blk);
#pragma unroll
  for (int k = 0; k < 8; ++k) out[L * 8 + k] = h[k];
}

// The leaves of two tables in one launch (the statement's inputs and
// outputs): one grid over both, so neither digest leaves SMs idle in its
// last wave.
__global__ void k_digest_leaves_table2(const uint32_t* __restrict__ ta, size_t na, uint32_t* __restrict__ oa,
                                       const uint32_t* __restrict__ tb, size_t nb, uint32_t* __restrict__ ob) {
  const size_t la = (na + 31) / 32, lb = (nb + 31) / 32;
  for (size_t L = blockIdx.x * (size_t)blockDim.x + threadIdx.x; L < la + lb; L += (size_t)gridDim.x * blockDim.x) {
    if (L < la) digest_leaf_table(ta, na, L, oa);
    else digest_leaf_table(tb, nb, L - la, ob);
  }
}

__global__ void k_digest_leaves_bytes(const uint8_t* __restrict__ data, size_t len, uint32_t* __restrict__ out) {
  const size_t nleaf = (len + 1023) / 1024;
  for (size_t L = blockIdx.x * (size_t)blockDim.x + threadIdx.x; L < nleaf; L += (size_t)gridDim.x * blockDim.x) {
    size_t off = L * 1024, m = min((size_t)1024, len - off);
    Sha256Stream h;
    h.begin();
    h.bytes(data + off, m);
    h.byte(0x00);
    uint32_t o[8];
    h.end(o);
    for (int k = 0; k < 8; ++k) out[L * 8 + k] = o[k];
  }
}

// node j of the next level over n nodes: H(left || right || 0x01), or the
// odd last node moved up
__device__ __forceinline__ void digest_node(const uint32_t* __restrict__ src, size_t n, size_t j,
                                            uint32_t* __restrict__ dst) {
  if (2 * j + 1 < n) {
    uint32_t h[8], blk[16];
    sha256_init(h);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      blk[k] = src[16 * j + k];
      blk[8 + k] = src[16 * j + 8 + k];
    }
    sha256_compress(h, blk);
    blk[0] = 0x01800000u;
#pragma unroll
    for (int k = 1; k < 15; ++k) blk[k] = 0;
    blk[15] = 65 * 8;
    sha256_compress(h, blk);
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[8 * j + k] = h[k];
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[8 * j + k] = src[16 * j + k];
  }
}

__global__ void k_digest_level(const uint32_t* __restrict__ src, size_t n, uint32_t* __restrict__ dst) {
  const size_t m = (n + 1) / 2;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < m; j += (size_t)gridDim.x * blockDim.x)
    digest_node(src, n, j, dst);
}

// one level of two trees (a tree already at its root has no nodes to add)
__global__ void k_digest_level2(const uint32_t* __restrict__ sa, size_t na, uint32_t* __restrict__ da,
                                const uint32_t* __restrict__ sb, size_t nb, uint32_t* __restrict__ db) {
  const size_t ma = na > 1 ? (na + 1) / 2 : 0, mb = nb > 1 ? (nb + 1) / 2 : 0;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < ma + mb; j += (size_t)gridDim.x * blockDim.x) {
    if (j < ma) digest_node(sa, na, j, da);
    else digest_node(sb, nb, j - ma, db);
  }
}

__device__ __forceinline__ void digest_finish(const uint32_t* root, uint64_t len, int empty, uint32_t* out) {
  uint32_t r[8], blk[16], h[8];
  if (empty) {
    sha256_init(r);
    blk[0] = 0x02800000u;
    for (int k = 1; k < 15; ++k) blk[k] = 0;
    blk[15] = 8;
    sha256_compress(r, blk);
  } else {
    for (int k = 0; k < 8; ++k) r[k] = root[k];
  }
  for (int k = 0; k < 8; ++k) blk[k] = r[k];
  blk[8] = bswap32((uint32_t)len);
  blk[9] = bswap32((uint32_t)(len >> 32));
  blk[10] = 0x03800000u;
  for (int k = 11; k < 15; ++k) blk[k] = 0;
  blk[15] = 41 * 8;
  sha256_init(h);
  sha256_compress(h, blk);
  for (int k = 0; k < 8; ++k) out[k] = h[k];
}

__global__ void k_digest_final(const uint32_t* root, uint64_t len, int empty, uint32_t* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  digest_finish(root, len, empty, out);
}

__global__ void k_digest_final2(const uint32_t* ra, uint64_t la, int ea, uint32_t* oa, const uint32_t* rb,
                                uint64_t lb, int eb, uint32_t* ob) {
  if (blockIdx.x != 0 || threadIdx.x >= 2) return;
  if (threadIdx.x == 0) digest_finish(ra, la, ea, oa);
  else digest_finish(rb, lb, eb, ob);
}

size_t digest_scratch_words(size_t len_bytes) { return 2 * 8 * ((len_bytes + 1023) / 1024) + 16; }

static int digest_tree(size_t nleaf, uint64_t len, uint32_t* scratch, uint32_t* out_words, cudaStream_t st) {
  uint32_t* a = scratch;
  uint32_t* b = scratch + 8 * nleaf + 8;
  size_t n = nleaf;
  while (n > 1) {
    size_t m = (n + 1) / 2;
    k_digest_level<<<grid_for(m, 128), 128, 0, st>>>(a, n, b);
    if (int e = post_launch()) return e;
    std::swap(a, b);
    n = m;
  }
  k_digest_final<<<1, 32, 0, st>>>(a, len, nleaf == 0, out_words);
  return post_launch();
}

int launch_digest_tables2(const uint32_t* ta, size_t na, const uint32_t* tb, size_t nb, uint32_t* scratch,
                          uint32_t* out_a, uint32_t* out_b, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const size_t la = (na + 31) / 32, lb = (nb + 31) / 32;
  // each tree ping-pongs between two halves of its own scratch
  uint32_t* a0 = scratch;
  uint32_t* a1 = a0 + 8 * la + 8;
  uint32_t* b0 = scratch + digest_scratch_words(na * 32);
  uint32_t* b1 = b0 + 8 * lb + 8;
  if (la + lb) {
    k_digest_leaves_table2<<<grid_for(la + lb, 128, 32), 128, 0, st>>>(ta, na, a0, tb, nb, b0);
    if (int e = post_launch()) return e;
  }
  size_t n_a = la, n_b = lb;
  while (n_a > 1 || n_b > 1) {
    const size_t m = (n_a > 1 ? (n_a + 1) / 2 : 0) + (n_b > 1 ? (n_b + 1) / 2 : 0);
    k_digest_level2<<<grid_for(m, 128), 128, 0, st>>>(a0, n_a, a1, b0, n_b, b1);
    if (int e = post_launch()) return e;
    if (n_a > 1) {
      std::swap(a0, a1);
      n_a = (n_a + 1) / 2;
    }
    if (n_b > 1) {
      std::swap(b0, b1);
      n_b = (n_b + 1) / 2;
    }
  }
  k_digest_final2<<<1, 32, 0, st>>>(a0, (uint64_t)na * 32, la == 0, out_a, b0, (uint64_t)nb * 32, lb == 0, out_b);
  return post_launch();
}

// Copy-sharded statement digests.  With W >= 32 elements a row (a whole
// number of 1 KiB chunks, a power of two) and a power-of-two copy count,
// the tree over a table is perfect and copy b's leaves form the subtree
// whose root is node b of level log2(W / 32): a rank can form the roots of
// its own copies, and the tree above them needs only those roots.

// The per-copy subtree roots of two tables of nc copies (widths wa, wb
// elements, both at least 32): roots_a[8 j .. 8 j + 7] for the rank's copy
// j, then roots_b likewise.  Scratch: digest_scratch_words of each table.
int launch_digest_copy_roots(const uint32_t* ta, uint32_t wa, const uint32_t* tb, uint32_t wb, uint32_t nc,
                             uint32_t* scratch, uint32_t* roots_a, uint32_t* roots_b, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const size_t na = (size_t)nc * wa, nb = (size_t)nc * wb;
  const size_t la = na / 32, lb = nb / 32;
  uint32_t* a0 = scratch;
  uint32_t* a1 = a0 + 8 * la + 8;
  uint32_t* b0 = scratch + digest_scratch_words(na * 32);
  uint32_t* b1 = b0 + 8 * lb + 8;
  k_digest_leaves_table2<<<grid_for(la + lb, 128, 32), 128, 0, st>>>(ta, na, a0, tb, nb, b0);
  if (int e = post_launch()) return e;
  size_t n_a = la, n_b = lb;
  while (n_a > nc || n_b > nc) {  // down to one node per copy in each tree
    const size_t m = (n_a > nc ? n_a / 2 : 0) + (n_b > nc ? n_b / 2 : 0);
    k_digest_level2<<<grid_for(m, 128), 128, 0, st>>>(a0, n_a > nc ? n_a : 1, a1, b0, n_b > nc ? n_b : 1, b1);
    if (int e = post_launch()) return e;
    if (n_a > nc) {
      std::swap(a0, a1);
      n_a /= 2;
    }
    if (n_b > nc) {
      std::swap(b0, b1);
      n_b /= 2;
    }
  }
  cudaError_t e = cudaMemcpyAsync(roots_a, a0, (size_t)nc * 32, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(roots_b, b0, (size_t)nc * 32, cudaMemcpyDeviceToDevice, st);
  return (int)e;
}

// roots gathered rank by rank (rank q's part: its nc roots of table a, then
// of table b) into copy order: copy b = j * world + q
__global__ void k_roots_to_copy_order(const uint32_t* __restrict__ all, uint32_t nc, uint32_t world,
                                      uint32_t* __restrict__ ra, uint32_t* __restrict__ rb) {
  const size_t total = (size_t)nc * world * 16;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t q = w / ((size_t)nc * 16), rest = w - q * nc * 16;
    const size_t tab = rest / ((size_t)nc * 8), r2 = rest - tab * nc * 8, j = r2 / 8, k = r2 - j * 8;
    (tab == 0 ? ra : rb)[(j * world + q) * 8 + k] = all[w];
  }
}

// The two statement digests from every rank's per-copy roots (all: world
// parts as above, nc copies a rank; tables of nc * world copies of wa and
// wb elements).  Scratch: 2 * digest_scratch_words(nc * world * 1024).
int launch_digest_from_roots(const uint32_t* all, uint32_t nc, uint32_t world, uint32_t wa, uint32_t wb,
                             uint32_t* scratch, uint32_t* out_a, uint32_t* out_b, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const size_t C = (size_t)nc * world;
  uint32_t* a0 = scratch;
  uint32_t* a1 = a0 + 8 * C + 8;
  uint32_t* b0 = scratch + digest_scratch_words(C * 1024);
  uint32_t* b1 = b0 + 8 * C + 8;
  k_roots_to_copy_order<<<grid_for(C * 16, 128), 128, 0, st>>>(all, nc, world, a0, b0);
  if (int e = post_launch()) return e;
  size_t n = C;
  while (n > 1) {
    k_digest_level2<<<grid_for(n, 128), 128, 0, st>>>(a0, n, a1, b0, n, b1);
    if (int e = post_launch()) return e;
    std::swap(a0, a1);
    std::swap(b0, b1);
    n = (n + 1) / 2;
  }
  k_digest_final2<<<1, 32, 0, st>>>(a0, (uint64_t)C * wa * 32, 0, out_a, b0, (uint64_t)C * wb * 32, 0, out_b);
  return post_launch();
}

int launch_digest_bytes(const uint8_t* data, size_t len, uint32_t* scratch, uint32_t* out_words, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  size_t nleaf = (len + 1023) / 1024;
  if (nleaf) {
    k_digest_leaves_bytes<<<grid_for(nleaf, 128, 32), 128, 0, st>>>(data, len, scratch);
    if (int e = post_launch()) return e;
  }
  return digest_tree(nleaf, (uint64_t)len, scratch, out_words, st);
}

}  // namespace sisu
