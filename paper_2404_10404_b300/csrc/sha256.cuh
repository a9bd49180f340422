// SHA-256 (FIPS 180-4) for host and device code of the library.
//
// sha256_compress works on big-endian message words, so the bulk Merkle
// kernels feed it field-element limbs directly (one byte swap per word).
// Sha256Stream hashes short byte strings one byte at a time; the prover's
// transcript runs it in a single thread.
#pragma once
#include <cstddef>
#include <cstdint>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace sisu {

#define SISU_SHA256_K                                                                                \
  0x428a2f98u, 0x71374491u, 0xb5c0fbcfu, 0xe9b5dba5u, 0x3956c25bu, 0x59f111f1u, 0x923f82a4u, 0xab1c5ed5u, \
  0xd807aa98u, 0x12835b01u, 0x243185beu, 0x550c7dc3u, 0x72be5d74u, 0x80deb1feu, 0x9bdc06a7u, 0xc19bf174u, \
  0xe49b69c1u, 0xefbe4786u, 0x0fc19dc6u, 0x240ca1ccu, 0x2de92c6fu, 0x4a7484aau, 0x5cb0a9dcu, 0x76f988dau, \
  0x983e5152u, 0xa831c66du, 0xb00327c8u, 0xbf597fc7u, 0xc6e00bf3u, 0xd5a79147u, 0x06ca6351u, 0x14292967u, \
  0x27b70a85u, 0x2e1b2138u, 0x4d2c6dfcu, 0x53380d13u, 0x650a7354u, 0x766a0abbu, 0x81c2c92eu, 0x92722c85u, \
  0xa2bfe8a1u, 0xa81a664bu, 0xc24b8b70u, 0xc76c51a3u, 0xd192e819u, 0xd6990624u, 0xf40e3585u, 0x106aa070u, \
  0x19a4c116u, 0x1e376c08u, 0x2748774cu, 0x34b0bcb5u, 0x391c0cb3u, 0x4ed8aa4au, 0x5b9cca4fu, 0x682e6ff3u, \
  0x748f82eeu, 0x78a5636fu, 0x84c87814u, 0x8cc70208u, 0x90befffau, 0xa4506cebu, 0xbef9a3f7u, 0xc67178f2u

// round constants of FIPS 180-4 Sec. 4.2.2: one copy in constant memory for
// device code, one for host code
#ifdef __CUDACC__
static __constant__ uint32_t c_sha256_k[64] = {SISU_SHA256_K};
#endif
static const uint32_t h_sha256_k[64] = {SISU_SHA256_K};

__host__ __device__ __forceinline__ void sha256_init(uint32_t h[8]) {
  h[0] = 0x6a09e667u; h[1] = 0xbb67ae85u; h[2] = 0x3c6ef372u; h[3] = 0xa54ff53au;
  h[4] = 0x510e527fu; h[5] = 0x9b05688cu; h[6] = 0x1f83d9abu; h[7] = 0x5be0cd19u;
}

__host__ __device__ __forceinline__ uint32_t sha_rotr(uint32_t x, int n) {
#ifdef __CUDA_ARCH__
  return __funnelshift_r(x, x, n);
#else
  return (x >> n) | (x << (32 - n));
#endif
}

__host__ __device__ __forceinline__ uint32_t bswap32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __byte_perm(x, 0, 0x0123);
#else
  return (x >> 24) | ((x >> 8) & 0xff00u) | ((x << 8) & 0xff0000u) | (x << 24);
#endif
}

// One compression of a 64-byte block given as 16 big-endian words.
__host__ __device__ __forceinline__ void sha256_compress(uint32_t h[8], const uint32_t blk[16]) {
  uint32_t w[16];
  for (int t = 0; t < 16; ++t) w[t] = blk[t];
  uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int t = 0; t < 64; ++t) {
    uint32_t wt;
    if (t < 16) {
      wt = w[t];
    } else {
      uint32_t w15 = w[(t - 15) & 15], w2 = w[(t - 2) & 15];
      uint32_t s0 = sha_rotr(w15, 7) ^ sha_rotr(w15, 18) ^ (w15 >> 3);
      uint32_t s1 = sha_rotr(w2, 17) ^ sha_rotr(w2, 19) ^ (w2 >> 10);
      wt = w[t & 15] + s0 + w[(t - 7) & 15] + s1;
      w[t & 15] = wt;
    }
    uint32_t S1 = sha_rotr(e, 6) ^ sha_rotr(e, 11) ^ sha_rotr(e, 25);
    uint32_t ch = (e & f) ^ (~e & g);
#ifdef __CUDA_ARCH__
    uint32_t t1 = hh + S1 + ch + c_sha256_k[t] + wt;
#else
    uint32_t t1 = hh + S1 + ch + h_sha256_k[t] + wt;
#endif
    uint32_t S0 = sha_rotr(a, 2) ^ sha_rotr(a, 13) ^ sha_rotr(a, 22);
    uint32_t maj = (a & b) ^ (a & c) ^ (b & c);
    hh = g; g = f; f = e; e = d + t1; d = c; c = b; b = a; a = t1 + S0 + maj;
  }
  h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}

// The same compression with only 16 rounds unrolled (four passes): a small
// code footprint for the single-thread transcript, which runs cold at the
// end of a round kernel.
__host__ __device__ __forceinline__ void sha256_compress_compact(uint32_t h[8], const uint32_t blk[16]) {
  uint32_t w[16];
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int t = 0; t < 16; ++t) w[t] = blk[t];
  uint32_t a = h[0], b = h[1], c = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
#ifdef __CUDA_ARCH__
#pragma unroll 1
#endif
  for (int r = 0; r < 64; r += 16) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
    for (int k = 0; k < 16; ++k) {
      uint32_t wt;
      if (r == 0) {
        wt = w[k];
      } else {
        uint32_t w15 = w[(k + 1) & 15], w2 = w[(k + 14) & 15];
        uint32_t s0 = sha_rotr(w15, 7) ^ sha_rotr(w15, 18) ^ (w15 >> 3);
        uint32_t s1 = sha_rotr(w2, 17) ^ sha_rotr(w2, 19) ^ (w2 >> 10);
        wt = w[k] + s0 + w[(k + 9) & 15] + s1;
        w[k] = wt;
      }
      uint32_t S1 = sha_rotr(e, 6) ^ sha_rotr(e, 11) ^ sha_rotr(e, 25);
      uint32_t ch = (e & f) ^ (~e & g);
#ifdef __CUDA_ARCH__
      uint32_t t1 = hh + S1 + ch + c_sha256_k[r + k] + wt;
#else
      uint32_t t1 = hh + S1 + ch + h_sha256_k[r + k] + wt;
#endif
      uint32_t S0 = sha_rotr(a, 2) ^ sha_rotr(a, 13) ^ sha_rotr(a, 22);
      uint32_t maj = (a & b) ^ (a & c) ^ (b & c);
      hh = g; g = f; f = e; e = d + t1; d = c; c = b; b = a; a = t1 + S0 + maj;
    }
  }
  h[0] += a; h[1] += b; h[2] += c; h[3] += d; h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}

// Chaining value and message block passed by value, so that an out-of-line
// compression keeps them in registers.
struct ShaWords8 {
  uint32_t w[8];
};
struct ShaWords16 {
  uint32_t w[16];
};

#ifdef __CUDACC__
// One out-of-line copy of the fully unrolled compression per translation
// unit for the single-thread transcript: with its code in the instruction
// caches the unrolled rounds run about 1.4x faster than the compact loop.
static __device__ __noinline__ ShaWords8 sha256_compress_v(ShaWords8 h, ShaWords16 blk) {
  sha256_compress(h.w, blk.w);
  return h;
}
// The compact loop (a quarter of the code) for a transcript that runs cold
// and once: there fetching the unrolled code costs more than the loop saves
// (measured in the copy-phase rounds before they warmed the unrolled code).
static __device__ __noinline__ ShaWords8 sha256_compress_small_v(ShaWords8 h, ShaWords16 blk) {
  sha256_compress_compact(h.w, blk.w);
  return h;
}
#endif

// Out-of-line compression for the byte-stream hasher: it is called from
// many single-thread call sites, where inlining the unrolled rounds would
// only grow the code.
#ifdef __CUDACC__
static __device__ __noinline__ void sha256_compress_call(uint32_t h[8], const uint32_t blk[16]) {
  sha256_compress_compact(h, blk);
}
__host__ __device__ __forceinline__ void sha256_compress_stream(uint32_t h[8], const uint32_t blk[16]) {
#ifdef __CUDA_ARCH__
  sha256_compress_call(h, blk);
#else
  sha256_compress(h, blk);
#endif
}
#else
inline void sha256_compress_stream(uint32_t h[8], const uint32_t blk[16]) { sha256_compress(h, blk); }
#endif

// Incremental hashing of a byte stream (small messages).
struct Sha256Stream {
  uint32_t h[8];
  uint32_t blk[16];
  uint32_t fill;   // bytes in the current block
  uint64_t total;  // bytes so far

  __host__ __device__ void begin() {
    sha256_init(h);
    fill = 0;
    total = 0;
    for (int i = 0; i < 16; ++i) blk[i] = 0;
  }
  __host__ __device__ void byte(uint8_t b) {
    blk[fill >> 2] |= (uint32_t)b << (24 - 8 * (fill & 3));
    ++fill;
    ++total;
    if (fill == 64) {
      sha256_compress_stream(h, blk);
      fill = 0;
      for (int i = 0; i < 16; ++i) blk[i] = 0;
    }
  }
  __host__ __device__ void bytes(const uint8_t* p, size_t n) {
    for (size_t i = 0; i < n; ++i) byte(p[i]);
  }
  // 32-bit word written little-endian (a field-element limb)
  __host__ __device__ void u32le(uint32_t v) {
    byte((uint8_t)v); byte((uint8_t)(v >> 8)); byte((uint8_t)(v >> 16)); byte((uint8_t)(v >> 24));
  }
  // 32-byte digest given as 8 big-endian words
  __host__ __device__ void digest_words(const uint32_t d[8]) {
    for (int i = 0; i < 8; ++i) {
      byte((uint8_t)(d[i] >> 24)); byte((uint8_t)(d[i] >> 16)); byte((uint8_t)(d[i] >> 8)); byte((uint8_t)d[i]);
    }
  }
  __host__ __device__ void end(uint32_t out[8]) {
    uint64_t bits = total * 8;
    byte(0x80);
    while (fill != 56) byte(0);
    for (int i = 7; i >= 0; --i) byte((uint8_t)(bits >> (8 * i)));
    for (int i = 0; i < 8; ++i) out[i] = h[i];
  }
};

}  // namespace sisu
