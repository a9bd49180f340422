// Field core: the BN254 scalar field F_r (the paper's choice of BN254,
// Sec. 4.1), for the sm_103a integer pipes.
//
// Representation: 8 x 32-bit little-endian limbs in Montgomery form,
// x_mont = x * 2^256 mod r.  Values are kept *lazily reduced* in [0, 2r):
// r < 2^254, so 4r < 2^256 and the CIOS product of two values below 2r is
// again below 2r without a final subtraction.  Additions and subtractions
// reduce once against 2r.  Canonical form ([0, r), not Montgomery) is used
// only at the boundary: inputs, proof bytes, transcript hashing.
//
// Multiplication is coarsely integrated operand scanning (CIOS, Koc, Acar
// and Kaliski 1996) written as PTX carry chains.  Every carry chain, with
// the instruction that consumes its final carry, sits inside one asm block:
// the carry flag is not preserved between separate asm statements.
#pragma once
#include <cstdint>

namespace sisu {

struct Fr {
  uint32_t v[8];
};

#ifdef __CUDACC__

#define SISU_FR_CONST(name, a0, a1, a2, a3, a4, a5, a6, a7) \
  __device__ __forceinline__ Fr name() {                     \
    Fr o;                                                    \
    o.v[0] = a0; o.v[1] = a1; o.v[2] = a2; o.v[3] = a3;      \
    o.v[4] = a4; o.v[5] = a5; o.v[6] = a6; o.v[7] = a7;      \
    return o;                                                \
  }

SISU_FR_CONST(fr_zero, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u)
// Montgomery form of 1: 2^256 mod r
SISU_FR_CONST(fr_one, 0x4ffffffbu, 0xac96341cu, 0x9f60cd29u, 0x36fc7695u, 0x7879462eu, 0x666ea36fu,
              0x9a07df2fu, 0x0e0a77c1u)
// 2^512 mod r: one product with it maps canonical -> Montgomery
SISU_FR_CONST(fr_r2, 0xae216da7u, 0x1bb8e645u, 0xe35c59e3u, 0x53fe3ab1u, 0x53bb8085u, 0x8c49833du,
              0x7f4e44a5u, 0x0216d0b1u)
// the integer 1 (a product with it maps Montgomery -> canonical)
SISU_FR_CONST(fr_int_one, 1u, 0u, 0u, 0u, 0u, 0u, 0u, 0u)
SISU_FR_CONST(fr_modulus, 0xf0000001u, 0x43e1f593u, 0x79b97091u, 0x2833e848u, 0x8181585du, 0xb85045b6u,
              0xe131a029u, 0x30644e72u)

// ---------------------------------------------------------------------------
// loads and stores of one 32-byte element (two 128-bit accesses)

__device__ __forceinline__ Fr fr_load(const uint32_t* __restrict__ base, size_t idx) {
  const uint4* p = reinterpret_cast<const uint4*>(base + 8 * idx);
  uint4 a = p[0], b = p[1];
  Fr x;
  x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
  x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
  return x;
}

// through L2 only: for data that other blocks of the same grid wrote
__device__ __forceinline__ Fr fr_load_cg(const uint32_t* base, size_t idx) {
  const uint4* p = reinterpret_cast<const uint4*>(base + 8 * idx);
  uint4 a = __ldcg(p), b = __ldcg(p + 1);
  Fr x;
  x.v[0] = a.x; x.v[1] = a.y; x.v[2] = a.z; x.v[3] = a.w;
  x.v[4] = b.x; x.v[5] = b.y; x.v[6] = b.z; x.v[7] = b.w;
  return x;
}

__device__ __forceinline__ void fr_store(uint32_t* __restrict__ base, size_t idx, const Fr& x) {
  uint4* p = reinterpret_cast<uint4*>(base + 8 * idx);
  p[0] = make_uint4(x.v[0], x.v[1], x.v[2], x.v[3]);
  p[1] = make_uint4(x.v[4], x.v[5], x.v[6], x.v[7]);
}

__device__ __forceinline__ void fr_store_cg(uint32_t* base, size_t idx, const Fr& x) {
  uint4* p = reinterpret_cast<uint4*>(base + 8 * idx);
  __stcg(p, make_uint4(x.v[0], x.v[1], x.v[2], x.v[3]));
  __stcg(p + 1, make_uint4(x.v[4], x.v[5], x.v[6], x.v[7]));
}

// ---------------------------------------------------------------------------
// addition and subtraction, inputs and outputs in [0, 2r)

__device__ __forceinline__ Fr fr_add(const Fr& a, const Fr& b) {
  Fr s = a, d;
  uint32_t keep;  // all ones when s < 2r
  asm("{\n\t"
      ".reg .u32 z;\n\t"
      "mov.u32 z, 0;\n\t"
      "add.cc.u32  %0, %0, %17;\n\t"
      "addc.cc.u32 %1, %1, %18;\n\t"
      "addc.cc.u32 %2, %2, %19;\n\t"
      "addc.cc.u32 %3, %3, %20;\n\t"
      "addc.cc.u32 %4, %4, %21;\n\t"
      "addc.cc.u32 %5, %5, %22;\n\t"
      "addc.cc.u32 %6, %6, %23;\n\t"
      "addc.u32    %7, %7, %24;\n\t"
      "sub.cc.u32  %8,  %0, 0xe0000002;\n\t"
      "subc.cc.u32 %9,  %1, 0x87c3eb27;\n\t"
      "subc.cc.u32 %10, %2, 0xf372e122;\n\t"
      "subc.cc.u32 %11, %3, 0x5067d090;\n\t"
      "subc.cc.u32 %12, %4, 0x0302b0ba;\n\t"
      "subc.cc.u32 %13, %5, 0x70a08b6d;\n\t"
      "subc.cc.u32 %14, %6, 0xc2634053;\n\t"
      "subc.cc.u32 %15, %7, 0x60c89ce5;\n\t"
      "subc.u32    %16, z, z;\n\t"
      "}"
      : "+r"(s.v[0]), "+r"(s.v[1]), "+r"(s.v[2]), "+r"(s.v[3]), "+r"(s.v[4]), "+r"(s.v[5]),
        "+r"(s.v[6]), "+r"(s.v[7]), "=r"(d.v[0]), "=r"(d.v[1]), "=r"(d.v[2]), "=r"(d.v[3]),
        "=r"(d.v[4]), "=r"(d.v[5]), "=r"(d.v[6]), "=r"(d.v[7]), "=r"(keep)
      : "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]), "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]),
        "r"(b.v[7]));
  Fr r;
#pragma unroll
  for (int i = 0; i < 8; ++i) r.v[i] = (s.v[i] & keep) | (d.v[i] & ~keep);
  return r;
}

__device__ __forceinline__ Fr fr_sub(const Fr& a, const Fr& b) {
  Fr d = a;
  asm("{\n\t"
      ".reg .u32 z, m, t0, t1, t2, t3, t4, t5, t6, t7;\n\t"
      "mov.u32 z, 0;\n\t"
      "sub.cc.u32  %0, %0, %8;\n\t"
      "subc.cc.u32 %1, %1, %9;\n\t"
      "subc.cc.u32 %2, %2, %10;\n\t"
      "subc.cc.u32 %3, %3, %11;\n\t"
      "subc.cc.u32 %4, %4, %12;\n\t"
      "subc.cc.u32 %5, %5, %13;\n\t"
      "subc.cc.u32 %6, %6, %14;\n\t"
      "subc.cc.u32 %7, %7, %15;\n\t"
      "subc.u32    m, z, z;\n\t"
      "and.b32 t0, m, 0xe0000002;\n\t"
      "and.b32 t1, m, 0x87c3eb27;\n\t"
      "and.b32 t2, m, 0xf372e122;\n\t"
      "and.b32 t3, m, 0x5067d090;\n\t"
      "and.b32 t4, m, 0x0302b0ba;\n\t"
      "and.b32 t5, m, 0x70a08b6d;\n\t"
      "and.b32 t6, m, 0xc2634053;\n\t"
      "and.b32 t7, m, 0x60c89ce5;\n\t"
      "add.cc.u32  %0, %0, t0;\n\t"
      "addc.cc.u32 %1, %1, t1;\n\t"
      "addc.cc.u32 %2, %2, t2;\n\t"
      "addc.cc.u32 %3, %3, t3;\n\t"
      "addc.cc.u32 %4, %4, t4;\n\t"
      "addc.cc.u32 %5, %5, t5;\n\t"
      "addc.cc.u32 %6, %6, t6;\n\t"
      "addc.u32    %7, %7, t7;\n\t"
      "}"
      : "+r"(d.v[0]), "+r"(d.v[1]), "+r"(d.v[2]), "+r"(d.v[3]), "+r"(d.v[4]), "+r"(d.v[5]),
        "+r"(d.v[6]), "+r"(d.v[7])
      : "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]), "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]),
        "r"(b.v[7]));
  return d;
}

__device__ __forceinline__ Fr fr_dbl(const Fr& a) { return fr_add(a, a); }

// ---------------------------------------------------------------------------
// Montgomery product a * b * 2^-256 mod r, inputs and output in [0, 2r).
//
// One CIOS step for limb bi of b: t += a * bi (9 words), m = t0 * (-r^-1),
// t += m * r, t >>= 32.  The products by the low limb of r, 0xf0000001 =
// 2^32 - 2^28 + 1, go without multiplies: m r_0 = m 2^32 - (m >> 4) 2^32 +
// (m - (m << 28) mod 2^32), the last term borrowing from the high word;
// t0 + m r_0 is 0 modulo 2^32 by the choice of m, so its low word only
// sets the carry (t0 != 0), and the high word m - (m >> 4) - borrow is added
// to t1 (2-3% more products a second in the microbenchmark, kinds 2 and
// 15).  With a < 2r and t < 3r at the start of a step the
// running value stays below 3r (1 + 2^32) < 2^288, so nine words never
// overflow and no tenth word is needed (this uses r < 2^254).

#define SISU_CIOS_STEP(BI)                                                                   \
  t8 = 0;                                                                                    \
  asm("{\n\t"                                                                                \
      ".reg .u32 m, s, q, hh;\n\t"                                                           \
      "mad.lo.cc.u32  %0, %9,  %17, %0;\n\t"                                                 \
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"                                                 \
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"                                                 \
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"                                                 \
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"                                                 \
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"                                                 \
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"                                                 \
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"                                                 \
      "addc.u32       %8, %8, 0;\n\t"                                                        \
      "mad.hi.cc.u32  %1, %9,  %17, %1;\n\t"                                                 \
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"                                                 \
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"                                                 \
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"                                                 \
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"                                                 \
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"                                                 \
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"                                                 \
      "madc.hi.u32    %8, %16, %17, %8;\n\t"                                                 \
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"                                                    \
      "shl.b32 s, m, 28;\n\t"                                                               \
      "sub.cc.u32 s, m, s;\n\t"                                                             \
      "shr.u32 q, m, 4;\n\t"                                                                \
      "subc.u32 hh, m, q;\n\t"                                                              \
      "add.cc.u32 %0, %0, 0xffffffff;\n\t"                                                  \
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"                                            \
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"                                            \
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"                                            \
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"                                            \
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"                                            \
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"                                            \
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"                                            \
      "addc.u32       %8, %8, 0;\n\t"                                                        \
      "add.cc.u32     %1, %1, hh;\n\t"                                                      \
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"                                            \
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"                                            \
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"                                            \
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"                                            \
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"                                            \
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"                                            \
      "madc.hi.u32    %8, m, 0x30644e72, %8;\n\t"                                            \
      "}"                                                                                    \
      : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7),      \
        "+r"(t8)                                                                             \
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),        \
        "r"(a.v[6]), "r"(a.v[7]), "r"(BI));                                                  \
  t0 = t1; t1 = t2; t2 = t3; t3 = t4; t4 = t5; t5 = t6; t6 = t7; t7 = t8;

// the same step with the products by r_0 as multiply-adds (kind 15)
#define SISU_CIOS_STEP_MADR0(BI)                                                                   \
  t8 = 0;                                                                                    \
  asm("{\n\t"                                                                                \
      ".reg .u32 m;\n\t"                                                                     \
      "mad.lo.cc.u32  %0, %9,  %17, %0;\n\t"                                                 \
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"                                                 \
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"                                                 \
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"                                                 \
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"                                                 \
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"                                                 \
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"                                                 \
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"                                                 \
      "addc.u32       %8, %8, 0;\n\t"                                                        \
      "mad.hi.cc.u32  %1, %9,  %17, %1;\n\t"                                                 \
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"                                                 \
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"                                                 \
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"                                                 \
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"                                                 \
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"                                                 \
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"                                                 \
      "madc.hi.u32    %8, %16, %17, %8;\n\t"                                                 \
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"                                                    \
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"                                            \
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"                                            \
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"                                            \
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"                                            \
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"                                            \
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"                                            \
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"                                            \
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"                                            \
      "addc.u32       %8, %8, 0;\n\t"                                                        \
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"                                            \
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"                                            \
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"                                            \
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"                                            \
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"                                            \
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"                                            \
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"                                            \
      "madc.hi.u32    %8, m, 0x30644e72, %8;\n\t"                                            \
      "}"                                                                                    \
      : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7),      \
        "+r"(t8)                                                                             \
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),        \
        "r"(a.v[6]), "r"(a.v[7]), "r"(BI));                                                  \
  t0 = t1; t1 = t2; t2 = t3; t3 = t4; t4 = t5; t5 = t6; t6 = t7; t7 = t8;

// the same step on named operand and accumulator words
#define SISU_CIOS_STEP_ON(A, BI, t0, t1, t2, t3, t4, t5, t6, t7, t8)                     \
  t8 = 0;                                                                                    \
  asm("{\n\t"                                                                                \
      ".reg .u32 m, s, q, hh;\n\t"                                                           \
      "mad.lo.cc.u32  %0, %9,  %17, %0;\n\t"                                                 \
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"                                                 \
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"                                                 \
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"                                                 \
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"                                                 \
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"                                                 \
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"                                                 \
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"                                                 \
      "addc.u32       %8, %8, 0;\n\t"                                                        \
      "mad.hi.cc.u32  %1, %9,  %17, %1;\n\t"                                                 \
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"                                                 \
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"                                                 \
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"                                                 \
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"                                                 \
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"                                                 \
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"                                                 \
      "madc.hi.u32    %8, %16, %17, %8;\n\t"                                                 \
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"                                                    \
      "shl.b32 s, m, 28;\n\t"                                                               \
      "sub.cc.u32 s, m, s;\n\t"                                                             \
      "shr.u32 q, m, 4;\n\t"                                                                \
      "subc.u32 hh, m, q;\n\t"                                                              \
      "add.cc.u32 %0, %0, 0xffffffff;\n\t"                                                  \
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"                                            \
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"                                            \
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"                                            \
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"                                            \
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"                                            \
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"                                            \
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"                                            \
      "addc.u32       %8, %8, 0;\n\t"                                                        \
      "add.cc.u32     %1, %1, hh;\n\t"                                                      \
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"                                            \
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"                                            \
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"                                            \
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"                                            \
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"                                            \
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"                                            \
      "madc.hi.u32    %8, m, 0x30644e72, %8;\n\t"                                            \
      "}"                                                                                    \
      : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7),      \
        "+r"(t8)                                                                             \
      : "r"(A.v[0]), "r"(A.v[1]), "r"(A.v[2]), "r"(A.v[3]), "r"(A.v[4]), "r"(A.v[5]),        \
        "r"(A.v[6]), "r"(A.v[7]), "r"(BI));                                                  \
  t0 = t1; t1 = t2; t2 = t3; t3 = t4; t4 = t5; t5 = t6; t6 = t7; t7 = t8;

__device__ __forceinline__ Fr fr_mul_inl(const Fr& a, const Fr& b) {
  uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0, t8;
  SISU_CIOS_STEP(b.v[0])
  SISU_CIOS_STEP(b.v[1])
  SISU_CIOS_STEP(b.v[2])
  SISU_CIOS_STEP(b.v[3])
  SISU_CIOS_STEP(b.v[4])
  SISU_CIOS_STEP(b.v[5])
  SISU_CIOS_STEP(b.v[6])
  SISU_CIOS_STEP(b.v[7])
  Fr r;
  r.v[0] = t0; r.v[1] = t1; r.v[2] = t2; r.v[3] = t3;
  r.v[4] = t4; r.v[5] = t5; r.v[6] = t6; r.v[7] = t7;
  return r;
}

// The product with r_0's products as multiply-adds (kind 15)
__device__ __forceinline__ Fr fr_mul_madr0_inl(const Fr& a, const Fr& b) {
  uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0, t8;
  SISU_CIOS_STEP_MADR0(b.v[0])
  SISU_CIOS_STEP_MADR0(b.v[1])
  SISU_CIOS_STEP_MADR0(b.v[2])
  SISU_CIOS_STEP_MADR0(b.v[3])
  SISU_CIOS_STEP_MADR0(b.v[4])
  SISU_CIOS_STEP_MADR0(b.v[5])
  SISU_CIOS_STEP_MADR0(b.v[6])
  SISU_CIOS_STEP_MADR0(b.v[7])
  Fr r;
  r.v[0] = t0; r.v[1] = t1; r.v[2] = t2; r.v[3] = t3;
  r.v[4] = t4; r.v[5] = t5; r.v[6] = t6; r.v[7] = t7;
  return r;
}
static __device__ __noinline__ Fr fr_mul_madr0_call(Fr a, Fr b) { return fr_mul_madr0_inl(a, b); }

// The same CIOS product with every 32x32 partial product formed as one
// 64-bit multiply (mul.wide.u32) and the carries in pure add chains.
#define SISU_ROW_ADD(P0, P1, P2, P3, P4, P5, P6, P7)                                          \
  asm("add.cc.u32  %0, %0, %9;\n\t"                                                          \
      "addc.cc.u32 %1, %1, %10;\n\t"                                                         \
      "addc.cc.u32 %2, %2, %11;\n\t"                                                         \
      "addc.cc.u32 %3, %3, %12;\n\t"                                                         \
      "addc.cc.u32 %4, %4, %13;\n\t"                                                         \
      "addc.cc.u32 %5, %5, %14;\n\t"                                                         \
      "addc.cc.u32 %6, %6, %15;\n\t"                                                         \
      "addc.cc.u32 %7, %7, %16;\n\t"                                                         \
      "addc.u32    %8, %8, 0;\n\t"                                                           \
      "add.cc.u32  %1, %1, %17;\n\t"                                                         \
      "addc.cc.u32 %2, %2, %18;\n\t"                                                         \
      "addc.cc.u32 %3, %3, %19;\n\t"                                                         \
      "addc.cc.u32 %4, %4, %20;\n\t"                                                         \
      "addc.cc.u32 %5, %5, %21;\n\t"                                                         \
      "addc.cc.u32 %6, %6, %22;\n\t"                                                         \
      "addc.cc.u32 %7, %7, %23;\n\t"                                                         \
      "addc.u32    %8, %8, %24;\n\t"                                                         \
      : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "+r"(t4), "+r"(t5), "+r"(t6), "+r"(t7), "+r"(t8) \
      : "r"((uint32_t)(P0)), "r"((uint32_t)(P1)), "r"((uint32_t)(P2)), "r"((uint32_t)(P3)),     \
        "r"((uint32_t)(P4)), "r"((uint32_t)(P5)), "r"((uint32_t)(P6)), "r"((uint32_t)(P7)),     \
        "r"((uint32_t)((P0) >> 32)), "r"((uint32_t)((P1) >> 32)), "r"((uint32_t)((P2) >> 32)), \
        "r"((uint32_t)((P3) >> 32)), "r"((uint32_t)((P4) >> 32)), "r"((uint32_t)((P5) >> 32)), \
        "r"((uint32_t)((P6) >> 32)), "r"((uint32_t)((P7) >> 32)))

#define SISU_CIOS_WIDE_STEP(BI)                                                               \
  {                                                                                          \
    const uint64_t bi_ = (BI);                                                               \
    t8 = 0;                                                                                  \
    SISU_ROW_ADD(a.v[0] * bi_, a.v[1] * bi_, a.v[2] * bi_, a.v[3] * bi_, a.v[4] * bi_,        \
                 a.v[5] * bi_, a.v[6] * bi_, a.v[7] * bi_);                                  \
    const uint64_t m_ = (uint32_t)(t0 * SISU_NINV_C);                                        \
    SISU_ROW_ADD(m_ * 0xf0000001ull, m_ * 0x43e1f593ull, m_ * 0x79b97091ull, m_ * 0x2833e848ull, \
                 m_ * 0x8181585dull, m_ * 0xb85045b6ull, m_ * 0xe131a029ull, m_ * 0x30644e72ull); \
    t0 = t1; t1 = t2; t2 = t3; t3 = t4; t4 = t5; t5 = t6; t6 = t7; t7 = t8;                   \
  }

#define SISU_NINV_C 0xefffffffu

__device__ __forceinline__ Fr fr_mul_wide_inl(const Fr& a, const Fr& b) {
  uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0, t8;
  SISU_CIOS_WIDE_STEP(b.v[0])
  SISU_CIOS_WIDE_STEP(b.v[1])
  SISU_CIOS_WIDE_STEP(b.v[2])
  SISU_CIOS_WIDE_STEP(b.v[3])
  SISU_CIOS_WIDE_STEP(b.v[4])
  SISU_CIOS_WIDE_STEP(b.v[5])
  SISU_CIOS_WIDE_STEP(b.v[6])
  SISU_CIOS_WIDE_STEP(b.v[7])
  Fr r;
  r.v[0] = t0; r.v[1] = t1; r.v[2] = t2; r.v[3] = t3;
  r.v[4] = t4; r.v[5] = t5; r.v[6] = t6; r.v[7] = t7;
  return r;
}

static __device__ __noinline__ Fr fr_mul_wide_call(Fr a, Fr b) { return fr_mul_wide_inl(a, b); }

// One out-of-line copy of the product per translation unit: a kernel that
// inlined every product would hold tens of kilobytes of straight-line code
// in its inner loop and stall on instruction fetch.  Operands and result
// travel in registers.
static __device__ __noinline__ Fr fr_mul_call(Fr a, Fr b) { return fr_mul_inl(a, b); }

__device__ __forceinline__ Fr fr_mul(const Fr& a, const Fr& b) { return fr_mul_call(a, b); }

// Two independent Montgomery products in one call, their CIOS steps
// interleaved (each step's carry chain stays inside its own asm block), so
// that the scheduler can issue one product's chain while the other waits:
// more instruction-level parallelism for kernels with few warps an SM.
struct Fr2 {
  Fr a, b;
};

__device__ __forceinline__ Fr2 fr_mul2_inl(const Fr& a, const Fr& b, const Fr& c, const Fr& d) {
  Fr2 o;
  {
    uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0, t7 = 0, t8;
    uint32_t u0 = 0, u1 = 0, u2 = 0, u3 = 0, u4 = 0, u5 = 0, u6 = 0, u7 = 0, u8;
#define SISU_CIOS_PAIR(I)                                                        \
  {                                                                              \
    SISU_CIOS_STEP(b.v[I])                                                       \
  }                                                                              \
  {                                                                              \
    uint32_t& q0 = u0; uint32_t& q1 = u1; uint32_t& q2 = u2; uint32_t& q3 = u3;  \
    uint32_t& q4 = u4; uint32_t& q5 = u5; uint32_t& q6 = u6; uint32_t& q7 = u7;  \
    uint32_t& q8 = u8;                                                           \
    SISU_CIOS_STEP_ON(c, d.v[I], q0, q1, q2, q3, q4, q5, q6, q7, q8)             \
  }
    SISU_CIOS_PAIR(0)
    SISU_CIOS_PAIR(1)
    SISU_CIOS_PAIR(2)
    SISU_CIOS_PAIR(3)
    SISU_CIOS_PAIR(4)
    SISU_CIOS_PAIR(5)
    SISU_CIOS_PAIR(6)
    SISU_CIOS_PAIR(7)
#undef SISU_CIOS_PAIR
    o.a.v[0] = t0; o.a.v[1] = t1; o.a.v[2] = t2; o.a.v[3] = t3;
    o.a.v[4] = t4; o.a.v[5] = t5; o.a.v[6] = t6; o.a.v[7] = t7;
    o.b.v[0] = u0; o.b.v[1] = u1; o.b.v[2] = u2; o.b.v[3] = u3;
    o.b.v[4] = u4; o.b.v[5] = u5; o.b.v[6] = u6; o.b.v[7] = u7;
  }
  return o;
}

static __device__ __noinline__ Fr2 fr_mul2_call(Fr a, Fr b, Fr c, Fr d) { return fr_mul2_inl(a, b, c, d); }

// a b 2^-256 and c d 2^-256 (mod r), inputs and outputs in [0, 2r)
__device__ __forceinline__ Fr2 fr_mul2(const Fr& a, const Fr& b, const Fr& c, const Fr& d) {
  return fr_mul2_call(a, b, c, d);
}

// Montgomery square a^2 2^-256 mod p, input and output in [0, 2p): the
// 512-bit square from its 28 off-diagonal products (doubled) and 8
// diagonal ones, then eight word-by-word Montgomery steps.  72 multiply
// halves for the square where a general product takes 128; the bound
// a^2 + m p < 4p^2 + 2^256 p < 2^511 keeps every carry inside 16 words and
// the result below 2p (4p < 2^256).
__device__ __forceinline__ Fr fr_sqr_inl(const Fr& a) {
  uint32_t t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = 0;
  asm("mad.lo.cc.u32 %0, %9, %10, %0;\n\t" "madc.lo.cc.u32 %1, %9, %11, %1;\n\t" "madc.lo.cc.u32 %2, %9, %12, %2;\n\t" "madc.lo.cc.u32 %3, %9, %13, %3;\n\t" "madc.lo.cc.u32 %4, %9, %14, %4;\n\t" "madc.lo.cc.u32 %5, %9, %15, %5;\n\t" "madc.lo.cc.u32 %6, %9, %16, %6;\n\t" "addc.cc.u32 %7, %7, 0;\n\t" "addc.u32 %8, %8, 0;\n\t" "mad.hi.cc.u32 %1, %9, %10, %1;\n\t" "madc.hi.cc.u32 %2, %9, %11, %2;\n\t" "madc.hi.cc.u32 %3, %9, %12, %3;\n\t" "madc.hi.cc.u32 %4, %9, %13, %4;\n\t" "madc.hi.cc.u32 %5, %9, %14, %5;\n\t" "madc.hi.cc.u32 %6, %9, %15, %6;\n\t" "madc.hi.cc.u32 %7, %9, %16, %7;\n\t" "addc.u32 %8, %8, 0;\n\t" : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]) : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  asm("mad.lo.cc.u32 %0, %8, %9, %0;\n\t" "madc.lo.cc.u32 %1, %8, %10, %1;\n\t" "madc.lo.cc.u32 %2, %8, %11, %2;\n\t" "madc.lo.cc.u32 %3, %8, %12, %3;\n\t" "madc.lo.cc.u32 %4, %8, %13, %4;\n\t" "madc.lo.cc.u32 %5, %8, %14, %5;\n\t" "addc.cc.u32 %6, %6, 0;\n\t" "addc.u32 %7, %7, 0;\n\t" "mad.hi.cc.u32 %1, %8, %9, %1;\n\t" "madc.hi.cc.u32 %2, %8, %10, %2;\n\t" "madc.hi.cc.u32 %3, %8, %11, %3;\n\t" "madc.hi.cc.u32 %4, %8, %12, %4;\n\t" "madc.hi.cc.u32 %5, %8, %13, %5;\n\t" "madc.hi.cc.u32 %6, %8, %14, %6;\n\t" "addc.u32 %7, %7, 0;\n\t" : "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]) : "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  asm("mad.lo.cc.u32 %0, %7, %8, %0;\n\t" "madc.lo.cc.u32 %1, %7, %9, %1;\n\t" "madc.lo.cc.u32 %2, %7, %10, %2;\n\t" "madc.lo.cc.u32 %3, %7, %11, %3;\n\t" "madc.lo.cc.u32 %4, %7, %12, %4;\n\t" "addc.cc.u32 %5, %5, 0;\n\t" "addc.u32 %6, %6, 0;\n\t" "mad.hi.cc.u32 %1, %7, %8, %1;\n\t" "madc.hi.cc.u32 %2, %7, %9, %2;\n\t" "madc.hi.cc.u32 %3, %7, %10, %3;\n\t" "madc.hi.cc.u32 %4, %7, %11, %4;\n\t" "madc.hi.cc.u32 %5, %7, %12, %5;\n\t" "addc.u32 %6, %6, 0;\n\t" : "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]) : "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  asm("mad.lo.cc.u32 %0, %6, %7, %0;\n\t" "madc.lo.cc.u32 %1, %6, %8, %1;\n\t" "madc.lo.cc.u32 %2, %6, %9, %2;\n\t" "madc.lo.cc.u32 %3, %6, %10, %3;\n\t" "addc.cc.u32 %4, %4, 0;\n\t" "addc.u32 %5, %5, 0;\n\t" "mad.hi.cc.u32 %1, %6, %7, %1;\n\t" "madc.hi.cc.u32 %2, %6, %8, %2;\n\t" "madc.hi.cc.u32 %3, %6, %9, %3;\n\t" "madc.hi.cc.u32 %4, %6, %10, %4;\n\t" "addc.u32 %5, %5, 0;\n\t" : "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]) : "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  asm("mad.lo.cc.u32 %0, %5, %6, %0;\n\t" "madc.lo.cc.u32 %1, %5, %7, %1;\n\t" "madc.lo.cc.u32 %2, %5, %8, %2;\n\t" "addc.cc.u32 %3, %3, 0;\n\t" "addc.u32 %4, %4, 0;\n\t" "mad.hi.cc.u32 %1, %5, %6, %1;\n\t" "madc.hi.cc.u32 %2, %5, %7, %2;\n\t" "madc.hi.cc.u32 %3, %5, %8, %3;\n\t" "addc.u32 %4, %4, 0;\n\t" : "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]) : "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  asm("mad.lo.cc.u32 %0, %4, %5, %0;\n\t" "madc.lo.cc.u32 %1, %4, %6, %1;\n\t" "addc.cc.u32 %2, %2, 0;\n\t" "addc.u32 %3, %3, 0;\n\t" "mad.hi.cc.u32 %1, %4, %5, %1;\n\t" "madc.hi.cc.u32 %2, %4, %6, %2;\n\t" "addc.u32 %3, %3, 0;\n\t" : "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]) : "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t" "addc.cc.u32 %1, %1, 0;\n\t" "addc.u32 %2, %2, 0;\n\t" "mad.hi.cc.u32 %1, %3, %4, %1;\n\t" "addc.u32 %2, %2, 0;\n\t" : "+r"(t[13]), "+r"(t[14]), "+r"(t[15]) : "r"(a.v[6]), "r"(a.v[7]));
  // doubling, then the diagonal squares
  asm("add.cc.u32 %0, %0, %0;\n\t" "addc.cc.u32 %1, %1, %1;\n\t" "addc.cc.u32 %2, %2, %2;\n\t" "addc.cc.u32 %3, %3, %3;\n\t" "addc.cc.u32 %4, %4, %4;\n\t" "addc.cc.u32 %5, %5, %5;\n\t" "addc.cc.u32 %6, %6, %6;\n\t" "addc.cc.u32 %7, %7, %7;\n\t" "addc.cc.u32 %8, %8, %8;\n\t" "addc.cc.u32 %9, %9, %9;\n\t" "addc.cc.u32 %10, %10, %10;\n\t" "addc.cc.u32 %11, %11, %11;\n\t" "addc.cc.u32 %12, %12, %12;\n\t" "addc.cc.u32 %13, %13, %13;\n\t" "addc.cc.u32 %14, %14, %14;\n\t" "addc.u32 %15, %15, %15;\n\t" : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]));
  asm("mad.lo.cc.u32 %0, %16, %16, %0;\n\t" "madc.hi.cc.u32 %1, %16, %16, %1;\n\t" "madc.lo.cc.u32 %2, %17, %17, %2;\n\t" "madc.hi.cc.u32 %3, %17, %17, %3;\n\t" "madc.lo.cc.u32 %4, %18, %18, %4;\n\t" "madc.hi.cc.u32 %5, %18, %18, %5;\n\t" "madc.lo.cc.u32 %6, %19, %19, %6;\n\t" "madc.hi.cc.u32 %7, %19, %19, %7;\n\t" "madc.lo.cc.u32 %8, %20, %20, %8;\n\t" "madc.hi.cc.u32 %9, %20, %20, %9;\n\t" "madc.lo.cc.u32 %10, %21, %21, %10;\n\t" "madc.hi.cc.u32 %11, %21, %21, %11;\n\t" "madc.lo.cc.u32 %12, %22, %22, %12;\n\t" "madc.hi.cc.u32 %13, %22, %22, %13;\n\t" "madc.lo.cc.u32 %14, %23, %23, %14;\n\t" "madc.hi.u32 %15, %23, %23, %15;\n\t" : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]) : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // Montgomery steps: m = t_i (-p^-1) mod 2^32, t += m p 2^(32 i); the
  // carry out of word i + 8 is held in cy and added into word i + 9 by the
  // next step (at most 2, so no word overflows unseen)
  uint32_t cy = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    asm("{\n\t" ".reg .u32 m;\n\t" "mul.lo.u32 m, %0, 0xefffffff;\n\t" "mad.lo.cc.u32 %0, m, 0xf0000001, %0;\n\t" "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t" "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t" "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t" "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t" "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t" "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t" "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t" "addc.cc.u32 %8, %8, %9;\n\t" "addc.u32 %9, %10, 0;\n\t" "mad.hi.cc.u32 %1, m, 0xf0000001, %1;\n\t" "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t" "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t" "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t" "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t" "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t" "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t" "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t" "addc.u32 %9, %9, 0;\n\t" "}"
        : "+r"(t[i]), "+r"(t[i + 1]), "+r"(t[i + 2]), "+r"(t[i + 3]), "+r"(t[i + 4]), "+r"(t[i + 5]), "+r"(t[i + 6]),
          "+r"(t[i + 7]), "+r"(t[i + 8]), "+r"(cy)
        : "r"(0u));
  }
  Fr r;
#pragma unroll
  for (int i = 0; i < 8; ++i) r.v[i] = t[8 + i];
  return r;
}

// one out-of-line copy per translation unit, as for the product
static __device__ __noinline__ Fr fr_sqr_call(Fr a) { return fr_sqr_inl(a); }

__device__ __forceinline__ Fr fr_sqr(const Fr& a) { return fr_sqr_call(a); }

// ---------------------------------------------------------------------------
// comparisons and conversions

// x < r for an integer given as 8 limbs
__device__ __forceinline__ bool fr_lt_modulus(const Fr& x) {
  uint32_t borrow;
  asm("{\n\t"
      ".reg .u32 z, t;\n\t"
      "mov.u32 z, 0;\n\t"
      "sub.cc.u32  t, %1, 0xf0000001;\n\t"
      "subc.cc.u32 t, %2, 0x43e1f593;\n\t"
      "subc.cc.u32 t, %3, 0x79b97091;\n\t"
      "subc.cc.u32 t, %4, 0x2833e848;\n\t"
      "subc.cc.u32 t, %5, 0x8181585d;\n\t"
      "subc.cc.u32 t, %6, 0xb85045b6;\n\t"
      "subc.cc.u32 t, %7, 0xe131a029;\n\t"
      "subc.cc.u32 t, %8, 0x30644e72;\n\t"
      "subc.u32    %0, z, z;\n\t"
      "}"
      : "=r"(borrow)
      : "r"(x.v[0]), "r"(x.v[1]), "r"(x.v[2]), "r"(x.v[3]), "r"(x.v[4]), "r"(x.v[5]), "r"(x.v[6]),
        "r"(x.v[7]));
  return borrow != 0;
}

// x - r when x >= r (x < 2r), else x
__device__ __forceinline__ Fr fr_reduce_once(const Fr& x) {
  Fr d = x;
  uint32_t keep;
  asm("{\n\t"
      ".reg .u32 z;\n\t"
      "mov.u32 z, 0;\n\t"
      "sub.cc.u32  %0, %0, 0xf0000001;\n\t"
      "subc.cc.u32 %1, %1, 0x43e1f593;\n\t"
      "subc.cc.u32 %2, %2, 0x79b97091;\n\t"
      "subc.cc.u32 %3, %3, 0x2833e848;\n\t"
      "subc.cc.u32 %4, %4, 0x8181585d;\n\t"
      "subc.cc.u32 %5, %5, 0xb85045b6;\n\t"
      "subc.cc.u32 %6, %6, 0xe131a029;\n\t"
      "subc.cc.u32 %7, %7, 0x30644e72;\n\t"
      "subc.u32    %8, z, z;\n\t"
      "}"
      : "+r"(d.v[0]), "+r"(d.v[1]), "+r"(d.v[2]), "+r"(d.v[3]), "+r"(d.v[4]), "+r"(d.v[5]),
        "+r"(d.v[6]), "+r"(d.v[7]), "=r"(keep));
  Fr r;
#pragma unroll
  for (int i = 0; i < 8; ++i) r.v[i] = (x.v[i] & keep) | (d.v[i] & ~keep);
  return r;
}

// Montgomery (lazy) -> canonical integer in [0, r)
__device__ __forceinline__ Fr fr_to_canonical(const Fr& a) {
  return fr_reduce_once(fr_mul(a, fr_int_one()));
}

// canonical integer (< r) -> Montgomery
__device__ __forceinline__ Fr fr_from_canonical(const Fr& a) { return fr_mul(a, fr_r2()); }

__device__ __forceinline__ bool fr_is_zero_lazy(const Fr& a) {
  // a in [0, 2r) represents 0 exactly when a == 0 or a == r
  Fr c = fr_reduce_once(a);
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) acc |= c.v[i];
  return acc == 0;
}

// a^e for a 256-bit exponent given as canonical limbs (square and multiply)
__device__ __forceinline__ Fr fr_pow(const Fr& a, const Fr& e) {
  Fr acc = fr_one();
  for (int i = 255; i >= 0; --i) {
    acc = fr_sqr(acc);
    if ((e.v[i >> 5] >> (i & 31)) & 1u) acc = fr_mul(acc, a);
  }
  return acc;
}

// Fermat inverse a^(r-2) (0 maps to 0)
__device__ __forceinline__ Fr fr_inv(const Fr& a) {
  Fr e = fr_modulus();
  e.v[0] -= 2u;  // r - 2 (no borrow: low limb of r is 0xf0000001)
  return fr_pow(a, e);
}

// warp-wide sum (result valid in lane 0)
__device__ __forceinline__ Fr fr_warp_sum(Fr x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Fr y;
#pragma unroll
    for (int i = 0; i < 8; ++i) y.v[i] = __shfl_down_sync(0xffffffffu, x.v[i], off);
    x = fr_add(x, y);
  }
  return x;
}

#endif  // __CUDACC__
}  // namespace sisu
