// Lazily reduced sums of field products (BN254 F_r, Montgomery form).
//
// A sum of many products a_i b_i needs only one Montgomery reduction when
// the full 512-bit products are added up first: the accumulator holds the
// exact integer T = sum a_i b_i in 17 words (544 bits), and one reduction at
// the end maps it into the field.  A full product costs 64 mad.lo and 64
// mad.hi, against 128 + 128 (+ 8 for the quotient digits) for a Montgomery
// product, so a dot product of n terms costs about half as much.
//
// The final reduction divides by 2^288 instead of 2^256 (nine quotient
// digits instead of eight), which keeps it exact for large sums: with
// m < 2^288 the result (T + m r) / 2^288 is below T / 2^288 + r, so any
// T < r 2^288 reduces to a value below 2r.  Operands below 2r give products
// below 4 r^2 < 2^510, so about 2^32 terms fit.  For Montgomery operands
// a = a' 2^256, b = b' 2^256 the result is a'b' 2^224 mod r: the Montgomery
// form of a'b' times 2^-32.  The caller multiplies by the Montgomery form
// of 2^32 once to undo that factor (or leaves it in a value that is scaled
// back later).
#pragma once
#include "fr.cuh"

namespace sisu {

struct FrAcc {
  uint32_t v[17];  // little-endian words of a 544-bit integer
};

#ifdef __CUDACC__

__device__ __forceinline__ FrAcc fracc_zero() {
  FrAcc z;
#pragma unroll
  for (int i = 0; i < 17; ++i) z.v[i] = 0;
  return z;
}

// Montgomery form of 2^32 (2^288 mod r): a product with it undoes the
// 2^-32 that fr_redc288 leaves
SISU_FR_CONST(fr_mont_2_32, 0x15b8b9dau, 0x93e78865u, 0xb05ea154u, 0x16df2426u, 0x302ab839u, 0x1271b743u,
              0xec6c226eu, 0x06bc037eu)
// 2^-32 in Montgomery form: 2^-32 2^256 mod p is the integer 2^224
SISU_FR_CONST(fr_mont_2_neg32, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 1u)
// the plain integer 2^32 (a Montgomery product by it multiplies by 2^32 R^-1)
SISU_FR_CONST(fr_int_2_32, 0u, 1u, 0u, 0u, 0u, 0u, 0u, 0u)

// acc += a * b (the full 512-bit product, no reduction)
__device__ __forceinline__ void fracc_mac_inl(FrAcc& acc, const Fr& a, const Fr& b) {
  uint32_t p[16];
  // row 0: p[0..8] = a * b_0
#pragma unroll
  for (int k = 0; k < 8; ++k) p[k] = a.v[k] * b.v[0];
  p[8] = __umulhi(a.v[7], b.v[0]);

  asm("mad.hi.cc.u32  %0, %8, %15, %0;\n\t"
      "madc.hi.cc.u32 %1, %9, %15, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, %15, %2;\n\t"
      "madc.hi.cc.u32 %3, %11, %15, %3;\n\t"
      "madc.hi.cc.u32 %4, %12, %15, %4;\n\t"
      "madc.hi.cc.u32 %5, %13, %15, %5;\n\t"
      "madc.hi.cc.u32 %6, %14, %15, %6;\n\t"
      "addc.u32       %7, %7, 0;"
      : "+r"(p[1]), "+r"(p[2]), "+r"(p[3]), "+r"(p[4]), "+r"(p[5]), "+r"(p[6]), "+r"(p[7]), "+r"(p[8])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(b.v[0]));
  // rows 1..7: p[i..i+8] += a * b_i (the top word of a row starts at 0)
  p[9] = 0;
  asm("mad.lo.cc.u32  %0, %9, %17, %0;\n\t"
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
      "addc.u32       %8, %8, 0;\n\t"
      "mad.hi.cc.u32  %1, %9, %17, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
      "madc.hi.u32    %8, %16, %17, %8;"
      : "+r"(p[1]), "+r"(p[2]), "+r"(p[3]), "+r"(p[4]), "+r"(p[5]), "+r"(p[6]), "+r"(p[7]), "+r"(p[8]), "+r"(p[9])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[1]));
  p[10] = 0;
  asm("mad.lo.cc.u32  %0, %9, %17, %0;\n\t"
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
      "addc.u32       %8, %8, 0;\n\t"
      "mad.hi.cc.u32  %1, %9, %17, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
      "madc.hi.u32    %8, %16, %17, %8;"
      : "+r"(p[2]), "+r"(p[3]), "+r"(p[4]), "+r"(p[5]), "+r"(p[6]), "+r"(p[7]), "+r"(p[8]), "+r"(p[9]), "+r"(p[10])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[2]));
  p[11] = 0;
  asm("mad.lo.cc.u32  %0, %9, %17, %0;\n\t"
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
      "addc.u32       %8, %8, 0;\n\t"
      "mad.hi.cc.u32  %1, %9, %17, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
      "madc.hi.u32    %8, %16, %17, %8;"
      : "+r"(p[3]), "+r"(p[4]), "+r"(p[5]), "+r"(p[6]), "+r"(p[7]), "+r"(p[8]), "+r"(p[9]), "+r"(p[10]), "+r"(p[11])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[3]));
  p[12] = 0;
  asm("mad.lo.cc.u32  %0, %9, %17, %0;\n\t"
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
      "addc.u32       %8, %8, 0;\n\t"
      "mad.hi.cc.u32  %1, %9, %17, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
      "madc.hi.u32    %8, %16, %17, %8;"
      : "+r"(p[4]), "+r"(p[5]), "+r"(p[6]), "+r"(p[7]), "+r"(p[8]), "+r"(p[9]), "+r"(p[10]), "+r"(p[11]), "+r"(p[12])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[4]));
  p[13] = 0;
  asm("mad.lo.cc.u32  %0, %9, %17, %0;\n\t"
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
      "addc.u32       %8, %8, 0;\n\t"
      "mad.hi.cc.u32  %1, %9, %17, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
      "madc.hi.u32    %8, %16, %17, %8;"
      : "+r"(p[5]), "+r"(p[6]), "+r"(p[7]), "+r"(p[8]), "+r"(p[9]), "+r"(p[10]), "+r"(p[11]), "+r"(p[12]), "+r"(p[13])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[5]));
  p[14] = 0;
  asm("mad.lo.cc.u32  %0, %9, %17, %0;\n\t"
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
      "addc.u32       %8, %8, 0;\n\t"
      "mad.hi.cc.u32  %1, %9, %17, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
      "madc.hi.u32    %8, %16, %17, %8;"
      : "+r"(p[6]), "+r"(p[7]), "+r"(p[8]), "+r"(p[9]), "+r"(p[10]), "+r"(p[11]), "+r"(p[12]), "+r"(p[13]), "+r"(p[14])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[6]));
  p[15] = 0;
  asm("mad.lo.cc.u32  %0, %9, %17, %0;\n\t"
      "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
      "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
      "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
      "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
      "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
      "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
      "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
      "addc.u32       %8, %8, 0;\n\t"
      "mad.hi.cc.u32  %1, %9, %17, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
      "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
      "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
      "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
      "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
      "madc.hi.u32    %8, %16, %17, %8;"
      : "+r"(p[7]), "+r"(p[8]), "+r"(p[9]), "+r"(p[10]), "+r"(p[11]), "+r"(p[12]), "+r"(p[13]), "+r"(p[14]), "+r"(p[15])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[7]));
  // acc += p
  asm("add.cc.u32  %0, %0, %17;\n\t"
      "addc.cc.u32 %1, %1, %18;\n\t"
      "addc.cc.u32 %2, %2, %19;\n\t"
      "addc.cc.u32 %3, %3, %20;\n\t"
      "addc.cc.u32 %4, %4, %21;\n\t"
      "addc.cc.u32 %5, %5, %22;\n\t"
      "addc.cc.u32 %6, %6, %23;\n\t"
      "addc.cc.u32 %7, %7, %24;\n\t"
      "addc.cc.u32 %8, %8, %25;\n\t"
      "addc.cc.u32 %9, %9, %26;\n\t"
      "addc.cc.u32 %10, %10, %27;\n\t"
      "addc.cc.u32 %11, %11, %28;\n\t"
      "addc.cc.u32 %12, %12, %29;\n\t"
      "addc.cc.u32 %13, %13, %30;\n\t"
      "addc.cc.u32 %14, %14, %31;\n\t"
      "addc.cc.u32 %15, %15, %32;\n\t"
      "addc.u32    %16, %16, 0;"
      : "+r"(acc.v[0]), "+r"(acc.v[1]), "+r"(acc.v[2]), "+r"(acc.v[3]), "+r"(acc.v[4]), "+r"(acc.v[5]), "+r"(acc.v[6]), "+r"(acc.v[7]), "+r"(acc.v[8]), "+r"(acc.v[9]), "+r"(acc.v[10]), "+r"(acc.v[11]), "+r"(acc.v[12]), "+r"(acc.v[13]), "+r"(acc.v[14]), "+r"(acc.v[15]), "+r"(acc.v[16])
      : "r"(p[0]), "r"(p[1]), "r"(p[2]), "r"(p[3]), "r"(p[4]), "r"(p[5]), "r"(p[6]), "r"(p[7]), "r"(p[8]), "r"(p[9]), "r"(p[10]), "r"(p[11]), "r"(p[12]), "r"(p[13]), "r"(p[14]), "r"(p[15]));
}

// p[0..7] = a[0..3] * b[0..3]: a 128 x 128-bit product, rows of four
// multiply halves as in the 256-bit product above.
__device__ __forceinline__ void mul128(const uint32_t* a, const uint32_t* b, uint32_t* p) {
#pragma unroll
  for (int k = 0; k < 4; ++k) p[k] = a[k] * b[0];
  p[4] = __umulhi(a[3], b[0]);
  asm("mad.hi.cc.u32  %0, %4, %7, %0;\n\t"
      "madc.hi.cc.u32 %1, %5, %7, %1;\n\t"
      "madc.hi.cc.u32 %2, %6, %7, %2;\n\t"
      "addc.u32       %3, %3, 0;"
      : "+r"(p[1]), "+r"(p[2]), "+r"(p[3]), "+r"(p[4])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(b[0]));
#pragma unroll
  for (int i = 1; i < 4; ++i) {
    p[i + 4] = 0;
    asm("mad.lo.cc.u32  %0, %5, %9, %0;\n\t"
        "madc.lo.cc.u32 %1, %6, %9, %1;\n\t"
        "madc.lo.cc.u32 %2, %7, %9, %2;\n\t"
        "madc.lo.cc.u32 %3, %8, %9, %3;\n\t"
        "addc.u32       %4, %4, 0;\n\t"
        "mad.hi.cc.u32  %1, %5, %9, %1;\n\t"
        "madc.hi.cc.u32 %2, %6, %9, %2;\n\t"
        "madc.hi.cc.u32 %3, %7, %9, %3;\n\t"
        "madc.hi.u32    %4, %8, %9, %4;"
        : "+r"(p[i]), "+r"(p[i + 1]), "+r"(p[i + 2]), "+r"(p[i + 3]), "+r"(p[i + 4])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[i]));
  }
}

// s = x + y (128-bit), returns the carry (0 or 1)
__device__ __forceinline__ uint32_t add128(const uint32_t* x, const uint32_t* y, uint32_t* s) {
  uint32_t c;
  asm("add.cc.u32  %0, %5, %9;\n\t"
      "addc.cc.u32 %1, %6, %10;\n\t"
      "addc.cc.u32 %2, %7, %11;\n\t"
      "addc.cc.u32 %3, %8, %12;\n\t"
      "addc.u32    %4, 0, 0;"
      : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(c)
      : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]));
  return c;
}

// acc += a * b by one level of Karatsuba (A. Karatsuba and Yu. Ofman, 1962):
// with a = a0 + a1 2^128 and b = b0 + b1 2^128,
//   a b = z0 + z1 2^128 + z2 2^256,  z0 = a0 b0,  z2 = a1 b1,
//   z1 = (a0 + a1)(b0 + b1) - z0 - z2 = a0 b1 + a1 b0 < 2^257,
// three 128 x 128-bit products (48 multiply halves each way) where the
// schoolbook product takes four.  The sums a0 + a1 and b0 + b1 have 129
// bits: their products are formed from the low 128 bits, and the carry
// bits add the other operand (masked) at 2^128 and their product at 2^256.
__device__ __forceinline__ void fracc_mac_kara_inl(FrAcc& acc, const Fr& a, const Fr& b) {
  uint32_t z0[8], z2[8], m[8], sa[4], sb[4];
  mul128(a.v, b.v, z0);
  mul128(a.v + 4, b.v + 4, z2);
  const uint32_t ca = add128(a.v, a.v + 4, sa), cb = add128(b.v, b.v + 4, sb);
  mul128(sa, sb, m);
  uint32_t z1[9];
#pragma unroll
  for (int k = 0; k < 8; ++k) z1[k] = m[k];
  z1[8] = ca & cb;
  const uint32_t ma = 0u - ca, mb = 0u - cb;  // all ones when the carry is set
  asm("add.cc.u32  %0, %0, %5;\n\t"
      "addc.cc.u32 %1, %1, %6;\n\t"
      "addc.cc.u32 %2, %2, %7;\n\t"
      "addc.cc.u32 %3, %3, %8;\n\t"
      "addc.u32    %4, %4, 0;\n\t"
      "add.cc.u32  %0, %0, %9;\n\t"
      "addc.cc.u32 %1, %1, %10;\n\t"
      "addc.cc.u32 %2, %2, %11;\n\t"
      "addc.cc.u32 %3, %3, %12;\n\t"
      "addc.u32    %4, %4, 0;"
      : "+r"(z1[4]), "+r"(z1[5]), "+r"(z1[6]), "+r"(z1[7]), "+r"(z1[8])
      : "r"(sb[0] & ma), "r"(sb[1] & ma), "r"(sb[2] & ma), "r"(sb[3] & ma), "r"(sa[0] & mb), "r"(sa[1] & mb),
        "r"(sa[2] & mb), "r"(sa[3] & mb));
  // z1 -= z0, z1 -= z2 (the difference is a0 b1 + a1 b0 >= 0)
  asm("sub.cc.u32  %0, %0, %9;\n\t"
      "subc.cc.u32 %1, %1, %10;\n\t"
      "subc.cc.u32 %2, %2, %11;\n\t"
      "subc.cc.u32 %3, %3, %12;\n\t"
      "subc.cc.u32 %4, %4, %13;\n\t"
      "subc.cc.u32 %5, %5, %14;\n\t"
      "subc.cc.u32 %6, %6, %15;\n\t"
      "subc.cc.u32 %7, %7, %16;\n\t"
      "subc.u32    %8, %8, 0;\n\t"
      "sub.cc.u32  %0, %0, %17;\n\t"
      "subc.cc.u32 %1, %1, %18;\n\t"
      "subc.cc.u32 %2, %2, %19;\n\t"
      "subc.cc.u32 %3, %3, %20;\n\t"
      "subc.cc.u32 %4, %4, %21;\n\t"
      "subc.cc.u32 %5, %5, %22;\n\t"
      "subc.cc.u32 %6, %6, %23;\n\t"
      "subc.cc.u32 %7, %7, %24;\n\t"
      "subc.u32    %8, %8, 0;"
      : "+r"(z1[0]), "+r"(z1[1]), "+r"(z1[2]), "+r"(z1[3]), "+r"(z1[4]), "+r"(z1[5]), "+r"(z1[6]), "+r"(z1[7]),
        "+r"(z1[8])
      : "r"(z0[0]), "r"(z0[1]), "r"(z0[2]), "r"(z0[3]), "r"(z0[4]), "r"(z0[5]), "r"(z0[6]), "r"(z0[7]), "r"(z2[0]),
        "r"(z2[1]), "r"(z2[2]), "r"(z2[3]), "r"(z2[4]), "r"(z2[5]), "r"(z2[6]), "r"(z2[7]));
  // p = z0 + z2 2^256 (side by side) + z1 2^128, then acc += p
  uint32_t p[16];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    p[k] = z0[k];
    p[8 + k] = z2[k];
  }
  asm("add.cc.u32  %0, %0, %12;\n\t"
      "addc.cc.u32 %1, %1, %13;\n\t"
      "addc.cc.u32 %2, %2, %14;\n\t"
      "addc.cc.u32 %3, %3, %15;\n\t"
      "addc.cc.u32 %4, %4, %16;\n\t"
      "addc.cc.u32 %5, %5, %17;\n\t"
      "addc.cc.u32 %6, %6, %18;\n\t"
      "addc.cc.u32 %7, %7, %19;\n\t"
      "addc.cc.u32 %8, %8, %20;\n\t"
      "addc.cc.u32 %9, %9, 0;\n\t"
      "addc.cc.u32 %10, %10, 0;\n\t"
      "addc.u32    %11, %11, 0;"
      : "+r"(p[4]), "+r"(p[5]), "+r"(p[6]), "+r"(p[7]), "+r"(p[8]), "+r"(p[9]), "+r"(p[10]), "+r"(p[11]),
        "+r"(p[12]), "+r"(p[13]), "+r"(p[14]), "+r"(p[15])
      : "r"(z1[0]), "r"(z1[1]), "r"(z1[2]), "r"(z1[3]), "r"(z1[4]), "r"(z1[5]), "r"(z1[6]), "r"(z1[7]), "r"(z1[8]));
  asm("add.cc.u32  %0, %0, %17;\n\t"
      "addc.cc.u32 %1, %1, %18;\n\t"
      "addc.cc.u32 %2, %2, %19;\n\t"
      "addc.cc.u32 %3, %3, %20;\n\t"
      "addc.cc.u32 %4, %4, %21;\n\t"
      "addc.cc.u32 %5, %5, %22;\n\t"
      "addc.cc.u32 %6, %6, %23;\n\t"
      "addc.cc.u32 %7, %7, %24;\n\t"
      "addc.cc.u32 %8, %8, %25;\n\t"
      "addc.cc.u32 %9, %9, %26;\n\t"
      "addc.cc.u32 %10, %10, %27;\n\t"
      "addc.cc.u32 %11, %11, %28;\n\t"
      "addc.cc.u32 %12, %12, %29;\n\t"
      "addc.cc.u32 %13, %13, %30;\n\t"
      "addc.cc.u32 %14, %14, %31;\n\t"
      "addc.cc.u32 %15, %15, %32;\n\t"
      "addc.u32    %16, %16, 0;"
      : "+r"(acc.v[0]), "+r"(acc.v[1]), "+r"(acc.v[2]), "+r"(acc.v[3]), "+r"(acc.v[4]), "+r"(acc.v[5]),
        "+r"(acc.v[6]), "+r"(acc.v[7]), "+r"(acc.v[8]), "+r"(acc.v[9]), "+r"(acc.v[10]), "+r"(acc.v[11]),
        "+r"(acc.v[12]), "+r"(acc.v[13]), "+r"(acc.v[14]), "+r"(acc.v[15]), "+r"(acc.v[16])
      : "r"(p[0]), "r"(p[1]), "r"(p[2]), "r"(p[3]), "r"(p[4]), "r"(p[5]), "r"(p[6]), "r"(p[7]), "r"(p[8]),
        "r"(p[9]), "r"(p[10]), "r"(p[11]), "r"(p[12]), "r"(p[13]), "r"(p[14]), "r"(p[15]));
}

// x += y (544-bit integers; the sum must fit)
__device__ __forceinline__ void fracc_add(FrAcc& x, const FrAcc& y) {

  asm("add.cc.u32  %0, %0, %17;\n\t"
      "addc.cc.u32 %1, %1, %18;\n\t"
      "addc.cc.u32 %2, %2, %19;\n\t"
      "addc.cc.u32 %3, %3, %20;\n\t"
      "addc.cc.u32 %4, %4, %21;\n\t"
      "addc.cc.u32 %5, %5, %22;\n\t"
      "addc.cc.u32 %6, %6, %23;\n\t"
      "addc.cc.u32 %7, %7, %24;\n\t"
      "addc.cc.u32 %8, %8, %25;\n\t"
      "addc.cc.u32 %9, %9, %26;\n\t"
      "addc.cc.u32 %10, %10, %27;\n\t"
      "addc.cc.u32 %11, %11, %28;\n\t"
      "addc.cc.u32 %12, %12, %29;\n\t"
      "addc.cc.u32 %13, %13, %30;\n\t"
      "addc.cc.u32 %14, %14, %31;\n\t"
      "addc.cc.u32 %15, %15, %32;\n\t"
      "addc.u32    %16, %16, %33;"
      : "+r"(x.v[0]), "+r"(x.v[1]), "+r"(x.v[2]), "+r"(x.v[3]), "+r"(x.v[4]), "+r"(x.v[5]), "+r"(x.v[6]), "+r"(x.v[7]), "+r"(x.v[8]), "+r"(x.v[9]), "+r"(x.v[10]), "+r"(x.v[11]), "+r"(x.v[12]), "+r"(x.v[13]), "+r"(x.v[14]), "+r"(x.v[15]), "+r"(x.v[16])
      : "r"(y.v[0]), "r"(y.v[1]), "r"(y.v[2]), "r"(y.v[3]), "r"(y.v[4]), "r"(y.v[5]), "r"(y.v[6]), "r"(y.v[7]), "r"(y.v[8]), "r"(y.v[9]), "r"(y.v[10]), "r"(y.v[11]), "r"(y.v[12]), "r"(y.v[13]), "r"(y.v[14]), "r"(y.v[15]), "r"(y.v[16]));
}

// T * 2^-288 mod r, in [0, 2r), for T < r 2^288: nine Montgomery steps, each
// adding the multiple m r of r that zeroes the lowest remaining word, with
// the carries rippling to the top word.  The result is the top eight words.
__device__ __forceinline__ Fr fr_redc288(const FrAcc& acc) {
  uint32_t t[17];
#pragma unroll
  for (int i = 0; i < 17; ++i) t[i] = acc.v[i];
  // step 0: zero t[0]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.cc.u32    %14, %14, 0;\n\t"
      "addc.cc.u32    %15, %15, 0;\n\t"
      "addc.u32       %16, %16, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.cc.u32    %14, %14, 0;\n\t"
      "addc.cc.u32    %15, %15, 0;\n\t"
      "addc.u32       %16, %16, 0;\n\t"
      "}"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 1: zero t[1]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.cc.u32    %14, %14, 0;\n\t"
      "addc.u32       %15, %15, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.cc.u32    %14, %14, 0;\n\t"
      "addc.u32       %15, %15, 0;\n\t"
      "}"
      : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 2: zero t[2]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.u32       %14, %14, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.u32       %14, %14, 0;\n\t"
      "}"
      : "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 3: zero t[3]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.u32       %13, %13, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.u32       %13, %13, 0;\n\t"
      "}"
      : "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 4: zero t[4]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.u32       %12, %12, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.u32       %12, %12, 0;\n\t"
      "}"
      : "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 5: zero t[5]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.u32       %11, %11, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.u32       %11, %11, 0;\n\t"
      "}"
      : "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 6: zero t[6]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.u32       %10, %10, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.u32       %10, %10, 0;\n\t"
      "}"
      : "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 7: zero t[7]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.u32       %9, %9, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.u32       %9, %9, 0;\n\t"
      "}"
      : "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 8: zero t[8]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.u32       %8, %8, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.u32    %8, m, 0x30644e72, %8;\n\t"
      "}"
      : "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  Fr o;
#pragma unroll
  for (int i = 0; i < 8; ++i) o.v[i] = t[9 + i];
  return o;
}

// T 2^-256 mod r, in [0, 2r), for T < 4 r^2 (a product of two values below
// 2r): eight Montgomery steps, each adding the multiple m r of r that zeroes
// the lowest remaining word, with the carries rippling to the top word.
// The result is words 8..15 (word 16 stays 0).
__device__ __forceinline__ Fr fr_redc256(const FrAcc& acc) {
  uint32_t t[17];
#pragma unroll
  for (int i = 0; i < 17; ++i) t[i] = acc.v[i];
  // step 0: zero t[0]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.cc.u32    %14, %14, 0;\n\t"
      "addc.cc.u32    %15, %15, 0;\n\t"
      "addc.u32       %16, %16, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.cc.u32    %14, %14, 0;\n\t"
      "addc.cc.u32    %15, %15, 0;\n\t"
      "addc.u32       %16, %16, 0;\n\t"
      "}"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 1: zero t[1]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.cc.u32    %14, %14, 0;\n\t"
      "addc.u32       %15, %15, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.cc.u32    %14, %14, 0;\n\t"
      "addc.u32       %15, %15, 0;\n\t"
      "}"
      : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 2: zero t[2]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.u32       %14, %14, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.cc.u32    %13, %13, 0;\n\t"
      "addc.u32       %14, %14, 0;\n\t"
      "}"
      : "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 3: zero t[3]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.u32       %13, %13, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.cc.u32    %12, %12, 0;\n\t"
      "addc.u32       %13, %13, 0;\n\t"
      "}"
      : "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 4: zero t[4]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.u32       %12, %12, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.cc.u32    %11, %11, 0;\n\t"
      "addc.u32       %12, %12, 0;\n\t"
      "}"
      : "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 5: zero t[5]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.u32       %11, %11, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.cc.u32    %10, %10, 0;\n\t"
      "addc.u32       %11, %11, 0;\n\t"
      "}"
      : "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 6: zero t[6]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.u32       %10, %10, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.cc.u32    %9, %9, 0;\n\t"
      "addc.u32       %10, %10, 0;\n\t"
      "}"
      : "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  // step 7: zero t[7]
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.u32       %9, %9, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.u32       %9, %9, 0;\n\t"
      "}"
      : "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]), "+r"(t[16]));
  Fr r;
#pragma unroll
  for (int i = 0; i < 8; ++i) r.v[i] = t[8 + i];
  return r;
}

// Montgomery product a b 2^-256 mod r by the Karatsuba 512-bit product and
// a separate reduction (inputs and output in [0, 2r))
__device__ __forceinline__ Fr fr_mul_kara_inl(const Fr& a, const Fr& b) {
  FrAcc t = fracc_zero();
  fracc_mac_kara_inl(t, a, b);
  return fr_redc256(t);
}


// one out-of-line copy per translation unit (see fr_mul_call); operands and
// result travel in registers
// The kernels' lazy product: one level of Karatsuba (three 128-bit
// products where the schoolbook form takes four; 130 against 84 G products
// a second in the microbenchmark, the multiply pipe being the busy one).
static __device__ __noinline__ FrAcc fracc_mac_call(FrAcc acc, Fr a, Fr b) {
  fracc_mac_kara_inl(acc, a, b);
  return acc;
}

// the schoolbook form out of line (microbenchmark kind 7)
static __device__ __noinline__ FrAcc fracc_mac_school_call(FrAcc acc, Fr a, Fr b) {
  fracc_mac_inl(acc, a, b);
  return acc;
}

__device__ __forceinline__ void fracc_mac(FrAcc& acc, const Fr& a, const Fr& b) { acc = fracc_mac_call(acc, a, b); }

// ---------------------------------------------------------------------------
// Products with one fixed multiplier (the fold of a table by a challenge).
//
// For a fixed rho (Montgomery form r) and K_i = rho 2^(32 i + 64) mod p,
// i = 0..7, the Montgomery form of D rho for d = D 2^256 (limbs d_i) is
//   sum_i d_i K_i  2^-64 mod p,
// because sum_i d_i K_i = d rho 2^64.  The sum is eight 32 x 256-bit rows
// added at the same offset (64 mad.lo and 64 mad.hi into ten words, below
// 8 2^32 2p < 2^291) and the factor 2^-64 is two Montgomery steps, whose
// result is below 2^291 / 2^64 + p < 2p.  That is 82 mad.lo and 80 mad.hi
// where a Montgomery product needs 136 and 128.  K_i = MontMul(r, X_i) for
// the plain constants X_i = 2^(32 i + 64) mod p.

// K_i for 0 <= i < 8 from the Montgomery form r of rho
__device__ __forceinline__ Fr fr_fixed_coeff(const Fr& r, int i) {
  Fr x = fr_zero();
  if (i < 6) {
    x.v[i + 2] = 1u;  // 2^(32 i + 64) < p
  } else {
    x = i == 6 ? fr_one() : fr_mont_2_32();  // 2^256 mod p, 2^288 mod p
  }
  return fr_mul(r, x);
}

// coefficient i of a table of eight (8 words each, 16-byte aligned)
__device__ __forceinline__ Fr fr_coeff_load(const uint32_t* K8, int i) {
  const uint4* p = reinterpret_cast<const uint4*>(K8 + 8 * i);
  const uint4 lo = p[0], hi = p[1];
  Fr k;
  k.v[0] = lo.x; k.v[1] = lo.y; k.v[2] = lo.z; k.v[3] = lo.w;
  k.v[4] = hi.x; k.v[5] = hi.y; k.v[6] = hi.z; k.v[7] = hi.w;
  return k;
}

// d rho (Montgomery forms, d < 2p) given the coefficients K_0..K_7 of
// fr_fixed_coeff as 64 words (16-byte aligned); only the rows of the first
// kRows limbs of d are summed (the others must be zero)
template <int kRows>
__device__ __forceinline__ Fr fr_mul_fixed_rows(const Fr& d, const uint32_t* K8) {
  uint32_t a[10];
#pragma unroll
  for (int i = 0; i < 10; ++i) a[i] = 0;
#pragma unroll
  for (int i = 0; i < kRows; ++i) {
    const Fr K = fr_coeff_load(K8, i);
    const uint32_t di = d.v[i];
    asm("mad.lo.cc.u32  %0, %11, %10, %0;\n\t"
        "madc.lo.cc.u32 %1, %12, %10, %1;\n\t"
        "madc.lo.cc.u32 %2, %13, %10, %2;\n\t"
        "madc.lo.cc.u32 %3, %14, %10, %3;\n\t"
        "madc.lo.cc.u32 %4, %15, %10, %4;\n\t"
        "madc.lo.cc.u32 %5, %16, %10, %5;\n\t"
        "madc.lo.cc.u32 %6, %17, %10, %6;\n\t"
        "madc.lo.cc.u32 %7, %18, %10, %7;\n\t"
        "addc.cc.u32    %8, %8, 0;\n\t"
        "addc.u32       %9, %9, 0;\n\t"
        "mad.hi.cc.u32  %1, %11, %10, %1;\n\t"
        "madc.hi.cc.u32 %2, %12, %10, %2;\n\t"
        "madc.hi.cc.u32 %3, %13, %10, %3;\n\t"
        "madc.hi.cc.u32 %4, %14, %10, %4;\n\t"
        "madc.hi.cc.u32 %5, %15, %10, %5;\n\t"
        "madc.hi.cc.u32 %6, %16, %10, %6;\n\t"
        "madc.hi.cc.u32 %7, %17, %10, %7;\n\t"
        "madc.hi.cc.u32 %8, %18, %10, %8;\n\t"
        "addc.u32       %9, %9, 0;"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9])
        : "r"(di), "r"(K.v[0]), "r"(K.v[1]), "r"(K.v[2]), "r"(K.v[3]), "r"(K.v[4]), "r"(K.v[5]), "r"(K.v[6]), "r"(K.v[7]));
  }
  // two Montgomery steps: divide by 2^64
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.cc.u32    %8, %8, 0;\n\t"
      "addc.u32       %9, %9, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.cc.u32 %8, m, 0x30644e72, %8;\n\t"
      "addc.u32       %9, %9, 0;\n\t"
      "}"
      : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]));
  asm("{\n\t"
      ".reg .u32 m;\n\t"
      "mul.lo.u32 m, %0, 0xefffffff;\n\t"
      "mad.lo.cc.u32  %0, m, 0xf0000001, %0;\n\t"
      "madc.lo.cc.u32 %1, m, 0x43e1f593, %1;\n\t"
      "madc.lo.cc.u32 %2, m, 0x79b97091, %2;\n\t"
      "madc.lo.cc.u32 %3, m, 0x2833e848, %3;\n\t"
      "madc.lo.cc.u32 %4, m, 0x8181585d, %4;\n\t"
      "madc.lo.cc.u32 %5, m, 0xb85045b6, %5;\n\t"
      "madc.lo.cc.u32 %6, m, 0xe131a029, %6;\n\t"
      "madc.lo.cc.u32 %7, m, 0x30644e72, %7;\n\t"
      "addc.u32       %8, %8, 0;\n\t"
      "mad.hi.cc.u32  %1, m, 0xf0000001, %1;\n\t"
      "madc.hi.cc.u32 %2, m, 0x43e1f593, %2;\n\t"
      "madc.hi.cc.u32 %3, m, 0x79b97091, %3;\n\t"
      "madc.hi.cc.u32 %4, m, 0x2833e848, %4;\n\t"
      "madc.hi.cc.u32 %5, m, 0x8181585d, %5;\n\t"
      "madc.hi.cc.u32 %6, m, 0xb85045b6, %6;\n\t"
      "madc.hi.cc.u32 %7, m, 0xe131a029, %7;\n\t"
      "madc.hi.u32    %8, m, 0x30644e72, %8;\n\t"
      "}"
      : "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]), "+r"(a[8]), "+r"(a[9]));
  Fr o;
#pragma unroll
  for (int i = 0; i < 8; ++i) o.v[i] = a[2 + i];
  return o;
}

__device__ __forceinline__ Fr fr_mul_fixed(const Fr& d, const uint32_t* K8) { return fr_mul_fixed_rows<8>(d, K8); }

#endif  // __CUDACC__
}  // namespace sisu
