// Arithmetic in F_p, p = 2^255 - 19 (the edwards25519 base field), as eight 32-bit limbs,
// little-endian.  Elements are kept "lazy": any value in [0, 2^256) that is congruent to
// the element; fe_canon() gives the unique representative in [0, p).
//
// Products are schoolbook 8x8 with mad.lo.cc / madc.hi.cc carry chains (IMAD pipe), and
// are folded with 2^256 = 38 (mod p).  The paper's GPU code used 4x64-bit words with
// add.cc.u64 (Sec. 7.4, "Finite Field Arithmetic with PTX Instructions"); on NVIDIA parts a
// 64-bit multiply is itself emulated with 32-bit IMADs, so 32-bit limbs are the native
// width here.
#pragma once
#include <cstdint>

// Implementation switches (build flags): squaring, multiplication, the 512-to-256-bit fold
// and addition/subtraction either as PTX carry chains or as 64-bit partial sums.  Measured on
// GB300: the 64-bit partial sums (independent wide products the scheduler overlaps) are
// faster than carry-flag chains for squaring and multiplication.
#ifndef POSLO_SQ_CHAINS
#define POSLO_SQ_CHAINS 0
#endif
#ifndef POSLO_MUL_WIDE
#define POSLO_MUL_WIDE 1
#endif
#ifndef POSLO_FOLD_WIDE
#define POSLO_FOLD_WIDE 0
#endif
#ifndef POSLO_ADD_WIDE
#define POSLO_ADD_WIDE 0
#endif

namespace poslo {

struct fe { uint32_t v[8]; };

__device__ __forceinline__ fe fe_zero() { fe r; for (int i = 0; i < 8; ++i) r.v[i] = 0; return r; }
__device__ __forceinline__ fe fe_one() { fe r = fe_zero(); r.v[0] = 1; return r; }

__device__ __forceinline__ fe fe_const(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t a4,
                                       uint32_t a5, uint32_t a6, uint32_t a7) {
  fe r; r.v[0] = a0; r.v[1] = a1; r.v[2] = a2; r.v[3] = a3; r.v[4] = a4; r.v[5] = a5; r.v[6] = a6; r.v[7] = a7;
  return r;
}

// d = -121665/121666 and 2d, sqrt(-1) = 2^((p-1)/4)  (RFC 8032 Sec. 5.1).
__device__ __forceinline__ fe fe_d() {
  return fe_const(0x135978a3u, 0x75eb4dcau, 0x4141d8abu, 0x00700a4du, 0x7779e898u, 0x8cc74079u, 0x2b6ffe73u, 0x52036ceeu);
}
__device__ __forceinline__ fe fe_d2() {
  return fe_const(0x26b2f159u, 0xebd69b94u, 0x8283b156u, 0x00e0149au, 0xeef3d130u, 0x198e80f2u, 0x56dffce7u, 0x2406d9dcu);
}
__device__ __forceinline__ fe fe_sqrtm1() {
  return fe_const(0x4a0ea0b0u, 0xc4ee1b27u, 0xad2fe478u, 0x2f431806u, 0x3dfbd7a7u, 0x2b4d0099u, 0x4fc1df0bu, 0x2b832480u);
}

#if POSLO_ADD_WIDE
// r = a + b, folding the carry out of bit 256 (2^256 = 38) until none is left.
__device__ __forceinline__ fe fe_add(const fe& a, const fe& b) {
  fe r;
  uint64_t c = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    c += (uint64_t)a.v[k] + b.v[k];
    r.v[k] = (uint32_t)c;
    c >>= 32;
  }
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    uint64_t d = (uint64_t)r.v[0] + c * 38u;
    r.v[0] = (uint32_t)d;
    d >>= 32;
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      d += r.v[k];
      r.v[k] = (uint32_t)d;
      d >>= 32;
    }
    c = d;
  }
  return r;
}

// r = a - b: a borrow out of bit 256 means the wrapped value is 38 too large mod p, so 38 is
// subtracted (twice at most).
__device__ __forceinline__ fe fe_sub(const fe& a, const fe& b) {
  fe r;
  int64_t c = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    c += (int64_t)a.v[k] - (int64_t)b.v[k];
    r.v[k] = (uint32_t)c;
    c >>= 32;   // 0 or -1
  }
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    int64_t d = (int64_t)r.v[0] + c * 38;
    r.v[0] = (uint32_t)d;
    d >>= 32;
#pragma unroll
    for (int k = 1; k < 8; ++k) {
      d += r.v[k];
      r.v[k] = (uint32_t)d;
      d >>= 32;
    }
    c = d;
  }
  return r;
}

#else
// r = a + b, folding the carry out of bit 256 twice (2^256 = 38).
__device__ __forceinline__ fe fe_add(const fe& a, const fe& b) {
  fe r;
  uint32_t c;
  asm("add.cc.u32 %0, %9, %17;\n\t"
      "addc.cc.u32 %1, %10, %18;\n\t"
      "addc.cc.u32 %2, %11, %19;\n\t"
      "addc.cc.u32 %3, %12, %20;\n\t"
      "addc.cc.u32 %4, %13, %21;\n\t"
      "addc.cc.u32 %5, %14, %22;\n\t"
      "addc.cc.u32 %6, %15, %23;\n\t"
      "addc.cc.u32 %7, %16, %24;\n\t"
      "addc.u32 %8, 0, 0;"
      : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]), "=r"(r.v[6]),
        "=r"(r.v[7]), "=r"(c)
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]),
        "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]), "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    const uint32_t k = c * 38u;
    asm("add.cc.u32 %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.cc.u32 %4, %4, 0;\n\t"
        "addc.cc.u32 %5, %5, 0;\n\t"
        "addc.cc.u32 %6, %6, 0;\n\t"
        "addc.cc.u32 %7, %7, 0;\n\t"
        "addc.u32 %8, 0, 0;"
        : "+r"(r.v[0]), "+r"(r.v[1]), "+r"(r.v[2]), "+r"(r.v[3]), "+r"(r.v[4]), "+r"(r.v[5]), "+r"(r.v[6]),
          "+r"(r.v[7]), "=r"(c)
        : "r"(k));
  }
  return r;
}

// r = a - b: on a borrow out of bit 256 the wrapped value is 2^256 too large, i.e. 38 too
// large mod p, so 38 is subtracted (twice at most).
__device__ __forceinline__ fe fe_sub(const fe& a, const fe& b) {
  fe r;
  uint32_t bo;
  asm("sub.cc.u32 %0, %9, %17;\n\t"
      "subc.cc.u32 %1, %10, %18;\n\t"
      "subc.cc.u32 %2, %11, %19;\n\t"
      "subc.cc.u32 %3, %12, %20;\n\t"
      "subc.cc.u32 %4, %13, %21;\n\t"
      "subc.cc.u32 %5, %14, %22;\n\t"
      "subc.cc.u32 %6, %15, %23;\n\t"
      "subc.cc.u32 %7, %16, %24;\n\t"
      "subc.u32 %8, 0, 0;"
      : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]), "=r"(r.v[6]),
        "=r"(r.v[7]), "=r"(bo)
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]),
        "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]), "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    const uint32_t k = bo & 38u;   // bo is 0 or 0xffffffff
    asm("sub.cc.u32 %0, %0, %9;\n\t"
        "subc.cc.u32 %1, %1, 0;\n\t"
        "subc.cc.u32 %2, %2, 0;\n\t"
        "subc.cc.u32 %3, %3, 0;\n\t"
        "subc.cc.u32 %4, %4, 0;\n\t"
        "subc.cc.u32 %5, %5, 0;\n\t"
        "subc.cc.u32 %6, %6, 0;\n\t"
        "subc.cc.u32 %7, %7, 0;\n\t"
        "subc.u32 %8, 0, 0;"
        : "+r"(r.v[0]), "+r"(r.v[1]), "+r"(r.v[2]), "+r"(r.v[3]), "+r"(r.v[4]), "+r"(r.v[5]), "+r"(r.v[6]),
          "+r"(r.v[7]), "=r"(bo)
        : "r"(k));
  }
  return r;
}

#endif

// Fold a 512-bit product t[0..15] to 256 bits: r = t_lo + 38 * t_hi, then fold the
// small top limb (and a possible last carry) the same way.
#if POSLO_FOLD_WIDE
__device__ __forceinline__ fe fe_fold512(const uint32_t t[16]) {
  fe r;
  uint64_t c = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    c += (uint64_t)t[8 + k] * 38u + t[k];
    r.v[k] = (uint32_t)c;
    c >>= 32;
  }
  // c < 38 + 1: fold again, then a possible last carry (at most 1) as 38
  uint64_t d = (uint64_t)r.v[0] + c * 38u;
  r.v[0] = (uint32_t)d;
  d >>= 32;
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    d += r.v[k];
    r.v[k] = (uint32_t)d;
    d >>= 32;
  }
  r.v[0] += (uint32_t)d * 38u;
  return r;
}
#else
__device__ __forceinline__ fe fe_fold512(const uint32_t t[16]) {
  fe r;
  uint32_t top;
  // r = lo + lo(38*hi); carry into top
  asm("mad.lo.cc.u32 %0, %9, 38, %17;\n\t"
      "madc.lo.cc.u32 %1, %10, 38, %18;\n\t"
      "madc.lo.cc.u32 %2, %11, 38, %19;\n\t"
      "madc.lo.cc.u32 %3, %12, 38, %20;\n\t"
      "madc.lo.cc.u32 %4, %13, 38, %21;\n\t"
      "madc.lo.cc.u32 %5, %14, 38, %22;\n\t"
      "madc.lo.cc.u32 %6, %15, 38, %23;\n\t"
      "madc.lo.cc.u32 %7, %16, 38, %24;\n\t"
      "addc.u32 %8, 0, 0;"
      : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]), "=r"(r.v[6]),
        "=r"(r.v[7]), "=r"(top)
      : "r"(t[8]), "r"(t[9]), "r"(t[10]), "r"(t[11]), "r"(t[12]), "r"(t[13]), "r"(t[14]), "r"(t[15]),
        "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(t[3]), "r"(t[4]), "r"(t[5]), "r"(t[6]), "r"(t[7]));
  // r[1..8] += hi(38*hi)
  asm("mad.hi.cc.u32 %0, %8, 38, %0;\n\t"
      "madc.hi.cc.u32 %1, %9, 38, %1;\n\t"
      "madc.hi.cc.u32 %2, %10, 38, %2;\n\t"
      "madc.hi.cc.u32 %3, %11, 38, %3;\n\t"
      "madc.hi.cc.u32 %4, %12, 38, %4;\n\t"
      "madc.hi.cc.u32 %5, %13, 38, %5;\n\t"
      "madc.hi.cc.u32 %6, %14, 38, %6;\n\t"
      "madc.hi.u32 %7, %15, 38, %7;"
      : "+r"(r.v[1]), "+r"(r.v[2]), "+r"(r.v[3]), "+r"(r.v[4]), "+r"(r.v[5]), "+r"(r.v[6]), "+r"(r.v[7]),
        "+r"(top)
      : "r"(t[8]), "r"(t[9]), "r"(t[10]), "r"(t[11]), "r"(t[12]), "r"(t[13]), "r"(t[14]), "r"(t[15]));
  // top < 2^6: fold top*38, then a final carry (at most 1) as 38.
  uint32_t c;
  asm("mad.lo.cc.u32 %0, %9, 38, %0;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.cc.u32 %3, %3, 0;\n\t"
      "addc.cc.u32 %4, %4, 0;\n\t"
      "addc.cc.u32 %5, %5, 0;\n\t"
      "addc.cc.u32 %6, %6, 0;\n\t"
      "addc.cc.u32 %7, %7, 0;\n\t"
      "addc.u32 %8, 0, 0;"
      : "+r"(r.v[0]), "+r"(r.v[1]), "+r"(r.v[2]), "+r"(r.v[3]), "+r"(r.v[4]), "+r"(r.v[5]), "+r"(r.v[6]),
        "+r"(r.v[7]), "=r"(c)
      : "r"(top));
  // If c = 1 the low 256 bits are < 38*64, so adding 38 cannot carry again.
  r.v[0] += c * 38u;
  return r;
}
#endif

// 8x8-limb schoolbook product.  Row i adds lo(a_i*b_j) into t[i+j] and hi(a_i*b_j) into
// t[i+j+1], each as one carry chain inside a single asm statement (the carry flag does not
// survive between statements).  Before row i, t[i+9..15] are still zero.
#define POSLO_MUL_ROW_LO                                   \
  "mad.lo.cc.u32 %0, %10, %11, %0;\n\t"                   \
  "madc.lo.cc.u32 %1, %10, %12, %1;\n\t"                  \
  "madc.lo.cc.u32 %2, %10, %13, %2;\n\t"                  \
  "madc.lo.cc.u32 %3, %10, %14, %3;\n\t"                  \
  "madc.lo.cc.u32 %4, %10, %15, %4;\n\t"                  \
  "madc.lo.cc.u32 %5, %10, %16, %5;\n\t"                  \
  "madc.lo.cc.u32 %6, %10, %17, %6;\n\t"                  \
  "madc.lo.cc.u32 %7, %10, %18, %7;\n\t"
#define POSLO_MUL_ROW_HI                                   \
  "mad.hi.cc.u32 %0, %9, %10, %0;\n\t"                    \
  "madc.hi.cc.u32 %1, %9, %11, %1;\n\t"                   \
  "madc.hi.cc.u32 %2, %9, %12, %2;\n\t"                   \
  "madc.hi.cc.u32 %3, %9, %13, %3;\n\t"                   \
  "madc.hi.cc.u32 %4, %9, %14, %4;\n\t"                   \
  "madc.hi.cc.u32 %5, %9, %15, %5;\n\t"                   \
  "madc.hi.cc.u32 %6, %9, %16, %6;\n\t"

__device__ __forceinline__ void mul_8x8(uint32_t t[16], const uint32_t a[8], const uint32_t b[8]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) t[k] = 0;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    asm(POSLO_MUL_ROW_LO
        "addc.cc.u32 %8, %8, 0;\n\t"
        "addc.u32 %9, 0, 0;"
        : "+r"(t[i + 0]), "+r"(t[i + 1]), "+r"(t[i + 2]), "+r"(t[i + 3]), "+r"(t[i + 4]), "+r"(t[i + 5]),
          "+r"(t[i + 6]), "+r"(t[i + 7]), "+r"(t[i + 8]), "=r"(t[i + 9])
        : "r"(a[i]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
    asm(POSLO_MUL_ROW_HI
        "madc.hi.cc.u32 %7, %9, %17, %7;\n\t"
        "addc.u32 %8, %8, 0;"
        : "+r"(t[i + 1]), "+r"(t[i + 2]), "+r"(t[i + 3]), "+r"(t[i + 4]), "+r"(t[i + 5]), "+r"(t[i + 6]),
          "+r"(t[i + 7]), "+r"(t[i + 8]), "+r"(t[i + 9])
        : "r"(a[i]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
  }
  // last row: the full product is < 2^512, so nothing carries out of t[15].  `unused`
  // keeps the operand numbering of the row macros.
  uint32_t unused;
  asm(POSLO_MUL_ROW_LO
      "addc.u32 %8, %8, 0;"
      : "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]),
        "+r"(t[15]), "=r"(unused)
      : "r"(a[7]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
  asm(POSLO_MUL_ROW_HI
      "madc.hi.u32 %7, %9, %17, %7;"
      : "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15]),
        "=r"(unused)
      : "r"(a[7]), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
}

__device__ __forceinline__ fe fe_mul(const fe& a, const fe& b) {
  uint32_t t[16];
#if POSLO_MUL_WIDE
  // operand scanning with 64-bit partial sums (independent wide products)
#pragma unroll
  for (int q = 0; q < 16; ++q) t[q] = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    uint64_t carry = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint64_t p = (uint64_t)a.v[i] * b.v[j] + t[i + j] + carry;
      t[i + j] = (uint32_t)p;
      carry = p >> 32;
    }
    t[i + 8] = (uint32_t)carry;
  }
#else
  mul_8x8(t, a.v, b.v);
#endif
  return fe_fold512(t);
}

#if POSLO_SQ_CHAINS
// Squaring: the 28 cross products a_i a_j (i < j) once, as row carry chains like mul_8x8
// (row i covers columns 2i+1 .. i+8), doubled by a funnel shift, plus the 8 diagonal
// squares a_i^2 at limb 2i in one multiply-add chain: 36 low + 36 high products instead of
// 64 + 64.
__device__ __forceinline__ fe fe_sq(const fe& a) {
  uint32_t t[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) t[k] = 0;
  uint32_t unused;
  // row 0: low halves of a_0 a_j, j = 1..7
  asm("mad.lo.cc.u32 %0, %9, %10, %0;\n\t"
      "madc.lo.cc.u32 %1, %9, %11, %1;\n\t"
      "madc.lo.cc.u32 %2, %9, %12, %2;\n\t"
      "madc.lo.cc.u32 %3, %9, %13, %3;\n\t"
      "madc.lo.cc.u32 %4, %9, %14, %4;\n\t"
      "madc.lo.cc.u32 %5, %9, %15, %5;\n\t"
      "madc.lo.cc.u32 %6, %9, %16, %6;\n\t"
      "addc.u32 %7, 0, 0;"
      : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "=r"(t[8]), "=r"(unused)
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 0: high halves
  asm("mad.hi.cc.u32 %0, %8, %9, %0;\n\t"
      "madc.hi.cc.u32 %1, %8, %10, %1;\n\t"
      "madc.hi.cc.u32 %2, %8, %11, %2;\n\t"
      "madc.hi.cc.u32 %3, %8, %12, %3;\n\t"
      "madc.hi.cc.u32 %4, %8, %13, %4;\n\t"
      "madc.hi.cc.u32 %5, %8, %14, %5;\n\t"
      "madc.hi.cc.u32 %6, %8, %15, %6;\n\t"
      "addc.u32 %7, %7, 0;"
      : "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 1: low halves of a_1 a_j, j = 2..7
  asm("mad.lo.cc.u32 %0, %8, %9, %0;\n\t"
      "madc.lo.cc.u32 %1, %8, %10, %1;\n\t"
      "madc.lo.cc.u32 %2, %8, %11, %2;\n\t"
      "madc.lo.cc.u32 %3, %8, %12, %3;\n\t"
      "madc.lo.cc.u32 %4, %8, %13, %4;\n\t"
      "madc.lo.cc.u32 %5, %8, %14, %5;\n\t"
      "addc.cc.u32 %6, %6, 0;\n\t"
      "addc.u32 %7, 0, 0;"
      : "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "=r"(t[10])
      : "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 1: high halves
  asm("mad.hi.cc.u32 %0, %7, %8, %0;\n\t"
      "madc.hi.cc.u32 %1, %7, %9, %1;\n\t"
      "madc.hi.cc.u32 %2, %7, %10, %2;\n\t"
      "madc.hi.cc.u32 %3, %7, %11, %3;\n\t"
      "madc.hi.cc.u32 %4, %7, %12, %4;\n\t"
      "madc.hi.cc.u32 %5, %7, %13, %5;\n\t"
      "addc.u32 %6, %6, 0;"
      : "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10])
      : "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 2: low halves of a_2 a_j, j = 3..7
  asm("mad.lo.cc.u32 %0, %7, %8, %0;\n\t"
      "madc.lo.cc.u32 %1, %7, %9, %1;\n\t"
      "madc.lo.cc.u32 %2, %7, %10, %2;\n\t"
      "madc.lo.cc.u32 %3, %7, %11, %3;\n\t"
      "madc.lo.cc.u32 %4, %7, %12, %4;\n\t"
      "addc.cc.u32 %5, %5, 0;\n\t"
      "addc.u32 %6, 0, 0;"
      : "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "=r"(t[11])
      : "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 2: high halves
  asm("mad.hi.cc.u32 %0, %6, %7, %0;\n\t"
      "madc.hi.cc.u32 %1, %6, %8, %1;\n\t"
      "madc.hi.cc.u32 %2, %6, %9, %2;\n\t"
      "madc.hi.cc.u32 %3, %6, %10, %3;\n\t"
      "madc.hi.cc.u32 %4, %6, %11, %4;\n\t"
      "addc.u32 %5, %5, 0;"
      : "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11])
      : "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 3: low halves of a_3 a_j, j = 4..7
  asm("mad.lo.cc.u32 %0, %6, %7, %0;\n\t"
      "madc.lo.cc.u32 %1, %6, %8, %1;\n\t"
      "madc.lo.cc.u32 %2, %6, %9, %2;\n\t"
      "madc.lo.cc.u32 %3, %6, %10, %3;\n\t"
      "addc.cc.u32 %4, %4, 0;\n\t"
      "addc.u32 %5, 0, 0;"
      : "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "=r"(t[12])
      : "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 3: high halves
  asm("mad.hi.cc.u32 %0, %5, %6, %0;\n\t"
      "madc.hi.cc.u32 %1, %5, %7, %1;\n\t"
      "madc.hi.cc.u32 %2, %5, %8, %2;\n\t"
      "madc.hi.cc.u32 %3, %5, %9, %3;\n\t"
      "addc.u32 %4, %4, 0;"
      : "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12])
      : "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 4: low halves of a_4 a_j, j = 5..7
  asm("mad.lo.cc.u32 %0, %5, %6, %0;\n\t"
      "madc.lo.cc.u32 %1, %5, %7, %1;\n\t"
      "madc.lo.cc.u32 %2, %5, %8, %2;\n\t"
      "addc.cc.u32 %3, %3, 0;\n\t"
      "addc.u32 %4, 0, 0;"
      : "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "=r"(t[13])
      : "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 4: high halves
  asm("mad.hi.cc.u32 %0, %4, %5, %0;\n\t"
      "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
      "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
      "addc.u32 %3, %3, 0;"
      : "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13])
      : "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 5: low halves of a_5 a_j, j = 6..7
  asm("mad.lo.cc.u32 %0, %4, %5, %0;\n\t"
      "madc.lo.cc.u32 %1, %4, %6, %1;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.u32 %3, 0, 0;"
      : "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "=r"(t[14])
      : "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 5: high halves
  asm("mad.hi.cc.u32 %0, %3, %4, %0;\n\t"
      "madc.hi.cc.u32 %1, %3, %5, %1;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(t[12]), "+r"(t[13]), "+r"(t[14])
      : "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  // row 6: low halves of a_6 a_j, j = 7..7
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.u32 %2, 0, 0;"
      : "+r"(t[13]), "+r"(t[14]), "=r"(t[15])
      : "r"(a.v[6]), "r"(a.v[7]));
  // row 6: high halves
  asm("mad.hi.cc.u32 %0, %2, %3, %0;\n\t"
      "addc.u32 %1, %1, 0;"
      : "+r"(t[14]), "+r"(t[15])
      : "r"(a.v[6]), "r"(a.v[7]));
  // double the cross products (their sum is below 2^511)
#pragma unroll
  for (int k = 15; k > 0; --k) t[k] = __funnelshift_l(t[k - 1], t[k], 1);
  t[0] = 0;
  asm("mad.lo.cc.u32 %0, %16, %16, %0;\n\t"
      "madc.hi.cc.u32 %1, %16, %16, %1;\n\t"
      "madc.lo.cc.u32 %2, %17, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %17, %17, %3;\n\t"
      "madc.lo.cc.u32 %4, %18, %18, %4;\n\t"
      "madc.hi.cc.u32 %5, %18, %18, %5;\n\t"
      "madc.lo.cc.u32 %6, %19, %19, %6;\n\t"
      "madc.hi.cc.u32 %7, %19, %19, %7;\n\t"
      "madc.lo.cc.u32 %8, %20, %20, %8;\n\t"
      "madc.hi.cc.u32 %9, %20, %20, %9;\n\t"
      "madc.lo.cc.u32 %10, %21, %21, %10;\n\t"
      "madc.hi.cc.u32 %11, %21, %21, %11;\n\t"
      "madc.lo.cc.u32 %12, %22, %22, %12;\n\t"
      "madc.hi.cc.u32 %13, %22, %22, %13;\n\t"
      "madc.lo.cc.u32 %14, %23, %23, %14;\n\t"
      "madc.hi.u32 %15, %23, %23, %15;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]),
        "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  (void)unused;
  return fe_fold512(t);
}

#else
// Squaring: the 28 cross products a_i a_j (i < j) once (operand scanning with 64-bit
// partial sums: independent wide products the scheduler can overlap), doubled by a funnel
// shift, plus the 8 diagonal squares a_i^2 at limb 2i in one carry chain.
__device__ __forceinline__ fe fe_sq(const fe& a) {
  uint32_t t[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) t[k] = 0;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    uint64_t carry = 0;
#pragma unroll
    for (int j = i + 1; j < 8; ++j) {
      const uint64_t p = (uint64_t)a.v[i] * a.v[j] + t[i + j] + carry;
      t[i + j] = (uint32_t)p;
      carry = p >> 32;
    }
    t[i + 8] = (uint32_t)carry;
  }
#pragma unroll
  for (int k = 15; k > 0; --k) t[k] = __funnelshift_l(t[k - 1], t[k], 1);
  t[0] = 0;
  asm("mad.lo.cc.u32 %0, %16, %16, %0;\n\t"
      "madc.hi.cc.u32 %1, %16, %16, %1;\n\t"
      "madc.lo.cc.u32 %2, %17, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %17, %17, %3;\n\t"
      "madc.lo.cc.u32 %4, %18, %18, %4;\n\t"
      "madc.hi.cc.u32 %5, %18, %18, %5;\n\t"
      "madc.lo.cc.u32 %6, %19, %19, %6;\n\t"
      "madc.hi.cc.u32 %7, %19, %19, %7;\n\t"
      "madc.lo.cc.u32 %8, %20, %20, %8;\n\t"
      "madc.hi.cc.u32 %9, %20, %20, %9;\n\t"
      "madc.lo.cc.u32 %10, %21, %21, %10;\n\t"
      "madc.hi.cc.u32 %11, %21, %21, %11;\n\t"
      "madc.lo.cc.u32 %12, %22, %22, %12;\n\t"
      "madc.hi.cc.u32 %13, %22, %22, %13;\n\t"
      "madc.lo.cc.u32 %14, %23, %23, %14;\n\t"
      "madc.hi.u32 %15, %23, %23, %15;"
      : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]),
        "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15])
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
  return fe_fold512(t);
}

#endif

// n successive squarings; the loop is kept rolled so the exponentiation chains of the
// inversion and square root stay small in the instruction cache.
__device__ __forceinline__ fe fe_sqn(fe a, int n) {
#pragma unroll 1
  for (int i = 0; i < n; ++i) a = fe_sq(a);
  return a;
}

// Multiply by a small constant k < 2^26 and fold.
__device__ __forceinline__ fe fe_mul_small(const fe& a, uint32_t k) {
  uint32_t t[16];
  uint32_t top;
  asm("mul.lo.u32 %0, %9, %17;\n\t"
      "mul.lo.u32 %1, %10, %17;\n\t"
      "mul.lo.u32 %2, %11, %17;\n\t"
      "mul.lo.u32 %3, %12, %17;\n\t"
      "mul.lo.u32 %4, %13, %17;\n\t"
      "mul.lo.u32 %5, %14, %17;\n\t"
      "mul.lo.u32 %6, %15, %17;\n\t"
      "mul.lo.u32 %7, %16, %17;\n\t"
      "mov.u32 %8, 0;"
      : "=r"(t[0]), "=r"(t[1]), "=r"(t[2]), "=r"(t[3]), "=r"(t[4]), "=r"(t[5]), "=r"(t[6]), "=r"(t[7]), "=r"(top)
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]),
        "r"(k));
  asm("mad.hi.cc.u32 %0, %9, %17, %0;\n\t"
      "madc.hi.cc.u32 %1, %10, %17, %1;\n\t"
      "madc.hi.cc.u32 %2, %11, %17, %2;\n\t"
      "madc.hi.cc.u32 %3, %12, %17, %3;\n\t"
      "madc.hi.cc.u32 %4, %13, %17, %4;\n\t"
      "madc.hi.cc.u32 %5, %14, %17, %5;\n\t"
      "madc.hi.cc.u32 %6, %15, %17, %6;\n\t"
      "madc.hi.u32 %7, %16, %17, %7;"
      : "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(top)
      : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]),
        "r"(k));
  t[8] = top;
#pragma unroll
  for (int i = 9; i < 16; ++i) t[i] = 0;
  return fe_fold512(t);
}

// Unique representative in [0, p): subtract p while the value is >= p (at most twice for
// a value below 2^256 = 2p + 38).
__device__ __forceinline__ fe fe_canon(fe a) {
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    fe r;
    uint32_t bo;
    asm("sub.cc.u32 %0, %9, 0xffffffed;\n\t"
        "subc.cc.u32 %1, %10, 0xffffffff;\n\t"
        "subc.cc.u32 %2, %11, 0xffffffff;\n\t"
        "subc.cc.u32 %3, %12, 0xffffffff;\n\t"
        "subc.cc.u32 %4, %13, 0xffffffff;\n\t"
        "subc.cc.u32 %5, %14, 0xffffffff;\n\t"
        "subc.cc.u32 %6, %15, 0xffffffff;\n\t"
        "subc.cc.u32 %7, %16, 0x7fffffff;\n\t"
        "subc.u32 %8, 0, 0;"
        : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]), "=r"(r.v[6]),
          "=r"(r.v[7]), "=r"(bo)
        : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]),
          "r"(a.v[7]));
    // keep r when no borrow (a >= p)
#pragma unroll
    for (int i = 0; i < 8; ++i) a.v[i] = bo ? a.v[i] : r.v[i];
  }
  return a;
}

__device__ __forceinline__ bool fe_is_zero(const fe& a) {
  const fe c = fe_canon(a);
  uint32_t o = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) o |= c.v[i];
  return o == 0;
}

__device__ __forceinline__ bool fe_eq(const fe& a, const fe& b) { return fe_is_zero(fe_sub(a, b)); }

__device__ __forceinline__ fe fe_neg(const fe& a) { return fe_sub(fe_zero(), a); }

__device__ __forceinline__ fe fe_select(const fe& a, const fe& b, bool pick_b) {
  fe r;
#pragma unroll
  for (int i = 0; i < 8; ++i) r.v[i] = pick_b ? b.v[i] : a.v[i];
  return r;
}

// z^(2^250 - 1) and z^11 share one addition chain (z^2, z^9, z^11, then runs of squarings
// building z^(2^k - 1) for k = 5, 10, 20, 40, 50, 100, 200, 250).
__device__ __forceinline__ fe fe_pow_2_250_1(const fe& z, fe* z11_out) {
  const fe z2 = fe_sq(z);
  const fe z8 = fe_sqn(z2, 2);
  const fe z9 = fe_mul(z8, z);
  const fe z11 = fe_mul(z9, z2);
  const fe z22 = fe_sq(z11);
  const fe z_5 = fe_mul(z22, z9);                 // 2^5 - 1
  const fe z_10 = fe_mul(fe_sqn(z_5, 5), z_5);     // 2^10 - 1
  const fe z_20 = fe_mul(fe_sqn(z_10, 10), z_10);  // 2^20 - 1
  const fe z_40 = fe_mul(fe_sqn(z_20, 20), z_20);  // 2^40 - 1
  const fe z_50 = fe_mul(fe_sqn(z_40, 10), z_10);  // 2^50 - 1
  const fe z_100 = fe_mul(fe_sqn(z_50, 50), z_50); // 2^100 - 1
  const fe z_200 = fe_mul(fe_sqn(z_100, 100), z_100);
  const fe z_250 = fe_mul(fe_sqn(z_200, 50), z_50);
  if (z11_out) *z11_out = z11;
  return z_250;
}

// z^(p-2) = z^(2^255 - 21) = (z^(2^250-1))^(2^5) * z^11  (Fermat inverse; 0 -> 0).
__device__ __forceinline__ fe fe_inv(const fe& z) {
  fe z11;
  const fe t = fe_pow_2_250_1(z, &z11);
  return fe_mul(fe_sqn(t, 5), z11);
}

// z^((p-5)/8) = z^(2^252 - 3) = (z^(2^250-1))^4 * z.
__device__ __forceinline__ fe fe_pow_p58(const fe& z) {
  const fe t = fe_pow_2_250_1(z, nullptr);
  return fe_mul(fe_sqn(t, 2), z);
}

__device__ __forceinline__ uint32_t fe_parity(const fe& a) { return fe_canon(a).v[0] & 1u; }

}  // namespace poslo
