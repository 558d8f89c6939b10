// Scalars modulo the edwards25519 group order q = 2^252 + 27742317777372353535851937790883648493,
// as eight 32-bit little-endian limbs.  Used for e = H(m || x) mod q (Fig. 3a AVer), the
// aggregates e~ = sum e and s~ = sum s mod q (POSLO-C.Agg, Fig. 3a), and the signer's
// s = r - e y mod q (test-data generation).
#pragma once
#include <cstdint>

namespace poslo {

struct sc { uint32_t v[8]; };

__device__ __forceinline__ uint32_t sc_q(int i) {
  const uint32_t q[8] = {0x5cf5d3edu, 0x5812631au, 0xa2f79cd6u, 0x14def9deu, 0u, 0u, 0u, 0x10000000u};
  return q[i];
}

// a - b over 8 limbs; returns the borrow (1 if a < b).
__device__ __forceinline__ uint32_t sub8(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
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
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(bo)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[0]),
        "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
  return bo & 1u;
}

// a + b over 8 limbs; returns the carry.
__device__ __forceinline__ uint32_t add8(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
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
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(c)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(b[0]),
        "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
  return c;
}

__device__ __forceinline__ void sc_qlimbs(uint32_t q[8]) {
  q[0] = 0x5cf5d3edu; q[1] = 0x5812631au; q[2] = 0xa2f79cd6u; q[3] = 0x14def9deu;
  q[4] = 0u; q[5] = 0u; q[6] = 0u; q[7] = 0x10000000u;
}

// 1 if a < q (a canonical scalar encoding).
__device__ __forceinline__ bool sc_is_canonical(const uint32_t a[8]) {
  uint32_t q[8], r[8];
  sc_qlimbs(q);
  return sub8(r, a, q) != 0;
}

// x mod q for x < 2^256: with t = floor(x / 2^252) <= 15, x - t q lies in (-15 q, q); one
// conditional addition of q finishes.  q - 2^252 = c < 2^125, so x - t q = (x mod 2^252) - t c.
__device__ __forceinline__ sc sc_reduce256(const uint32_t x[8]) {
  const uint32_t t = x[7] >> 28;
  uint32_t lo[8];
#pragma unroll
  for (int i = 0; i < 7; ++i) lo[i] = x[i];
  lo[7] = x[7] & 0x0fffffffu;
  // tc = t * c  (c = limbs 0..3 of q), 5 limbs
  uint32_t tc[8];
  tc[0] = t * 0x5cf5d3edu;  tc[1] = __umulhi(t, 0x5cf5d3edu);
  uint32_t h1 = __umulhi(t, 0x5812631au), h2 = __umulhi(t, 0xa2f79cd6u), h3 = __umulhi(t, 0x14def9deu);
  asm("mad.lo.cc.u32 %0, %5, 0x5812631a, %0;\n\t"
      "madc.lo.cc.u32 %1, %5, 0xa2f79cd6, %6;\n\t"
      "madc.lo.cc.u32 %2, %5, 0x14def9de, %7;\n\t"
      "addc.cc.u32 %3, %8, 0;\n\t"
      "addc.u32 %4, 0, 0;"
      : "+r"(tc[1]), "=r"(tc[2]), "=r"(tc[3]), "=r"(tc[4]), "=r"(tc[5])
      : "r"(t), "r"(h1), "r"(h2), "r"(h3));
  tc[6] = 0; tc[7] = 0;
  sc r;
  const uint32_t bo = sub8(r.v, lo, tc);
  if (bo) {
    uint32_t q[8];
    sc_qlimbs(q);
    add8(r.v, r.v, q);
  }
  return r;
}

// (a + b) mod q for canonical a, b.
__device__ __forceinline__ sc sc_add(const sc& a, const sc& b) {
  sc r, s;
  uint32_t q[8];
  sc_qlimbs(q);
  add8(r.v, a.v, b.v);   // < 2q < 2^254: no carry
  const uint32_t bo = sub8(s.v, r.v, q);
  return bo ? r : s;
}

// (a - b) mod q for canonical a, b.
__device__ __forceinline__ sc sc_sub(const sc& a, const sc& b) {
  sc r;
  uint32_t q[8];
  sc_qlimbs(q);
  if (sub8(r.v, a.v, b.v)) add8(r.v, r.v, q);
  return r;
}

// Barrett reduction (Menezes, van Oorschot, Vanstone, Handbook of Applied Cryptography,
// Algorithm 14.42) of a 512-bit x with base b = 2^32, k = 8 and mu = floor(2^512 / q).
__device__ __forceinline__ sc sc_reduce512(const uint32_t x[16]) {
  const uint32_t mu[9] = {0x0a2c131bu, 0xed9ce5a3u, 0x086329a7u, 0x2106215du, 0xffffffebu,
                          0xffffffffu, 0xffffffffu, 0xffffffffu, 0x0000000fu};
  // q1 = floor(x / b^7): limbs x[7..15] (9 limbs)
  // q2 = q1 * mu (18 limbs); q3 = floor(q2 / b^9)
  uint32_t q2[18];
#pragma unroll
  for (int k = 0; k < 18; ++k) q2[k] = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    uint64_t carry = 0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const uint64_t p = (uint64_t)x[7 + i] * mu[j] + q2[i + j] + carry;
      q2[i + j] = (uint32_t)p;
      carry = p >> 32;
    }
    q2[i + 9] = (uint32_t)carry;
  }
  // r2 = (q3 * q) mod b^9, q3 = q2[9..17]
  uint32_t q[8];
  sc_qlimbs(q);
  uint32_t r2[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) r2[k] = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    uint64_t carry = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (i + j < 9) {
        const uint64_t p = (uint64_t)q2[9 + i] * q[j] + r2[i + j] + carry;
        r2[i + j] = (uint32_t)p;
        carry = p >> 32;
      }
    }
    if (i + 8 < 9) r2[i + 8] = (uint32_t)carry;
  }
  // r = (x mod b^9) - r2 mod b^9, then subtract q while r >= q (at most twice)
  uint32_t r[9];
  uint64_t borrow = 0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const uint64_t d = (uint64_t)x[k] - r2[k] - borrow;
    r[k] = (uint32_t)d;
    borrow = (d >> 32) & 1u;
  }
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    uint32_t s[9];
    uint64_t bb = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const uint64_t d = (uint64_t)r[k] - (k < 8 ? q[k] : 0u) - bb;
      s[k] = (uint32_t)d;
      bb = (d >> 32) & 1u;
    }
    if (!bb) {
#pragma unroll
      for (int k = 0; k < 9; ++k) r[k] = s[k];
    }
  }
  sc out;
#pragma unroll
  for (int k = 0; k < 8; ++k) out.v[k] = r[k];
  return out;
}

// (a * b) mod q.
__device__ __forceinline__ sc sc_mul(const sc& a, const sc& b) {
  uint32_t t[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) t[k] = 0;
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
  return sc_reduce512(t);
}

// Unreduced accumulator of up to 2^32 terms below 2^384: 13 limbs (416 bits).
struct acc13 { uint32_t v[13]; };

__device__ __forceinline__ void acc_zero(acc13& a) {
#pragma unroll
  for (int k = 0; k < 13; ++k) a.v[k] = 0;
}

// a += x (x has n limbs, n <= 12)
template <int N>
__device__ __forceinline__ void acc_add(acc13& a, const uint32_t x[N]) {
  uint64_t carry = 0;
#pragma unroll
  for (int k = 0; k < 13; ++k) {
    const uint64_t s = (uint64_t)a.v[k] + (k < N ? x[k] : 0u) + carry;
    a.v[k] = (uint32_t)s;
    carry = s >> 32;
  }
}

// z (4 limbs, 128-bit weight) times x (8 limbs) -> 12 limbs.
__device__ __forceinline__ void mul_4x8(uint32_t r[12], const uint32_t z[4], const uint32_t x[8]) {
#pragma unroll
  for (int k = 0; k < 12; ++k) r[k] = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    uint64_t carry = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint64_t p = (uint64_t)z[i] * x[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)p;
      carry = p >> 32;
    }
    r[i + 8] = (uint32_t)carry;
  }
}

__device__ __forceinline__ sc acc_reduce(const acc13& a) {
  uint32_t x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = k < 13 ? a.v[k] : 0u;
  return sc_reduce512(x);
}

}  // namespace poslo
