// edwards25519 group operations: -x^2 + y^2 = 1 + d x^2 y^2 over F_p, extended coordinates
// (X:Y:Z:T) with x = X/Z, y = Y/Z, xy = T/Z (Hisil, Wong, Carter, Dawson, "Twisted Edwards
// curves revisited", ASIACRYPT 2008).  The paper writes its group multiplicatively
// (alpha^x mod p, products of commitments); here alpha^x is [x]G and a product is a sum.
#pragma once
#include "fe25519.cuh"
#include "sc25519.cuh"

namespace poslo {

struct ge { fe X, Y, Z, T; };

__device__ __forceinline__ ge ge_identity() {
  ge r; r.X = fe_zero(); r.Y = fe_one(); r.Z = fe_one(); r.T = fe_zero(); return r;
}

// Base point G: y = 4/5, x even (RFC 8032 Sec. 5.1).
__device__ __forceinline__ ge ge_base() {
  ge r;
  r.X = fe_const(0x8f25d51au, 0xc9562d60u, 0x9525a7b2u, 0x692cc760u, 0xfdd6dc5cu, 0xc0a4e231u, 0xcd6e53feu, 0x216936d3u);
  r.Y = fe_const(0x66666658u, 0x66666666u, 0x66666666u, 0x66666666u, 0x66666666u, 0x66666666u, 0x66666666u, 0x66666666u);
  r.Z = fe_one();
  r.T = fe_const(0xa5b7dda3u, 0x6dde8ab3u, 0x775152f5u, 0x20f09f80u, 0x64abe37du, 0x66ea4e8eu, 0xd78b7665u, 0x67875f0fu);
  return r;
}

// Unified addition (add-2008-hwcd-3 with a = -1, k = 2d): complete on this curve because d
// is not a square in F_p.  9M.
__device__ __forceinline__ ge ge_add(const ge& p, const ge& q) {
  const fe A = fe_mul(fe_sub(p.Y, p.X), fe_sub(q.Y, q.X));
  const fe B = fe_mul(fe_add(p.Y, p.X), fe_add(q.Y, q.X));
  const fe C = fe_mul(fe_mul(p.T, fe_d2()), q.T);
  const fe Zp = fe_mul(p.Z, q.Z);
  const fe D = fe_add(Zp, Zp);
  const fe E = fe_sub(B, A), F = fe_sub(D, C), G = fe_add(D, C), H = fe_add(B, A);
  ge r;
  r.X = fe_mul(E, F); r.Y = fe_mul(G, H); r.Z = fe_mul(F, G); r.T = fe_mul(E, H);
  return r;
}

// Doubling (dbl-2008-hwcd with a = -1).  4M + 4S; T of the input is not used.
__device__ __forceinline__ ge ge_dbl(const ge& p) {
  const fe A = fe_sq(p.X);
  const fe B = fe_sq(p.Y);
  const fe Z2 = fe_sq(p.Z);
  const fe C = fe_add(Z2, Z2);
  const fe E = fe_sub(fe_sub(fe_sq(fe_add(p.X, p.Y)), A), B);
  const fe G = fe_sub(B, A);          // D + B with D = -A
  const fe F = fe_sub(G, C);
  const fe H = fe_neg(fe_add(A, B));  // D - B
  ge r;
  r.X = fe_mul(E, F); r.Y = fe_mul(G, H); r.Z = fe_mul(F, G); r.T = fe_mul(E, H);
  return r;
}

__device__ __forceinline__ ge ge_neg(const ge& p) {
  ge r = p; r.X = fe_neg(p.X); r.T = fe_neg(p.T); return r;
}

__device__ __forceinline__ ge ge_sub(const ge& p, const ge& q) { return ge_add(p, ge_neg(q)); }

__device__ __forceinline__ ge ge_select(const ge& a, const ge& b, bool pick_b) {
  ge r;
  r.X = fe_select(a.X, b.X, pick_b); r.Y = fe_select(a.Y, b.Y, pick_b);
  r.Z = fe_select(a.Z, b.Z, pick_b); r.T = fe_select(a.T, b.T, pick_b);
  return r;
}

// P = O  <=>  X = 0 and Y = Z.
__device__ __forceinline__ bool ge_is_identity(const ge& p) { return fe_is_zero(p.X) && fe_eq(p.Y, p.Z); }

__device__ __forceinline__ ge ge_mul_cofactor(const ge& p) { return ge_dbl(ge_dbl(ge_dbl(p))); }

// Strict decoding of a 32-byte compressed point (RFC 8032 Sec. 5.1.3): reject y >= p,
// reject when (y^2 - 1)/(d y^2 + 1) has no square root, reject x = 0 with the sign bit set.
// The root of u/v is u v^3 (u v^7)^((p-5)/8), corrected by sqrt(-1) when needed.
__device__ __forceinline__ bool ge_decode(const uint32_t b[8], ge& out) {
  fe y;
#pragma unroll
  for (int i = 0; i < 8; ++i) y.v[i] = b[i];
  const uint32_t sign = b[7] >> 31;
  y.v[7] &= 0x7fffffffu;
  // y < p  <=>  canon(y) == y
  const fe yc = fe_canon(y);
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 8; ++i) ok &= (yc.v[i] == y.v[i]);
  const fe y2 = fe_sq(y);
  const fe u = fe_sub(y2, fe_one());
  const fe v = fe_add(fe_mul(fe_d(), y2), fe_one());
  const fe v3 = fe_mul(fe_sq(v), v);
  const fe v7 = fe_mul(fe_sq(v3), v);
  fe x = fe_mul(fe_mul(u, v3), fe_pow_p58(fe_mul(u, v7)));
  const fe vx2 = fe_mul(v, fe_sq(x));
  const bool root = fe_eq(vx2, u);
  const bool root_neg = fe_eq(vx2, fe_neg(u));
  x = fe_select(x, fe_mul(x, fe_sqrtm1()), !root && root_neg);
  ok &= (root || root_neg);
  x = fe_canon(x);
  bool xzero = true;
#pragma unroll
  for (int i = 0; i < 8; ++i) xzero &= (x.v[i] == 0);
  ok &= !(xzero && sign);
  x = fe_select(x, fe_neg(x), (x.v[0] & 1u) != sign);
  out.X = x;
  out.Y = y;
  out.Z = fe_one();
  out.T = fe_mul(x, y);
  return ok;
}

// Compressed encoding: y with the parity of x in bit 255.
__device__ __forceinline__ void ge_encode(const ge& p, uint32_t b[8]) {
  const fe zi = fe_inv(p.Z);
  const fe x = fe_canon(fe_mul(p.X, zi));
  const fe y = fe_canon(fe_mul(p.Y, zi));
#pragma unroll
  for (int i = 0; i < 8; ++i) b[i] = y.v[i];
  b[7] |= (x.v[0] & 1u) << 31;
}

// Mixed addition with an affine point given as (x, y, t2d = 2d x y): the "precomputed"
// form of the unified addition, 7M (Hisil et al. 2008, Sec. 3.1 with Z2 = 1).
__device__ __forceinline__ ge ge_madd(const ge& p, const fe& x, const fe& y, const fe& t2d) {
  const fe A = fe_mul(fe_sub(p.Y, p.X), fe_sub(y, x));
  const fe B = fe_mul(fe_add(p.Y, p.X), fe_add(y, x));
  const fe C = fe_mul(p.T, t2d);
  const fe D = fe_add(p.Z, p.Z);
  const fe E = fe_sub(B, A), F = fe_sub(D, C), G = fe_add(D, C), H = fe_add(B, A);
  ge r;
  r.X = fe_mul(E, F); r.Y = fe_mul(G, H); r.Z = fe_mul(F, G); r.T = fe_mul(E, H);
  return r;
}

// ge_madd of P or of -P = (-x, y, -t2d): negation swaps y - x with y + x and negates t2d.
__device__ __forceinline__ ge ge_madd_signed(const ge& p, const fe& x, const fe& y, const fe& t2d, bool neg) {
  const fe ym = fe_sub(y, x), yp = fe_add(y, x);
  const fe A = fe_mul(fe_sub(p.Y, p.X), fe_select(ym, yp, neg));
  const fe B = fe_mul(fe_add(p.Y, p.X), fe_select(yp, ym, neg));
  const fe C = fe_mul(p.T, fe_select(t2d, fe_neg(t2d), neg));
  const fe D = fe_add(p.Z, p.Z);
  const fe E = fe_sub(B, A), F = fe_sub(D, C), G = fe_add(D, C), H = fe_add(B, A);
  ge r;
  r.X = fe_mul(E, F); r.Y = fe_mul(G, H); r.Z = fe_mul(F, G); r.T = fe_mul(E, H);
  return r;
}

// ---- quad-cooperative point operations ------------------------------------------------
// Four consecutive lanes of a warp (a quad) hold the same point and split the field
// multiplications of one group operation between them, then exchange the results by
// shuffles: a doubling costs the latency of 2 multiplications instead of 8, an addition
// 3 instead of 9.  Every lane of the warp must take part (full-mask shuffles); each quad
// works on its own point.
__device__ __forceinline__ fe fe_shfl(const fe& a, int src) {
  fe r;
#pragma unroll
  for (int i = 0; i < 8; ++i) r.v[i] = __shfl_sync(0xffffffffu, a.v[i], src);
  return r;
}

__device__ __forceinline__ ge ge_dbl_quad(const ge& p) {
  const int lane = threadIdx.x & 31, q = lane & 3, base = lane & ~3;
  fe in = fe_select(p.X, p.Y, q == 1);
  in = fe_select(in, p.Z, q == 2);
  in = fe_select(in, fe_add(p.X, p.Y), q == 3);
  const fe sq = fe_sq(in);
  const fe A = fe_shfl(sq, base), B = fe_shfl(sq, base + 1), Z2 = fe_shfl(sq, base + 2), S = fe_shfl(sq, base + 3);
  const fe C = fe_add(Z2, Z2);
  const fe E = fe_sub(fe_sub(S, A), B);
  const fe G = fe_sub(B, A);
  const fe F = fe_sub(G, C);
  const fe H = fe_neg(fe_add(A, B));
  // X3 = E F, Y3 = G H, Z3 = F G, T3 = E H
  fe m1 = fe_select(E, G, q == 1), m2 = fe_select(F, H, q == 1);
  m1 = fe_select(m1, F, q == 2); m2 = fe_select(m2, G, q == 2);
  m2 = fe_select(m2, H, q == 3);
  const fe r = fe_mul(m1, m2);
  ge o;
  o.X = fe_shfl(r, base); o.Y = fe_shfl(r, base + 1); o.Z = fe_shfl(r, base + 2); o.T = fe_shfl(r, base + 3);
  return o;
}

__device__ __forceinline__ ge ge_add_quad(const ge& p, const ge& qq) {
  const int lane = threadIdx.x & 31, q = lane & 3, base = lane & ~3;
  // phase 1: A = (Y1-X1)(Y2-X2), B = (Y1+X1)(Y2+X2), TT = T1 T2, ZZ = Z1 Z2
  fe a = fe_select(fe_sub(p.Y, p.X), fe_add(p.Y, p.X), q == 1);
  fe b = fe_select(fe_sub(qq.Y, qq.X), fe_add(qq.Y, qq.X), q == 1);
  a = fe_select(a, p.T, q == 2); b = fe_select(b, qq.T, q == 2);
  a = fe_select(a, p.Z, q == 3); b = fe_select(b, qq.Z, q == 3);
  fe r = fe_mul(a, b);
  // lane 2 turns T1 T2 into C = 2d T1 T2
  r = fe_select(r, fe_mul(r, fe_d2()), q == 2);
  const fe A = fe_shfl(r, base), B = fe_shfl(r, base + 1), C = fe_shfl(r, base + 2), ZZ = fe_shfl(r, base + 3);
  const fe D = fe_add(ZZ, ZZ);
  const fe E = fe_sub(B, A), F = fe_sub(D, C), G = fe_add(D, C), H = fe_add(B, A);
  fe m1 = fe_select(E, G, q == 1), m2 = fe_select(F, H, q == 1);
  m1 = fe_select(m1, F, q == 2); m2 = fe_select(m2, G, q == 2);
  m2 = fe_select(m2, H, q == 3);
  const fe s = fe_mul(m1, m2);
  ge o;
  o.X = fe_shfl(s, base); o.Y = fe_shfl(s, base + 1); o.Z = fe_shfl(s, base + 2); o.T = fe_shfl(s, base + 3);
  return o;
}

// Signed 4-bit recoding of a scalar below 2^253: 64 digits in [-8, 8), sum d_i 16^i = k.
__device__ __forceinline__ int sc_digit4(const uint32_t k[8], int w, int& carry) {
  int d = (int)((k[w >> 3] >> ((w & 7) * 4)) & 15u) + carry;
  carry = d >= 8 ? 1 : 0;
  return d - (carry << 4);
}

// Plain left-to-right double-and-add [k]P for a scalar of `bits` bits (used off the hot
// path: key generation, table construction, single-entry checks in tests).
__device__ __forceinline__ ge ge_scalarmult(const uint32_t k[8], const ge& P, int bits) {
  ge acc = ge_identity();
  for (int i = bits - 1; i >= 0; --i) {
    acc = ge_dbl(acc);
    const bool bit = (k[i >> 5] >> (i & 31)) & 1u;
    const ge s = ge_add(acc, P);
    acc = ge_select(acc, s, bit);
  }
  return acc;
}

}  // namespace poslo
