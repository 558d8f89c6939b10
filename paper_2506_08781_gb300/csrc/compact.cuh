// Point arithmetic for the single-block kernels that run once per call (the combined check of
// shard records, the finishing steps): their instructions are fetched from a cold instruction
// cache on every launch, so inlined copies of the field multiplication at every call site
// (tens of kilobytes of straight-line code) cost more than the arithmetic.  The same formulas
// as ge25519.cuh, built from one out-of-line copy of each field operation.
#pragma once
#include "ge25519.cuh"

namespace poslo {
namespace compact {

static __device__ __noinline__ fe mul(const fe& a, const fe& b) { return fe_mul(a, b); }
static __device__ __noinline__ fe sq(const fe& a) { return fe_sq(a); }
static __device__ __noinline__ fe canon(const fe& a) { return fe_canon(a); }

// Unified addition (add-2008-hwcd-3, a = -1, k = 2d), as ge_add.
static __device__ __noinline__ ge add(const ge& p, const ge& q) {
  const fe A = mul(fe_sub(p.Y, p.X), fe_sub(q.Y, q.X));
  const fe B = mul(fe_add(p.Y, p.X), fe_add(q.Y, q.X));
  const fe C = mul(mul(p.T, fe_d2()), q.T);
  const fe Zp = mul(p.Z, q.Z);
  const fe D = fe_add(Zp, Zp);
  const fe E = fe_sub(B, A), F = fe_sub(D, C), G = fe_add(D, C), H = fe_add(B, A);
  ge r;
  r.X = mul(E, F);
  r.Y = mul(G, H);
  r.Z = mul(F, G);
  r.T = mul(E, H);
  return r;
}

// Doubling (dbl-2008-hwcd, a = -1), as ge_dbl.
static __device__ __noinline__ ge dbl(const ge& p) {
  const fe A = sq(p.X);
  const fe B = sq(p.Y);
  const fe Z2 = sq(p.Z);
  const fe C = fe_add(Z2, Z2);
  const fe E = fe_sub(fe_sub(sq(fe_add(p.X, p.Y)), A), B);
  const fe G = fe_sub(B, A);
  const fe F = fe_sub(G, C);
  const fe H = fe_neg(fe_add(A, B));
  ge r;
  r.X = mul(E, F);
  r.Y = mul(G, H);
  r.Z = mul(F, G);
  r.T = mul(E, H);
  return r;
}

static __device__ __forceinline__ ge sub(const ge& p, const ge& q) { return add(p, ge_neg(q)); }

static __device__ __noinline__ fe sqn(fe a, int n) {
#pragma unroll 1
  for (int i = 0; i < n; ++i) a = sq(a);
  return a;
}

// z^(p-2), Fermat's inverse (0 -> 0), by the addition chain of fe_inv.
static __device__ __noinline__ fe inv(const fe& z) {
  const fe z2 = sq(z);
  const fe z9 = mul(sqn(z2, 2), z);
  const fe z11 = mul(z9, z2);
  const fe z_5 = mul(sq(z11), z9);                 // 2^5 - 1
  const fe z_10 = mul(sqn(z_5, 5), z_5);           // 2^10 - 1
  const fe z_20 = mul(sqn(z_10, 10), z_10);        // 2^20 - 1
  const fe z_40 = mul(sqn(z_20, 20), z_20);        // 2^40 - 1
  const fe z_50 = mul(sqn(z_40, 10), z_10);        // 2^50 - 1
  const fe z_100 = mul(sqn(z_50, 50), z_50);       // 2^100 - 1
  const fe z_200 = mul(sqn(z_100, 100), z_100);    // 2^200 - 1
  const fe z_250 = mul(sqn(z_200, 50), z_50);      // 2^250 - 1
  return mul(sqn(z_250, 5), z11);
}

// The compressed encoding (y with the parity of x in bit 255), as ge_encode.
static __device__ __noinline__ void encode(const ge& p, uint32_t b[8]) {
  const fe zi = inv(p.Z);
  const fe x = canon(mul(p.X, zi));
  const fe y = canon(mul(p.Y, zi));
#pragma unroll
  for (int i = 0; i < 8; ++i) b[i] = y.v[i];
  b[7] |= (x.v[0] & 1u) << 31;
}

static __device__ __forceinline__ ge mul_cofactor(ge p) {
#pragma unroll 1
  for (int i = 0; i < 3; ++i) p = dbl(p);
  return p;
}

// The sum of the 128 points terms[0..127] (32 words each, in shared memory) by a block of
// 128 threads: quad q adds terms 4q .. 4q + 3 (quad-cooperative additions), then a tree over
// the 32 quads' sums in qs; the sum ends in qs[0].  Every thread calls it (full-mask
// shuffles, barriers inside); the caller has stored the terms and synchronised.
__device__ __forceinline__ void quad_sum128(uint32_t (*terms)[32], uint32_t (*qs)[32]) {
  constexpr int kQuads = 32;
  const int tid = threadIdx.x, quad = tid >> 2;
  ge acc = ge_identity();
#pragma unroll 1
  for (int k = 0; k < 4; ++k) acc = ge_add_quad(acc, ge_load(terms[4 * quad + k]));
  if ((tid & 3) == 0) ge_store(qs[quad], acc);
  __syncthreads();
#pragma unroll 1
  for (int h = kQuads / 2; h > 0; h >>= 1) {
    const ge sum = ge_add_quad(ge_load(qs[quad]), ge_load(qs[(quad + h) % kQuads]));
    __syncthreads();
    if ((tid & 3) == 0 && quad < h) ge_store(qs[quad], sum);
    __syncthreads();
  }
}

}  // namespace compact
}  // namespace poslo
