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

static __device__ __forceinline__ ge mul_cofactor(ge p) {
#pragma unroll 1
  for (int i = 0; i < 3; ++i) p = dbl(p);
  return p;
}

}  // namespace compact
}  // namespace poslo
