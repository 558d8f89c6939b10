// Distill / SeBVer at entry granularity (Fig. 3b semantics, Sec. 4.3): find every entry that
// fails its own check by recursively re-verifying subset aggregates on the device.
//
// The subsets are the nodes of a segment tree over the entries: node (l, k) aggregates
// entries [k 2^l, (k+1) 2^l) as (sum R_t, sum e_t mod q, sum s_t mod q).  A node is checked
// with the paper's aggregate equation [8](R - eY - sG) = O; the children of failing nodes
// form the next frontier, down to single entries.  Unit sums can hide a pair of invalid
// entries whose errors cancel, so the host confirms the rest of the batch with the weighted
// check afterwards and falls back to per-entry checks of everything when that fails.
#include "common.cuh"

namespace poslo {

__device__ __forceinline__ bool flagged(const uint8_t* a, const uint8_t* b, uint64_t t) {
  return (a && a[t]) || (b && b[t]);
}

__device__ __forceinline__ sc sc_load(const uint8_t* p) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
  const uint4 a = q[0], b = q[1];
  sc r;
  r.v[0] = a.x; r.v[1] = a.y; r.v[2] = a.z; r.v[3] = a.w; r.v[4] = b.x; r.v[5] = b.y; r.v[6] = b.z; r.v[7] = b.w;
  return r;
}

__device__ __forceinline__ void sc_store(uint8_t* p, const sc& r) {
  uint4* q = reinterpret_cast<uint4*>(p);
  q[0] = make_uint4(r.v[0], r.v[1], r.v[2], r.v[3]);
  q[1] = make_uint4(r.v[4], r.v[5], r.v[6], r.v[7]);
}

__device__ __forceinline__ sc sc_zero() {
  sc r;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.v[k] = 0;
  return r;
}

// Leaf t as (point, e, s); flagged or padding leaves are (O, 0, 0).
__device__ __forceinline__ void leaf(const TreeArgs& a, uint64_t t, ge& P, sc& e, sc& s) {
  if (t >= a.n || flagged(a.skip1, a.skip2, t)) {
    P = ge_identity();
    e = sc_zero();
    s = sc_zero();
    return;
  }
  fe t2d;
  pts_load(a.pts + (size_t)kPtsWords * t, P.X, P.Y, t2d);
  P.Z = fe_one();
  P.T = fe_mul(P.X, P.Y);
  e = sc_load(a.e + 32 * t);
  s = sc_load(a.s + 32 * t);
}

// Level 1 of the tree from the leaves.
__global__ void __launch_bounds__(128) k_tree_leaves(const TreeArgs a) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.M / 2) return;
  ge P0, P1;
  sc e0, e1, s0, s1;
  leaf(a, 2 * k, P0, e0, s0);
  leaf(a, 2 * k + 1, P1, e1, s1);
  ge_store(a.tree_pts + 32 * k, ge_add(P0, P1));
  sc_store(a.tree_e + 32 * k, sc_add(e0, e1));
  sc_store(a.tree_s + 32 * k, sc_add(s0, s1));
}

// Level l+1 from level l: node k = child 2k + child 2k+1.
__global__ void __launch_bounds__(128) k_tree_level(const TreeArgs a, uint64_t in_off, uint64_t out_off,
                                                    uint64_t count) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const uint64_t c0 = in_off + 2 * k, c1 = c0 + 1, o = out_off + k;
  ge_store(a.tree_pts + 32 * o, ge_add(ge_load(a.tree_pts + 32 * c0), ge_load(a.tree_pts + 32 * c1)));
  sc_store(a.tree_e + 32 * o, sc_add(sc_load(a.tree_e + 32 * c0), sc_load(a.tree_e + 32 * c1)));
  sc_store(a.tree_s + 32 * o, sc_add(sc_load(a.tree_s + 32 * c0), sc_load(a.tree_s + 32 * c1)));
}

// Signed 4-bit digit of window w (carry recomputed from the low windows).
__device__ __forceinline__ int digit_at(const uint32_t k[8], int w) {
  int carry = 0, d = 0;
  for (int i = 0; i <= w; ++i) d = sc_digit4(k, i, carry);
  return d;
}

// [8](P - eY - sG) = O evaluated by one warp: lane l adds the table terms of windows 2l and
// 2l+1, a shuffle tree sums the 32 partial points.  Every lane returns the same answer.
__device__ __forceinline__ bool warp_check(const ge& P, const sc& e, const sc& s, const uint32_t* tY,
                                           const uint32_t* tG) {
  const int lane = threadIdx.x & 31;
  const int w0 = 2 * lane, w1 = w0 + 1;
  ge acc = ge_add(table_pick(tY, w0, digit_at(e.v, w0)), table_pick(tY, w1, digit_at(e.v, w1)));
  acc = ge_add(acc, table_pick(tG, w0, digit_at(s.v, w0)));
  acc = ge_add(acc, table_pick(tG, w1, digit_at(s.v, w1)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ge other;
    other.X = fe_shfl(acc.X, lane ^ o); other.Y = fe_shfl(acc.Y, lane ^ o);
    other.Z = fe_shfl(acc.Z, lane ^ o); other.T = fe_shfl(acc.T, lane ^ o);
    acc = ge_add(acc, other);
  }
  return ge_is_identity(ge_mul_cofactor(ge_sub(P, acc)));
}

// One frontier level: each warp checks nodes of level `lvl`; failing nodes push their
// children (level lvl-1) to the next frontier, or their entries to the leaf frontier when
// lvl == 1.
__global__ void __launch_bounds__(128) k_bisect(const TreeArgs a, int lvl, uint64_t lvl_off, const uint64_t* front,
                                                const uint64_t* front_cnt, uint64_t* next, uint64_t* next_cnt,
                                                const uint32_t* tY, const uint32_t* tG) {
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t cnt = *front_cnt;
  for (uint64_t f = warp; f < cnt; f += nwarps) {
    const uint64_t k = front[f];
    const uint64_t node = lvl_off + k;
    const ge P = ge_load(a.tree_pts + 32 * node);
    const sc e = sc_load(a.tree_e + 32 * node), s = sc_load(a.tree_s + 32 * node);
    const bool ok = warp_check(P, e, s, tY, tG);
    if (!ok && (threadIdx.x & 31) == 0) {
      const uint64_t pos = atomicAdd(reinterpret_cast<unsigned long long*>(next_cnt), 2ull);
      next[pos] = 2 * k;
      next[pos + 1] = 2 * k + 1;
    }
  }
  (void)lvl;
}

// Leaf frontier: single-entry checks; failing entries are marked invalid.
__global__ void __launch_bounds__(128) k_bisect_leaves(const TreeArgs a, const uint64_t* front,
                                                       const uint64_t* front_cnt, const uint32_t* tY,
                                                       const uint32_t* tG, uint8_t* invalid) {
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t cnt = *front_cnt;
  for (uint64_t f = warp; f < cnt; f += nwarps) {
    const uint64_t t = front[f];
    ge P;
    sc e, s;
    leaf(a, t, P, e, s);
    const bool ok = warp_check(P, e, s, tY, tG);
    if (!ok && (threadIdx.x & 31) == 0 && t < a.n) invalid[t] = 1;
  }
}

// Weighted scalar sums sum z_t e_t, sum z_t s_t over the entries not flagged (same partial
// layout as k_hash).
__global__ void __launch_bounds__(kHashThreads) k_weighted_sums(const uint8_t* e, const uint8_t* s, const uint32_t* z,
                                                               const uint8_t* skip1, const uint8_t* skip2, uint64_t n,
                                                               unsigned long long* partial) {
  acc13 acc_e, acc_s;
  acc_zero(acc_e);
  acc_zero(acc_s);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    if (flagged(skip1, skip2, t)) continue;
    const uint4 zz = __ldg(reinterpret_cast<const uint4*>(z) + t);
    const uint32_t zw[4] = {zz.x, zz.y, zz.z, zz.w};
    const sc ev = sc_load(e + 32 * t), sv = sc_load(s + 32 * t);
    uint32_t p[12];
    mul_4x8(p, zw, ev.v);
    acc_add<12>(acc_e, p);
    mul_4x8(p, zw, sv.v);
    acc_add<12>(acc_s, p);
  }
  __shared__ unsigned long long red[kHashThreads / 32][kPartialWords];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kPartialWords; ++k) {
    unsigned long long v = k < 13 ? acc_e.v[k] : (k < 26 ? acc_s.v[k - 13] : 0ull);
    warp_sum_u64(v);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kPartialWords) {
    unsigned long long v = 0;
    for (int w = 0; w < kHashThreads / 32; ++w) v += red[w][threadIdx.x];
    partial[(uint64_t)blockIdx.x * kPartialWords + threadIdx.x] = v;
  }
}

// Unit sum of the stored points not flagged (partials in the k_points layout).
__global__ void __launch_bounds__(kPointThreads) k_pts_sum(const uint32_t* pts, const uint8_t* skip1,
                                                          const uint8_t* skip2, uint64_t n, uint32_t* partial) {
  ge acc = ge_identity();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    if (flagged(skip1, skip2, t)) continue;
    fe x, y, t2d;
    pts_load(pts + (size_t)kPtsWords * t, x, y, t2d);
    acc = ge_madd(acc, x, y, t2d);
  }
  __shared__ uint32_t sp[kPointThreads][32];
  ge_store(sp[threadIdx.x], acc);
  __syncthreads();
  for (int h = kPointThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) ge_store(sp[threadIdx.x], ge_add(ge_load(sp[threadIdx.x]), ge_load(sp[threadIdx.x + h])));
    __syncthreads();
  }
  if (threadIdx.x < 32) partial[(uint64_t)blockIdx.x * kPointPartialWords + threadIdx.x] = sp[0][threadIdx.x];
  if (threadIdx.x == 0) partial[(uint64_t)blockIdx.x * kPointPartialWords + 32] = 0;
}

// out[t] = a[t] | b[t] | c[t] (NULL arrays count as zero).
__global__ void k_flags_or(const uint8_t* a, const uint8_t* b, const uint8_t* c, uint64_t n, uint8_t* out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
    out[t] = (uint8_t)(((a && a[t]) || (b && b[t]) || (c && c[t])) ? 1 : 0);
}

}  // namespace poslo
