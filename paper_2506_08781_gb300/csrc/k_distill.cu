// Distill / SeBVer at entry granularity (Fig. 3b semantics, Sec. 4.3): find every entry that
// fails its own check by recursively re-verifying subset aggregates on the device.
//
// The subsets are the nodes of a segment tree over the entries: node (l, k) aggregates
// entries [k 2^l, (k+1) 2^l) as (sum R_t, sum e_t mod q, sum s_t mod q).  A node is checked
// with the paper's aggregate equation [8](R - eY - sG) = O; the descendants of failing nodes
// (one or several levels down) are checked next, down to single entries.  Unit sums can hide a pair of invalid
// entries whose errors cancel, so the host confirms the rest of the batch with the weighted
// check afterwards and falls back to per-entry checks of everything when that fails.
#include "common.cuh"
#include "compact.cuh"

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

// Lane l's two signed 4-bit digits (windows 2l and 2l+1) of the recoding of sc_digit4, with
// the carries of the lower windows from a warp scan instead of a walk over them: a window
// generates a carry when its nibble is 8 or more and propagates the incoming one when it is
// 7, so the carry into lane l is the scan of (generate, propagate) over lanes 0 .. l-1.
__device__ __forceinline__ void lane_digits(const uint32_t k[8], int lane, int& d0, int& d1) {
  uint32_t word = 0;                                         // windows 2l, 2l+1 = byte (l & 3) of word l / 4
#pragma unroll
  for (int i = 0; i < 8; ++i) word = i == (lane >> 2) ? k[i] : word;   // (no dynamic register index)
  const int n0 = (int)((word >> (8 * (lane & 3))) & 15u), n1 = (int)((word >> (8 * (lane & 3) + 4)) & 15u);
  uint32_t G = (n1 >= 8) | ((n1 == 7) & (n0 >= 8)), P = (n1 == 7) & (n0 == 7);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t Gp = __shfl_up_sync(0xffffffffu, G, o), Pp = __shfl_up_sync(0xffffffffu, P, o);
    if (lane >= o) {
      G = G | (P & Gp);
      P = P & Pp;
    }
  }
  const uint32_t up = __shfl_up_sync(0xffffffffu, G, 1);
  int carry = lane ? (int)up : 0;
  d0 = n0 + carry;
  carry = d0 >= 8 ? 1 : 0;
  d0 -= carry << 4;
  d1 = n1 + carry;
  d1 -= (d1 >= 8 ? 1 : 0) << 4;
}

// [8](P - eY - sG) = O evaluated by one warp: lane l adds the table terms of windows 2l and
// 2l+1, a shuffle tree sums the 32 partial points.  Every lane returns the same answer.
__device__ __forceinline__ bool warp_check(const ge& P, const sc& e, const sc& s, const uint32_t* tY,
                                           const uint32_t* tG) {
  const int lane = threadIdx.x & 31;
  const int w0 = 2 * lane, w1 = w0 + 1;
  int de0, de1, ds0, ds1;
  lane_digits(e.v, lane, de0, de1);
  lane_digits(s.v, lane, ds0, ds1);
  ge acc = ge_add(table_pick(tY, w0, de0), table_pick(tY, w1, de1));
  acc = ge_add(acc, table_pick(tG, w0, ds0));
  acc = ge_add(acc, table_pick(tG, w1, ds1));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ge other;
    other.X = fe_shfl(acc.X, lane ^ o); other.Y = fe_shfl(acc.Y, lane ^ o);
    other.Z = fe_shfl(acc.Z, lane ^ o); other.T = fe_shfl(acc.T, lane ^ o);
    acc = ge_add(acc, other);
  }
  return ge_is_identity(ge_mul_cofactor(ge_sub(P, acc)));
}

// [8](P - eY - sG) = O evaluated by a group of 8 lanes (lanes 8g .. 8g+7 of the warp hold the
// same P, e, s; four groups check four nodes at once).  Lane r of the group takes word r of
// each scalar, i.e. the 8 windows 8r .. 8r+7: it recodes them into signed 4-bit digits (the
// carry into its first window from a scan over the group's lower lanes, as in lane_digits),
// adds their 16 table terms, and a shuffle tree over the group sums the 8 partial points.
// Fewer lanes per check than warp_check, so fewer instructions per check: each lane's chain is
// longer (15 additions instead of 3), but the work of the tree and of the final check is shared
// by 8 lanes instead of 32.  Every lane of the group returns the same answer.
__device__ __forceinline__ void group8_digits(uint32_t word, int r, int8_t d[8]) {
  uint32_t G = 0, Pp = 1;   // carry out of this lane's 8 windows with no carry in; all-7 propagate
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t n = (word >> (4 * i)) & 15u;
    G = (n >= 8) | ((n == 7) & G);
    Pp &= (n == 7);
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) {
    const uint32_t Gu = __shfl_up_sync(0xffffffffu, G, o, 8), Pu = __shfl_up_sync(0xffffffffu, Pp, o, 8);
    if (r >= o) {
      G = G | (Pp & Gu);
      Pp = Pp & Pu;
    }
  }
  const uint32_t up = __shfl_up_sync(0xffffffffu, G, 1, 8);
  int carry = r ? (int)up : 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int v = (int)((word >> (4 * i)) & 15u) + carry;
    carry = v >= 8 ? 1 : 0;
    d[i] = (int8_t)(v - (carry << 4));
  }
}

__device__ __forceinline__ bool group8_check(const ge& P, const sc& e, const sc& s, const uint32_t* tY,
                                             const uint32_t* tG) {
  const int lane = threadIdx.x & 31, r = lane & 7;
  uint32_t we = 0, ws = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {   // word r of each scalar (no dynamic register index)
    we = i == r ? e.v[i] : we;
    ws = i == r ? s.v[i] : ws;
  }
  int8_t dg[16];   // the 8 digits of e, then the 8 of s
  group8_digits(we, r, dg);
  group8_digits(ws, r, dg + 8);
  // loops, not unrolled: one copy of the point addition in the code keeps the kernel inside
  // the instruction cache (unrolled, the warps stalled mostly on instruction fetch)
  ge acc = ge_identity();
#pragma unroll 1
  for (int i = 0; i < 16; ++i) acc = ge_add(acc, table_pick(i < 8 ? tY : tG, 8 * r + (i & 7), dg[i]));
#pragma unroll 1
  for (int o = 4; o > 0; o >>= 1) {
    ge other;
    other.X = fe_shfl(acc.X, lane ^ o); other.Y = fe_shfl(acc.Y, lane ^ o);
    other.Z = fe_shfl(acc.Z, lane ^ o); other.T = fe_shfl(acc.T, lane ^ o);
    acc = ge_add(acc, other);
  }
  return ge_is_identity(ge_mul_cofactor(ge_sub(P, acc)));
}

// One step of the descent, several levels at a time.  The step reads the failing nodes of
// level l (state.fail[s % 3], count state.cnt[s % 3], level state.level[s % 2]) and checks
// their descendants j levels further down, j the largest depth for which all of them fit in
// one pass of the grid's check slots (4 per warp; at least 1, at most l): with few failing nodes a step jumps
// many levels, with many it descends one.  Failing descendants go to the next list
// (state.fail[(s+1) % 3]); at level 0 the descendants are entries, checked on their own, and
// failing ones are marked invalid.  Each step also clears the counter the step after it will
// fill, and block 0 publishes the level it reached; a step that starts at level 0 (done)
// returns at once, so the host issues as many steps as the tree has levels without reading
// anything back.  Checking the descendants of a failing node directly, instead of its
// children first, only adds checks of nodes whose ancestors failed: every entry that fails
// its own check is still found, and entries are flagged only by their own check.
__global__ void __launch_bounds__(128, POSLO_BISECT_MINB) k_bisect_step(const TreeArgs a, BisectState st, int step,
                                                     const uint32_t* tY, const uint32_t* tG, uint8_t* invalid) {
  const int l = st.level[step & 1];
  const uint64_t* fail_in = st.fail[step % 3];
  uint64_t* fail_out = st.fail[(step + 1) % 3];
  unsigned long long* cnt_out = reinterpret_cast<unsigned long long*>(st.cnt + (step + 1) % 3);
  if (blockIdx.x == 0 && threadIdx.x == 0) st.cnt[(step + 2) % 3] = 0;
  if (l <= 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st.level[(step + 1) & 1] = l;
    return;
  }
  const uint64_t F = st.cnt[step % 3];
  // four checks per warp (one per group of 8 lanes)
  const uint64_t slots = ((uint64_t)gridDim.x * blockDim.x) >> 3;
  int j = 1;
  while (j < l && (F << (j + 1)) <= slots) ++j;
  const int tl = l - j;
  if (blockIdx.x == 0 && threadIdx.x == 0) st.level[(step + 1) & 1] = tl;
  const uint64_t total = F << j;
  const uint64_t mask = (1ull << j) - 1;
  // the loop runs the same number of times for all lanes of a warp (the check shuffles across
  // the warp); a group past the end checks the identity and records nothing
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t grp = (threadIdx.x & 31) >> 3;
  for (uint64_t w0 = 4 * warp; w0 < total; w0 += 4 * nwarps) {
    const uint64_t w = w0 + grp;
    const bool live = w < total;
    const uint64_t k = live ? ((fail_in[w >> j] << j) | (w & mask)) : 0;
    ge P = ge_identity();
    sc e = sc_zero(), s = sc_zero();
    if (live) {
      if (tl > 0) {
        const uint64_t node = a.M - (a.M >> (tl - 1)) + k;   // levels 1 .. tl-1 hold M/2 + ... + M/2^(tl-1) nodes
        P = ge_load(a.tree_pts + 32 * node);
        e = sc_load(a.tree_e + 32 * node);
        s = sc_load(a.tree_s + 32 * node);
      } else {
        leaf(a, k, P, e, s);
      }
    }
    const bool ok = group8_check(P, e, s, tY, tG);
    if (live && !ok && (threadIdx.x & 7) == 0) {
      if (tl > 0) fail_out[atomicAdd(cnt_out, 1ull)] = k;
      else if (k < a.n) invalid[k] = 1;
    }
  }
}

// The flagged entries' rows for the MSM of the confirmation: decoded point (kPtsWords words),
// weight z_t (4 words) and "point did not decode" (the MSM leaves those out), at the local
// indices idx[0 .. cnt).
__global__ void k_gather_flagged(const uint32_t* pts, const uint32_t* z, const uint8_t* badR, const uint64_t* idx,
                                 uint64_t cnt, uint32_t* gp, uint32_t* gz, uint8_t* gs) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const uint64_t k = idx[t];
  const uint4* src = reinterpret_cast<const uint4*>(pts + (size_t)kPtsWords * k);
  uint4* dst = reinterpret_cast<uint4*>(gp + (size_t)kPtsWords * t);
#pragma unroll
  for (int i = 0; i < kPtsWords / 4; ++i) dst[i] = src[i];
  reinterpret_cast<uint4*>(gz)[t] = reinterpret_cast<const uint4*>(z)[k];
  gs[t] = badR ? badR[k] : 0;
}

// ccd^v's point: the batch's unit sum of its decodable R_t (unit, 32 words) minus the flagged
// entries' decodable R_t (local indices idx[0 .. *nf_dev), the count left in device memory by
// the compaction), encoded to enc_out (32 bytes).  One block: the flagged points are few next
// to the batch.
__global__ void __launch_bounds__(256) k_ccd_points(const uint32_t* pts, const uint8_t* badR, const uint64_t* idx,
                                                    const uint64_t* nf_dev, const uint32_t* unit, uint8_t* enc_out) {
  __shared__ uint32_t sp[256][32];
  ge acc = ge_identity();
  const uint64_t nf = *nf_dev;
  for (uint64_t i = threadIdx.x; i < nf; i += blockDim.x) {
    const uint64_t t = idx[i];
    if (badR && badR[t]) continue;
    fe x, y, t2d;
    pts_load(pts + (size_t)kPtsWords * t, x, y, t2d);
    acc = ge_madd(acc, x, y, t2d);
  }
  ge_store(sp[threadIdx.x], acc);
  __syncthreads();
  // once per call: compact (out-of-line) point operations, the code being fetched cold
#pragma unroll 1
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) ge_store(sp[threadIdx.x], compact::add(ge_load(sp[threadIdx.x]), ge_load(sp[threadIdx.x + h])));
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    uint32_t w[8];
    compact::encode(compact::sub(ge_load(unit), ge_load(sp[0])), w);
    for (int k = 0; k < 8; ++k) {
      enc_out[4 * k] = (uint8_t)w[k]; enc_out[4 * k + 1] = (uint8_t)(w[k] >> 8);
      enc_out[4 * k + 2] = (uint8_t)(w[k] >> 16); enc_out[4 * k + 3] = (uint8_t)(w[k] >> 24);
    }
  }
}

// out = a - b (b = nullptr: out = a), extended points of 32 words.
__global__ void k_point_diff(const uint32_t* a, const uint32_t* b, uint32_t* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ge_store(out, b ? ge_sub(ge_load(a), ge_load(b)) : ge_load(a));
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

// out[t] = a[t] | b[t] | c[t] (NULL arrays count as zero).
__global__ void k_flags_or(const uint8_t* a, const uint8_t* b, const uint8_t* c, uint64_t n, uint8_t* out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
    out[t] = (uint8_t)(((a && a[t]) || (b && b[t]) || (c && c[t])) ? 1 : 0);
}

}  // namespace poslo
