// Pippenger bucket multi-scalar multiplication sum_t [z_t] P_t (128- or 256-bit scalars) for the
// weighted aggregate check: the verifier's random linear combination of the entries'
// equations R_t = e_t Y + s_t G (an extension of AVer, Fig. 4; the paper aggregates with
// unit coefficients only).
#include "common.cuh"

namespace poslo {

// Counting sort, pass 1: rank of every (window, entry) inside its bucket.
__global__ void k_msm_count(const uint32_t* z, const uint8_t* skip, uint64_t n, MsmPlan pl, uint32_t* cnt,
                            uint32_t* rank) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    if (skip && skip[t]) continue;
    uint32_t zw[8];
    z_load(z, pl.sw, t, zw);
    uint32_t carry = 0;
    bool neg;
    for (int w = 0; w < pl.windows; ++w) {
      const uint32_t d = z_sdigit(zw, pl.sw, w, pl.c, carry, neg);
      if (d) rank[(size_t)w * n + t] = atomicAdd(&cnt[(size_t)w * pl.nb + d], 1u);
    }
  }
}

// Counting sort, pass 2: exclusive scan of the bucket counts, one block per window.
__global__ void __launch_bounds__(1024) k_msm_scan(const uint32_t* cnt, uint32_t* off, MsmPlan pl) {
  __shared__ uint32_t warp_sums[32];
  const int w = blockIdx.x;
  const uint32_t per = (pl.nb + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = threadIdx.x * per;
  const uint32_t* c = cnt + (size_t)w * pl.nb;
  uint32_t local = 0;
  for (uint32_t d = lo; d < lo + per && d < pl.nb; ++d) local += c[d];
  // block-wide exclusive scan of `local`
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    warp_sums[lane] = v;   // inclusive over warps
  }
  __syncthreads();
  uint32_t base = (incl - local) + (warp > 0 ? warp_sums[warp - 1] : 0u);
  uint32_t* o = off + (size_t)w * pl.nb;
  for (uint32_t d = lo; d < lo + per && d < pl.nb; ++d) {
    o[d] = base;
    base += c[d];
  }
}

// Counting sort, pass 3: entry indices in bucket order, per window.
__global__ void k_msm_scatter(const uint32_t* z, const uint8_t* skip, uint64_t n, MsmPlan pl, const uint32_t* off,
                              const uint32_t* rank, uint32_t* idx, uint16_t* bkt) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    if (skip && skip[t]) continue;
    uint32_t zw[8];
    z_load(z, pl.sw, t, zw);
    uint32_t carry = 0;
    bool neg;
    for (int w = 0; w < pl.windows; ++w) {
      const uint32_t d = z_sdigit(zw, pl.sw, w, pl.c, carry, neg);
      if (d) {
        const size_t pos = (size_t)w * n + off[(size_t)w * pl.nb + d] + rank[(size_t)w * n + t];
        idx[pos] = (uint32_t)t;
        bkt[pos] = (uint16_t)((d - 1u) | (neg ? kBktNeg : 0u));
      }
    }
  }
}

// Bucket sums B_{w,d} = sum of sign(digit) P_t over the entries whose digit in window w has
// magnitude d, load-balanced: thread (w, tau) adds exactly the S = 2^seg_log2 sorted entries
// at positions [tau S, (tau+1) S) of window w (range tau), cutting its run wherever the
// bucket changes.  A bucket lying strictly inside the range is written directly; the first
// run goes to A[w][tau], the last (when different) to B[w][tau], and k_msm_combine joins
// the pieces of buckets that cross range boundaries.
__global__ void __launch_bounds__(128, POSLO_ACCUM_MINB) k_msm_accum(const uint32_t* pts, const uint32_t* idx, const uint16_t* bkt,
                                                   const uint32_t* off, const uint32_t* cnt, uint64_t n, MsmPlan pl,
                                                   const uint8_t* skip, uint32_t* buckets, uint32_t* A, uint32_t* B) {
  const uint64_t seg = 1ull << pl.seg_log2;
  const uint64_t nseg = (n + seg - 1) >> pl.seg_log2;
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (uint64_t)pl.windows * nseg) return;
  const uint32_t w = (uint32_t)(g / nseg);
  const uint64_t tau = g % nseg;
  const size_t last = (size_t)w * pl.nb + pl.nb - 1;
  const uint64_t nnz = (uint64_t)off[last] + cnt[last];
  const uint64_t p0 = tau << pl.seg_log2;
  if (p0 >= nnz) return;
  const uint64_t p1 = min(p0 + seg, nnz);
  const uint32_t* li = idx + (size_t)w * n;
  const uint16_t* lb = bkt + (size_t)w * n;
  // Entry p's bucket code, point and skip flag are fetched during entry p - 1's addition: the
  // point and the flag are gathers at a random index, whose latency the addition hides.
  uint32_t code = lb[p0];
  uint32_t cur = code & kBktMask;
  bool first = true;
  ge acc = ge_identity();
  fe x, y, t2d;
  const uint32_t t0 = __ldg(li + p0);
  pts_load(pts + (size_t)kPtsWords * t0, x, y, t2d);
  bool skip_c = skip && skip[t0];
  for (uint64_t p = p0; p < p1; ++p) {
    const uint32_t d = code & kBktMask;
    if (d != cur) {
      uint32_t* dst = first ? A + 32 * g : buckets + 32 * ((size_t)w * pl.nb + cur + 1);
      ge_store(dst, acc);
      first = false;
      acc = ge_identity();
      cur = d;
    }
    fe nx = x, ny = y, nt = t2d;
    uint32_t ncode = code;
    bool nskip = skip_c;
    if (p + 1 < p1) {
      const uint32_t tn = __ldg(li + p + 1);
      ncode = lb[p + 1];
      pts_load(pts + (size_t)kPtsWords * tn, nx, ny, nt);
      nskip = skip && __ldg(skip + tn);
    }
    // entries whose point did not decode are sorted but never added
    if (!skip_c) acc = ge_madd_signed(acc, x, y, t2d, (code & kBktNeg) != 0);
    x = nx; y = ny; t2d = nt;
    code = ncode;
    skip_c = nskip;
  }
  ge_store(first ? A + 32 * g : B + 32 * g, acc);
}

// Buckets that were not written whole by k_msm_accum: the run in the range holding the
// bucket's first entry (A or B of that range) plus the first runs of the following ranges.
// Buckets spanning more than kCombineSpan ranges (a narrow window can put thousands of
// entries into one digit) are listed for k_msm_combine_big instead of summed here.
constexpr uint64_t kCombineSpan = 8;

struct CombineSpan {
  uint64_t ts, te;       // first and last range of the bucket
  bool starts_range;     // the first run is range ts's A (else its B)
  bool whole;            // strictly inside one range: k_msm_accum wrote it
};

__device__ __forceinline__ CombineSpan combine_span(const uint32_t* off, const uint32_t* cnt, const MsmPlan& pl,
                                                    uint64_t b) {
  const uint32_t w = (uint32_t)(b / pl.nb);
  const size_t last = (size_t)w * pl.nb + pl.nb - 1;
  const uint64_t nnz = (uint64_t)off[last] + cnt[last];
  const uint64_t s = off[b], e = s + cnt[b] - 1;
  CombineSpan c;
  c.ts = s >> pl.seg_log2;
  c.te = e >> pl.seg_log2;
  const uint64_t r_end = min((c.ts + 1) << pl.seg_log2, nnz) - 1;   // last position of range ts
  c.starts_range = s == c.ts << pl.seg_log2;
  c.whole = !c.starts_range && e < r_end;
  return c;
}

__global__ void __launch_bounds__(128) k_msm_combine(const uint32_t* off, const uint32_t* cnt, uint64_t n, MsmPlan pl,
                                                     const uint32_t* A, const uint32_t* B, uint32_t* buckets,
                                                     uint32_t* big_list, uint32_t* big_count) {
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= (uint64_t)pl.windows * pl.nb) return;
  const uint32_t w = (uint32_t)(b / pl.nb), d = (uint32_t)(b % pl.nb);
  const uint32_t len = d ? cnt[b] : 0u;
  if (len == 0) {
    ge_store(buckets + 32 * b, ge_identity());
    return;
  }
  const CombineSpan c = combine_span(off, cnt, pl, b);
  if (c.whole) return;
  if (c.te - c.ts > kCombineSpan) {
    big_list[atomicAdd(big_count, 1u)] = (uint32_t)b;
    return;
  }
  const uint64_t g0 = (uint64_t)w * ((n + (1ull << pl.seg_log2) - 1) >> pl.seg_log2);
  ge acc = ge_load((c.starts_range ? A : B) + 32 * (g0 + c.ts));
  for (uint64_t t = c.ts + 1; t <= c.te; ++t) acc = ge_add(acc, ge_load(A + 32 * (g0 + t)));
  ge_store(buckets + 32 * b, acc);
}

__device__ __forceinline__ ge ge_shfl_down(const ge& p, int delta) {
  ge r;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    r.X.v[i] = __shfl_down_sync(0xffffffffu, p.X.v[i], delta);
    r.Y.v[i] = __shfl_down_sync(0xffffffffu, p.Y.v[i], delta);
    r.Z.v[i] = __shfl_down_sync(0xffffffffu, p.Z.v[i], delta);
    r.T.v[i] = __shfl_down_sync(0xffffffffu, p.T.v[i], delta);
  }
  return r;
}

// The listed wide buckets, one warp each: the lanes sum the ranges' first runs with a
// stride of 32 (lane 0 starting from the bucket's first run), and a shuffle tree joins the
// lanes.  The grid is fixed; warps stride over the list (the trip count is uniform across a
// warp, so every lane takes part in every shuffle).
__global__ void __launch_bounds__(kCombineBigThreads) k_msm_combine_big(const uint32_t* off, const uint32_t* cnt,
                                                                        uint64_t n, MsmPlan pl, const uint32_t* A,
                                                                        const uint32_t* B, uint32_t* buckets,
                                                                        const uint32_t* big_list,
                                                                        const uint32_t* big_count) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warp = ((uint32_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = ((uint32_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t total = *big_count;
  const uint64_t nseg = (n + (1ull << pl.seg_log2) - 1) >> pl.seg_log2;
  for (uint32_t i = warp; i < total; i += nwarps) {
    const uint64_t b = big_list[i];
    const uint32_t w = (uint32_t)(b / pl.nb);
    const CombineSpan c = combine_span(off, cnt, pl, b);
    const uint64_t g0 = (uint64_t)w * nseg;
    ge acc = lane == 0 ? ge_load((c.starts_range ? A : B) + 32 * (g0 + c.ts)) : ge_identity();
    for (uint64_t t = c.ts + 1 + lane; t <= c.te; t += 32) acc = ge_add(acc, ge_load(A + 32 * (g0 + t)));
    for (int delta = 16; delta > 0; delta >>= 1) acc = ge_add(acc, ge_shfl_down(acc, delta));
    if (lane == 0) ge_store(buckets + 32 * b, acc);
  }
}

// Chunk j of window w holds buckets d = 16j .. 16j+15: L = sum_r r B_{16j+r} by running
// sums, T = sum_r B_{16j+r}.  One quad of lanes per chunk (quad-cooperative additions: the
// 31 dependent additions are latency-bound).
__global__ void __launch_bounds__(128) k_msm_chunk(const uint32_t* buckets, MsmPlan pl, uint32_t* L, uint32_t* T) {
  const uint64_t total = (uint64_t)pl.windows * pl.nchunks;
  const uint64_t quad = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const uint64_t g = quad < total ? quad : total - 1;   // surplus quads repeat the last chunk
  const uint32_t w = (uint32_t)(g / pl.nchunks), j = (uint32_t)(g % pl.nchunks);
  const uint32_t* B = buckets + 32 * ((size_t)w * pl.nb + (size_t)j * kMsmChunk);
  ge run = ge_identity(), acc = ge_identity();
  for (int r = kMsmChunk - 1; r >= 1; --r) {
    run = ge_add_quad(run, ge_load(B + 32 * r));
    acc = ge_add_quad(acc, run);
  }
  run = ge_add_quad(run, ge_load(B));
  if ((threadIdx.x & 3) == 0 && quad < total) {
    ge_store(L + 32 * g, acc);
    ge_store(T + 32 * g, run);
  }
}

// Narrow windows (c <= 8, the plans of batches of a few thousand entries): the window sum
// W_w = sum_d d B_d directly, one block per window and one quad per bucket d = 1 .. 2^(c-1):
// d B_d by double-and-add over c bits (the same c steps for every quad, the addition taken or
// not by a select: quad operations need every lane of the warp), then a tree over the
// buckets.  W_w goes to group 0 of window w and O to its other groups, which the window
// kernels read as G_0 + 16 sum_k 2^k G_{1+k} = W_w.  It replaces the running sums over chunks
// and the group sums, whose chains of dependent additions set the latency at these sizes.
__global__ void __launch_bounds__(512) k_msm_direct_groups(const uint32_t* buckets, MsmPlan pl, uint32_t* groups) {
  extern __shared__ uint32_t sp[];   // one point (32 words) per quad
  const int w = blockIdx.x;
  const int quad = threadIdx.x >> 2, nq = blockDim.x >> 2;   // nq = 2^(c-1)
  const uint32_t d = (uint32_t)quad + 1;
  const ge B = ge_load(buckets + 32 * ((size_t)w * pl.nb + d));
  ge acc = ge_identity();
#pragma unroll 1
  for (int bit = pl.c - 1; bit >= 0; --bit) {
    acc = ge_dbl_quad(acc);
    const ge sum = ge_add_quad(acc, B);
    acc = ge_select(acc, sum, ((d >> bit) & 1u) != 0);
  }
  if ((threadIdx.x & 3) == 0) ge_store(sp + 32 * quad, acc);
  __syncthreads();
#pragma unroll 1
  for (int h = nq / 2; h > 0; h >>= 1) {
    const ge sum = ge_add_quad(ge_load(sp + 32 * quad), ge_load(sp + 32 * ((quad + h) % nq)));
    __syncthreads();
    if ((threadIdx.x & 3) == 0 && quad < h) ge_store(sp + 32 * quad, sum);
    __syncthreads();
  }
  const int ng = 1 + pl.jbits;
  uint32_t* G = groups + 32 * (size_t)w * ng;
  for (int i = threadIdx.x; i < 32 * ng; i += blockDim.x) {
    const int g = i >> 5, k = i & 31;
    uint32_t v;
    if (g == 0) {
      v = sp[k];
    } else {   // the identity (0 : 1 : 1 : 0), word k of the extended point
      v = (k == 8 || k == 16) ? 1u : 0u;
    }
    G[i] = v;
  }
}

// Group sums per window: group 0 = sum_j L_j; group 1+k = sum of T_j over chunks j whose
// bit k is set.  One block of 256 quads per (window, group); every quad takes part in every
// addition of the tree (quad operations need all lanes), only the surviving half keeps it.
constexpr int kGroupThreads = 512;
__global__ void __launch_bounds__(512) k_msm_groups(const uint32_t* L, const uint32_t* T, MsmPlan pl,
                                                     uint32_t* groups) {
  const int ng = 1 + pl.jbits;
  const int w = blockIdx.x / ng, grp = blockIdx.x % ng;
  const uint32_t* base = (grp == 0 ? L : T) + 32 * (size_t)w * pl.nchunks;
  const int quad = threadIdx.x >> 2, nq = kGroupThreads / 4;
  ge acc = ge_identity();
  for (uint32_t j0 = 0; j0 < pl.nchunks; j0 += nq) {
    const uint32_t j = j0 + quad;
    const bool take = j < pl.nchunks && (grp == 0 || ((j >> (grp - 1)) & 1u));
    const ge p = take ? ge_load(base + 32 * (size_t)j) : ge_identity();
    acc = ge_add_quad(acc, p);
  }
  __shared__ uint32_t sp[kGroupThreads / 4][32];
  if ((threadIdx.x & 3) == 0) ge_store(sp[quad], acc);
  __syncthreads();
  for (int h = nq / 2; h > 0; h >>= 1) {
    const ge other = ge_load(sp[(quad + h) % nq]);
    const ge sum = ge_add_quad(ge_load(sp[quad]), other);
    __syncthreads();
    if ((threadIdx.x & 3) == 0 && quad < h) ge_store(sp[quad], sum);
    __syncthreads();
  }
  if (threadIdx.x < 32) groups[32 * (size_t)blockIdx.x + threadIdx.x] = sp[0][threadIdx.x];
}

// Window sums W_w = G_0 + 16 sum_k 2^k G_{1+k} (quad w computes window w), then
// sum_w 2^{c w} W_w by Horner's rule in quad 0.  One warp; windows are processed in rounds
// of eight quads.
__global__ void __launch_bounds__(32) k_msm_final(const uint32_t* groups, MsmPlan pl, uint32_t* out) {
  __shared__ uint32_t wsum[kMsmMaxWindows][32];
  const int lane = threadIdx.x & 31, quad = lane >> 2;
  const int ng = 1 + pl.jbits;
  for (int r0 = 0; r0 < pl.windows; r0 += 8) {
    const int w = r0 + quad;
    const int wc = w < pl.windows ? w : pl.windows - 1;
    const uint32_t* G = groups + 32 * (size_t)wc * ng;
    ge acc = ge_load(G + 32 * pl.jbits);       // top bit group
    for (int k = pl.jbits - 2; k >= 0; --k) acc = ge_add_quad(ge_dbl_quad(acc), ge_load(G + 32 * (1 + k)));
    for (int s = 0; s < 4; ++s) acc = ge_dbl_quad(acc);   // times kMsmChunk = 16
    acc = ge_add_quad(acc, ge_load(G));
    if ((lane & 3) == 0 && w < pl.windows) ge_store(wsum[w], acc);
    __syncwarp();
  }
  ge acc = ge_load(wsum[pl.windows - 1]);
  for (int w = pl.windows - 2; w >= 0; --w) {
    for (int s = 0; s < pl.c; ++s) acc = ge_dbl_quad(acc);
    acc = ge_add_quad(acc, ge_load(wsum[w]));
  }
  if (lane == 0) ge_store(out, acc);
}

// Window sum W_w = G_0 + 16 sum_k 2^k G_{1+k} of window w from its group sums (quad-cooperative
// Horner over the group bits; every lane of the quad ends with the whole point).
__device__ __forceinline__ ge window_sum_quad(const uint32_t* groups, const MsmPlan& pl, int w) {
  const int ng = 1 + pl.jbits;
  const uint32_t* G = groups + 32 * (size_t)w * ng;
  ge acc = ge_load(G + 32 * pl.jbits);
  for (int k = pl.jbits - 2; k >= 0; --k) acc = ge_add_quad(ge_dbl_quad(acc), ge_load(G + 32 * (1 + k)));
  for (int i = 0; i < 4; ++i) acc = ge_dbl_quad(acc);   // times kMsmChunk = 16
  return ge_add_quad(acc, ge_load(G));
}

// The window sums W_w of every window into W (32 words each): quad w per window, in rounds
// of eight quads.  One warp.
__global__ void __launch_bounds__(32) k_msm_windows(const uint32_t* groups, MsmPlan pl, uint32_t* W) {
  const int lane = threadIdx.x & 31, quad = lane >> 2;
  for (int r0 = 0; r0 < pl.windows; r0 += 8) {
    const int w = r0 + quad;
    const ge acc = window_sum_quad(groups, pl, w < pl.windows ? w : pl.windows - 1);
    if ((lane & 3) == 0 && w < pl.windows) ge_store(W + 32 * (size_t)w, acc);
  }
}

// Per-window weighted check, group side: quad w forms the window sum W_w and tests
// [8](W_w - P_w) = O against P_w = [E_w] Y + [S_w] G (k_window_prep); windows are processed in
// rounds of eight quads.  accept = every window holds, no malformed s (*bad), no undecodable
// R (*point_bad) and a decodable key.  One warp.
__global__ void __launch_bounds__(32) k_msm_window_check(const uint32_t* groups, MsmPlan pl, const uint32_t* Pw,
                                                         const uint32_t* bad, const uint32_t* point_bad,
                                                         const uint32_t* status, uint8_t* accept) {
  const int lane = threadIdx.x & 31, quad = lane >> 2;
  bool ok = true;
  for (int r0 = 0; r0 < pl.windows; r0 += 8) {
    const int w = r0 + quad;
    const int wc = w < pl.windows ? w : pl.windows - 1;
    const ge acc = window_sum_quad(groups, pl, wc);
    ge diff = ge_add_quad(acc, ge_neg(ge_load(Pw + 32 * (size_t)wc)));
    for (int i = 0; i < 3; ++i) diff = ge_dbl_quad(diff);   // cofactor 8
    if (w < pl.windows) ok = ok && ge_is_identity(diff);
  }
  const bool all = __all_sync(0xffffffffu, ok);
  if (lane == 0) *accept = (all && *bad == 0 && !(point_bad && *point_bad) && (*status & kErrKey) == 0) ? 1 : 0;
}

// Synthetic input for timing window widths: every point is G (the cost of a complete
// addition does not depend on its operands) and the scalars are SplitMix64 output with the
// top bit of a 4-word weight, or the top 3 bits of an 8-word scalar, cleared.
__global__ void k_msm_tune_fill(uint32_t* pts, uint32_t* z, uint64_t n, int sw) {
  const ge G = ge_base();
  const fe t2d = fe_mul(G.T, fe_d2());
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    uint32_t* dst = pts + (size_t)kPtsWords * t;
#pragma unroll
    for (int i = 0; i < 8; ++i) { dst[i] = G.X.v[i]; dst[8 + i] = G.Y.v[i]; dst[16 + i] = t2d.v[i]; }
    for (int k = 0; k < sw / 2; ++k) {
      uint64_t x = (t * 8 + k) + 0x9e3779b97f4a7c15ull;
      x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
      x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
      x ^= x >> 31;
      z[(size_t)sw * t + 2 * k] = (uint32_t)x;
      z[(size_t)sw * t + 2 * k + 1] = (uint32_t)(x >> 32);
    }
    z[(size_t)sw * t + sw - 1] &= sw == 4 ? 0x7fffffffu : 0x1fffffffu;
  }
}

}  // namespace poslo
