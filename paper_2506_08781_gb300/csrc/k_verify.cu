// Verification kernels: epoch seeds, hashing and scalar aggregation, point decoding and sums,
// window tables and the final cofactored check.
#include "common.cuh"
#include "compact.cuh"

namespace poslo {

template <int INST>
__global__ void k_epoch_seeds(const DsNode* __restrict__ ds, int nds, uint64_t e0, uint64_t ne,
                              uint32_t* __restrict__ x0_out, uint32_t* __restrict__ status) {
  AesCtx c{};
  if constexpr (INST == kInstAes) {
    __shared__ AesShared sh;
    aes_tables_init(sh);
    c = aes_ctx(&sh);
  }
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ne) return;
  const uint64_t target = e0 + k;
  // pop from the top of the stack until a node covers leaf `target`
  int top = nds - 1;
  bool ok = top >= 0;
  if (ok) {
    const DsNode& n = ds[top];
    ok = target < (((uint64_t)n.i + 1) << n.d);
  }
  while (ok && target < ((uint64_t)ds[top].i << ds[top].d)) {
    --top;
    ok = top >= 0;
  }
  uint32_t x[4] = {0, 0, 0, 0};
  if (ok) {
    const DsNode n = ds[top];
    x[0] = n.seed[0]; x[1] = n.seed[1]; x[2] = n.seed[2]; x[3] = n.seed[3];
    const uint64_t off = target - ((uint64_t)n.i << n.d);
    for (int j = (int)n.d - 1; j >= 0; --j) {
      uint32_t y[4];
      prf_node_i<INST>(c, x, (uint32_t)(off >> j) & 1u, y);
      x[0] = y[0]; x[1] = y[1]; x[2] = y[2]; x[3] = y[3];
    }
  } else {
    atomicOr(status, kErrSeed);
  }
  uint4* o = reinterpret_cast<uint4*>(x0_out) + k;
  *o = make_uint4(x[0], x[1], x[2], x[3]);
}

// Entries are processed in tiles of kHashTile; inside a tile they are reordered by the
// number of SHA-256 blocks of m_t || x_t (a counting sort in shared memory), so the lanes of
// a warp run the same number of compressions.  Per entry, one loop drives every
// compression (the PRF block, the message blocks, and the weight block in weighted mode)
// through a single inlined copy of the compression function.
constexpr int kHashTile = 256;
constexpr int kHashClasses = 8;

// z_t = SHA-256("POSLO-Z" || verifier_seed || le64(t)): the single padded block.
__device__ __forceinline__ void weight_block(const uint32_t zpre[10], uint64_t zi, uint32_t w[16]) {
  const uint32_t lo = (uint32_t)zi, hi = (uint32_t)(zi >> 32);
#pragma unroll
  for (int q = 0; q < 9; ++q) w[q] = zpre[q];
  w[9] = zpre[9] | (lo & 0xffu);
  w[10] = ((lo >> 8) & 0xffu) << 24 | ((lo >> 16) & 0xffu) << 16 | ((lo >> 24) & 0xffu) << 8 | (hi & 0xffu);
  w[11] = ((hi >> 8) & 0xffu) << 24 | ((hi >> 16) & 0xffu) << 16 | ((hi >> 24) & 0xffu) << 8 | 0x80u;
  w[12] = 0; w[13] = 0; w[14] = 0; w[15] = 47 * 8;
}

// The verifier's weights alone: z_t for entries first .. first + n - 1 (one SHA-256 block
// each), so that the MSM's counting sort need not wait for the message hashing.
__global__ void k_weights(const ZPre zp, uint64_t n, uint64_t first, uint32_t* z_out) {
  uint32_t pre[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) pre[q] = zp.w[q];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    uint32_t w[16], st[8];
    weight_block(pre, first + t, w);
    sha256_init(st);
    sha256_compress(st, w);
    reinterpret_cast<uint4*>(z_out)[t] =
        make_uint4(bswap32(st[0]), bswap32(st[1]), bswap32(st[2]), bswap32(st[3]) & 0x7fffffffu);
  }
}

// MINB: resident blocks per SM the kernel is compiled for -- POSLO_HASH_MIN_BLOCKS when it runs
// on its own, kCoresidentMinBlocks (128 registers) when it is to share the SMs with the
// decoding of a multi-device batch.
template <int INST, int MINB>
__global__ void __launch_bounds__(kHashThreads, MINB) k_hash(const HashArgs a) {
  AesCtx c{};
  if constexpr (INST == kInstAes) {
    __shared__ AesShared sh;
    aes_tables_init(sh);
    c = aes_ctx(&sh);
  }
  acc13 acc_e, acc_s;
  acc_zero(acc_e);
  acc_zero(acc_s);
  uint32_t bad = 0;
  __shared__ uint16_t s_order[kHashTile];
  __shared__ uint32_t s_cnt[kHashClasses], s_off[kHashClasses];
  constexpr int kPer = kHashTile / kHashThreads;
  const uint64_t ntiles = (a.n + kHashTile - 1) / kHashTile;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t base = tile * kHashTile;
    const uint64_t rem = a.n - base;
    const uint32_t m = rem < (uint64_t)kHashTile ? (uint32_t)rem : (uint32_t)kHashTile;
    if (threadIdx.x < kHashClasses) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    uint32_t cls[kPer], pos[kPer];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const uint32_t k = threadIdx.x + r * kHashThreads;
      if (k < m) {
        const uint64_t lo = a.offs[base + k], hi = a.offs[base + k + 1];
        if (hi < lo || lo < a.base_off || hi - lo > 0xffffffffull) atomicOr(a.status, kErrInput);
        const uint64_t L = hi >= lo ? hi - lo : 0;
        const uint64_t c = (L + 88) >> 6;
        cls[r] = c < (uint64_t)(kHashClasses - 1) ? (uint32_t)c : (uint32_t)(kHashClasses - 1);
        pos[r] = atomicAdd(&s_cnt[cls[r]], 1u);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t acc = 0;
      for (int c = 0; c < kHashClasses; ++c) { s_off[c] = acc; acc += s_cnt[c]; }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const uint32_t k = threadIdx.x + r * kHashThreads;
      if (k < m) s_order[s_off[cls[r]] + pos[r]] = (uint16_t)k;
    }
    __syncthreads();
#pragma unroll 1
    for (int r = 0; r < kPer; ++r) {
      const uint32_t k = threadIdx.x + r * kHashThreads;
      if (k >= m) continue;
      const uint64_t t = base + s_order[k];
      uint64_t gi, i, j, seed_idx, zi;
      if (a.n_seg) {
        const uint32_t d = segment_of(a.seg_start, a.n_seg, t);
        gi = a.seg_first[d] + (t - a.seg_start[d]);
        const uint32_t n2 = a.seg_n2[d];
        i = gi / n2;
        j = gi - i * n2;
        seed_idx = a.seg_seed_off[d] + (i - a.seg_e0[d]);
        zi = t;
      } else {
        gi = a.first_index + t;
        if (a.n2_log2 != 0xffffffffu) {
          i = gi >> a.n2_log2;
          j = gi & ((1ull << a.n2_log2) - 1);
        } else {
          i = gi / a.n2;
          j = gi - i * a.n2;
        }
        seed_idx = i - a.e0;
        zi = gi;
      }
      const uint4 xs = __ldg(reinterpret_cast<const uint4*>(a.seeds) + seed_idx);
      const uint64_t o0 = a.offs[t] - a.base_off, o1 = a.offs[t + 1] - a.base_off;
      // malformed offsets (flagged above) hash as empty messages and never read memory
      const uint32_t L = (o1 >= o0 && o1 - o0 <= 0xffffffffull && a.offs[t] >= a.base_off) ? (uint32_t)(o1 - o0) : 0u;
      uint32_t st[8], dig[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if constexpr (INST == kInstAes) {
        // x_t = MMO-AES-128 PRF, e_t from MDC-2-AES-128 over m || x_t, then z_t by SHA-256
        const uint32_t x0[4] = {xs.x, xs.y, xs.z, xs.w};
        uint32_t x[4];
        prf_entry_aes(c, x0, (uint32_t)j, x);
        mdc2_stream(c, entry_stream(a.msgs + o0, L, x), dig);
        if (a.weighted && !a.z_in) {
          uint32_t w[16];
          weight_block(a.zpre, zi, w);
          sha256_init(st);
          sha256_compress(st, w);
        }
      } else {
        // padded stream of m || x (x is known after the PRF block)
        EntryStream es;
        {
          const uintptr_t p = reinterpret_cast<uintptr_t>(a.msgs + o0);
          const uint32_t sh = (uint32_t)(p & 3u);
          es.base = reinterpret_cast<const uint32_t*>(p - sh);
          es.sel = (sh + 3) | ((sh + 2) << 4) | ((sh + 1) << 8) | (sh << 12);
          es.sh_nz = sh != 0;
          es.L = L;
          es.kmax = L > 0 ? (int32_t)((L + sh - 1) >> 2) : 0;
          es.a = L & ~3u;
        }
        const uint32_t total = L + 16;
        const uint32_t nb = (total + 9 + 63) >> 6;
        const uint32_t iters = 1 + nb + (a.weighted && !a.z_in ? 1u : 0u);
        sha256_init(st);
#pragma unroll 1
        for (uint32_t it = 0; it < iters; ++it) {
          uint32_t w[16];
          if (it == 0) {
            // PRF_0(x_0[i] || le32(j)): x0 || le32(j) || 0x00 || 0x80 ... || bitlen(21 bytes)
            w[0] = xs.x; w[1] = xs.y; w[2] = xs.z; w[3] = xs.w;
            w[4] = bswap32((uint32_t)j);
            w[5] = 0x00800000u;
#pragma unroll
            for (int q = 6; q < 15; ++q) w[q] = 0;
            w[15] = 21 * 8;
          } else if (it <= nb) {
            const uint32_t o = (it - 1) << 6;
            if (o + 64 <= L) {
#pragma unroll
              for (int q = 0; q < 16; ++q) w[q] = load_msg_word(es, (o >> 2) + q);
            } else {
#pragma unroll
              for (int q = 0; q < 16; ++q) w[q] = stream_word(es, o + 4 * q);
              if (it == nb) {
                w[14] |= total >> 29;
                w[15] |= total << 3;
              }
            }
          } else {
            weight_block(a.zpre, zi, w);
          }
          sha256_compress(st, w);
          if (it == 0) {
            // x = first 16 bytes of the PRF digest, shifted into the stream after m
            const uint32_t sr = 8u * (L & 3u);
            es.S[0] = __funnelshift_r(st[0], 0u, sr);
            es.S[1] = __funnelshift_r(st[1], st[0], sr);
            es.S[2] = __funnelshift_r(st[2], st[1], sr);
            es.S[3] = __funnelshift_r(st[3], st[2], sr);
            es.S[4] = __funnelshift_r(0x80000000u, st[3], sr);
            sha256_init(st);
          } else if (it == nb) {
#pragma unroll
            for (int q = 0; q < 8; ++q) dig[q] = bswap32(st[q]);
            sha256_init(st);
          }
        }
      }
      const sc e = sc_reduce256(dig);
      if (a.e_out) {
        uint4* eo = reinterpret_cast<uint4*>(a.e_out + 32 * t);
        eo[0] = make_uint4(e.v[0], e.v[1], e.v[2], e.v[3]);
        eo[1] = make_uint4(e.v[4], e.v[5], e.v[6], e.v[7]);
      }
      uint32_t s[8];
      if (a.s) {
        const uint4* sp = reinterpret_cast<const uint4*>(a.s + 32 * t);
        const uint4 s0 = __ldg(sp), s1 = __ldg(sp + 1);
        s[0] = s0.x; s[1] = s0.y; s[2] = s0.z; s[3] = s0.w; s[4] = s1.x; s[5] = s1.y; s[6] = s1.z; s[7] = s1.w;
        const bool canon = sc_is_canonical(s);
        bad += canon ? 0u : 1u;
        if (a.sbad_out) a.sbad_out[t] = canon ? 0 : 1;
      }
      if (a.weighted) {
        // z_t: the first 16 digest bytes as a little-endian integer, bit 127 cleared
        uint32_t z[4];
        if (a.z_in) {
          const uint4 zz = __ldg(reinterpret_cast<const uint4*>(a.z_in) + t);
          z[0] = zz.x; z[1] = zz.y; z[2] = zz.z; z[3] = zz.w;
        } else {
          z[0] = bswap32(st[0]); z[1] = bswap32(st[1]); z[2] = bswap32(st[2]); z[3] = bswap32(st[3]) & 0x7fffffffu;
        }
        if (a.z_out) reinterpret_cast<uint4*>(a.z_out)[t] = make_uint4(z[0], z[1], z[2], z[3]);
        uint32_t pr[12];
        mul_4x8(pr, z, e.v);
        acc_add<12>(acc_e, pr);
        if (a.s) {
          mul_4x8(pr, z, s);
          acc_add<12>(acc_s, pr);
        }
      } else {
        acc_add<8>(acc_e, e.v);
        if (a.s) acc_add<8>(acc_s, s);
      }
    }
    __syncthreads();
  }
  // block reduction of the limb values as 64-bit sums
  __shared__ unsigned long long red[kHashThreads / 32][kPartialWords];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kPartialWords; ++k) {
    unsigned long long v = k < 13 ? acc_e.v[k] : (k < 26 ? acc_s.v[k - 13] : bad);
    warp_sum_u64(v);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kPartialWords) {
    unsigned long long v = 0;
    for (int w = 0; w < kHashThreads / 32; ++w) v += red[w][threadIdx.x];
    a.partial[(uint64_t)blockIdx.x * kPartialWords + threadIdx.x] = v;
  }
}

#ifndef POSLO_POINTS_DYNAMIC
#define POSLO_POINTS_DYNAMIC 1
#endif

// Strict decoding of R_t, its affine form for the MSM and its decode flag, and its addition
// into the thread's unit sum.
__device__ __forceinline__ void decode_one(const PointArgs& a, uint64_t t, ge& acc, uint32_t& bad) {
  const uint4* rp = reinterpret_cast<const uint4*>(a.R + 32 * t);
  const uint4 r0 = __ldg(rp), r1 = __ldg(rp + 1);
  const uint32_t b[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
  ge P;
  const bool ok = ge_decode(b, P);
  bad += ok ? 0u : 1u;
  if (a.bad_out) a.bad_out[t] = ok ? 0 : 1;
  const fe t2d = fe_mul(P.T, fe_d2());
  if (a.pts_out) {
    uint4* dst = reinterpret_cast<uint4*>(a.pts_out + (size_t)kPtsWords * t);
    dst[0] = make_uint4(P.X.v[0], P.X.v[1], P.X.v[2], P.X.v[3]);
    dst[1] = make_uint4(P.X.v[4], P.X.v[5], P.X.v[6], P.X.v[7]);
    dst[2] = make_uint4(P.Y.v[0], P.Y.v[1], P.Y.v[2], P.Y.v[3]);
    dst[3] = make_uint4(P.Y.v[4], P.Y.v[5], P.Y.v[6], P.Y.v[7]);
    dst[4] = make_uint4(t2d.v[0], t2d.v[1], t2d.v[2], t2d.v[3]);
    dst[5] = make_uint4(t2d.v[4], t2d.v[5], t2d.v[6], t2d.v[7]);
  }
  if (ok && !(a.skip && a.skip[t])) acc = ge_madd(acc, P.X, P.Y, t2d);
}

// Every R_t: blocks take chunks of kPointChunk points from a shared counter, so a block that
// starts late (its SM busy with the hashing beside it) simply takes fewer chunks; then the
// block's unit sum and decode-failure count.
// MINB: 1 when the decoding runs on its own (146 registers), kCoresidentMinBlocks (128
// registers) when three of its blocks share each SM with a hashing block.
template <int MINB>
__global__ void __launch_bounds__(kPointThreads, MINB) k_points(const PointArgs a) {
  ge acc = ge_identity();
  uint32_t bad = 0;
#if POSLO_POINTS_DYNAMIC
  __shared__ uint64_t s_base;
  for (;;) {
    if (threadIdx.x == 0) s_base = (uint64_t)atomicAdd(a.work, 1u) * kPointChunk;
    __syncthreads();
    const uint64_t base = s_base;
    __syncthreads();
    if (base >= a.count) break;
    const uint64_t end = min(base + kPointChunk, a.count);
    for (uint64_t t = base + threadIdx.x; t < end; t += blockDim.x) decode_one(a, t, acc, bad);
  }
#else
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.count; t += stride)
    decode_one(a, t, acc, bad);
#endif
  // tree reduction in shared memory
  __shared__ uint32_t sp[kPointThreads][32];
  __shared__ uint32_t sbad[kPointThreads];
  ge_store(sp[threadIdx.x], acc);
  sbad[threadIdx.x] = bad;
  __syncthreads();
  for (int h = kPointThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      const ge o = ge_load(sp[threadIdx.x + h]);
      const ge m = ge_load(sp[threadIdx.x]);
      ge_store(sp[threadIdx.x], ge_add(m, o));
      sbad[threadIdx.x] += sbad[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x < 32) a.partial[(uint64_t)blockIdx.x * kPointPartialWords + threadIdx.x] = sp[0][threadIdx.x];
  if (threadIdx.x == 0) a.partial[(uint64_t)blockIdx.x * kPointPartialWords + 32] = sbad[0];
}

// Fixed-window tables table[w][d-1] = d 16^w P (w = 0..63, d = 1..8) of n keys, in two
// launches.  k_table_chain: one quad of lanes per key walks P, 16P, ..., 16^63 P with
// quad-cooperative doublings (252 of them, at a quarter of a doubling's dependent
// multiplications each) and writes each 16^w P as table[w][0].  k_table_fill: one quad per
// (key, window) forms d 16^w P for d = 2..8 by quad-cooperative additions.  The key of
// index k is the encoding enc + 8 k, the decoded point pts + kPtsWords * list[k] (affine
// x, y; k itself without a list), or G (use_base).  An encoding that does not decode gives
// the identity's table and sets bad_out[k] (when given) or the kErrKey status bit.
__global__ void __launch_bounds__(128) k_table_chain(const uint32_t* __restrict__ enc,
                                                     const uint32_t* __restrict__ pts,
                                                     const uint32_t* __restrict__ list, uint32_t n,
                                                     uint32_t* __restrict__ tables, uint32_t* const* dst,
                                                     uint32_t* __restrict__ status, int use_base,
                                                     uint8_t* __restrict__ bad_out) {
  const uint32_t quad = ((uint32_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const uint32_t k = quad < n ? quad : n - 1;   // surplus quads repeat the last key, unwritten
  const bool writer = quad < n && (threadIdx.x & 3) == 0;
  ge P;
  if (use_base) {
    P = ge_base();
  } else if (pts) {
    fe t2d;
    pts_load(pts + (size_t)kPtsWords * (list ? list[k] : k), P.X, P.Y, t2d);
    P.Z = fe_one();
    P.T = fe_mul(P.X, P.Y);
  } else {
    uint32_t b[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) b[i] = enc[8 * (size_t)k + i];
    const bool ok = ge_decode(b, P);
    if (!ok) P = ge_identity();
    if (writer) {
      if (bad_out) bad_out[k] = ok ? 0 : 1;   // the caller reports which key failed
      else if (!ok) atomicOr(status, kErrKey);
    }
  }
  uint32_t* table = dst ? dst[k] : tables + (size_t)k * kTableWords;
  // every lane runs every quad doubling (full-mask shuffles)
  for (int w = 0; w < kTableWindows; ++w) {
    if (writer) ge_store(table + (size_t)w * kTableDigits * 32, P);
    if (w + 1 < kTableWindows)
      for (int i = 0; i < 4; ++i) P = ge_dbl_quad(P);
  }
}

__global__ void __launch_bounds__(128) k_table_fill(uint32_t n, uint32_t* __restrict__ tables, uint32_t* const* dst) {
  const uint64_t total = (uint64_t)n * kTableWindows;
  const uint64_t quad = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const uint64_t q = quad < total ? quad : total - 1;
  const bool writer = quad < total && (threadIdx.x & 3) == 0;
  const uint64_t key = q / kTableWindows;
  uint32_t* row = (dst ? dst[key] : tables + key * kTableWords) + (q % kTableWindows) * kTableDigits * 32;
  const ge Pw = ge_load(row);
  ge acc = Pw;
  for (int d = 2; d <= kTableDigits; ++d) {
    acc = ge_add_quad(acc, Pw);
    if (writer) ge_store(row + (d - 1) * 32, acc);
  }
}

// Runs once per call: its point operations are the compact (out-of-line) ones, its code being
// fetched cold on every launch.
__global__ void __launch_bounds__(kFinalThreads) k_finalize(const FinalArgs a) {
  __shared__ unsigned long long sums[kPartialWords];
  __shared__ uint32_t pts[kFinalThreads][32];
  __shared__ uint32_t pbad;
  __shared__ int8_t dig_e[64], dig_s[64];
  __shared__ uint32_t sh_e[8], sh_s[8];
  __shared__ uint32_t bad_flag;
  const int tid = threadIdx.x;
  if (tid < kPartialWords) sums[tid] = 0;
  if (tid == 0) { pbad = 0; bad_flag = 0; }
  __syncthreads();
  // scalar partial sums: word w of every block's partial, the blocks split over
  // kFinalThreads / kPartialWords threads per word (a chain of dependent loads per word was the
  // kernel's longest part)
  constexpr int kLanesPerWord = kFinalThreads / kPartialWords;
  if (tid < kLanesPerWord * kPartialWords) {
    const int w = tid % kPartialWords, lane = tid / kPartialWords;
    unsigned long long v = 0;
    for (uint32_t b = lane; b < a.nhash; b += kLanesPerWord) v += a.hash_partial[(size_t)b * kPartialWords + w];
    atomicAdd(&sums[w], v);
  }
  // point partials
  ge acc = ge_identity();
  uint32_t bad = 0;
  for (uint32_t b = tid; b < a.npoint; b += kFinalThreads) {
    acc = compact::add(acc, ge_load(a.point_partial + (size_t)b * kPointPartialWords));
    bad += a.point_partial[(size_t)b * kPointPartialWords + 32];
  }
  ge_store(pts[tid], acc);
  atomicAdd(&pbad, bad);
  __syncthreads();
  for (int h = kFinalThreads / 2; h > 0; h >>= 1) {
    if (tid < h) ge_store(pts[tid], compact::add(ge_load(pts[tid]), ge_load(pts[tid + h])));
    __syncthreads();
  }
  if (tid == 0) {
    const sc e = limb_sums_to_scalar(sums);
    sc s;
    uint32_t bf = (sums[26] != 0 || pbad != 0) ? 1u : 0u;
    if (a.s_given) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        s.v[k] = a.s_given[4 * k] | (a.s_given[4 * k + 1] << 8) | (a.s_given[4 * k + 2] << 16) |
                 ((uint32_t)a.s_given[4 * k + 3] << 24);
      if (!sc_is_canonical(s.v)) bf = 1;
    } else {
      s = limb_sums_to_scalar(sums + 13);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) { sh_e[k] = e.v[k]; sh_s[k] = s.v[k]; }
    recode4(e.v, dig_e);
    recode4(s.v, dig_s);
    bad_flag = bf;
  }
  __syncthreads();
  // R is the reduced point sum unless given
  ge R = a.R_given ? ge_load(a.R_given) : ge_load(pts[0]);
  __syncthreads();
  // window terms: thread w adds dig_e[w] 16^w Y + dig_s[w] 16^w G
  ge term = ge_identity();
  if (tid < kTableWindows) {
    term = compact::add(table_pick(a.tableY, tid, dig_e[tid]), table_pick(a.tableG, tid, dig_s[tid]));
  }
  ge_store(pts[tid], term);
  __syncthreads();
  for (int h = kTableWindows / 2; h > 0; h >>= 1) {
    if (tid < h) ge_store(pts[tid], compact::add(ge_load(pts[tid]), ge_load(pts[tid + h])));
    __syncthreads();
  }
  if (tid == 0) {
    const ge eYsG = ge_load(pts[0]);
    const ge diff = compact::sub(R, eYsG);
    const bool ok = ge_is_identity(compact::mul_cofactor(diff)) && !bad_flag;
    const bool key_bad = (*a.status & kErrKey) != 0;
    a.accept[0] = (ok && !key_bad) ? 1 : 0;
    if (a.out_words) {
      for (int k = 0; k < 8; ++k) { a.out_words[k] = sh_e[k]; a.out_words[8 + k] = sh_s[k]; }
      ge_store(a.out_words + 16, R);
    }
  }
}

// The final check split in two so that its expensive half overlaps the MSM:
// k_final_prep (side stream, after hashing and the window table of Y) reduces the scalar
// partials to e and s and evaluates [e]Y + [s]G from the two window tables (128 terms
// summed by a shared-memory tree); k_final_check (after the MSM) only forms
// [8](R - ([e]Y + [s]G)) and tests it for the identity.
constexpr int kPrepThreads = 128;
__global__ void __launch_bounds__(128) k_final_prep(const PrepArgs a) {
  __shared__ unsigned long long sums[kPartialWords];
  __shared__ int8_t dig_e[64], dig_s[64];
  __shared__ uint32_t pts_[kPrepThreads][32];
  __shared__ uint32_t bad_flag;
  const int tid = threadIdx.x;
  if (tid < kPartialWords) sums[tid] = 0;
  __syncthreads();
  constexpr int kLanesPerWord = kPrepThreads / kPartialWords;   // blocks split over lanes per word
  if (tid < kLanesPerWord * kPartialWords) {
    const int w = tid % kPartialWords, lane = tid / kPartialWords;
    unsigned long long v = 0;
    for (uint32_t b = lane; b < a.nhash; b += kLanesPerWord) v += a.hash_partial[(size_t)b * kPartialWords + w];
    atomicAdd(&sums[w], v);
  }
  __syncthreads();
  if (tid == 0) {
    const sc e = limb_sums_to_scalar(sums);
    sc s;
    uint32_t bf = sums[26] != 0 ? 1u : 0u;
    if (a.s_given) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        s.v[k] = a.s_given[4 * k] | (a.s_given[4 * k + 1] << 8) | (a.s_given[4 * k + 2] << 16) |
                 ((uint32_t)a.s_given[4 * k + 3] << 24);
      if (!sc_is_canonical(s.v)) bf = 1;
    } else {
      s = limb_sums_to_scalar(sums + 13);
    }
    recode4(e.v, dig_e);
    recode4(s.v, dig_s);
    bad_flag = bf;
  }
  __syncthreads();
  const ge term = tid < 64 ? table_pick(a.tableY, tid, dig_e[tid]) : table_pick(a.tableG, tid - 64, dig_s[tid - 64]);
  ge_store(pts_[tid], term);
  __syncthreads();
  static_assert(kPrepThreads == 128 && kWindowThreads == 128, "quad_sum128 takes one term per thread of 128");
  __shared__ uint32_t qs_[32][32];
  compact::quad_sum128(pts_, qs_);
  if (tid < 32) a.prep[tid] = qs_[0][tid];
  if (tid == 0) a.prep[32] = bad_flag;
}

// Per-window weighted check, scalar side.  With z_t = sum_w d_{t,w} 2^(c w) in the MSM's
// signed window digits, window w of the batch equation is
//   sum_t d_{t,w} R_t = [E_w] Y + [S_w] G,  E_w = sum_t d_{t,w} e_t,  S_w = sum_t d_{t,w} s_t (mod q).
// k_window_sums: grid (x, windows), blockIdx.y = w; each thread recodes the weights of its
// entries up to window w and adds |d| x, with x = e_t (s_t) for a positive digit and q - x for
// a negative one, into exact 416-bit accumulators; per block 13 limb sums of E_w and 13 of
// S_w (26 u64 at partial[(w * gridDim.x + blockIdx.x) * 26]).
__global__ void __launch_bounds__(kWindowThreads) k_window_sums(const uint8_t* e, const uint8_t* s, const uint32_t* z,
                                                                uint64_t n, MsmPlan pl,
                                                                unsigned long long* partial) {
  const int w = blockIdx.y;
  acc13 ae, as;
  acc_zero(ae);
  acc_zero(as);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    bool neg;
    const uint32_t d = weight_digit(z, t, w, pl.c, neg);
    if (d) add_window_terms(ae, as, e + 32 * t, s + 32 * t, d, neg);
  }
  __shared__ unsigned long long red[kWindowThreads / 32][26];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 26; ++k) {
    unsigned long long v = k < 13 ? ae.v[k] : as.v[k - 13];
    warp_sum_u64(v);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 26) {
    unsigned long long v = 0;
    for (int i = 0; i < kWindowThreads / 32; ++i) v += red[i][threadIdx.x];
    partial[((size_t)w * gridDim.x + blockIdx.x) * 26 + threadIdx.x] = v;
  }
}

// One block per window: E_w and S_w from the partials of k_window_sums, then
// P_w = [E_w] Y + [S_w] G from the two window tables (128 terms, shared-memory tree) into
// Pw[w] (32 words).  Block 0 also writes the malformed-s flag of the hashing partials to *bad.
__global__ void __launch_bounds__(kWindowThreads) k_window_prep(const unsigned long long* partial, uint32_t nblocks,
                                                                const unsigned long long* hash_partial, uint32_t nhash,
                                                                const uint32_t* tableY, const uint32_t* tableG,
                                                                uint32_t* Pw, uint32_t* bad) {
  __shared__ unsigned long long sums[26];
  __shared__ int8_t dig_e[64], dig_s[64];
  __shared__ uint32_t pts_[kWindowThreads][32];
  const int w = blockIdx.x, tid = threadIdx.x;
  if (tid < 26) {
    unsigned long long v = 0;
    for (uint32_t b = 0; b < nblocks; ++b) v += partial[((size_t)w * nblocks + b) * 26 + tid];
    sums[tid] = v;
  }
  if (w == 0 && tid == 32) {
    unsigned long long v = 0;
    for (uint32_t b = 0; b < nhash; ++b) v += hash_partial[(size_t)b * kPartialWords + 26];
    *bad = v != 0 ? 1u : 0u;
  }
  __syncthreads();
  if (tid == 0) {
    const sc E = limb_sums_to_scalar(sums), S = limb_sums_to_scalar(sums + 13);
    recode4(E.v, dig_e);
    recode4(S.v, dig_s);
  }
  __syncthreads();
  const ge term = tid < 64 ? table_pick(tableY, tid, dig_e[tid]) : table_pick(tableG, tid - 64, dig_s[tid - 64]);
  ge_store(pts_[tid], term);
  __syncthreads();
  static_assert(kPrepThreads == 128 && kWindowThreads == 128, "quad_sum128 takes one term per thread of 128");
  __shared__ uint32_t qs_[32][32];
  compact::quad_sum128(pts_, qs_);
  if (tid < 32) Pw[32 * w + tid] = qs_[0][tid];
}

// One warp (quad operations: every lane takes part).
__global__ void k_final_check(const uint32_t* prep, const uint32_t* R, const uint32_t* point_bad,
                              const uint32_t* status, uint8_t* accept) {
  if (blockIdx.x != 0) return;
  ge d = ge_add_quad(ge_load(R), ge_neg(ge_load(prep)));
#pragma unroll 1
  for (int i = 0; i < 3; ++i) d = ge_dbl_quad(d);
  const bool ok = ge_is_identity(d) && prep[32] == 0 && !(point_bad && *point_bad) && (*status & kErrKey) == 0;
  if (threadIdx.x == 0) accept[0] = ok ? 1 : 0;
}

// Host launchers (kernel templates are launched from the translation unit that defines them).
void launch_epoch_seeds(int inst, unsigned grid, unsigned block, cudaStream_t st, const DsNode* ds, int nds,
                        uint64_t e0, uint64_t ne, uint32_t* x0_out, uint32_t* status) {
  if (inst == kInstAes) k_epoch_seeds<kInstAes><<<grid, block, 0, st>>>(ds, nds, e0, ne, x0_out, status);
  else k_epoch_seeds<kInstSha><<<grid, block, 0, st>>>(ds, nds, e0, ne, x0_out, status);
}

void launch_hash(int inst, unsigned grid, cudaStream_t st, const HashArgs& a, bool coresident) {
  if (coresident) {
    if (inst == kInstAes) k_hash<kInstAes, kCoresidentMinBlocks><<<grid, kHashThreads, 0, st>>>(a);
    else k_hash<kInstSha, kCoresidentMinBlocks><<<grid, kHashThreads, 0, st>>>(a);
  } else {
    if (inst == kInstAes) k_hash<kInstAes, POSLO_HASH_MIN_BLOCKS><<<grid, kHashThreads, 0, st>>>(a);
    else k_hash<kInstSha, POSLO_HASH_MIN_BLOCKS><<<grid, kHashThreads, 0, st>>>(a);
  }
}

void launch_points(unsigned grid, cudaStream_t st, const PointArgs& a, bool coresident) {
  if (coresident) k_points<kCoresidentMinBlocks><<<grid, kPointThreads, 0, st>>>(a);
  else k_points<1><<<grid, kPointThreads, 0, st>>>(a);
}

}  // namespace poslo
