// Multi-device batches: many signers' logs verified in one pass of each stage over a segment
// table (device d owns entries [seg_start[d], seg_start[d+1]) of the concatenated batch).
// The paper verifies one signer at a time (single-signer aggregation, Sec. 5); here every
// stage is one launch for all devices, and one random linear combination checks them all
// at once: sum_t z_t R_t - sum_d (sum_{t in d} z_t e_t) Y_d - (sum_t z_t s_t) G = O.
#include "common.cuh"

namespace poslo {

// SRet for every (device, epoch) pair of the batch: seeds[s] for s in
// [seed_off[d], seed_off[d+1]) is x_0[e0[d] + s - seed_off[d]] under device d's ds.
template <int INST>
__global__ void k_epoch_seeds_multi(const DsNode* ds_all, const uint32_t* ds_off, const uint64_t* seed_off,
                                    const uint64_t* e0, uint32_t n_dev, uint32_t* seeds, uint32_t* status) {
  AesCtx c{};
  if constexpr (INST == kInstAes) {
    __shared__ AesShared sh;
    aes_tables_init(sh);
    c = aes_ctx(&sh);
  }
  const uint64_t total = seed_off[n_dev];
  const uint64_t sidx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (sidx >= total) return;
  const uint32_t d = segment_of(seed_off, n_dev, sidx);
  const uint64_t target = e0[d] + (sidx - seed_off[d]);
  const DsNode* ds = ds_all + ds_off[d];
  int top = (int)(ds_off[d + 1] - ds_off[d]) - 1;
  bool ok = top >= 0 && target < (((uint64_t)ds[top].i + 1) << ds[top].d);
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
  reinterpret_cast<uint4*>(seeds)[sidx] = make_uint4(x[0], x[1], x[2], x[3]);
}

// offs[t] -= base for t < n (a chunk's offsets made relative to its first message byte).
__global__ void k_offs_sub(uint64_t* offs, uint64_t n, uint64_t base) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) offs[t] -= base;   // a decreasing offset wraps and is flagged by k_hash
}

// Concatenated offsets: raw holds each device's n_d + 1 offsets at slot[d]; entry k of
// device d becomes msg_base[d] + raw[slot[d] + k] - raw[slot[d]] at position start[d] + k.
__global__ void k_rebase_offs(const uint64_t* raw, const uint64_t* slot, const uint64_t* start,
                              const uint64_t* msg_base, uint32_t n_dev, uint64_t* out, uint32_t* status) {
  const uint64_t total = slot[n_dev];
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= total) return;
  const uint32_t d = segment_of(slot, n_dev, r);
  const uint64_t k = r - slot[d];
  const uint64_t v = raw[r], v0 = raw[slot[d]];
  if (v < v0) atomicOr(status, kErrInput);
  out[start[d] + k] = msg_base[d] + (v >= v0 ? v - v0 : 0);
}

namespace {

__device__ __forceinline__ uint64_t seg_pieces(uint64_t n) { return n == 0 ? 1 : (n + kSegPiece - 1) / kSegPiece; }

// The shared-memory tree over the block's points (one per thread of kThreads); the sum ends
// in sp_[0].
template <int kThreads = kSegThreads>
__device__ __forceinline__ void seg_point_tree(uint32_t (*sp_)[32]) {
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) ge_store(sp_[threadIdx.x], ge_add(ge_load(sp_[threadIdx.x]), ge_load(sp_[threadIdx.x + h])));
    __syncthreads();
  }
}

// Device d's results from its exact limb sums (four 13-limb sums, then the bad count) and
// its point sum R (32 words): the scalars reduced mod q.  kPart selects what is written.
template <int kPart>
__device__ __forceinline__ void seg_write(const unsigned long long* tot, const uint32_t* R, uint32_t d, SegSums out) {
  if (kPart & kSegScalars) {
    if (threadIdx.x < 4) {
      unsigned long long sums[13];
      for (int k = 0; k < 13; ++k) sums[k] = tot[13 * threadIdx.x + k];
      const sc r = limb_sums_to_scalar(sums);
      uint32_t* dst = threadIdx.x == 0 ? out.Ew : threadIdx.x == 1 ? out.Sw : threadIdx.x == 2 ? out.Eu : out.Su;
      for (int k = 0; k < 8; ++k) dst[8 * (size_t)d + k] = r.v[k];
    }
    if (threadIdx.x == 0) out.bad[d] = (uint32_t)tot[kSegLimbWords - 1];
  }
  if (kPart & kSegPoints) {
    if (threadIdx.x < 32) out.Ru[32 * (size_t)d + threadIdx.x] = R[threadIdx.x];
  }
}

}  // namespace

// Per-device sums: weighted E_d = sum z e, S_d = sum z s (mod q), unit Eu_d, Su_d and the
// count of malformed entries (kPart = kSegScalars), or the unit point sum Ru_d (kSegPoints):
// two launches, each light enough for two blocks per SM.  One block per piece of at most
// kSegPiece entries of one device: a device of one piece gets its results here, the others
// leave exact partials (limb sums, which add without loss, and a point) for
// k_segment_combine.
template <int kPart, int kThreads>
__global__ void __launch_bounds__(kThreads, 512 / kThreads) k_segment_sums(const uint8_t* e, const uint8_t* s, const uint32_t* z,
                                                                 const uint32_t* pts, const uint8_t* badR,
                                                                 const uint8_t* badS, const uint64_t* start,
                                                                 const uint64_t* pieces,
                                                                 unsigned long long* piece_limbs, uint32_t* piece_R,
                                                                 SegSums out) {
  const uint64_t pc = pieces[blockIdx.x];
  const uint32_t d = (uint32_t)pc, piece = (uint32_t)(pc >> 32);
  const uint64_t dlo = start[d], dhi = start[d + 1];
  const uint64_t lo = dlo + (uint64_t)piece * kSegPiece, hi = min(lo + kSegPiece, dhi);
  const bool whole = seg_pieces(dhi - dlo) == 1;   // block-uniform
  if (kPart == kSegPoints) {
    __shared__ uint32_t sp_[kThreads][32];
    ge acc = ge_identity();
    for (uint64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
      if (badR[t] || badS[t]) continue;
      fe x, y, t2d;
      pts_load(pts + (size_t)kPtsWords * t, x, y, t2d);
      acc = ge_madd(acc, x, y, t2d);
    }
    ge_store(sp_[threadIdx.x], acc);
    seg_point_tree<kThreads>(sp_);
    if (!whole) {
      if (threadIdx.x < 32) piece_R[32 * (size_t)blockIdx.x + threadIdx.x] = sp_[0][threadIdx.x];
      return;
    }
    seg_write<kSegPoints>(nullptr, sp_[0], d, out);
    return;
  }
  acc13 Ew, Sw, Eu, Su;
  acc_zero(Ew); acc_zero(Sw); acc_zero(Eu); acc_zero(Su);
  uint32_t bad = 0;
  for (uint64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    if (badR[t] || badS[t]) {
      ++bad;
      continue;
    }
    const uint4* ep = reinterpret_cast<const uint4*>(e + 32 * t);
    const uint4* sp = reinterpret_cast<const uint4*>(s + 32 * t);
    const uint4 e0 = ep[0], e1 = ep[1], s0 = __ldg(sp), s1 = __ldg(sp + 1);
    const uint32_t ev[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
    const uint32_t sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
    const uint4 zz = __ldg(reinterpret_cast<const uint4*>(z) + t);
    const uint32_t zw[4] = {zz.x, zz.y, zz.z, zz.w};
    uint32_t pr[12];
    mul_4x8(pr, zw, ev);
    acc_add<12>(Ew, pr);
    mul_4x8(pr, zw, sv);
    acc_add<12>(Sw, pr);
    acc_add<8>(Eu, ev);
    acc_add<8>(Su, sv);
  }
  // 4 x 13 limb sums and the bad count: warp shuffles, then shared memory
  __shared__ unsigned long long red[kThreads / 32][kSegLimbWords];
  __shared__ unsigned long long tot[kSegLimbWords];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kSegLimbWords; ++k) {
    unsigned long long v;
    if (k < 13) v = Ew.v[k];
    else if (k < 26) v = Sw.v[k - 13];
    else if (k < 39) v = Eu.v[k - 26];
    else if (k < 52) v = Su.v[k - 39];
    else v = bad;
    warp_sum_u64(v);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kSegLimbWords; k += blockDim.x) {
    unsigned long long v = 0;
    for (int w = 0; w < kThreads / 32; ++w) v += red[w][k];
    tot[k] = v;
    if (!whole) piece_limbs[(size_t)blockIdx.x * kSegLimbWords + k] = v;
  }
  if (!whole) return;
  __syncthreads();
  seg_write<kSegScalars>(tot, nullptr, d, out);
}

void launch_segment_sums(unsigned n_pieces, cudaStream_t st, const uint8_t* e, const uint8_t* s, const uint32_t* z,
                         const uint32_t* pts, const uint8_t* badR, const uint8_t* badS, const uint64_t* start,
                         const uint64_t* pieces, unsigned long long* piece_limbs, uint32_t* piece_R, SegSums out) {
  // the point sums in blocks of 128 threads (four per SM by registers), so that other blocks
  // keep the SM busy through each block's tree
  k_segment_sums<kSegScalars, kSegThreads><<<n_pieces, kSegThreads, 0, st>>>(e, s, z, pts, badR, badS, start, pieces,
                                                                              piece_limbs, piece_R, out);
  k_segment_sums<kSegPoints, 128><<<n_pieces, 128, 0, st>>>(e, s, z, pts, badR, badS, start, pieces, piece_limbs,
                                                            piece_R, out);
}

// One block per device; devices of one piece have their results already.
__global__ void __launch_bounds__(kSegThreads) k_segment_combine(const uint64_t* start, const uint64_t* pfirst,
                                                                 const unsigned long long* piece_limbs,
                                                                 const uint32_t* piece_R, uint32_t n_dev,
                                                                 SegSums out) {
  const uint32_t d = blockIdx.x;
  if (d >= n_dev) return;
  const uint64_t np = seg_pieces(start[d + 1] - start[d]);
  if (np == 1) return;   // block-uniform
  const uint64_t p0 = pfirst[d];
  __shared__ unsigned long long tot[kSegLimbWords];
  for (int k = threadIdx.x; k < kSegLimbWords; k += blockDim.x) {
    unsigned long long v = 0;   // below 2^40 per piece: no overflow for any 32-bit entry count
    for (uint64_t j = 0; j < np; ++j) v += piece_limbs[(p0 + j) * kSegLimbWords + k];
    tot[k] = v;
  }
  ge acc = ge_identity();
  for (uint64_t j = threadIdx.x; j < np; j += blockDim.x) acc = ge_add(acc, ge_load(piece_R + 32 * (p0 + j)));
  __shared__ uint32_t sp_[kSegThreads][32];
  ge_store(sp_[threadIdx.x], acc);
  seg_point_tree(sp_);
  seg_write<kSegScalars | kSegPoints>(tot, sp_[0], d, out);
}

// Per-device, per-window weighted sums (the per-window form of the combined check, used for
// batches small enough that the MSM's Horner over windows is a large share of the latency):
// block b = d windows + w adds d_{t,w} e_t and d_{t,w} s_t over the well-formed entries of
// device d (a negative digit adds |d| (q - x)) and writes them reduced mod q to
// Ewd[8 (w n_dev + d)] and Swd[8 (w n_dev + d)].  The blocks of one device are consecutive,
// so its entries come from DRAM once and from L2 for the other windows.
__global__ void __launch_bounds__(kSegThreads) k_segment_window_sums(const uint8_t* e, const uint8_t* s,
                                                                     const uint32_t* z, const uint8_t* badR,
                                                                     const uint8_t* badS, const uint64_t* start,
                                                                     const uint64_t* order, uint32_t n_dev,
                                                                     MsmPlan pl, uint32_t* Ewd, uint32_t* Swd) {
  const uint32_t d = (uint32_t)order[blockIdx.x / (uint32_t)pl.windows];
  const int w = (int)(blockIdx.x % (uint32_t)pl.windows);
  acc13 ae, as;
  acc_zero(ae);
  acc_zero(as);
  for (uint64_t t = start[d] + threadIdx.x; t < start[d + 1]; t += blockDim.x) {
    if (badR[t] || badS[t]) continue;
    bool neg;
    const uint32_t dg = weight_digit(z, t, w, pl.c, neg);
    if (dg) add_window_terms(ae, as, e + 32 * t, s + 32 * t, dg, neg);
  }
  __shared__ unsigned long long red[kSegThreads / 32][26];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 26; ++k) {
    unsigned long long v = k < 13 ? ae.v[k] : as.v[k - 13];
    warp_sum_u64(v);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    unsigned long long sums[13];
    for (int k = 0; k < 13; ++k) {
      unsigned long long v = 0;
      for (int i = 0; i < kSegThreads / 32; ++i) v += red[i][13 * threadIdx.x + k];
      sums[k] = v;
    }
    const sc r = limb_sums_to_scalar(sums);
    uint32_t* dst = (threadIdx.x == 0 ? Ewd : Swd) + 8 * ((size_t)w * n_dev + d);
    for (int k = 0; k < 8; ++k) dst[k] = r.v[k];
  }
}

// Combined weighted check of window w over the devices not flagged (block w):
// [8](W_w - Wsub_w - P2_w - (sum_d S_{d,w}) G) = O, with W_w = sum_t d_{t,w} R_t over the whole
// batch, Wsub_w the same sum over the flagged devices' entries (none when Wsub is null) and
// P2_w = sum_d E_{d,w} Y_d already restricted to the devices not flagged.  A window that fails
// clears accept[0] (set to 1 beforehand).  The windows together imply the check with the full
// weights z_t.
__global__ void __launch_bounds__(kFinalThreads) k_multi_window_check(const uint32_t* W, const uint32_t* Wsub,
                                                                      const uint32_t* P2w, const uint32_t* Swd,
                                                                      const uint8_t* dev_flag, uint32_t n_dev,
                                                                      const uint32_t* tableG, uint8_t* accept) {
  const int w = blockIdx.x;
  __shared__ unsigned long long red[kFinalThreads / 32][13];
  __shared__ int8_t dig[64];
  __shared__ uint32_t pts_[kFinalThreads][32];
  acc13 a;
  acc_zero(a);
  for (uint32_t d = threadIdx.x; d < n_dev; d += blockDim.x)
    if (!(dev_flag && dev_flag[d])) acc_add<8>(a, Swd + 8 * ((size_t)w * n_dev + d));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 13; ++k) {
    unsigned long long v = a.v[k];
    warp_sum_u64(v);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long sums[13];
    for (int k = 0; k < 13; ++k) {
      unsigned long long v = 0;
      for (int i = 0; i < kFinalThreads / 32; ++i) v += red[i][k];
      sums[k] = v;
    }
    const sc S = limb_sums_to_scalar(sums);
    recode4(S.v, dig);
  }
  __syncthreads();
  ge term = threadIdx.x < kTableWindows ? table_pick(tableG, threadIdx.x, dig[threadIdx.x]) : ge_identity();
  ge_store(pts_[threadIdx.x], term);
  __syncthreads();
  for (int h = kTableWindows / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) ge_store(pts_[threadIdx.x], ge_add(ge_load(pts_[threadIdx.x]), ge_load(pts_[threadIdx.x + h])));
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ge p1 = ge_load(W + 32 * (size_t)w);
    if (Wsub) p1 = ge_sub(p1, ge_load(Wsub + 32 * (size_t)w));
    const ge diff = ge_sub(ge_sub(p1, ge_load(P2w + 32 * (size_t)w)), ge_load(pts_[0]));
    if (!ge_is_identity(ge_mul_cofactor(diff))) accept[0] = 0;
  }
}

// sum over the devices not skipped of [k_{d,w}] Y_d for every window w, from the devices'
// fixed-window tables: block (x, w) adds the table terms of its share of the (device, table
// window) pairs for the scalars k + 8 (w n + d), no doublings; per block one partial point
// at partial[33 (w gridDim.x + x)].
__global__ void __launch_bounds__(kPointThreads) k_table_msm_windows(const uint32_t* const* tabs, const uint32_t* k,
                                                                     const uint8_t* skip, uint32_t n,
                                                                     uint32_t* partial) {
  const int win = blockIdx.y;
  ge acc = ge_identity();
  const uint64_t total = (uint64_t)n * kTableWindows;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += stride) {
    const uint32_t d = (uint32_t)(p / kTableWindows);
    const int w = (int)(p % kTableWindows);
    if (skip && skip[d]) continue;
    const uint32_t* kd = k + 8 * ((size_t)win * n + d);
    int carry = 0, digit = 0;
    for (int i = 0; i <= w; ++i) digit = sc_digit4(kd, i, carry);
    if (digit) acc = ge_add(acc, table_pick(tabs[d], w, digit));
  }
  __shared__ uint32_t sp[kPointThreads][32];
  ge_store(sp[threadIdx.x], acc);
  __syncthreads();
  for (int h = kPointThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) ge_store(sp[threadIdx.x], ge_add(ge_load(sp[threadIdx.x]), ge_load(sp[threadIdx.x + h])));
    __syncthreads();
  }
  const size_t o = ((size_t)win * gridDim.x + blockIdx.x) * kPointPartialWords;
  if (threadIdx.x < 32) partial[o + threadIdx.x] = sp[0][threadIdx.x];
  if (threadIdx.x == 0) partial[o + 32] = 0;
}

// out[w] = the sum of the nblocks partial points of window w (block w).
__global__ void __launch_bounds__(kPointThreads) k_window_point_sums(const uint32_t* partial, uint32_t nblocks,
                                                                     uint32_t* out) {
  const int w = blockIdx.x;
  ge acc = ge_identity();
  for (uint32_t b = threadIdx.x; b < nblocks; b += blockDim.x)
    acc = ge_add(acc, ge_load(partial + ((size_t)w * nblocks + b) * kPointPartialWords));
  __shared__ uint32_t sp[kPointThreads][32];
  ge_store(sp[threadIdx.x], acc);
  __syncthreads();
  for (int h = kPointThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) ge_store(sp[threadIdx.x], ge_add(ge_load(sp[threadIdx.x]), ge_load(sp[threadIdx.x + h])));
    __syncthreads();
  }
  if (threadIdx.x < 32) out[32 * (size_t)w + threadIdx.x] = sp[0][threadIdx.x];
}

// Combined weighted check over the devices not flagged:
// [8](P1 - P2 - (sum_d S_d) G) = O, with P1 = sum_t z_t R_t and P2 = sum_d E_d Y_d already
// restricted to those devices.  One block.
__global__ void __launch_bounds__(kFinalThreads) k_multi_check(const uint32_t* P1, const uint32_t* P1sub,
                                                               const uint32_t* P2,
                                                               const uint32_t* Sw, const uint8_t* dev_flag,
                                                               uint32_t n_dev, const uint32_t* tableG,
                                                               uint8_t* accept) {
  __shared__ unsigned long long red[kFinalThreads / 32][13];
  __shared__ int8_t dig[64];
  __shared__ uint32_t pts_[kFinalThreads][32];
  acc13 a;
  acc_zero(a);
  for (uint32_t d = threadIdx.x; d < n_dev; d += blockDim.x)
    if (!(dev_flag && dev_flag[d])) acc_add<8>(a, Sw + 8 * (size_t)d);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 13; ++k) {
    unsigned long long v = a.v[k];
    warp_sum_u64(v);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long sums[13];
    for (int k = 0; k < 13; ++k) {
      unsigned long long v = 0;
      for (int w = 0; w < kFinalThreads / 32; ++w) v += red[w][k];
      sums[k] = v;
    }
    const sc S = limb_sums_to_scalar(sums);
    recode4(S.v, dig);
  }
  __syncthreads();
  ge term = threadIdx.x < kTableWindows ? table_pick(tableG, threadIdx.x, dig[threadIdx.x]) : ge_identity();
  ge_store(pts_[threadIdx.x], term);
  __syncthreads();
  for (int h = kTableWindows / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) ge_store(pts_[threadIdx.x], ge_add(ge_load(pts_[threadIdx.x]), ge_load(pts_[threadIdx.x + h])));
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ge p1 = ge_load(P1);
    if (P1sub) p1 = ge_sub(p1, ge_load(P1sub));
    const ge diff = ge_sub(ge_sub(p1, ge_load(P2)), ge_load(pts_[0]));
    accept[0] = ge_is_identity(ge_mul_cofactor(diff)) ? 1 : 0;
  }
}

// Per-device unit check [8](Ru - Eu Y_d - Su G) = O, one quad of lanes per device: 64 + 64
// quad-cooperative additions of entries of the window tables of Y_d and of G.  Devices that
// fail, or hold malformed entries, are flagged.
__global__ void __launch_bounds__(128) k_device_unit_check(const uint32_t* const* tabs, SegSums ss, uint32_t n_dev,
                                                           const uint32_t* tableG, uint8_t* dev_flag) {
  const uint32_t quad = ((uint32_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2;
  const uint32_t d = quad < n_dev ? quad : n_dev - 1;   // surplus quads repeat the last device
  const uint32_t* tY = tabs[d];
  const uint32_t* eu = ss.Eu + 8 * (size_t)d;
  const uint32_t* su = ss.Su + 8 * (size_t)d;
  // every lane runs every quad operation (full-mask shuffles)
  ge acc = ge_identity();
  int ce = 0, cs = 0;
  for (int w = 0; w < 64; ++w) {
    acc = ge_add_quad(acc, table_pick(tY, w, sc_digit4(eu, w, ce)));
    acc = ge_add_quad(acc, table_pick(tableG, w, sc_digit4(su, w, cs)));
  }
  const ge diff = ge_sub(ge_load(ss.Ru + 32 * (size_t)d), acc);
  const bool ok = ge_is_identity(ge_mul_cofactor(diff)) && ss.bad[d] == 0;
  if ((threadIdx.x & 3) == 0 && quad < n_dev) dev_flag[d] = ok ? 0 : 1;
}

// sum_d [k_d] Y_d over the keys not skipped, from their window tables: one (key, window)
// pair per step, 64 table entries per key, no doublings.  Per block: the partial sum in the
// decode kernel's partial format (kPointPartialWords, bad count 0).
__global__ void __launch_bounds__(kPointThreads) k_table_msm(const uint32_t* const* tabs, const uint32_t* k,
                                                             const uint8_t* skip, uint32_t n, uint32_t* partial) {
  ge acc = ge_identity();
  const uint64_t total = (uint64_t)n * kTableWindows;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += stride) {
    const uint32_t d = (uint32_t)(p / kTableWindows);
    const int w = (int)(p % kTableWindows);
    if (skip && skip[d]) continue;
    const uint32_t* kd = k + 8 * (size_t)d;
    int carry = 0, digit = 0;
    for (int i = 0; i <= w; ++i) digit = sc_digit4(kd, i, carry);
    if (digit) acc = ge_add(acc, table_pick(tabs[d], w, digit));
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

// Entry flags from device flags (entries of flagged devices are left out) or'ed with the
// malformed-point flags.  One block per device.
__global__ void k_device_to_entries(const uint8_t* dev_flag, const uint64_t* start, const uint8_t* badR,
                                    uint8_t* skip, int keep_flagged) {
  const uint32_t d = blockIdx.x;
  const uint8_t f = keep_flagged ? !dev_flag[d] : dev_flag[d];
  for (uint64_t t = start[d] + threadIdx.x; t < start[d + 1]; t += blockDim.x) skip[t] = (f || badR[t]) ? 1 : 0;
}

// Single-entry checks [8](R_t - e_t Y_d - s_t G) = O (Fig. 4 with |m| = 1) for every entry of
// the flagged devices, plus s_t canonical and R_t decodable.  Thread t belongs to flagged
// device k = the last k with fstart[k] <= t (binary search); R_t comes from the decoded point
// buffer and [e]Y_d from the table of device fl[k].
__global__ void __launch_bounds__(128) k_multi_entry_check(const MultiCheckArgs a) {
  const uint64_t total = a.fstart[a.nfl];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    uint32_t lo = 0, hi = a.nfl;   // fstart[lo] <= t < fstart[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (a.fstart[mid] <= t) lo = mid; else hi = mid;
    }
    const uint64_t g = a.seg_start[a.fl[lo]] + (t - a.fstart[lo]);
    bool ok = !a.badR[g] && !a.badS[g];
    if (ok) {
      const uint4* ep = reinterpret_cast<const uint4*>(a.e + 32 * g);
      const uint4* sp = reinterpret_cast<const uint4*>(a.s + 32 * g);
      const uint4 e0 = ep[0], e1 = ep[1], s0 = __ldg(sp), s1 = __ldg(sp + 1);
      const uint32_t e[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
      const uint32_t s[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
      ge R;
      fe t2d;
      pts_load(a.pts + (size_t)kPtsWords * g, R.X, R.Y, t2d);
      R.Z = fe_one();
      R.T = fe_mul(R.X, R.Y);
      const ge d = ge_sub(R, double_scalar_tables(e, s, a.tabs[a.fl[lo]], a.tableG));
      ok = ge_is_identity(ge_mul_cofactor(d));
    }
    a.inv[g] = ok ? 0 : 1;
  }
}

// k_multi_entry_check with eight lanes per entry; surplus groups repeat the last entry and
// do not write.
__global__ void __launch_bounds__(128) k_multi_entry_check_group(const MultiCheckArgs a) {
  const uint64_t total = a.fstart[a.nfl];
  if (total == 0) return;   // grid-uniform
  const uint64_t grp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  const uint64_t t = grp < total ? grp : total - 1;
  uint32_t lo = 0, hi = a.nfl;   // fstart[lo] <= t < fstart[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a.fstart[mid] <= t) lo = mid; else hi = mid;
  }
  const uint64_t g = a.seg_start[a.fl[lo]] + (t - a.fstart[lo]);
  const bool ok = entry_check8(a.e + 32 * g, a.s + 32 * g, a.pts + (size_t)kPtsWords * g, a.badR[g] || a.badS[g],
                               a.tabs[a.fl[lo]], a.tableG);
  if ((threadIdx.x & 7) == 0 && grp < total) a.inv[g] = ok ? 0 : 1;
}

// Per flagged device k: 1 if any of its entries is flagged in inv.
__global__ void k_segment_any(const uint8_t* inv, const uint64_t* seg_start, const uint32_t* fl, uint8_t* out) {
  const uint32_t d = fl[blockIdx.x];
  int any = 0;
  for (uint64_t t = seg_start[d] + threadIdx.x; t < seg_start[d + 1]; t += blockDim.x) any |= inv[t];
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) out[blockIdx.x] = any ? 1 : 0;
}

void launch_epoch_seeds_multi(int inst, unsigned grid, unsigned block, cudaStream_t st, const DsNode* ds_all,
                              const uint32_t* ds_off, const uint64_t* seed_off, const uint64_t* e0, uint32_t n_dev,
                              uint32_t* seeds, uint32_t* status) {
  if (inst == kInstAes)
    k_epoch_seeds_multi<kInstAes><<<grid, block, 0, st>>>(ds_all, ds_off, seed_off, e0, n_dev, seeds, status);
  else
    k_epoch_seeds_multi<kInstSha><<<grid, block, 0, st>>>(ds_all, ds_off, seed_off, e0, n_dev, seeds, status);
}

// Staging of requests whose inputs are page-locked host memory the device reads directly:
// the blocks stride over a table of chunks (source, destination, bytes; no chunk is longer
// than kGatherChunk, so a large request spreads over many blocks), each copying its chunk in
// 16-byte words where source and destination agree modulo 16, 8-byte words where they agree
// modulo 8, and otherwise in 4-byte destination words, each assembled from the two aligned
// source words it straddles.  (The entries of consecutive requests are back to back in the
// batch, so the destination's alignment is not the source's in general.)
template <typename W>
__device__ __forceinline__ void copy_words(uint8_t* dst, const uint8_t* src, uint64_t len) {
  constexpr uint64_t B = sizeof(W);
  const uint64_t lead = (B - (reinterpret_cast<uintptr_t>(dst) & (B - 1))) & (B - 1);
  const uint64_t head = len < lead ? len : lead;
  if (threadIdx.x < head) dst[threadIdx.x] = src[threadIdx.x];
  const uint64_t words = (len - head) / B;
  const W* s = reinterpret_cast<const W*>(src + head);
  W* d = reinterpret_cast<W*>(dst + head);
  uint64_t i = threadIdx.x;
  for (; i + 3 * blockDim.x < words; i += 4 * blockDim.x) {   // four loads in flight per thread
    const W a = s[i], b = s[i + blockDim.x], c = s[i + 2 * blockDim.x], e = s[i + 3 * blockDim.x];
    d[i] = a;
    d[i + blockDim.x] = b;
    d[i + 2 * blockDim.x] = c;
    d[i + 3 * blockDim.x] = e;
  }
  for (; i < words; i += blockDim.x) d[i] = s[i];
  const uint64_t done = head + words * B;
  if (threadIdx.x < len - done) dst[done + threadIdx.x] = src[done + threadIdx.x];
}

// dst in aligned 4-byte words whatever the source's alignment: word w of the destination is
// bytes m .. m+3 of the source's aligned words w, w+1 (m = the source's misalignment).  The
// second word may extend past the source's last byte, but never past its aligned 4-byte word,
// so it stays on the same page.
__device__ __forceinline__ void copy_shifted(uint8_t* dst, const uint8_t* src, uint64_t len) {
  const uint64_t lead = (4 - (reinterpret_cast<uintptr_t>(dst) & 3)) & 3;
  const uint64_t head = len < lead ? len : lead;
  if (threadIdx.x < head) dst[threadIdx.x] = src[threadIdx.x];
  dst += head;
  src += head;
  len -= head;
  const uint32_t m = (uint32_t)(reinterpret_cast<uintptr_t>(src) & 3);
  const uint32_t* s0 = reinterpret_cast<const uint32_t*>(src - m);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  const uint64_t words = len >> 2;
  for (uint64_t w = threadIdx.x; w < words; w += blockDim.x) {
    const uint32_t lo = s0[w];
    d[w] = m ? __funnelshift_r(lo, s0[w + 1], 8 * m) : lo;
  }
  const uint64_t done = words << 2;
  if (threadIdx.x < len - done) dst[done + threadIdx.x] = src[done + threadIdx.x];
}

__global__ void __launch_bounds__(256) k_stage_gather(const GatherRegion* regions, uint32_t n_regions) {
  for (uint32_t g = blockIdx.x; g < n_regions; g += gridDim.x) {
    const GatherRegion r = regions[g];
    const uintptr_t x = reinterpret_cast<uintptr_t>(r.src) ^ reinterpret_cast<uintptr_t>(r.dst);
    if ((x & 15) == 0) {
      copy_words<uint4>(r.dst, r.src, r.bytes);
    } else if ((x & 7) == 0) {
      copy_words<uint2>(r.dst, r.src, r.bytes);
    } else {
      copy_shifted(r.dst, r.src, r.bytes);
    }
  }
}

}  // namespace poslo
