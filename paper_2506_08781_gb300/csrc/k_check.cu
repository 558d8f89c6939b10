// Per-entry checks, the reference multi-scalar multiplication, masked sums and ordered compaction used by Distill.
#include "common.cuh"
#include "compact.cuh"

namespace poslo {

__global__ void __launch_bounds__(128) k_entry_check(const CheckArgs a) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.n; t += stride) {
    const uint4* ep = reinterpret_cast<const uint4*>(a.e + 32 * t);
    const uint4* sp = reinterpret_cast<const uint4*>(a.s + 32 * t);
    const uint4* rp = reinterpret_cast<const uint4*>(a.R + 32 * t);
    const uint4 e0 = ep[0], e1 = ep[1], s0 = __ldg(sp), s1 = __ldg(sp + 1), r0 = __ldg(rp), r1 = __ldg(rp + 1);
    const uint32_t e[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
    const uint32_t s[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
    const uint32_t rb[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    ge R;
    bool ok = ge_decode(rb, R);
    ok &= sc_is_canonical(s);
    if (ok) {
      const ge d = ge_sub(R, double_scalar_tables(e, s, a.tableY, a.tableG));
      ok = ge_is_identity(ge_mul_cofactor(d));
    }
    a.invalid[t] = ok ? 0 : 1;
  }
}

// Eight lanes per entry (entry_check8); surplus groups repeat the last entry and do not write.
__global__ void __launch_bounds__(128) k_entry_check_group(const DirectCheckArgs a) {
  const uint64_t grp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  if (a.n == 0) return;   // grid-uniform
  const uint64_t t = grp < a.n ? grp : a.n - 1;
  const bool ok = entry_check8(a.e + 32 * t, a.s + 32 * t, a.pts + (size_t)kPtsWords * t, a.badR[t] || a.badS[t],
                               a.tableY, a.tableG);
  if ((threadIdx.x & 7) == 0 && grp < a.n) a.invalid[t] = ok ? 0 : 1;
}

__global__ void __launch_bounds__(kHashThreads) k_sum_scalars(const uint8_t* s, uint64_t n, const uint8_t* skip,
                                                             unsigned long long* partial) {
  acc13 acc;
  acc_zero(acc);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    if (skip && skip[t]) continue;
    const uint4* sp = reinterpret_cast<const uint4*>(s + 32 * t);
    const uint4 s0 = __ldg(sp), s1 = __ldg(sp + 1);
    const uint32_t v[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
    acc_add<8>(acc, v);
  }
  __shared__ unsigned long long red[kHashThreads / 32][13];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 13; ++k) {
    unsigned long long v = acc.v[k];
    warp_sum_u64(v);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 13) {
    unsigned long long v = 0;
    for (int w = 0; w < kHashThreads / 32; ++w) v += red[w][threadIdx.x];
    partial[(uint64_t)blockIdx.x * 13 + threadIdx.x] = v;
  }
}

__global__ void k_reduce_scalars(const unsigned long long* partial, uint32_t nparts, uint8_t* out) {
  __shared__ unsigned long long sums[13];
  if (threadIdx.x < 13) sums[threadIdx.x] = 0;
  __syncthreads();
  // word w of every part, the parts split over blockDim.x / 13 threads per word
  const uint32_t lanes = blockDim.x / 13;
  if (threadIdx.x < lanes * 13) {
    const uint32_t w = threadIdx.x % 13, lane = threadIdx.x / 13;
    unsigned long long v = 0;
    for (uint32_t b = lane; b < nparts; b += lanes) v += partial[(size_t)b * 13 + w];
    atomicAdd(&sums[w], v);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const sc r = limb_sums_to_scalar(sums);
    for (int k = 0; k < 8; ++k) {
      out[4 * k] = (uint8_t)r.v[k]; out[4 * k + 1] = (uint8_t)(r.v[k] >> 8);
      out[4 * k + 2] = (uint8_t)(r.v[k] >> 16); out[4 * k + 3] = (uint8_t)(r.v[k] >> 24);
    }
  }
}

__global__ void k_sum_encode(const uint32_t* partial, uint32_t nparts, uint32_t* point_out, uint8_t* enc_out,
                             uint32_t* bad_out) {
  __shared__ uint32_t sp[kFinalThreads][32];
  __shared__ uint32_t sbad;
  const int tid = threadIdx.x;
  if (tid == 0) sbad = 0;
  __syncthreads();
  // once per call: compact (out-of-line) point operations, the code being fetched cold
  ge acc = ge_identity();
  uint32_t bad = 0;
#pragma unroll 1
  for (uint32_t b = tid; b < nparts; b += kFinalThreads) {
    acc = compact::add(acc, ge_load(partial + (size_t)b * kPointPartialWords));
    bad += partial[(size_t)b * kPointPartialWords + 32];
  }
  ge_store(sp[tid], acc);
  atomicAdd(&sbad, bad);
  __syncthreads();
#pragma unroll 1
  for (int h = kFinalThreads / 2; h > 0; h >>= 1) {
    if (tid < h) ge_store(sp[tid], compact::add(ge_load(sp[tid]), ge_load(sp[tid + h])));
    __syncthreads();
  }
  if (tid == 0) {
    const ge r = ge_load(sp[0]);
    if (point_out) ge_store(point_out, r);
    if (enc_out) {
      uint32_t w[8];
      compact::encode(r, w);
      for (int k = 0; k < 8; ++k) {
        enc_out[4 * k] = (uint8_t)w[k]; enc_out[4 * k + 1] = (uint8_t)(w[k] >> 8);
        enc_out[4 * k + 2] = (uint8_t)(w[k] >> 16); enc_out[4 * k + 3] = (uint8_t)(w[k] >> 24);
      }
    }
    if (bad_out) *bad_out = sbad;
  }
}

// Encode one extended point (32 words) to its 32-byte compressed form.
__global__ void k_encode_ext(const uint32_t* point, uint8_t* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t w[8];
  compact::encode(ge_load(point), w);
  for (int k = 0; k < 8; ++k) {
    out[4 * k] = (uint8_t)w[k]; out[4 * k + 1] = (uint8_t)(w[k] >> 8);
    out[4 * k + 2] = (uint8_t)(w[k] >> 16); out[4 * k + 3] = (uint8_t)(w[k] >> 24);
  }
}

// Ordered compaction across many blocks: block b owns flags [b*kFlagChunk, (b+1)*kFlagChunk).
// Pass 1 counts, pass 2 scans the counts (one block), pass 3 writes first_index + t of
// every flagged t in ascending order.
__global__ void __launch_bounds__(1024) k_flag_count(const uint8_t* flags, uint64_t n, uint32_t* blockcnt) {
  __shared__ uint32_t tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  const uint64_t lo = (uint64_t)blockIdx.x * kFlagChunk;
  uint32_t c = 0;
  for (uint64_t t = lo + threadIdx.x; t < lo + kFlagChunk && t < n; t += blockDim.x) c += flags[t] ? 1u : 0u;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) atomicAdd(&tot, c);
  __syncthreads();
  if (threadIdx.x == 0) blockcnt[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_flag_scan(const uint32_t* blockcnt, uint32_t nblocks, uint64_t* blockoff,
                                                   uint64_t* total) {
  __shared__ uint64_t warp_sums[32];
  __shared__ uint64_t base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t c0 = 0; c0 < nblocks; c0 += blockDim.x) {
    const uint32_t b = c0 + threadIdx.x;
    const uint64_t v = b < nblocks ? blockcnt[b] : 0;
    uint64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    const uint64_t excl = base + (warp ? warp_sums[warp - 1] : 0) + incl - v;
    if (b < nblocks) blockoff[b] = excl;
    __syncthreads();
    if (threadIdx.x == 0) base += warp_sums[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = base;
}

__global__ void __launch_bounds__(1024) k_flag_scatter(const uint8_t* flags, uint64_t n, uint64_t first_index,
                                                      const uint64_t* blockoff, uint64_t* out, uint64_t cap) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint64_t base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) base = blockoff[blockIdx.x];
  __syncthreads();
  const uint64_t lo = (uint64_t)blockIdx.x * kFlagChunk;
  for (uint64_t c0 = lo; c0 < lo + kFlagChunk && c0 < n; c0 += blockDim.x) {
    const uint64_t t = c0 + threadIdx.x;
    const bool f = t < n && t < lo + kFlagChunk && flags[t] != 0;
    const uint32_t m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_tot[warp] = __popc(m);
    __syncthreads();
    uint64_t off = base;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    off += __popc(m & ((1u << lane) - 1u));
    if (f && off < cap) out[off] = first_index + t;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t tot = 0;
      for (int w = 0; w < 32; ++w) tot += warp_tot[w];
      base += tot;
    }
    __syncthreads();
  }
}

}  // namespace poslo
