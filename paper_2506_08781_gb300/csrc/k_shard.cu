// Partials of one shard of a log and their combination (a log split over several GPUs).
//
// A log of one signer split into contiguous index ranges is verified shard by shard: each
// shard reduces its entries to the aggregate of Fig. 3a / Fig. 4 AVer before the group check,
//   e~ = sum_t e_t mod q,  s~ = sum_t s_t mod q,  R~ = sum_t R_t
// (weighted: every term times the verifier's z_t of its global index), and the check itself
// runs once over the sum of the shards' partials.  Scalar sums mod q and point sums are not
// reductions a collective library offers, so the shards exchange these records and each
// combines them.
//
// Record (54 words, the layout of poslo_partial): e~ (8 words, LE limbs), s~ (8), R~ as an
// extended point X, Y, Z, T (8 each, every coordinate fully reduced below p), then
// first_index (2), n (2), malformed (1), agg_mode (1); the kernels read and write e~, s~, R~
// (words 0..47) and malformed (word kShardBadWord = 52); the host fills in the rest.
#include "common.cuh"
#include "compact.cuh"

namespace poslo {

// One block: the shard's record from the hashing partials (e~, s~ and the count of
// non-canonical s_t), the summed point R (unit sum or MSM result, 32 words) and the count
// of undecodable R_t.  For POSLO-C the aggregate s~ is given instead (s_given, 32 bytes;
// non-canonical counts as malformed).
__global__ void __launch_bounds__(kShardThreads) k_partial_out(const unsigned long long* hash_partial, uint32_t nhash,
                                                              const uint8_t* s_given, const uint32_t* R,
                                                              const uint32_t* point_bad, uint32_t* out) {
  __shared__ unsigned long long sums[kPartialWords];
  const int tid = threadIdx.x;
  if (tid < kPartialWords) sums[tid] = 0;
  __syncthreads();
  // word w of every block's partial, the blocks split over kShardThreads / kPartialWords threads
  constexpr int kLanesPerWord = kShardThreads / kPartialWords;
  if (tid < kLanesPerWord * kPartialWords) {
    const int w = tid % kPartialWords, lane = tid / kPartialWords;
    unsigned long long v = 0;
    for (uint32_t b = lane; b < nhash; b += kLanesPerWord) v += hash_partial[(size_t)b * kPartialWords + w];
    atomicAdd(&sums[w], v);
  }
  __syncthreads();
  if (tid == 0) {
    const sc e = limb_sums_to_scalar(sums);
    sc s;
    unsigned long long bad = sums[26] + (point_bad ? *point_bad : 0u);
    if (s_given) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        s.v[k] = s_given[4 * k] | (s_given[4 * k + 1] << 8) | (s_given[4 * k + 2] << 16) |
                 ((uint32_t)s_given[4 * k + 3] << 24);
      if (!sc_is_canonical(s.v)) {
        bad += 1;
#pragma unroll
        for (int k = 0; k < 8; ++k) s.v[k] = 0;
      }
    } else {
      s = limb_sums_to_scalar(sums + 13);
    }
    const ge P = ge_load(R);
    const fe X = fe_canon(P.X), Y = fe_canon(P.Y), Z = fe_canon(P.Z), T = fe_canon(P.T);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      out[k] = e.v[k];
      out[8 + k] = s.v[k];
      out[16 + k] = X.v[k];
      out[24 + k] = Y.v[k];
      out[32 + k] = Z.v[k];
      out[40 + k] = T.v[k];
    }
    out[kShardBadWord] = bad > 0xffffffffull ? 0xffffffffu : (uint32_t)bad;
  }
}

// One block: sums the records of nparts shards (e~ and s~ mod q, R~ by point addition, the
// malformed counts), writes the total as a record, and evaluates the cofactored check
// [8](R~ - [e~]Y - [s~]G) = O with the two fixed-window tables (128 terms summed by a
// shared-memory tree).  accept[0] = 1 iff no shard had a malformed entry, every record's
// point coordinates are below p with Z != 0 and lies on the curve, the key decoded, and the
// equation holds.
__global__ void __launch_bounds__(kShardThreads) k_combine_check(const uint32_t* parts, uint32_t nparts,
                                                                const uint32_t* tableY, const uint32_t* tableG,
                                                                const uint32_t* status, uint32_t* total,
                                                                uint8_t* accept) {
  __shared__ int8_t dig_e[64], dig_s[64];
  __shared__ uint32_t pts_[kShardThreads][32];
  __shared__ uint32_t sR[32];
  __shared__ uint32_t well_formed;
  const int tid = threadIdx.x;
  // a single call's worth of arithmetic from compact (out-of-line) field and point
  // operations: the kernel's code is fetched cold on every launch.  Thread 0 sums the
  // records, thread 32 (another warp, so the two run side by side) checks them.
  __shared__ uint32_t valid_records;
  if (tid == 32) {
    bool ok = true;
#pragma unroll 1
    for (uint32_t i = 0; i < nparts; ++i) {
      const uint32_t* p = parts + (size_t)i * kShardWords;
      if (!sc_is_canonical(p) || !sc_is_canonical(p + 8)) ok = false;
      // coordinates below p, Z != 0, XY = ZT and -X^2 + Y^2 = Z^2 + d T^2 (the extended curve)
      fe c[4];
      bool canon = true;
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int k = 0; k < 8; ++k) c[q].v[k] = p[16 + 8 * q + k];
        const fe r = compact::canon(c[q]);
#pragma unroll
        for (int k = 0; k < 8; ++k) canon &= r.v[k] == c[q].v[k];
      }
      const fe XX = compact::sq(c[0]), YY = compact::sq(c[1]), ZZ = compact::sq(c[2]), TT = compact::sq(c[3]);
      const bool on = !fe_is_zero(c[2]) && fe_eq(compact::mul(c[0], c[1]), compact::mul(c[2], c[3])) &&
                      fe_eq(fe_sub(YY, XX), fe_add(ZZ, compact::mul(fe_d(), TT)));
      if (!canon || !on) ok = false;
    }
    valid_records = ok ? 1u : 0u;
  }
  __shared__ unsigned long long bad_sum;
  if (tid == 0) {
    sc e, s;
#pragma unroll
    for (int k = 0; k < 8; ++k) e.v[k] = s.v[k] = 0;
    ge R = ge_identity();
    unsigned long long bad = 0;
#pragma unroll 1
    for (uint32_t i = 0; i < nparts; ++i) {
      const uint32_t* p = parts + (size_t)i * kShardWords;
      sc ei, si;
      ge Pi;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        ei.v[k] = p[k];
        si.v[k] = p[8 + k];
        Pi.X.v[k] = p[16 + k];
        Pi.Y.v[k] = p[24 + k];
        Pi.Z.v[k] = p[32 + k];
        Pi.T.v[k] = p[40 + k];
      }
      e = sc_add(e, ei);
      s = sc_add(s, si);
      R = i == 0 ? Pi : compact::add(R, Pi);
      bad += p[kShardBadWord];
    }
    recode4(e.v, dig_e);
    recode4(s.v, dig_s);
    ge_store(sR, R);
    bad_sum = bad;
    if (total) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        total[k] = e.v[k];
        total[8 + k] = s.v[k];
      }
      total[kShardBadWord] = bad > 0xffffffffull ? 0xffffffffu : (uint32_t)bad;
    }
  }
  __syncthreads();
  if (tid < 4 && total) {   // R~ in canonical coordinates, one coordinate per thread
    fe c;
#pragma unroll
    for (int k = 0; k < 8; ++k) c.v[k] = sR[8 * tid + k];
    const fe r = compact::canon(c);
#pragma unroll
    for (int k = 0; k < 8; ++k) total[16 + 8 * tid + k] = r.v[k];
  }
  if (tid == 0) well_formed = (valid_records && bad_sum == 0) ? 1u : 0u;
  __syncthreads();
  const ge term = tid < 64 ? table_pick(tableY, tid, dig_e[tid]) : table_pick(tableG, tid - 64, dig_s[tid - 64]);
  ge_store(pts_[tid], term);
  __syncthreads();
  // e~Y + s~G: the 128 terms summed by quads
  static_assert(kShardThreads == 128, "one term per thread");
  __shared__ uint32_t qs_[32][32];
  compact::quad_sum128(pts_, qs_);
  // [8](R~ - e~Y - s~G) by the first warp's quads (all of them compute it)
  if (tid < 32) {
    ge d = ge_add_quad(ge_load(sR), ge_neg(ge_load(qs_[0])));
#pragma unroll 1
    for (int i = 0; i < 3; ++i) d = ge_dbl_quad(d);
    if (tid == 0) accept[0] = (ge_is_identity(d) && well_formed && (*status & kErrKey) == 0) ? 1 : 0;
  }
}

}  // namespace poslo
