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
  if (tid == 0) {
    sc e, s;
#pragma unroll
    for (int k = 0; k < 8; ++k) e.v[k] = s.v[k] = 0;
    ge R = ge_identity();
    unsigned long long bad = 0;
    bool ok = true;
    for (uint32_t i = 0; i < nparts; ++i) {
      const uint32_t* p = parts + (size_t)i * kShardWords;
      sc ei, si;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        ei.v[k] = p[k];
        si.v[k] = p[8 + k];
      }
      if (!sc_is_canonical(ei.v) || !sc_is_canonical(si.v)) ok = false;
      ge Pi;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        Pi.X.v[k] = p[16 + k];
        Pi.Y.v[k] = p[24 + k];
        Pi.Z.v[k] = p[32 + k];
        Pi.T.v[k] = p[40 + k];
      }
      // coordinates below p, Z != 0, XY = ZT and -X^2 + Y^2 = Z^2 + d T^2 (the extended curve)
      const fe X = Pi.X, Y = Pi.Y, Z = Pi.Z, T = Pi.T;
      bool canon = true;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        canon &= fe_canon(X).v[k] == X.v[k] && fe_canon(Y).v[k] == Y.v[k] && fe_canon(Z).v[k] == Z.v[k] &&
                 fe_canon(T).v[k] == T.v[k];
      }
      const fe XX = fe_sq(X), YY = fe_sq(Y), ZZ = fe_sq(Z), TT = fe_sq(T);
      const bool on = !fe_is_zero(Z) && fe_eq(fe_mul(X, Y), fe_mul(Z, T)) &&
                      fe_eq(fe_sub(YY, XX), fe_add(ZZ, fe_mul(fe_d(), TT)));
      if (!canon || !on) ok = false;
      e = sc_add(e, ei);
      s = sc_add(s, si);
      R = ge_add(R, Pi);
      bad += p[kShardBadWord];
    }
    recode4(e.v, dig_e);
    recode4(s.v, dig_s);
    ge_store(sR, R);
    well_formed = (ok && bad == 0) ? 1u : 0u;
    if (total) {
      const fe X = fe_canon(R.X), Y = fe_canon(R.Y), Z = fe_canon(R.Z), T = fe_canon(R.T);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        total[k] = e.v[k];
        total[8 + k] = s.v[k];
        total[16 + k] = X.v[k];
        total[24 + k] = Y.v[k];
        total[32 + k] = Z.v[k];
        total[40 + k] = T.v[k];
      }
      total[kShardBadWord] = bad > 0xffffffffull ? 0xffffffffu : (uint32_t)bad;
    }
  }
  __syncthreads();
  const ge term = tid < 64 ? table_pick(tableY, tid, dig_e[tid]) : table_pick(tableG, tid - 64, dig_s[tid - 64]);
  ge_store(pts_[tid], term);
  __syncthreads();
  for (int h = kShardThreads / 2; h > 0; h >>= 1) {
    if (tid < h) ge_store(pts_[tid], ge_add(ge_load(pts_[tid]), ge_load(pts_[tid + h])));
    __syncthreads();
  }
  if (tid == 0) {
    const ge diff = ge_sub(ge_load(sR), ge_load(pts_[0]));
    const bool ok = ge_is_identity(ge_mul_cofactor(diff)) && well_formed && (*status & kErrKey) == 0;
    accept[0] = ok ? 1 : 0;
  }
}

}  // namespace poslo
