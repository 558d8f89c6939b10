// Shared device code of the POSLO verification path (sm_103a): argument structs, per-entry
// helpers and the declarations of every kernel (defined in k_verify.cu, k_check.cu,
// k_signer.cu).
//
//   k_epoch_seeds   x_0[i] = SRet(ds, i), hoisted once per epoch (Fig. 2a; the paper's
//                   Agg-eKeys recomputes it in every thread, Fig. 6)
//   k_hash          x_t = PRF_0(x_0[i] || j), e_t = H(m_t || x_t) mod q, and the scalar
//                   aggregates sum e_t, sum s_t (or their weighted forms)
//   k_points        strict decoding of R_t and the unit aggregate sum R_t
//   k_table_*       fixed-window tables {d 16^w P : d = 1..8, w = 0..63} for the check
//   k_finalize      reduce the partial aggregates and evaluate [8](R - eY - sG) = O
#pragma once
#include <cstdint>

#include "aes128.cuh"
#include "ge25519.cuh"
#include "sc25519.cuh"
#include "sha256.cuh"

namespace poslo {


constexpr int kHashThreads = 128;
#ifndef POSLO_HASH_MIN_BLOCKS
#define POSLO_HASH_MIN_BLOCKS 3   // resident blocks per SM the hash kernel is compiled for
#endif
constexpr int kPointThreads = 128;
// Block size of the short kernels that run beside the decoding (weights, counting sort):
// small enough that one of their blocks fits in the registers the three resident decoding
// blocks of an SM leave free, so they progress during the decoding instead of after it.
#ifndef POSLO_SIDE_THREADS
#define POSLO_SIDE_THREADS 128
#endif
constexpr int kSideThreads = POSLO_SIDE_THREADS;
constexpr int kTableWindows = 64;   // 4-bit windows over 256 bits
constexpr int kTableDigits = 8;     // signed digits |d| in 1..8
constexpr int kTableWords = kTableWindows * kTableDigits * 32;   // one table: 64 KB

// Device-side error codes written to the context's status word.
enum : uint32_t { kErrNone = 0, kErrSeed = 1, kErrKey = 2, kErrPoint = 4, kErrTimeout = 8, kErrInput = 16 };

struct DsNode { uint32_t d, i; uint32_t seed[4]; };   // seed as 4 big-endian words

// ----------------------------------------------------------------------------------------
// Epoch seeds: SRet per epoch.
// ----------------------------------------------------------------------------------------


// ----------------------------------------------------------------------------------------
// Per-entry hashing and scalar aggregation.
// ----------------------------------------------------------------------------------------
struct HashArgs {
  const uint8_t* msgs;
  const uint64_t* offs;        // n+1
  uint64_t base_off;           // offs[] value that corresponds to msgs[0]
  uint64_t n;
  uint64_t first_index;        // global index of entry 0
  uint64_t e0;                 // epoch of seeds[0]
  uint32_t n2;
  uint32_t n2_log2;            // log2(n2) if n2 is a power of two, else 0xffffffff
  const uint32_t* seeds;       // x_0 per epoch, 4 BE words each
  uint8_t* e_out;              // optional: n*32 bytes
  const uint8_t* s;            // optional (F): n*32 scalars to check and aggregate
  uint32_t weighted;           // 1: aggregate z_t e_t and z_t s_t
  uint32_t zpre[10];           // weighted: BE words of "POSLO-Z" || verifier_seed || (byte 39 = 0)
  uint32_t* z_out;             // optional (weighted): n*4 words of z_t
  const uint32_t* z_in;        // optional (weighted): z_t already computed (k_weights); read, not hashed
  uint8_t* sbad_out;           // optional: n bytes, 1 = s_t is not canonical
  unsigned long long* partial; // per block: 13 u64 limb sums of e, 13 of s, 1 bad count (27 u64)
  uint32_t* status;            // device status word (kErrInput for decreasing offsets)
  // multi-device batches (n_seg > 0): entry t belongs to the device d with
  // seg_start[d] <= t < seg_start[d+1]; its index in that signer's log is
  // seg_first[d] + t - seg_start[d], and its epoch seeds start at seeds[seg_seed_off[d]]
  // (epoch seg_e0[d]).  The weight z_t then uses the batch position t, unique across devices.
  uint32_t n_seg;
  const uint64_t* seg_start;
  const uint64_t* seg_first;
  const uint64_t* seg_seed_off;
  const uint64_t* seg_e0;
  const uint32_t* seg_n2;
};

// Largest d with start[d] <= t, for start[0] = 0 <= t < start[n].
__device__ __forceinline__ uint32_t segment_of(const uint64_t* start, uint32_t n, uint64_t t) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (start[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

constexpr int kPartialWords = 27;

// Big-endian word at byte offset o (a multiple of 4) of the padded SHA-256 input
// m || x || 0x80 || 0.. || bitlen, for the blocks that are not wholly message bytes.
struct EntryStream {
  const uint32_t* base;   // 4-byte aligned pointer at or before the first message byte
  uint32_t sel;           // PRMT selector realigning two loaded words to the message
  uint32_t sh_nz;         // 1 if the message is not 4-byte aligned
  uint32_t L;             // message length in bytes
  int32_t kmax;           // last loadable word index (the word holding the last byte)
  uint32_t a;             // L rounded down to a multiple of 4
  uint32_t S[5];          // x || 0x80 shifted by L mod 4 bytes, as the words at a, a+4, ...
};

__device__ __forceinline__ uint32_t load_msg_word(const EntryStream& es, uint32_t k) {
  const uint32_t lo = __ldg(es.base + k);
  const uint32_t hi = __ldg(es.base + k + es.sh_nz);
  return __byte_perm(lo, hi, es.sel);
}

__device__ __forceinline__ uint32_t stream_word(const EntryStream& es, uint32_t o) {
  uint32_t mw = 0;
  if (es.L > 0) {
    const int32_t k = (int32_t)(o >> 2);
    const uint32_t k0 = (uint32_t)min(k, es.kmax);
    const uint32_t k1 = (uint32_t)min(k + (int32_t)es.sh_nz, es.kmax);
    mw = __byte_perm(__ldg(es.base + k0), __ldg(es.base + k1), es.sel);
    // keep the leading min(4, max(0, L - o)) bytes
    const int32_t keep = min(4, max(0, (int32_t)es.L - (int32_t)o));
    mw &= __funnelshift_lc(0u, 0xffffffffu, 8u * (uint32_t)(4 - keep));
  }
  const int32_t kk = ((int32_t)o - (int32_t)es.a) >> 2;
  uint32_t tw = 0;
  tw = kk == 0 ? es.S[0] : tw;
  tw = kk == 1 ? es.S[1] : tw;
  tw = kk == 2 ? es.S[2] : tw;
  tw = kk == 3 ? es.S[3] : tw;
  tw = kk == 4 ? es.S[4] : tw;
  return mw | tw;
}

// The stream m || x || 0x80 || 0... of one entry (x given as 4 big-endian words).
__device__ __forceinline__ EntryStream entry_stream(const uint8_t* m, uint32_t L, const uint32_t x[4]) {
  EntryStream es;
  const uintptr_t p = reinterpret_cast<uintptr_t>(m);
  const uint32_t sh = (uint32_t)(p & 3u);
  es.base = reinterpret_cast<const uint32_t*>(p - sh);
  es.sel = (sh + 3) | ((sh + 2) << 4) | ((sh + 1) << 8) | (sh << 12);
  es.sh_nz = sh != 0;
  es.L = L;
  es.kmax = L > 0 ? (int32_t)((L + sh - 1) >> 2) : 0;
  const uint32_t r = L & 3u;
  es.a = L - r;
  const uint32_t sr = 8u * r;
  es.S[0] = __funnelshift_r(x[0], 0u, sr);
  es.S[1] = __funnelshift_r(x[1], x[0], sr);
  es.S[2] = __funnelshift_r(x[2], x[1], sr);
  es.S[3] = __funnelshift_r(x[3], x[2], sr);
  es.S[4] = __funnelshift_r(0x80000000u, x[3], sr);
  return es;
}

// SHA-256(m || x) for one entry; returns the 8 state words.
__device__ __forceinline__ void hash_entry(const uint8_t* m, uint32_t L, const uint32_t x[4], uint32_t st[8]) {
  const EntryStream es = entry_stream(m, L, x);
  const uint32_t total = L + 16;
  const uint32_t nb = (total + 9 + 63) >> 6;
  sha256_init(st);
  for (uint32_t b = 0; b < nb; ++b) {
    uint32_t w[16];
    const uint32_t o0 = b << 6;
    if (o0 + 64 <= L) {
#pragma unroll
      for (int i = 0; i < 16; ++i) w[i] = load_msg_word(es, (o0 >> 2) + i);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) w[i] = stream_word(es, o0 + 4 * i);
      if (b == nb - 1) {
        w[14] |= total >> 29;
        w[15] |= total << 3;
      }
    }
    sha256_compress(st, w);
  }
}

// ----------------------------------------------------------------------------------------
// Instantiations of PRF and H (Sec. 7.2): POSLO = SHA-256 for both, POSLO+ = MMO-AES-128
// (kappa = 127) and MDC-2-AES-128.  Kernels that hash are templates on the instantiation;
// a POSLO+ kernel builds its AES table in shared memory first (aes_tables_init).
// ----------------------------------------------------------------------------------------
enum : int { kInstSha = 0, kInstAes = 1 };

template <int INST>
__device__ __forceinline__ void prf_node_i(const AesCtx& c, const uint32_t z[4], uint32_t bit, uint32_t out[4]) {
  if constexpr (INST == kInstAes) prf_node_aes(c, z, bit, out);
  else prf_node(z, bit, out);
}

template <int INST>
__device__ __forceinline__ void prf_entry_i(const AesCtx& c, const uint32_t x0[4], uint32_t j, uint32_t out[4]) {
  if constexpr (INST == kInstAes) prf_entry_aes(c, x0, j, out);
  else prf_entry(x0, j, out);
}

// MDC-2-AES-128 over the padded stream: (L + 16 + 16) / 16 blocks (the 0x80 byte always
// fits, a whole-block input gains a block).  dig = the 32-byte digest as 8 little-endian
// words (the integer H(m || x) before reduction mod q).
__device__ __forceinline__ void mdc2_stream(const AesCtx& c, const EntryStream& es, uint32_t dig[8]) {
  uint32_t h[4] = {kIvA, kIvA, kIvA, kIvA}, g[4] = {kIvB, kIvB, kIvB, kIvB};
  const uint32_t nb = (es.L + 32) >> 4;
#pragma unroll 1
  for (uint32_t b = 0; b < nb; ++b) {
    const uint32_t o = b << 4;
    uint32_t m[4];
    if (o + 16 <= es.L) {
#pragma unroll
      for (int q = 0; q < 4; ++q) m[q] = load_msg_word(es, (o >> 2) + q);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) m[q] = stream_word(es, o + 4 * q);
    }
    mdc2_step(c, h, g, m);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) { dig[q] = bswap32(h[q]); dig[4 + q] = bswap32(g[q]); }
}

// H(m || x) as 8 little-endian digest words for the instantiation.
template <int INST>
__device__ __forceinline__ void entry_digest(const AesCtx& c, const uint8_t* m, uint32_t L, const uint32_t x[4],
                                             uint32_t dig[8]) {
  if constexpr (INST == kInstAes) {
    mdc2_stream(c, entry_stream(m, L, x), dig);
  } else {
    uint32_t st[8];
    hash_entry(m, L, x, st);
#pragma unroll
    for (int q = 0; q < 8; ++q) dig[q] = bswap32(st[q]);
  }
}

__device__ __forceinline__ void warp_sum_u64(unsigned long long& v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
}


// ----------------------------------------------------------------------------------------
// Unit aggregation of the commitments: decode R_t, flag malformed ones, sum the rest.
// ----------------------------------------------------------------------------------------
struct PointArgs {
  const uint8_t* R;       // count*32
  uint64_t count;
  uint32_t* partial;      // per block: ge (32 words) + bad count (1 word), 33 words
  uint32_t* pts_out;      // optional: count*24 words (x, y, 2d x y) of decoded points
  uint8_t* bad_out;       // optional: count bytes, 1 = undecodable
  const uint8_t* skip;    // optional: count bytes, 1 = leave the point out of the sum
  uint32_t* work;         // chunk counter, zero at launch: blocks take kPointChunk points at a time
};

constexpr int kPtsWords = 24;   // stored decoded point: x, y, t2d = 2d x y (8 words each)
constexpr uint32_t kPointChunk = kPointThreads;   // one point per thread per grab: small batches keep their parallelism

constexpr int kPointPartialWords = 33;

__device__ __forceinline__ void ge_store(uint32_t* dst, const ge& p) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    dst[i] = p.X.v[i]; dst[8 + i] = p.Y.v[i]; dst[16 + i] = p.Z.v[i]; dst[24 + i] = p.T.v[i];
  }
}

__device__ __forceinline__ ge ge_load(const uint32_t* src) {
  ge p;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    p.X.v[i] = src[i]; p.Y.v[i] = src[8 + i]; p.Z.v[i] = src[16 + i]; p.T.v[i] = src[24 + i];
  }
  return p;
}


// ----------------------------------------------------------------------------------------
// Fixed-window tables: table[w][d-1] = d * 16^w * P for w = 0..63, d = 1..8 (k_table_*).
// ----------------------------------------------------------------------------------------


// Recode k (< 2^253) into 64 signed digits in [-8, 8).
__device__ __forceinline__ void recode4(const uint32_t k[8], int8_t dig[64]) {
  int carry = 0;
  for (int w = 0; w < 64; ++w) dig[w] = (int8_t)sc_digit4(k, w, carry);
}

__device__ __forceinline__ ge table_pick(const uint32_t* table, int w, int d) {
  if (d == 0) return ge_identity();
  const ge p = ge_load(table + ((size_t)w * kTableDigits + (abs(d) - 1)) * 32);
  return d < 0 ? ge_neg(p) : p;
}

// ----------------------------------------------------------------------------------------
// Combine the partial aggregates and evaluate the cofactored check.
// ----------------------------------------------------------------------------------------
struct FinalArgs {
  const unsigned long long* hash_partial;   // nhash blocks * kPartialWords
  uint32_t nhash;
  const uint32_t* point_partial;            // npoint blocks * kPointPartialWords (unit R sum)
  uint32_t npoint;
  const uint32_t* R_given;                  // optional: an extended point (32 words) used as R
  const uint8_t* s_given;                   // optional: aggregate s (C), 32 bytes
  const uint32_t* tableY;
  const uint32_t* tableG;
  uint8_t* accept;                          // 1 byte
  uint32_t* out_words;                      // optional: e~ (8), s~ (8), R (32) for inspection
  uint32_t* status;
};

constexpr int kFinalThreads = 256;

__device__ __forceinline__ sc limb_sums_to_scalar(const unsigned long long* sums13) {
  // value = sum_k sums13[k] * 2^(32k); propagate carries into 16 limbs and reduce mod q
  uint32_t x[16];
  unsigned long long carry = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const unsigned long long v = (k < 13 ? sums13[k] : 0ull) + carry;
    x[k] = (uint32_t)v;
    carry = v >> 32;
  }
  return sc_reduce512(x);
}


// ---- per-entry checks (see k_check.cu) ----
//
//   k_entry_check  the single-entry POSLO-F check of Fig. 4 (|m| = 1) for every entry:
//                  s_t canonical, R_t decodable, [8](R_t - e_t Y - s_t G) = O, with
//                  [e]Y + [s]G taken from the two fixed-window tables (128 additions)


//   k_entry_check_group  the same check, eight lanes per entry (two quads summing the Y and
//                  the G terms side by side with quad-cooperative additions), on the decoded
//                  points and malformed flags of the first stage: the direct localisation of
//                  small batches, where the latency of one entry is the latency of the launch
struct DirectCheckArgs {
  const uint8_t* e;          // n*32 (from k_hash)
  const uint8_t* s;          // n*32
  const uint32_t* pts;       // n*kPtsWords decoded R_t (from k_points)
  const uint8_t* badR;       // n: R_t does not decode
  const uint8_t* badS;       // n: s_t not canonical
  uint64_t n;
  const uint32_t* tableY;
  const uint32_t* tableG;
  uint8_t* invalid;          // n bytes: 1 = entry fails its own check
};
__global__ void __launch_bounds__(128) k_entry_check_group(const DirectCheckArgs a);


__device__ __forceinline__ ge double_scalar_tables(const uint32_t e[8], const uint32_t s[8],
                                                   const uint32_t* tableY, const uint32_t* tableG) {
  int8_t de[64], ds_[64];
  recode4(e, de);
  recode4(s, ds_);
  ge acc = ge_identity();
  for (int w = 0; w < 64; ++w) {
    acc = ge_add(acc, table_pick(tableY, w, de[w]));
    acc = ge_add(acc, table_pick(tableG, w, ds_[w]));
  }
  return acc;
}

struct CheckArgs {
  const uint8_t* e;          // n*32 (from k_hash)
  const uint8_t* s;          // n*32
  const uint8_t* R;          // n*32 compressed
  uint64_t n;
  const uint32_t* tableY;
  const uint32_t* tableG;
  uint8_t* invalid;          // n bytes: 1 = entry fails its own check
};


// Masked scalar sum: per block, 13 u64 limb sums of the s_t whose skip byte is 0.


// Reduce scalar partials (13 u64 limb sums per block) to one canonical scalar.




// Sum point partials (one block) and encode the result.


// ---- signer helpers (see k_signer.cu) ----
// Signer-side kernels: key generation and signing of synthetic logs (POSLO-C.Kg/Sig of
// Fig. 3a, POSLO-F.Kg/Sig of Fig. 4 with the BPV generator of Definition 3).  They produce
// workloads for the verifier; they are not on the verification path.


__device__ __forceinline__ void load_sc_bytes(const uint8_t* b, uint32_t v[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k)
    v[k] = b[4 * k] | (b[4 * k + 1] << 8) | (b[4 * k + 2] << 16) | ((uint32_t)b[4 * k + 3] << 24);
}

__device__ __forceinline__ void store_words_bytes(uint8_t* b, const uint32_t v[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    b[4 * k] = (uint8_t)v[k]; b[4 * k + 1] = (uint8_t)(v[k] >> 8);
    b[4 * k + 2] = (uint8_t)(v[k] >> 16); b[4 * k + 3] = (uint8_t)(v[k] >> 24);
  }
}

// r_i^j = SHA-256(r || le32(i) || le32(j) || 0x00) mod q: one block of 41 bytes.
__device__ __forceinline__ sc nonce_c(const uint32_t rw[8], uint32_t i, uint32_t j) {
  uint32_t w[16];
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = rw[k];
  w[8] = bswap32(i);
  w[9] = bswap32(j);
  w[10] = 0x00800000u;   // byte 40 = 0x00, byte 41 = 0x80
#pragma unroll
  for (int k = 11; k < 15; ++k) w[k] = 0;
  w[15] = 41 * 8;
  uint32_t st[8];
  sha256_init(st);
  sha256_compress(st, w);
  uint32_t d[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) d[k] = bswap32(st[k]);
  return sc_reduce256(d);
}

// [k]G for a scalar below 2^256 via the fixed-window table of G (64 table additions).
__device__ __forceinline__ ge base_mult_table(const uint32_t k[8], const uint32_t* tableG) {
  int8_t dig[64];
  recode4(k, dig);
  ge acc = ge_identity();
  for (int w = 0; w < 64; ++w) acc = ge_add(acc, table_pick(tableG, w, dig[w]));
  return acc;
}

// Y = [y]G (one thread).


// POSLO-C.Kg steps 5-7: R~_i = [sum_j r_i^j mod q]G, one thread per epoch.


// BPV.Offline: R_k = [r_k]G, one thread per table entry.


// Decode the BPV commitment table once into extended points.


struct SignFArgs {
  const uint8_t* msgs;
  const uint64_t* offs;
  uint64_t base_off;
  uint64_t n;
  uint64_t first_index;
  uint64_t e0;
  uint32_t n2;
  const uint32_t* seeds;     // x_0 per epoch (BE words)
  const uint8_t* y;          // 32 bytes
  const uint8_t* bpv_r;      // v*32
  const uint32_t* bpv_pts;   // v decoded points (32 words each)
  uint32_t v, k;
  const uint16_t* subsets;   // n*k
  uint8_t* s_out;
  uint8_t* R_out;
  uint8_t* x_out;            // optional
};

// POSLO-F.Sig: (r_t, R_t) = BPV.Online, e_t = H(m_t || x_t), s_t = r_t - e_t y.


struct SignCArgs {
  const uint8_t* msgs;
  const uint64_t* offs;
  uint64_t base_off;
  uint64_t n_epochs;
  uint64_t first_epoch;
  uint32_t n2;
  const uint32_t* seeds;     // x_0 per epoch of the range (BE words)
  const uint8_t* y;
  const uint8_t* r;
  uint8_t* s_out;            // n_epochs*32
};

// POSLO-C.Sig: s~_i = sum_j (r_i^j - e_i^j y) mod q, one thread per epoch.


// ---- Pippenger multi-scalar multiplication (k_msm.cu) ----
// sum_t [z_t] P_t for scalars z_t of 4 words (the verifier's weights, below 2^127) or 8
// words (any 256-bit value) and stored points P_t (kPtsWords each).  Scalars are cut into
// signed windows of c bits covering the width plus one bit (for the last carry); in
// window w every point goes to bucket |digit_w(z_t)|, found by a counting sort (count with atomics, scan, scatter).  Bucket sums
// B_{w,d} come from a load-balanced pass over the sorted entries; the window sum sum_d d B_{w,d} from chunks of
// kMsmChunk buckets (running sums inside a chunk, then a binary decomposition of the chunk
// index), and the windows are joined by Horner's rule in one warp with quad-cooperative
// doublings.
constexpr int kMsmChunk = 16;
constexpr int kMsmSegLog2Min = 4;    // sorted entries per accumulation thread: 2^4 .. 2^8
constexpr int kMsmSegLog2Max = 8;

// Pippenger plan with signed window digits.  Scalars of `sw` words hold at most `bits` bits
// (127 for the 4-word weights z_t, whose top bit is clear; 256 for 8-word scalars); windows =
// ceil((bits + 1) / c), so the last window never carries out.  A digit lies in
// [-(2^(c-1) - 1), 2^(c-1)]; its bucket is |digit| in 1 .. 2^(c-1), and the bucket array of a
// window is padded to nb = 2^(c-1) + kMsmChunk so that it splits into whole chunks.
struct MsmPlan {
  int c;              // window bits (8..16)
  int sw;             // scalar words: 4 (weights below 2^127) or 8 (256-bit scalars)
  int windows;        // ceil((bits + 1) / c)
  uint32_t nb;        // buckets per window, 2^(c-1) + kMsmChunk (bucket 0 and the padding stay empty)
  uint32_t nchunks;   // nb / kMsmChunk = 2^(c-5) + 1
  int jbits;          // bits of the largest chunk index 2^(c-5): c - 4
  int seg_log2;       // each accumulation thread adds 2^seg_log2 sorted entries (a range)
};

// Unsigned c-bit field w of the scalar (0 past its last word).
__device__ __forceinline__ uint32_t z_digit(const uint32_t* z, int sw, int w, int c) {
  const int bit = w * c;
  if (bit >= 32 * sw) return 0;
  const int word = bit >> 5, off = bit & 31;
  uint64_t v = z[word];
  if (word + 1 < sw) v |= (uint64_t)z[word + 1] << 32;
  return (uint32_t)(v >> off) & ((1u << c) - 1u);
}

// Signed recoding, windows taken in increasing order: r = field + carry in [0, 2^c]; above
// 2^(c-1) the digit is r - 2^c (negative) and 1 carries into the next window.  Returns the
// bucket |digit| (0: no entry in this window) and its sign.
__device__ __forceinline__ uint32_t z_sdigit(const uint32_t* z, int sw, int w, int c, uint32_t& carry, bool& neg) {
  const uint32_t r = z_digit(z, sw, w, c) + carry;
  neg = r > (1u << (c - 1));
  carry = neg ? 1u : 0u;
  return neg ? (1u << c) - r : r;
}

// Sorted bucket codes: bits 0..14 = bucket - 1, bit 15 = the digit is negative.
constexpr uint32_t kBktNeg = 0x8000u, kBktMask = 0x7fffu;
constexpr int kMsmMaxWindows = 40;   // c >= 8: at most ceil(257 / 8) = 33 windows

__device__ __forceinline__ void z_load(const uint32_t* z, int sw, uint64_t t, uint32_t zw[8]) {
  const uint4* p = reinterpret_cast<const uint4*>(z + (size_t)sw * t);
  const uint4 a = __ldg(p);
  zw[0] = a.x; zw[1] = a.y; zw[2] = a.z; zw[3] = a.w;
  if (sw == 8) {
    const uint4 b = __ldg(p + 1);
    zw[4] = b.x; zw[5] = b.y; zw[6] = b.z; zw[7] = b.w;
  } else {
    zw[4] = zw[5] = zw[6] = zw[7] = 0;
  }
}

// Window w of entry t's weight in the MSM's signed digits: magnitude d and sign neg.
__device__ __forceinline__ uint32_t weight_digit(const uint32_t* z, uint64_t t, int w, int c, bool& neg) {
  uint32_t zw[8];
  z_load(z, 4, t, zw);
  uint32_t carry = 0, d = 0;
  neg = false;
  for (int k = 0; k <= w; ++k) d = z_sdigit(zw, 4, k, c, carry, neg);
  return d;
}

// ae += digit e_t, as += digit s_t (mod q, exactly in 416-bit accumulators) for the digit of
// magnitude d and sign neg: a negative digit adds d (q - x).
__device__ __forceinline__ void add_window_terms(acc13& ae, acc13& as, const uint8_t* e32, const uint8_t* s32,
                                                 uint32_t d, bool neg) {
  const uint4* ep = reinterpret_cast<const uint4*>(e32);
  const uint4* sp = reinterpret_cast<const uint4*>(s32);
  const uint4 e0 = ep[0], e1 = ep[1], s0 = sp[0], s1 = sp[1];
  uint32_t x[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
  uint32_t y[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
  if (neg) {
    uint32_t q[8];
    sc_qlimbs(q);
    int64_t bx = 0, by = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      bx += (int64_t)q[k] - x[k];
      by += (int64_t)q[k] - y[k];
      x[k] = (uint32_t)bx;
      y[k] = (uint32_t)by;
      bx >>= 32;
      by >>= 32;
    }
  }
  uint32_t r[9];
  uint64_t c0 = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    c0 += (uint64_t)d * x[k];
    r[k] = (uint32_t)c0;
    c0 >>= 32;
  }
  r[8] = (uint32_t)c0;
  acc_add<9>(ae, r);
  uint64_t c1 = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    c1 += (uint64_t)d * y[k];
    r[k] = (uint32_t)c1;
    c1 >>= 32;
  }
  r[8] = (uint32_t)c1;
  acc_add<9>(as, r);
}

__device__ __forceinline__ void pts_load(const uint32_t* src, fe& x, fe& y, fe& t2d) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4 v[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) v[i] = __ldg(s4 + i);
  x = fe_const(v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y, v[1].z, v[1].w);
  y = fe_const(v[2].x, v[2].y, v[2].z, v[2].w, v[3].x, v[3].y, v[3].z, v[3].w);
  t2d = fe_const(v[4].x, v[4].y, v[4].z, v[4].w, v[5].x, v[5].y, v[5].z, v[5].w);
}

// [8](R_t - e_t Y - s_t G) = O for entry t by the eight lanes of a group (lanes 8g .. 8g+7 of
// the warp): the first quad sums the 64 terms of [e]Y from Y's window table, the second the
// 64 of [s]G from G's, each fetching the next window's entry during the current addition;
// the two sums meet by shuffles and every lane returns the verdict.  Every lane of the warp
// must call it (full-mask shuffles).
__device__ __forceinline__ bool entry_check8(const uint8_t* e32, const uint8_t* s32, const uint32_t* pts_t,
                                             bool malformed, const uint32_t* tableY, const uint32_t* tableG) {
  const bool g_half = (threadIdx.x & 4) != 0;
  const uint4* kp = reinterpret_cast<const uint4*>(g_half ? s32 : e32);
  const uint4 k0 = __ldg(kp), k1 = __ldg(kp + 1);
  const uint32_t k[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
  const uint32_t* tab = g_half ? tableG : tableY;
  ge acc = ge_identity();
  int carry = 0;
  ge next = table_pick(tab, 0, sc_digit4(k, 0, carry));
  for (int w = 0; w < kTableWindows; ++w) {
    const ge cur = next;
    if (w + 1 < kTableWindows) next = table_pick(tab, w + 1, sc_digit4(k, w + 1, carry));
    acc = ge_add_quad(acc, cur);
  }
  ge other;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    other.X.v[i] = __shfl_xor_sync(0xffffffffu, acc.X.v[i], 4);
    other.Y.v[i] = __shfl_xor_sync(0xffffffffu, acc.Y.v[i], 4);
    other.Z.v[i] = __shfl_xor_sync(0xffffffffu, acc.Z.v[i], 4);
    other.T.v[i] = __shfl_xor_sync(0xffffffffu, acc.T.v[i], 4);
  }
  acc = ge_add_quad(acc, other);
  ge R;
  fe t2d;
  pts_load(pts_t, R.X, R.Y, t2d);
  R.Z = fe_one();
  R.T = fe_mul(R.X, R.Y);
  const ge d = ge_sub(R, acc);
  return !malformed && ge_is_identity(ge_dbl_quad(ge_dbl_quad(ge_dbl_quad(d))));
}

// ---- Distill segment tree (k_distill.cu) ----
struct TreeArgs {
  const uint32_t* pts;       // n*kPtsWords decoded points
  const uint8_t* e;          // n*32 e_t
  const uint8_t* s;          // n*32 s_t
  const uint8_t* skip1;      // malformed R_t (undecodable)
  const uint8_t* skip2;      // malformed s_t (non-canonical)
  uint64_t n;                // entries
  uint64_t M;                // leaves, the next power of two >= max(n, 2)
  uint32_t* tree_pts;        // M-1 nodes (levels 1..log2 M), 32 words each
  uint8_t* tree_e;           // M-1 scalars
  uint8_t* tree_s;           // M-1 scalars
};

// ---- multi-device batches (k_multi.cu) ----
struct SegSums {
  uint32_t* Ew;    // n_dev * 8: sum z e mod q
  uint32_t* Sw;    // n_dev * 8: sum z s mod q
  uint32_t* Eu;    // n_dev * 8: sum e mod q
  uint32_t* Su;    // n_dev * 8: sum s mod q
  uint32_t* Ru;    // n_dev * 32: sum R (extended)
  uint32_t* bad;   // n_dev: malformed entries
};

struct PrepArgs {
  const unsigned long long* hash_partial;   // nhash blocks * kPartialWords
  uint32_t nhash;
  const uint8_t* s_given;                   // optional: aggregate s (POSLO-C), 32 bytes
  const uint32_t* tableY;
  const uint32_t* tableG;
  uint32_t* prep;                           // out: [e]Y + [s]G (32 words), malformed-s flag (1 word)
};

// ---- kernel declarations ----
void launch_epoch_seeds(int inst, unsigned grid, unsigned block, cudaStream_t st, const DsNode* ds, int nds,
                        uint64_t e0, uint64_t ne, uint32_t* x0_out, uint32_t* status);
// Multi-device batches compile their decoding and hashing for this many blocks per SM (128
// registers a thread), so that three decoding blocks and one hashing block share an SM and
// the hashing (ALU pipe) runs during the decoding (IMAD pipe) instead of after it.
constexpr int kCoresidentMinBlocks = 4;
void launch_hash(int inst, unsigned grid, cudaStream_t st, const HashArgs& a, bool coresident = false);
void launch_points(unsigned grid, cudaStream_t st, const PointArgs& a, bool coresident = false);
struct ZPre { uint32_t w[10]; };   // BE words of "POSLO-Z" || verifier_seed || (byte 39 = 0)
__global__ void k_weights(const ZPre zp, uint64_t n, uint64_t first, uint32_t* z_out);

// (Key k's table is dst[k] when a destination list is given -- tables scattered over a
// cache -- else tables + k kTableWords.)
__global__ void __launch_bounds__(128) k_table_chain(const uint32_t* __restrict__ enc,
                                                     const uint32_t* __restrict__ pts,
                                                     const uint32_t* __restrict__ list, uint32_t n,
                                                     uint32_t* __restrict__ tables, uint32_t* const* dst,
                                                     uint32_t* __restrict__ status, int use_base,
                                                     uint8_t* __restrict__ bad_out);
__global__ void __launch_bounds__(128) k_table_fill(uint32_t n, uint32_t* __restrict__ tables, uint32_t* const* dst);
__global__ void __launch_bounds__(kFinalThreads) k_finalize(const FinalArgs a);
__global__ void __launch_bounds__(128) k_final_prep(const PrepArgs a);
__global__ void k_final_check(const uint32_t* prep, const uint32_t* R, const uint32_t* point_bad,
                              const uint32_t* status, uint8_t* accept);
__global__ void __launch_bounds__(128) k_entry_check(const CheckArgs a);
__global__ void __launch_bounds__(kHashThreads) k_sum_scalars(const uint8_t* s, uint64_t n, const uint8_t* skip,
                                                             unsigned long long* partial);
__global__ void k_reduce_scalars(const unsigned long long* partial, uint32_t nparts, uint8_t* out);
__global__ void k_sum_encode(const uint32_t* partial, uint32_t nparts, uint32_t* point_out, uint8_t* enc_out,
                             uint32_t* bad_out);
__global__ void k_keygen_y(const uint8_t* y, const uint32_t* tableG, uint8_t* Y_out);
__global__ void k_keygen_c_epochs(const uint8_t* r, uint32_t n1, uint32_t n2, const uint32_t* tableG,
                                  uint8_t* epoch_R);
__global__ void k_keygen_bpv(const uint8_t* bpv_r, uint32_t v, const uint32_t* tableG, uint8_t* bpv_R);
__global__ void k_decode_table(const uint8_t* enc, uint32_t v, uint32_t* out, uint32_t* status);
void launch_sign_f(int inst, unsigned grid, unsigned block, cudaStream_t st, const SignFArgs& a);
void launch_sign_c(int inst, unsigned grid, unsigned block, cudaStream_t st, const SignCArgs& a);
__global__ void k_msm_count(const uint32_t* z, const uint8_t* skip, uint64_t n, MsmPlan pl, uint32_t* cnt,
                            uint32_t* rank);
__global__ void __launch_bounds__(1024) k_msm_scan(const uint32_t* cnt, uint32_t* off, MsmPlan pl);
__global__ void k_msm_scatter(const uint32_t* z, const uint8_t* skip, uint64_t n, MsmPlan pl, const uint32_t* off,
                              const uint32_t* rank, uint32_t* idx, uint16_t* bkt);
__global__ void k_msm_tune_fill(uint32_t* pts, uint32_t* z, uint64_t n, int sw);
#ifndef POSLO_ACCUM_MINB
#define POSLO_ACCUM_MINB 4   // resident blocks per SM the bucket accumulation is compiled for (128 registers)
#endif
__global__ void __launch_bounds__(128, POSLO_ACCUM_MINB) k_msm_accum(const uint32_t* pts, const uint32_t* idx, const uint16_t* bkt,
                                                   const uint32_t* off, const uint32_t* cnt, uint64_t n, MsmPlan pl,
                                                   const uint8_t* skip, uint32_t* buckets, uint32_t* A, uint32_t* B);
__global__ void __launch_bounds__(128) k_msm_combine(const uint32_t* off, const uint32_t* cnt, uint64_t n, MsmPlan pl,
                                                     const uint32_t* A, const uint32_t* B, uint32_t* buckets,
                                                     uint32_t* big_list, uint32_t* big_count);
constexpr int kCombineBigThreads = 128;
__global__ void __launch_bounds__(kCombineBigThreads) k_msm_combine_big(const uint32_t* off, const uint32_t* cnt,
                                                                        uint64_t n, MsmPlan pl, const uint32_t* A,
                                                                        const uint32_t* B, uint32_t* buckets,
                                                                        const uint32_t* big_list,
                                                                        const uint32_t* big_count);
__global__ void __launch_bounds__(128) k_msm_chunk(const uint32_t* buckets, MsmPlan pl, uint32_t* L, uint32_t* T);
__global__ void __launch_bounds__(512) k_msm_groups(const uint32_t* L, const uint32_t* T, MsmPlan pl, uint32_t* groups);
constexpr int kMsmDirectMaxC = 8;   // windows up to this width skip the chunk and group sums (512 threads)
__global__ void __launch_bounds__(512) k_msm_direct_groups(const uint32_t* buckets, MsmPlan pl, uint32_t* groups);
__global__ void __launch_bounds__(32) k_msm_final(const uint32_t* groups, MsmPlan pl, uint32_t* out);
__global__ void __launch_bounds__(32) k_msm_windows(const uint32_t* groups, MsmPlan pl, uint32_t* W);
__global__ void __launch_bounds__(32) k_msm_window_check(const uint32_t* groups, MsmPlan pl, const uint32_t* Pw,
                                                         const uint32_t* bad, const uint32_t* point_bad,
                                                         const uint32_t* status, uint8_t* accept);
constexpr int kWindowThreads = 128;
__global__ void __launch_bounds__(kWindowThreads) k_window_sums(const uint8_t* e, const uint8_t* s, const uint32_t* z,
                                                                uint64_t n, MsmPlan pl, unsigned long long* partial);
__global__ void __launch_bounds__(kWindowThreads) k_window_prep(const unsigned long long* partial, uint32_t nblocks,
                                                                const unsigned long long* hash_partial, uint32_t nhash,
                                                                const uint32_t* tableY, const uint32_t* tableG,
                                                                uint32_t* Pw, uint32_t* bad);
__global__ void __launch_bounds__(128) k_tree_leaves(const TreeArgs a);
__global__ void __launch_bounds__(128) k_tree_level(const TreeArgs a, uint64_t in_off, uint64_t out_off,
                                                    uint64_t count);
// The descent's state on the device: three failing-node lists with their counters (rotated
// by step), two level words.  Node (l, k) of the tree, l >= 1, is at M - (M >> (l - 1)) + k
// in the node arrays (levels 1 .. l-1 come first).
struct BisectState {
  uint64_t* fail[3];
  uint64_t* cnt;     // 3 counters
  int* level;        // 2 words
};
// Resident blocks per SM the descent is compiled for (its checks are latency-bound chains of
// point additions: more warps per SM hide more of it, at the cost of registers).
#ifndef POSLO_BISECT_MINB
#define POSLO_BISECT_MINB 2
#endif
#ifndef POSLO_BISECT_WAVES
#define POSLO_BISECT_WAVES 1   // the descent's grid: this many waves of resident blocks
#endif
__global__ void __launch_bounds__(128, POSLO_BISECT_MINB) k_bisect_step(const TreeArgs a, BisectState st, int step,
                                                     const uint32_t* tY, const uint32_t* tG, uint8_t* invalid);
__global__ void k_gather_flagged(const uint32_t* pts, const uint32_t* z, const uint8_t* badR, const uint64_t* idx,
                                 uint64_t cnt, uint32_t* gp, uint32_t* gz, uint8_t* gs);
__global__ void k_point_diff(const uint32_t* a, const uint32_t* b, uint32_t* out);
__global__ void __launch_bounds__(256) k_ccd_points(const uint32_t* pts, const uint8_t* badR, const uint64_t* idx,
                                                    const uint64_t* nf_dev, const uint32_t* unit, uint8_t* enc_out);
__global__ void __launch_bounds__(kHashThreads) k_weighted_sums(const uint8_t* e, const uint8_t* s, const uint32_t* z, const uint8_t* skip1,
                                const uint8_t* skip2, uint64_t n, unsigned long long* partial);
__global__ void k_flags_or(const uint8_t* a, const uint8_t* b, const uint8_t* c, uint64_t n, uint8_t* out);
__global__ void k_encode_ext(const uint32_t* point, uint8_t* out);
void launch_epoch_seeds_multi(int inst, unsigned grid, unsigned block, cudaStream_t st, const DsNode* ds_all,
                              const uint32_t* ds_off, const uint64_t* seed_off, const uint64_t* e0, uint32_t n_dev,
                              uint32_t* seeds, uint32_t* status);
constexpr uint64_t kGatherChunk = 1ull << 16;   // bytes of one chunk of the staging gather
#ifndef POSLO_GATHER_MAX_REQUEST
#define POSLO_GATHER_MAX_REQUEST (1ull << 20)
#endif
constexpr uint64_t kGatherMaxRequestBytes = POSLO_GATHER_MAX_REQUEST;   // larger requests: copy engines
struct GatherRegion {
  const uint8_t* src;   // device-readable (mapped page-locked host memory)
  uint8_t* dst;         // device memory
  uint64_t bytes;
};
__global__ void __launch_bounds__(256) k_stage_gather(const GatherRegion* regions, uint32_t n_regions);
__global__ void k_rebase_offs(const uint64_t* raw, const uint64_t* slot, const uint64_t* start,
                              const uint64_t* msg_base, uint32_t n_dev, uint64_t* out, uint32_t* status);
#ifndef POSLO_SEG_THREADS
#define POSLO_SEG_THREADS 256
#endif
constexpr int kSegThreads = POSLO_SEG_THREADS;   // threads per block of the segment sums
// Entries per piece of the segment sums: a device's entries are cut into pieces of this size
// (one block each), so a device of 65,536 entries no longer runs as one long block at the end.
constexpr uint64_t kSegPiece = 2048;
constexpr int kSegLimbWords = 4 * 13 + 1;          // a piece's partial: four 13-limb sums and its bad count
// The pieces of a call: pieces[p] = device | (piece index within the device << 32), devices
// largest first and a device's pieces consecutive; pfirst[d] = index of device d's first piece.
constexpr int kSegScalars = 1, kSegPoints = 2;     // the two launches of the segment sums
// k_segment_sums<kSegScalars> then k_segment_sums<kSegPoints>, one block per piece, on st.
void launch_segment_sums(unsigned n_pieces, cudaStream_t st, const uint8_t* e, const uint8_t* s, const uint32_t* z,
                         const uint32_t* pts, const uint8_t* badR, const uint8_t* badS, const uint64_t* start,
                         const uint64_t* pieces, unsigned long long* piece_limbs, uint32_t* piece_R, SegSums out);
// Devices of more than one piece: their pieces' limb sums, bad counts and points added up.
__global__ void __launch_bounds__(kSegThreads) k_segment_combine(const uint64_t* start, const uint64_t* pfirst,
                                                         const unsigned long long* piece_limbs,
                                                         const uint32_t* piece_R, uint32_t n_dev, SegSums out);
__global__ void __launch_bounds__(kFinalThreads) k_multi_check(const uint32_t* P1, const uint32_t* P1sub, const uint32_t* P2,
                                                               const uint32_t* Sw, const uint8_t* dev_flag,
                                                               uint32_t n_dev, const uint32_t* tableG,
                                                               uint8_t* accept);
__global__ void __launch_bounds__(kPointThreads) k_table_msm(const uint32_t* const* tabs, const uint32_t* k,
                                                             const uint8_t* skip, uint32_t n, uint32_t* partial);
__global__ void __launch_bounds__(kSegThreads) k_segment_window_sums(const uint8_t* e, const uint8_t* s, const uint32_t* z,
                                                             const uint8_t* badR, const uint8_t* badS,
                                                             const uint64_t* start, const uint64_t* order,
                                                             uint32_t n_dev, MsmPlan pl, uint32_t* Ewd, uint32_t* Swd);
__global__ void __launch_bounds__(kFinalThreads) k_multi_window_check(const uint32_t* W, const uint32_t* Wsub,
                                                                      const uint32_t* P2w, const uint32_t* Swd,
                                                                      const uint8_t* dev_flag, uint32_t n_dev,
                                                                      const uint32_t* tableG, uint8_t* accept);
__global__ void __launch_bounds__(kPointThreads) k_table_msm_windows(const uint32_t* const* tabs, const uint32_t* k,
                                                                     const uint8_t* skip, uint32_t n,
                                                                     uint32_t* partial);
__global__ void __launch_bounds__(kPointThreads) k_window_point_sums(const uint32_t* partial, uint32_t nblocks,
                                                                     uint32_t* out);
__global__ void __launch_bounds__(128) k_device_unit_check(const uint32_t* const* tabs, SegSums ss, uint32_t n_dev,
                                                           const uint32_t* tableG, uint8_t* dev_flag);
struct MultiCheckArgs {
  const uint32_t* pts;        // decoded R_t of the whole batch (kPtsWords each)
  const uint8_t* e;           // e_t, 32 bytes each
  const uint8_t* s;           // s_t, 32 bytes each
  const uint8_t* badR;        // 1 = R_t does not decode
  const uint8_t* badS;        // 1 = s_t is not canonical
  const uint64_t* seg_start;  // n_dev + 1 entry offsets of the devices
  const uint32_t* fl;         // the flagged devices, nfl of them
  const uint64_t* fstart;     // nfl + 1: prefix sums of their entry counts
  uint32_t nfl;
  const uint32_t* const* tabs;   // window table of each device's key (kTableWords words each)
  const uint32_t* tableG;
  uint8_t* inv;               // out: 1 = entry invalid (written for the flagged devices' entries)
};
__global__ void __launch_bounds__(128) k_multi_entry_check(const MultiCheckArgs a);
// The same checks with eight lanes per entry (as k_entry_check_group): for few flagged
// entries, where one entry's latency is the launch's.
__global__ void __launch_bounds__(128) k_multi_entry_check_group(const MultiCheckArgs a);
constexpr uint64_t kMultiGroupCheckMax = 16384;   // flagged entries up to which the group form runs
__global__ void k_segment_any(const uint8_t* inv, const uint64_t* seg_start, const uint32_t* fl, uint8_t* out);
// ---- POSLO-C distillation and SeBVer (k_ccd.cu) ----
constexpr int kCcdThreads = 128;
__global__ void __launch_bounds__(kCcdThreads) k_scalar_group_sums(const uint8_t* x, uint64_t G, uint64_t n,
                                                                   const uint8_t* skip, uint32_t* out);
__global__ void __launch_bounds__(kCcdThreads) k_point_group_sums(const uint32_t* pts, const uint8_t* bad, uint64_t G,
                                                                  uint64_t n, const uint8_t* skip, uint8_t* enc);
__global__ void __launch_bounds__(128) k_check_list(const uint32_t* e, const uint8_t* s, const uint32_t* pts,
                                                    const uint8_t* bad, uint32_t n, const uint32_t* tableY,
                                                    const uint32_t* tableG, uint8_t* ok);
__global__ void k_gather32(const uint8_t* src, const uint64_t* idx, uint64_t n, uint8_t* dst);
__global__ void k_flip(const uint8_t* ok, uint64_t n, uint8_t* flag);
__global__ void k_offs_sub(uint64_t* offs, uint64_t n, uint64_t base);
__global__ void k_device_to_entries(const uint8_t* dev_flag, const uint64_t* start, const uint8_t* badR,
                                    uint8_t* skip, int keep_flagged);
constexpr uint32_t kFlagChunk = 8192;
__global__ void __launch_bounds__(1024) k_flag_count(const uint8_t* flags, uint64_t n, uint32_t* blockcnt);
__global__ void __launch_bounds__(1024) k_flag_scan(const uint32_t* blockcnt, uint32_t nblocks, uint64_t* blockoff,
                                                   uint64_t* total);
__global__ void __launch_bounds__(1024) k_flag_scatter(const uint8_t* flags, uint64_t n, uint64_t first_index,
                                                      const uint64_t* blockoff, uint64_t* out, uint64_t cap);
// ---- shard partials and their combination (k_shard.cu) ----
constexpr int kShardWords = 54;     // one poslo_partial record in 32-bit words
constexpr int kShardBadWord = 52;   // its malformed count (after e~, s~, R~, first_index, n)
constexpr int kShardThreads = 128;
__global__ void __launch_bounds__(kShardThreads) k_partial_out(const unsigned long long* hash_partial, uint32_t nhash,
                                                              const uint8_t* s_given, const uint32_t* R,
                                                              const uint32_t* point_bad, uint32_t* out);
__global__ void __launch_bounds__(kShardThreads) k_combine_check(const uint32_t* parts, uint32_t nparts,
                                                                const uint32_t* tableY, const uint32_t* tableG,
                                                                const uint32_t* status, uint32_t* total,
                                                                uint8_t* accept);

}  // namespace poslo
