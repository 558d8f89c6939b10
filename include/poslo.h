/*
 * libposlo — GB300 (sm_103a) batch verification of POSLO signed logs.
 *
 * C ABI over the cold-storage verification path of POSLO (Nouma and Yavuz, "Lightweight and
 * High-Throughput Secure Logging for Internet of Things and Cold Cloud Continuum",
 * arXiv 2506.08781).  Section, figure and equation numbers below refer to that paper.
 *
 * Instantiation: "POSLO" of Sec. 7.2 (Table 2): SHA-256 for both PRF and H; the group is the
 * prime-order subgroup of edwards25519 (the paper names FourQ with |q| = 256, which is not
 * self-consistent; edwards25519 is the reading used throughout).
 *
 * Encodings (all little-endian):
 *   scalar  32 bytes, canonical (< q = 2^252 + 27742317777372353535851937790883648493);
 *   point   32 bytes, edwards25519 compressed encoding (y with the parity of x in bit 255);
 *   seed    16 bytes (kappa = 128);
 *   ds node 24 bytes: le32 depth d, le32 index i, 16-byte seed x_d[i]; a disclosed-seed stack
 *           (ds, Sec. 4.1) is an array of nodes with the bottom of the stack first.
 *   messages: one byte buffer plus n+1 uint64 offsets; entry t is msgs[offs[t] .. offs[t+1]).
 *
 * Derivations (Sec. 4.1 and Fig. 3a; byte layouts are this library's reading of the paper):
 *   PRF_b(z)      = SHA-256(z || byte b)[0..16)            seed-tree children (Eq. 1)
 *   x_i^j         = SHA-256(x_0[i] || le32(j) || 0x00)[0..16)  one-time seed, j = t mod n2
 *   e_t           = SHA-256(m_t || x_t) as a little-endian integer, mod q
 *   verification  [8](R - e Y - s G) = O  (cofactored)
 *
 * Ownership and errors.  The caller owns every buffer it passes.  Unless a call says
 * otherwise, pointers are host pointers; batch pointers marked "device-capable" may be
 * device pointers when poslo_batch.on_device = 1 (they must then stay valid and unmodified
 * until the call returns).  Device-resident offsets must be 8-byte aligned and device-resident
 * s, R, e_out, points and scalars 16-byte aligned (every cudaMalloc or torch allocation is);
 * misaligned ones are refused with POSLO_EINVAL before any device work.  Messages may start at
 * any byte.  Every call is synchronous: it returns when its outputs are in
 * the caller's buffers.  Calls on one context must not overlap (they share its streams and
 * workspace); different contexts are independent.  A call returns POSLO_OK or a negative
 * poslo_status; poslo_last_error() then describes the failure.  "Signature invalid" is not
 * an error: it is an output bit or index.
 */
#ifndef POSLO_H_
#define POSLO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define POSLO_ABI_VERSION 1

typedef enum {
  POSLO_OK = 0,
  POSLO_EINVAL = -1,    /* malformed argument: sizes, bad public key, seed not disclosed (SRet bottom) */
  POSLO_ENOMEM = -2,    /* device memory could not be allocated or the context budget is exceeded */
  POSLO_EDEVICE = -3,   /* CUDA error (no device, launch failure) */
  POSLO_ETIMEOUT = -4,  /* a bounded device-side wait expired.  Reserved: no kernel of this
                           library waits on a flag or on another block (every step is its own
                           launch, ordered by streams and events), so no call returns it */
  POSLO_EBUFSMALL = -5, /* an output buffer is too small; the needed count is still reported */
  POSLO_EBUSY = -6,     /* serving: admission refused by the memory budget */
  POSLO_ENOTFOUND = -7, /* serving: unknown key id or ticket */
  POSLO_PENDING = 1     /* serving: the request is not verified yet (not an error) */
} poslo_status;

enum { POSLO_VARIANT_C = 0, POSLO_VARIANT_F = 1 };
enum { POSLO_AGG_UNIT = 0, POSLO_AGG_WEIGHTED = 1 };
/* Instantiations of PRF and H (Sec. 7.2, table of instantiations):
 *   POSLO_INST_SHA256  "POSLO": SHA-256 for both; seeds kappa = 128 bits.
 *   POSLO_INST_AES     "POSLO+": PRF = MMO over AES-128 with kappa = 127 (a node and its
 *                      child bit fill one AES block), H = MDC-2 over AES-128.  Seeds are 16
 *                      bytes whose least significant bit (bit 0 of byte 15) is not part of
 *                      the seed.  Initial values 16 x 0x52 (MMO, first MDC-2 chain) and
 *                      16 x 0x25 (second chain); MDC-2 pads with 0x80 then zeros to whole
 *                      blocks, always; the one-time seed x_i^j is MMO over the seed (bit 0)
 *                      and le32(j), 20 bytes padded the same way.
 * POSLO-C nonces and the verifier's weights z_t use SHA-256 in both. */
enum { POSLO_INST_SHA256 = 0, POSLO_INST_AES = 1 };

typedef struct poslo_ctx poslo_ctx;

typedef struct {
  int device;                 /* CUDA device ordinal */
  uint32_t msm_window;        /* Pippenger window in bits, 8..16; 0 = autotune */
  uint64_t mem_budget;        /* bytes of device memory the context may hold; 0 = no limit */
  uint8_t verifier_seed[32];  /* secret randomness of the verifier for the weights z_t */
  uint32_t instantiation;     /* POSLO_INST_SHA256 (0) or POSLO_INST_AES; every call on the
                                 context (keys, signing, verification, serving) uses it */
} poslo_params;

/*
 * One batch of signed log entries of a single signer.
 *   POSLO-F (Fig. 4): entry t (global index first_index + t) carries (s_t, R_t); s and R
 *     hold n scalars and n points.  R_count must equal n.
 *   POSLO-C (Fig. 3a): the batch is whole epochs: first_index and n are multiples of n2.
 *     s is the aggregate s~ (one scalar); R is either the aggregate R~ (R_count = 1) or the
 *     per-epoch commitments R~_i of pk for the batch's epochs (R_count = n / n2).
 * msgs, offs, s and R are device-capable; Y and ds are always host memory.
 */
typedef struct {
  uint32_t variant;      /* POSLO_VARIANT_C or POSLO_VARIANT_F */
  uint32_t n2;           /* entries per epoch, >= 1 */
  const uint8_t* Y;      /* 32-byte public key */
  const uint8_t* msgs;   /* message bytes */
  const uint64_t* offs;  /* n+1 non-decreasing offsets into msgs */
  uint64_t n;            /* number of entries */
  uint64_t first_index;  /* global index of entry 0 */
  const uint8_t* s;      /* F: n*32; C: 32 */
  const uint8_t* R;      /* F: n*32; C: R_count*32 */
  uint64_t R_count;
  const uint8_t* ds;     /* disclosed seeds (24 bytes per node), or the root as one node at depth D */
  uint32_t ds_nodes;
  uint32_t on_device;    /* 1: msgs, offs, s, R are device pointers */
} poslo_batch;

/* Context: device memory, streams, the fixed-base table of G and the Pippenger settings.
 * Returns POSLO_EDEVICE when the device is missing or not an sm_103 part. */
int poslo_create(const poslo_params* params, poslo_ctx** out);
void poslo_destroy(poslo_ctx* ctx);
const char* poslo_last_error(const poslo_ctx* ctx);
/* The CUDA stream (cudaStream_t) the context launches its hot kernels on. */
void* poslo_stream(poslo_ctx* ctx);

/* ---- test-data side (signer): deterministic from the caller's secret bytes ---------- */

/* POSLO-C.Kg (Fig. 3a) for n1 = 2^D epochs: Y = [y]G and R~_i = [sum_j r_i^j]G with
 * r_i^j = SHA-256(r || le32(i) || le32(j) || 0x00) mod q.  y: 32-byte scalar, 0 < y < q.
 * epoch_R_out: n1*32 bytes. */
int poslo_keygen_c(poslo_ctx* ctx, const uint8_t y[32], const uint8_t r[32], uint32_t D, uint32_t n2,
                   uint8_t Y_out[32], uint8_t* epoch_R_out);

/* POSLO-F.Kg (Fig. 4) with the BPV table of Definition 3: Y = [y]G, R_k = [r_k]G for the
 * v table scalars bpv_r (v*32 bytes, canonical).  bpv_R_out: v*32 bytes. */
int poslo_keygen_f(poslo_ctx* ctx, const uint8_t y[32], const uint8_t* bpv_r, uint32_t v, uint8_t Y_out[32],
                   uint8_t* bpv_R_out);

/* POSLO-C.Sig (Fig. 3a) for n_epochs whole epochs starting at first_epoch: msgs/offs hold
 * n_epochs*n2 entries; s_out receives one aggregate scalar s~_i per epoch (n_epochs*32). */
int poslo_sign_c(poslo_ctx* ctx, const uint8_t y[32], const uint8_t r[32], const uint8_t root[16], uint32_t D,
                 uint32_t n2, const uint8_t* msgs, const uint64_t* offs, uint64_t first_epoch,
                 uint64_t n_epochs, uint8_t* s_out);

/* POSLO-F.Sig (Fig. 4) for entries first_index .. first_index+n-1.  subsets: n*k uint16
 * indices into the BPV table (the online step's random choice, supplied by the caller);
 * outputs s_t (n*32), R_t (n*32, compressed) and optionally x_t (n*16, may be NULL). */
int poslo_sign_f(poslo_ctx* ctx, const uint8_t y[32], const uint8_t root[16], uint32_t D, uint32_t n2,
                 const uint8_t* bpv_r, const uint8_t* bpv_R, uint32_t v, uint32_t k, const uint16_t* subsets,
                 const uint8_t* msgs, const uint64_t* offs, uint64_t n, uint64_t first_index, uint8_t* s_out,
                 uint8_t* R_out, uint8_t* x_out);

/* Agg (Fig. 3a C.Agg, Fig. 4 F.Agg): s~ = sum of the n scalars mod q (each taken as the
 * integer its 32 bytes encode) and R~ = sum of the n points, both encoded.  scalars and
 * points are n*32 bytes, device-capable per on_device.  n = 0 gives s~ = 0 and R~ = O.
 * Errors: EINVAL if a point does not decode (the outputs are then not written). */
int poslo_agg(poslo_ctx* ctx, const uint8_t* scalars, const uint8_t* points, uint64_t n, uint32_t on_device,
              uint8_t s_out[32], uint8_t R_out[32]);

/* SSO (Fig. 2a) run for epochs 0..i from an empty stack: writes ds_i (24 bytes per node,
 * bottom first) to ds_out (capacity cap_nodes) and its node count to *nodes. */
int poslo_disclose(poslo_ctx* ctx, const uint8_t root[16], uint32_t D, uint64_t i, uint8_t* ds_out,
                   uint32_t cap_nodes, uint32_t* nodes);

/* ---- verifier side (device) ----------------------------------------------------------- */

/* POSLO.AVer / PAVer (Fig. 3a, Fig. 4, Fig. 6): one accept bit for the whole batch.
 *   agg_mode = POSLO_AGG_UNIT: the paper's equation with unit coefficients,
 *     [8](sum R - (sum e) Y - (sum s) G) = O, plus "every s_t canonical, every R_t decodable".
 *   agg_mode = POSLO_AGG_WEIGHTED (POSLO-F only): each entry weighted by a secret 127-bit z_t,
 *     accepts iff every entry passes its own check, except with probability <= 2^-127.
 * Errors: EINVAL for malformed sizes, more than 2^32 - 1 entries (longer logs: the streaming
 * call below), an undecodable Y, or a seed the ds does not disclose. */
int poslo_aver(poslo_ctx* ctx, const poslo_batch* batch, uint32_t agg_mode, uint8_t* accept);

/* POSLO-F Distill / SeBVer at entry granularity (Fig. 3b semantics, Sec. 4.3): the sorted
 * global indices of every entry that fails its own check (malformed s_t or R_t included),
 * and ccd^v = (sum of valid s_t, sum of valid R_t).  invalid_idx has room for cap indices;
 * *n_invalid is the full count (EBUFSMALL if it exceeds cap).  At most 2^32 - 1 entries per
 * call (EINVAL beyond). */
int poslo_distill(poslo_ctx* ctx, const poslo_batch* batch, uint64_t* invalid_idx, uint64_t cap,
                  uint64_t* n_invalid, uint8_t ccd_s[32], uint8_t ccd_R[32]);

/*
 * Many signers (IoT devices) verified together.  The entries of all devices are concatenated
 * (device d owns entries dev_start[d] .. dev_start[d+1]-1); msgs, offs (N+1 offsets into
 * msgs), s and R (N*32 each) are device-capable; the per-device arrays are host memory.
 * Each device is a POSLO-F signer with its own key Y_d, epoch size n2[d], disclosed seeds
 * (ds nodes ds_off[d] .. ds_off[d+1]-1 of ds) and index of its first entry first_index[d].
 */
typedef struct {
  uint32_t n_dev;
  const uint8_t* Y;             /* n_dev*32 public keys */
  const uint64_t* dev_start;    /* n_dev+1 entry starts, dev_start[0] = 0 */
  const uint64_t* first_index;  /* n_dev */
  const uint32_t* n2;           /* n_dev */
  const uint8_t* ds;            /* all devices' ds nodes, 24 bytes each */
  const uint32_t* ds_off;       /* n_dev+1 node offsets, ds_off[0] = 0 */
  const uint8_t* msgs;
  const uint64_t* offs;
  const uint8_t* s;
  const uint8_t* R;
  uint32_t on_device;           /* 1: msgs, offs, s, R are device pointers */
} poslo_multi_batch;

/* Per-device AVer + Distill for a multi-device batch: accept[d] = 1 iff every entry of
 * device d passes its own check (except with probability <= 2^-127); invalid_pairs receives
 * (device, global index) pairs of the failing entries, 2 uint64 per pair, sorted by device
 * then index, room for cap pairs; *n_invalid is the full count (EBUFSMALL if it exceeds cap).
 * Every stage is one launch over the segment table; one random linear combination checks
 * all devices at once, and only devices that fail their unit aggregate are localised.
 * At most 2^32 - 1 entries over all devices (EINVAL beyond). */
int poslo_aver_multi(poslo_ctx* ctx, const poslo_multi_batch* mb, uint8_t* accept, uint64_t* invalid_pairs,
                     uint64_t cap, uint64_t* n_invalid);

/* ---- one log split over several GPUs -------------------------------------------------------
 * A log of one signer split into contiguous ranges of global indices (shards, e.g. one per
 * GPU) is checked by aggregating each shard on its own GPU and combining the aggregates: AVer
 * (Fig. 3a, Fig. 4) needs only the sums e~ = sum e_t, s~ = sum s_t mod q and R~ = sum R_t
 * before its single group check, so a shard's contribution is these three values.  Sums mod q
 * and point sums are not reductions a collective library provides: the shards exchange the
 * fixed-size records below (an all-gather of 216 bytes per shard) and each runs the combined
 * check on its own device.  The localisation of invalid entries (poslo_distill) stays local to
 * each shard; since shards are contiguous and in index order, the concatenation of their
 * ascending lists is the log's list.  Not in the paper, whose verifier is one machine; the
 * paper does split 1 TB logs into chunks aggregated separately (Sec. 7.4). */
typedef struct {
  uint8_t e[32];           /* e~ = sum of e_t mod q (weighted: of z_t e_t), canonical LE */
  uint8_t s[32];           /* s~ = sum of s_t mod q (weighted: of z_t s_t); POSLO-C: the batch's s~ */
  uint8_t R[128];          /* R~ = sum of R_t (weighted: of [z_t]R_t) in extended coordinates X, Y, Z, T
                              (x = X/Z, y = Y/Z, xy = T/Z), 32 bytes LE each, every one below p */
  uint64_t first_index;    /* global index of the shard's first entry */
  uint64_t n;              /* entries in the shard */
  uint32_t malformed;      /* non-canonical s_t plus undecodable R_t of the shard (left out of the
                              sums; any makes the combined check fail); saturates at 2^32 - 1 */
  uint32_t agg_mode;       /* POSLO_AGG_UNIT or POSLO_AGG_WEIGHTED */
} poslo_partial;           /* 216 bytes, no padding */

/* The record of one shard: the aggregate of poslo_aver over the batch, before its group check.
 * agg_mode as for poslo_aver; for weighted records every shard's context must hold the same
 * verifier_seed (z_t depends on it and on the global index t, not on the shard).  Y is not
 * read.  Errors as poslo_aver (EINVAL for malformed sizes or an undisclosed seed). */
int poslo_aver_partial(poslo_ctx* ctx, const poslo_batch* batch, uint32_t agg_mode, poslo_partial* out);

/* The combined check of a log from its shards' records (host memory, n_parts >= 1, in index
 * order, each starting where the previous ends, all of one agg_mode): sums them on the device
 * and evaluates [8](R~ - e~ Y - s~ G) = O there.  *accept = 1 iff no shard reported a malformed
 * entry, every record is well formed (scalars below q, point coordinates below p on the curve)
 * and the equation holds -- the bit poslo_aver gives for the whole log.  total (optional)
 * receives the summed record (first_index of the first shard, n of all).  EINVAL for records
 * out of order, gaps, mixed modes or a Y that does not decode. */
int poslo_combine_check(poslo_ctx* ctx, const uint8_t Y[32], const poslo_partial* parts, uint32_t n_parts,
                        uint8_t* accept, poslo_partial* total);

/* ---- serving: continuous batching over registered keys ------------------------------------
 * Not in the paper (which verifies one signer's log at a time); built on poslo_aver_multi.
 * poslo_serve_start starts `workers` host threads (1..8), each with its own internal context
 * on the same device.  Requests are copied at submission (unless flagged POSLO_REQ_BORROW)
 * and admitted against the context's mem_budget (POSLO_EBUSY when the device memory they
 * would need does not fit; 0 = no limit).  A worker copies each request of a batch straight
 * from its buffers into device staging (no host concatenation): lent page-locked requests
 * below 1 MiB are read in place by one gather kernel, larger ones and copied requests by one
 * DMA copy per array (asynchronous when the buffers are page-locked).
 * A free worker takes the oldest pending requests, up to max_batch_devices requests and
 * max_batch_entries entries, and verifies them as one multi-device batch; requests arriving
 * meanwhile join the next batch.  While no worker is idle, a worker also takes its next batch
 * before verifying the current one and stages it in the background (a second set of device
 * buffers), and when fewer entries wait than the workers' next batches would hold, each takes
 * an even share.  Each result is what poslo_distill gives for that request alone.  All
 * serving calls on one context may be made from any host thread. */
typedef struct {
  uint32_t key_id;        /* from poslo_register_key */
  uint32_t n2;
  uint64_t first_index;
  const uint8_t* msgs;    /* host memory, copied at submission */
  const uint64_t* offs;   /* n+1 */
  uint64_t n;
  const uint8_t* s;       /* n*32 */
  const uint8_t* R;       /* n*32 */
  const uint8_t* ds;      /* ds_nodes*24 (always copied) */
  uint32_t ds_nodes;
  uint32_t flags;         /* POSLO_REQ_BORROW: msgs, offs, s and R are not copied at submission;
                             the caller keeps them alive and unchanged until the request's
                             result has been read by poslo_poll */
} poslo_request;
enum { POSLO_REQ_BORROW = 1 };

int poslo_serve_start(poslo_ctx* ctx, uint32_t workers, uint32_t max_batch_devices, uint64_t max_batch_entries);
int poslo_serve_stop(poslo_ctx* ctx);
/* Keys are kept by the service for its lifetime; key ids count from 0.  Registration decodes
 * Y once and keeps its fixed-window table resident on the device (64 KiB per key, outside
 * mem_budget), so batches of registered keys neither decode nor tabulate them again.
 * POSLO_EINVAL if Y does not decode (no id is assigned). */
int poslo_register_key(poslo_ctx* ctx, const uint8_t Y[32], uint32_t* key_id);
/* POSLO_EBUSY: over the memory budget (nothing queued); POSLO_ENOTFOUND: unknown key id. */
int poslo_submit(poslo_ctx* ctx, const poslo_request* req, uint64_t* ticket);
/* Waits up to wait_ms for the result.  POSLO_PENDING if not ready; otherwise the accept bit
 * and the invalid entries' global indices (ascending, room for cap) are written, the time the
 * request spent in the service (from the start of poslo_submit to its result, in ns) goes
 * to *latency_ns (may be NULL), the ticket is retired (unless EBUFSMALL, which keeps it so it
 * can be polled again with more room) and the request's own status is returned (POSLO_OK, or
 * the error its verification met). */
int poslo_poll(poslo_ctx* ctx, uint64_t ticket, uint32_t wait_ms, uint8_t* accept, uint64_t* invalid_idx,
               uint64_t cap, uint64_t* n_invalid, uint64_t* latency_ns);
/* Batches run, requests verified in them, budget bytes held by requests not yet polled. */
int poslo_serve_stats(poslo_ctx* ctx, uint64_t* batches, uint64_t* requests, uint64_t* bytes_in_use);
/* Per-batch timeline of the service (no counterpart in the paper), times in ns since
 * poslo_serve_start on the host's monotonic clock: the worker took the batch (t_take), the
 * copies of its requests' inputs into device staging were issued (t_staged; they run while
 * the worker's previous batch is verified), the inputs had landed and the worker began to
 * verify it (t_verify), the multi-device verification returned (t_checked), every result was
 * published (t_done).  poslo_serve_timeline moves the oldest
 * min(cap, held) records to out (in the order batches finished) and sets *n to that count; the
 * service holds at most 2^20 unread records (later batches are not recorded).  EINVAL without
 * a running service. */
typedef struct {
  uint32_t worker;          /* 0 .. workers - 1 */
  uint32_t requests;
  uint64_t entries;
  uint64_t t_take_ns, t_staged_ns, t_verify_ns, t_checked_ns, t_done_ns;
} poslo_batch_record;
int poslo_serve_timeline(poslo_ctx* ctx, poslo_batch_record* out, uint64_t cap, uint64_t* n);

/* ---- inspection entry points (single steps of the path, for parity tests) ---------------- */

/* SRet (Fig. 2a) for epochs first_epoch .. first_epoch+n_epochs-1: x_0[i] (16 bytes each). */
int poslo_epoch_seeds(poslo_ctx* ctx, const uint8_t* ds, uint32_t ds_nodes, uint64_t first_epoch,
                      uint64_t n_epochs, uint8_t* x0_out);

/* e_t = H(m_t || x_t) mod q for every entry of the batch (Fig. 6 Agg-eKeys, per entry);
 * e_out: n*32 bytes, host or device memory as batch->on_device says. */
int poslo_hash_entries(poslo_ctx* ctx, const poslo_batch* batch, uint8_t* e_out);

/* sum_t [k_t]P_t for n compressed points and n 32-byte scalars (any value below 2^256 is
 * taken as the integer it encodes).  Host or device memory per on_device.  EINVAL if a
 * point does not decode or n > 2^32 - 1. */
int poslo_msm(poslo_ctx* ctx, const uint8_t* points, const uint8_t* scalars, uint64_t n, uint32_t on_device,
              uint8_t out[32]);

/* Window autotuner for the bucket MSM (no counterpart in the paper, whose aggregate uses unit
 * coefficients): times every window width c in [max(8, lg - 8), min(16, lg - 1)], lg =
 * floor(log2 n), on n synthetic points with random scalars of scalar_words 32-bit words (4:
 * the 127-bit verification weights; 8: 256-bit scalars) and keeps the fastest for every later
 * MSM of that size class and scalar width on this context, unless poslo_params.msm_window
 * fixes c; with each width it also times the accumulation's range lengths (see
 * poslo_msm_get_plan).  Untuned classes use c = min(16, max(8, lg - 4)).  Writes the chosen c to
 * window_out (optional).  Allocates about (96 + 4 scalar_words + 16 windows) bytes per point
 * of grow-only scratch.  EINVAL for n = 0, n > 2^32 or another scalar width.  Blocks until
 * the timing runs finish; takes tens of milliseconds per width at n = 2^20. */
int poslo_msm_autotune(poslo_ctx* ctx, uint64_t n, uint32_t scalar_words, uint32_t* window_out);

/* The bucket-MSM plan of a size class (no counterpart in the paper).  A plan is the window
 * width c and the range length 2^range_log2: each thread of the bucket accumulation adds
 * 2^range_log2 consecutive entries of the digit-sorted list, and the pieces of a bucket that
 * crosses ranges are joined afterwards.  poslo_msm_autotune times every range length from
 * 2^4 up to the average bucket size (at most 2^8) beside every width; untuned classes take
 * 2^4, doubled while a bucket averages at least two ranges of the doubled length and the
 * accumulation keeps 1,024 threads per SM.
 * poslo_msm_get_plan writes the plan the next MSM of n entries with scalar_words-word scalars
 * would use (either output may be NULL).  poslo_msm_set_plan stores a plan for n's size class
 * floor(log2 n), e.g. one that an earlier process's autotuner found; a width fixed by
 * poslo_params.msm_window still wins over it.  Both only touch the context's host-side
 * table: no device work, no allocation.  EINVAL for another scalar width, c outside
 * [8, 16] or range_log2 outside [4, 8]. */
int poslo_msm_get_plan(poslo_ctx* ctx, uint64_t n, uint32_t scalar_words, uint32_t* window_out,
                       uint32_t* range_log2_out);
int poslo_msm_set_plan(poslo_ctx* ctx, uint64_t n, uint32_t scalar_words, uint32_t window, uint32_t range_log2);

/* ---- out-of-core verification --------------------------------------------------------- */

/* AVer + Distill of a POSLO-F batch held in HOST memory, chunk_entries entries at a time
 * (the last chunk shorter), for logs larger than device memory (Sec. 7.4 verifies 1 TB of
 * log data chunk by chunk).  While chunk k is verified, chunk k+1 is copied on a separate
 * stream into the other of two staging buffers; with pinned host memory the copies overlap
 * the verification, with pageable memory they are correct but serialised.  The result equals
 * poslo_distill over the whole batch: the invalid entries' global indices, ascending (room
 * for cap; EBUFSMALL after counting them all if more), and *accept = 1 iff there are none.
 * Device memory: two chunks of inputs plus poslo_distill's workspace for one chunk.  EINVAL
 * for a device-resident or POSLO-C batch, chunk_entries = 0 or decreasing offsets. */
int poslo_distill_stream(poslo_ctx* ctx, const poslo_batch* batch, uint64_t chunk_entries, uint8_t* accept,
                         uint64_t* invalid_idx, uint64_t cap, uint64_t* n_invalid);

/* ---- POSLO-C distillation and selective batch verification (Fig. 3b) ------------------- */

/* The distilled record ccd of a POSLO-C batch: the aggregate of its valid epochs (ccd^v),
 * one umbrella aggregate per group of g = n1 / n_umbrella consecutive epochs over the
 * group's valid epochs (ccd^u; a group with no valid epoch holds s = 0, R = identity), and
 * the invalid epochs (ccd^i; their sigma~_i are the batch's own s~_i, R~_i).  All buffers
 * belong to the caller (host memory). */
typedef struct {
  uint8_t* s_v;           /* 32 B: s~^v */
  uint8_t* R_v;           /* 32 B: R~^v, encoded */
  uint8_t* umbrellas;     /* n_umbrella * 64 B: s~^u || R~^u of group l at l * 64 */
  uint64_t* invalid;      /* global epoch indices of ccd^i, ascending; room for cap */
  uint64_t cap;
  uint64_t n_invalid;     /* set by poslo_distill_c; read by poslo_sebver_c */
} poslo_ccd_c;

/* C.Distill (Fig. 3b) over a POSLO-C batch of n1 = n / n2 whole epochs, every epoch checked
 * on its own: b_i = C.AVer(m_i, s~_i, R~_i).  batch->s holds the n1 per-epoch signatures
 * s~_i (32 B each, epoch order) and batch->R the n1 R~_i of pk (R_count = n1).  n_umbrella
 * must divide n1.  valid: n1 bytes (b_i).  EINVAL on a malformed batch or n_umbrella;
 * EBUFSMALL (after filling everything else) if more than ccd->cap epochs are invalid. */
int poslo_distill_c(poslo_ctx* ctx, const poslo_batch* batch, uint32_t n_umbrella, uint8_t* valid,
                    poslo_ccd_c* ccd);

/* SeBVer (Fig. 3b) of the same batch layout against a ccd: mode 'V' writes one bit (every
 * epoch outside ccd^i against ccd^v), 'U' one bit per umbrella (its group's epochs outside
 * ccd^i against the umbrella), 'I' one bit per invalid epoch (its messages against its own
 * s~_i, R~_i from the batch).  bits: room for 1, n_umbrella or ccd->n_invalid bytes. */
enum { POSLO_SEBVER_V = 'V', POSLO_SEBVER_U = 'U', POSLO_SEBVER_I = 'I' };
int poslo_sebver_c(poslo_ctx* ctx, const poslo_batch* batch, uint32_t n_umbrella, const poslo_ccd_c* ccd,
                   uint32_t mode, uint8_t* bits);

/* ---- allocation-free variant ---------------------------------------------------------- */

/* The paper has no counterpart to this entry point: it exists for callers that cannot
 * allocate device memory, such as a process whose device memory is owned by another
 * allocator that has reserved all of it (a framework's caching allocator, a fixed pool
 * sized at start-up) or a service that forbids allocation after its initialisation.
 *
 * It computes what poslo_hash_entries computes on a context of the POSLO_INST_SHA256
 * instantiation (e_t = SHA-256(m_t || x_t) mod q for every entry, n*32 bytes to e_out)
 * without a context and without allocating: no cudaMalloc, no cudaFree, no allocating library
 * routine.  It has no POSLO+ (AES) form: a batch has no instantiation field, and a log signed
 * under POSLO_INST_AES must be hashed through poslo_hash_entries on a POSLO+ context.  Its
 * scratch memory is one file-scope device array of about 1.3 MiB that every GPU loading the
 * library keeps until the process exits.
 *   - batch->on_device must be 1: msgs, offs (and e_out) are device pointers; Y, s and R are
 *     not read; batch->ds is host memory with at most 64 nodes.  The variant and, for
 *     POSLO-C, the whole-epoch rule are checked as poslo_hash_entries checks them; n = 0
 *     returns POSLO_OK without device work.
 *   - Limits: the batch may span at most 65,536 epochs; larger batches return POSLO_EINVAL
 *     before any work is queued.  A seed that ds does not disclose returns POSLO_EINVAL.
 *   - stream: the cudaStream_t to run on (NULL = the legacy default stream).  The call is
 *     synchronous: it returns after that stream has finished its work.
 *   - The first call on each device looks up the scratch array's device address (with that
 *     device current); make that first call before any stream capture.
 *   - Every call on a device shares the one scratch array.  Calls that overlap on the GPU
 *     (from several host threads or streams at once) race on it and must be serialised by
 *     the caller.
 * Returns POSLO_OK, POSLO_EINVAL or POSLO_EDEVICE. */
int poslo_hash_entries_noalloc(const poslo_batch* batch, uint8_t* e_out, void* stream);

/* ---- profiling -------------------------------------------------------------------------- */

/* When enabled, the context brackets each hot kernel with CUDA events on its own stream and
 * accumulates the durations: poslo_kernel_time() returns total milliseconds and launch count
 * for kernel `name` ("hash", "points", "msm", "finalize", ...); poslo_reset_kernel_times()
 * clears them. */
int poslo_set_profiling(poslo_ctx* ctx, int enabled);
int poslo_kernel_time(poslo_ctx* ctx, const char* name, double* total_ms, uint64_t* launches);
void poslo_reset_kernel_times(poslo_ctx* ctx);

/* ---- CUDA-graph replay (no counterpart in the paper) ------------------------------------ */

/* poslo_aver_multi and poslo_distill run their work up to the first host decision (the
 * combined weighted check) as a fixed sequence of launches.  When a call has the same shape
 * as the previous call of that entry point on this context -- for poslo_aver_multi the
 * device count, segment tables, seeds layout, batch pointers (device-resident inputs) and
 * MSM plan; for poslo_distill a device-resident batch with the same pointers, n, n2,
 * first_index and ds layout -- the sequence is captured into a CUDA graph, and later calls of
 * that shape launch the graph instead of the individual kernels.  The contents of every
 * input (messages, signatures, keys, seeds) are read afresh on each call; the uploads of
 * host-side tables happen before the graph runs.  A workspace reallocation in between, or
 * profiling (poslo_set_profiling), makes the call run its launches directly.  Enabled by
 * default; poslo_set_graphs(ctx, 0) turns it off and frees the graphs.
 * poslo_graph_stats reports how many graphs were captured and how many replays ran. */
int poslo_set_graphs(poslo_ctx* ctx, int enabled);

/* Form of poslo_aver_multi's combined weighted check (no counterpart in the paper).  Batches
 * of at most max_entries entries (default 0: none) check it window by window of the weights'
 * signed digits -- sum_t d_{t,w} R_t = sum_d (sum_{t in d} d_{t,w} e_t) Y_d + (sum_t d_{t,w} s_t) G
 * for every window w, which together imply the check with the full weights -- and so skip the
 * MSM's doublings between windows on their critical path, at the cost of per-device,
 * per-window scalar sums (one block per device and window).  Results are the same either way.
 * EINVAL for a null context. */
int poslo_set_multi_window_limit(poslo_ctx* ctx, uint64_t max_entries);

/* Key cache (no counterpart in the paper).  poslo_distill and poslo_aver_multi (without
 * resident tables) need the fixed-window table of every public key they check, whose
 * construction is a chain of 252 dependent point doublings (about 0.3 ms, however many keys
 * are built at once).  The context keeps the tables of the `capacity` most recently used keys
 * (64 KiB each, device memory allocated in blocks of 256 keys, counted against
 * poslo_params.mem_budget; default 4,096 keys) and builds only the keys it misses.  A key
 * whose encoding does not decode, or whose call fails, is not kept.  A call with more keys
 * than the capacity builds all of its tables without the cache.  poslo_set_key_cache drops
 * every cached table and sets the capacity (0 turns the cache off); poslo_key_cache_stats
 * counts lookups that hit and missed.  EINVAL for a null context. */
int poslo_set_key_cache(poslo_ctx* ctx, uint32_t capacity);
int poslo_key_cache_stats(poslo_ctx* ctx, uint64_t* hits, uint64_t* misses);
int poslo_graph_stats(poslo_ctx* ctx, uint64_t* captures, uint64_t* replays);

#ifdef __cplusplus
}
#endif

#endif /* POSLO_H_ */
