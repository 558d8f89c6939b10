// libposlo: host orchestration and the C ABI declared in include/poslo.h.
//
// One context owns its CUDA streams: the main stream runs the seeds, weights, counting sort
// and MSM and the final check; a side stream builds the window table of the public key Y
// while hashing runs; a third stream decodes and sums the commitments R_t; a fourth hashes
// the messages during the decoding.  The hash kernel is
// bound by the integer ALU pipe (SHA-256) and the point kernel by the IMAD pipe (field
// multiplication), so running them concurrently lets both pipes issue on every SM.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/poslo.h"
#include "common.cuh"

using namespace poslo;


#include "ctx.h"

using poslo_host::DevBuf;
using poslo_host::KernelTimer;
using poslo_host::kSmallHostBytes;

namespace {

int fail(poslo_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CU(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(ctx, POSLO_EDEVICE, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Internal status: a workspace buffer would have to grow during a stream capture.
constexpr int kCaptureGrow = -100;

// Grow-only named workspace buffers.
int ensure(poslo_ctx* ctx, const char* name, size_t bytes, void** out) {
  DevBuf& b = ctx->bufs[name];
  if (bytes == 0) bytes = 16;
  if (b.cap < bytes) {
    // no allocation (and none of its synchronisation) inside a stream capture: the caller
    // abandons the capture and runs the sequence directly
    if (ctx->capturing) return kCaptureGrow;
    ++ctx->alloc_gen;
    size_t want = std::max(bytes, b.cap + b.cap / 2);
    want = (want + 255) & ~size_t(255);
    if (ctx->mem_budget && ctx->mem_used - b.cap + want > ctx->mem_budget)
      return fail(ctx, POSLO_ENOMEM, "workspace '%s' of %zu bytes exceeds the memory budget", name, want);
    if (b.p) {
      cudaStreamSynchronize(ctx->s_main);
      cudaStreamSynchronize(ctx->s_table);
      cudaStreamSynchronize(ctx->s_points);
      cudaFree(b.p);
      ctx->mem_used -= b.cap;
      b.p = nullptr;
      b.cap = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) return fail(ctx, POSLO_ENOMEM, "cudaMalloc(%zu) for '%s': %s", want, name, cudaGetErrorString(e));
    b.cap = want;
    ctx->mem_used += want;
  }
  *out = b.p;
  return POSLO_OK;
}

template <class T>
int ensure_t(poslo_ctx* ctx, const char* name, size_t bytes, T** out) {
  void* p;
  int rc = ensure(ctx, name, bytes, &p);
  *out = static_cast<T*>(p);
  return rc;
}

// Device view of a caller buffer: either the caller's device pointer or a copy.
int stage(poslo_ctx* ctx, const char* name, const void* src, size_t bytes, bool on_device, cudaStream_t st,
          const void** out) {
  if (on_device || bytes == 0) {
    *out = src;
    if (bytes == 0 && !src) {
      void* p;
      int rc = ensure(ctx, name, 16, &p);
      if (rc) return rc;
      *out = p;
    }
    return POSLO_OK;
  }
  void* p;
  int rc = ensure(ctx, name, bytes, &p);
  if (rc) return rc;
  CU(cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, st));
  *out = p;
  return POSLO_OK;
}

void timer_begin(poslo_ctx* ctx, const char* name, cudaStream_t st, cudaEvent_t* b, cudaEvent_t* e) {
  *b = *e = nullptr;
  if (!ctx->profiling) return;
  auto take = [&]() {
    cudaEvent_t ev;
    if (!ctx->event_pool.empty()) {
      ev = ctx->event_pool.back();
      ctx->event_pool.pop_back();
    } else {
      cudaEventCreate(&ev);
    }
    return ev;
  };
  *b = take();
  *e = take();
  cudaEventRecord(*b, st);
  (void)name;
}

void timer_end(poslo_ctx* ctx, const char* name, cudaStream_t st, cudaEvent_t b, cudaEvent_t e) {
  if (!ctx->profiling || !b) return;
  cudaEventRecord(e, st);
  ctx->pending.push_back({name, {b, e}});
}

void timers_collect(poslo_ctx* ctx) {
  for (auto& p : ctx->pending) {
    cudaEventSynchronize(p.second.second);
    float ms = 0;
    cudaEventElapsedTime(&ms, p.second.first, p.second.second);
    KernelTimer& t = ctx->timers[p.first];
    t.total_ms += ms;
    t.launches += 1;
    ctx->event_pool.push_back(p.second.first);
    ctx->event_pool.push_back(p.second.second);
  }
  ctx->pending.clear();
}

uint32_t load_be32(const uint8_t* b) {
  return ((uint32_t)b[0] << 24) | ((uint32_t)b[1] << 16) | ((uint32_t)b[2] << 8) | b[3];
}

int parse_ds(poslo_ctx* ctx, const uint8_t* ds, uint32_t nodes, std::vector<DsNode>& out) {
  if (nodes == 0 || !ds) return fail(ctx, POSLO_EINVAL, "empty disclosed-seed stack");
  out.resize(nodes);
  for (uint32_t k = 0; k < nodes; ++k) {
    const uint8_t* b = ds + 24 * (size_t)k;
    DsNode n;
    n.d = b[0] | (b[1] << 8) | (b[2] << 16) | ((uint32_t)b[3] << 24);
    n.i = b[4] | (b[5] << 8) | (b[6] << 16) | ((uint32_t)b[7] << 24);
    if (n.d > 40) return fail(ctx, POSLO_EINVAL, "ds node %u: depth %u too large", k, n.d);
    for (int w = 0; w < 4; ++w) n.seed[w] = load_be32(b + 8 + 4 * w);
    out[k] = n;
  }
  return POSLO_OK;
}

int grid_for(const poslo_ctx* ctx, uint64_t n, int threads, int per_sm) {
  const uint64_t need = (n + threads - 1) / threads;
  const uint64_t cap = (uint64_t)ctx->sm_count * per_sm;
  return (int)std::max<uint64_t>(1, std::min(need, cap));
}

int check_status(poslo_ctx* ctx) {
  CU(cudaMemcpyAsync(ctx->h_status, ctx->status, 4, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaStreamSynchronize(ctx->s_main));
  const uint32_t st = *ctx->h_status;
  if (st & kErrSeed) return fail(ctx, POSLO_EINVAL, "a requested epoch seed is not disclosed by ds (SRet bottom)");
  if (st & kErrKey) return fail(ctx, POSLO_EINVAL, "public key Y does not decode");
  if (st & kErrTimeout) return fail(ctx, POSLO_ETIMEOUT, "device-side wait expired");
  if (st & kErrInput) return fail(ctx, POSLO_EINVAL, "message offsets decrease (or precede msgs)");
  return POSLO_OK;
}

int reset_status(poslo_ctx* ctx) {
  CU(cudaMemsetAsync(ctx->status, 0, 4, ctx->s_main));
  return POSLO_OK;
}

void graph_reset(poslo_host::GraphSlot& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  g.sig.clear();
}

// Runs launch() -- a sequence of launches, device-side copies and event waits that starts
// and ends on s_main, allocates nothing and does not synchronise -- or replays it.  The
// first call of a shape runs it directly; a second call of the same shape in a row captures
// it into a CUDA graph (thread-local capture on s_main; the side streams join through their
// events) and launches the graph; later calls of that shape launch the graph again.  A
// workspace reallocation since the capture, profiling (whose timers are host-side events)
// or graphs switched off fall back to running it directly.
template <class F>
int run_replayable(poslo_ctx* ctx, poslo_host::GraphSlot& g, const std::vector<uint64_t>& sig, F&& launch) {
  if (!ctx->graphs || ctx->profiling) {
    graph_reset(g);
    g.last_sig.clear();
    return launch();
  }
  if (g.exec && g.sig == sig && g.gen == ctx->alloc_gen) {
    CU(cudaGraphLaunch(g.exec, ctx->s_main));
    ctx->launch_count += g.launches;
    ++ctx->graph_replays;
    return POSLO_OK;
  }
  if (g.last_sig != sig) {
    g.last_sig = sig;
    return launch();
  }
  graph_reset(g);
  const uint64_t launches0 = ctx->launch_count;
  CU(cudaStreamBeginCapture(ctx->s_main, cudaStreamCaptureModeThreadLocal));
  ctx->capturing = true;
  int rc = launch();
  ctx->capturing = false;
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(ctx->s_main, &graph);
  if (rc != POSLO_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();   // a failed capture leaves its error behind
    g.last_sig.clear();
    ctx->launch_count = launches0;
    return launch();   // run it directly (a genuine error shows there again)
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    g.last_sig.clear();
    ctx->launch_count = launches0;
    return launch();
  }
  g.exec = exec;
  g.sig = sig;
  g.gen = ctx->alloc_gen;
  g.launches = ctx->launch_count - launches0;
  ++ctx->graph_captures;
  CU(cudaGraphLaunch(g.exec, ctx->s_main));
  return POSLO_OK;
}

uint32_t log2_exact(uint32_t n) {
  if (n == 0 || (n & (n - 1))) return 0xffffffffu;
  uint32_t l = 0;
  while ((1u << l) < n) ++l;
  return l;
}

// Epoch seeds for global entries [first, first+n) into buffer "seeds"; returns e0.
int run_epoch_seeds(poslo_ctx* ctx, const uint8_t* ds, uint32_t nodes, uint64_t first_epoch, uint64_t n_epochs,
                    uint32_t** seeds_out) {
  std::vector<DsNode> h;
  int rc = parse_ds(ctx, ds, nodes, h);
  if (rc) return rc;
  DsNode* d_ds;
  if ((rc = ensure_t(ctx, "ds", h.size() * sizeof(DsNode), &d_ds))) return rc;
  CU(cudaMemcpyAsync(d_ds, h.data(), h.size() * sizeof(DsNode), cudaMemcpyHostToDevice, ctx->s_main));
  uint32_t* seeds;
  if ((rc = ensure_t(ctx, "seeds", std::max<uint64_t>(1, n_epochs) * 16, &seeds))) return rc;
  if (n_epochs) {
    const int threads = 128;
    const uint64_t blocks = (n_epochs + threads - 1) / threads;
    cudaEvent_t b, e;
    timer_begin(ctx, "seeds", ctx->s_main, &b, &e);
    launch_epoch_seeds((int)ctx->inst, (unsigned)blocks, threads, ctx->s_main, d_ds, (int)h.size(), first_epoch,
                       n_epochs, seeds, ctx->status);
    ++ctx->launch_count;
    CU(cudaGetLastError());
    timer_end(ctx, "seeds", ctx->s_main, b, e);
  }
  *seeds_out = seeds;
  return POSLO_OK;
}

struct Staged {
  const uint8_t* msgs = nullptr;
  const uint64_t* offs = nullptr;
  uint64_t base_off = 0;
  const uint8_t* s = nullptr;
  const uint8_t* R = nullptr;
  bool packed = false;   // a host batch that went up as one copy before any launch
};

// Host batches up to this many bytes (R_t, offsets, messages, s_t) are packed into page-locked
// memory and go up as one copy: fewer, asynchronous copies, and every input is on the device
// before the first launch, so the launch sequence can be replayed from a CUDA graph as for
// device-resident batches.  Larger host batches are copied array by array, R_t first, so that
// the decoding starts while the messages are still in flight (and page-locked callers' arrays
// go by DMA without a host copy).
constexpr size_t kPackMaxBytes = 1u << 20;

bool device_aligned(const void* offs, const void* s, const void* R) {
  return !(reinterpret_cast<uintptr_t>(offs) & 7) && !(reinterpret_cast<uintptr_t>(s) & 15) &&
         !(reinterpret_cast<uintptr_t>(R) & 15);
}

int validate_batch(poslo_ctx* ctx, const poslo_batch* b) {
  if (!b) return fail(ctx, POSLO_EINVAL, "null batch");
  if (b->variant != POSLO_VARIANT_C && b->variant != POSLO_VARIANT_F) return fail(ctx, POSLO_EINVAL, "bad variant");
  if (b->n2 == 0) return fail(ctx, POSLO_EINVAL, "n2 must be >= 1");
  if (!b->Y) return fail(ctx, POSLO_EINVAL, "missing public key");
  if (b->n && (!b->offs || !b->s || !b->R)) return fail(ctx, POSLO_EINVAL, "missing batch arrays");
  if (b->variant == POSLO_VARIANT_C) {
    if (b->n % b->n2 || b->first_index % b->n2)
      return fail(ctx, POSLO_EINVAL, "POSLO-C batches hold whole epochs of n2 entries");
    if (!b->s || !b->R) return fail(ctx, POSLO_EINVAL, "POSLO-C needs s~ and R");
    if (b->R_count != 1 && b->R_count != b->n / b->n2)
      return fail(ctx, POSLO_EINVAL, "POSLO-C R_count must be 1 or n/n2");
  } else {
    if (b->R_count != b->n) return fail(ctx, POSLO_EINVAL, "POSLO-F R_count must equal n");
  }
  // the kernels read device-resident offsets as 8-byte words and s, R as 16-byte vectors
  if (b->on_device && b->n && !device_aligned(b->offs, b->s, b->R))
    return fail(ctx, POSLO_EINVAL, "device-resident offs must be 8-byte aligned, s and R 16-byte aligned");
  return POSLO_OK;
}

// One verification call indexes its entries with 32-bit indices inside the MSM and the
// localisation; longer logs go through poslo_distill_stream in chunks.
constexpr uint64_t kMaxCallEntries = (1ull << 32) - 1;
// Distill batches up to this many entries are localised by every entry's own check (one
// launch, eight lanes per entry) rather than by the descent over the segment tree: measured
// on GB300, 0.18 ms of checking at 4,096 entries and 0.56 ms at 16,384 against 1.0 ms of
// tree, descent and confirmation; the two meet near 32,768.
constexpr uint64_t kDirectCheckMax = 16384;

// Host inputs are copied R_t first: ev_staged marks their arrival, so the decoding (the
// longest stage) starts while the messages are still on their way.
int stage_batch(poslo_ctx* ctx, const poslo_batch* b, Staged& sb, size_t s_bytes_override = 0) {
  int rc;
  const bool dev = b->on_device != 0;
  const void* p;
  const size_t s_bytes = s_bytes_override ? s_bytes_override : (b->variant == POSLO_VARIANT_F ? 32 * b->n : 32);
  const size_t R_bytes = 32 * (b->variant == POSLO_VARIANT_F ? b->n : b->R_count);
  if (!dev && b->n) {
    const uint64_t lo = b->offs[0], hi = b->offs[b->n];
    if (hi < lo) return fail(ctx, POSLO_EINVAL, "offsets decrease");
    const size_t offs_bytes = 8 * (b->n + 1), msg_bytes = hi - lo;
    auto up16 = [](size_t x) { return (x + 15) & ~size_t(15); };
    const size_t oR = 0, oO = up16(R_bytes), oM = oO + up16(offs_bytes), oS = oM + up16(msg_bytes);
    const size_t total = oS + up16(s_bytes);
    if (total <= kPackMaxBytes) {
      if (ctx->h_pack_cap < total) {
        if (ctx->h_pack) cudaFreeHost(ctx->h_pack);
        ctx->h_pack = nullptr;
        ctx->h_pack_cap = 0;
        const size_t want = std::max<size_t>(total, 1 << 20);
        if (cudaMallocHost(&ctx->h_pack, want) != cudaSuccess) {
          cudaGetLastError();
          return fail(ctx, POSLO_ENOMEM, "page-locked staging of %zu bytes", want);
        }
        ctx->h_pack_cap = want;
      }
      uint8_t* d;
      if ((rc = ensure_t(ctx, "packed_in", total, &d))) return rc;
      // the previous call's copy out of h_pack has completed: every call ends synchronised
      memcpy(ctx->h_pack + oR, b->R, R_bytes);
      memcpy(ctx->h_pack + oO, b->offs, offs_bytes);
      if (msg_bytes) memcpy(ctx->h_pack + oM, b->msgs + lo, msg_bytes);
      memcpy(ctx->h_pack + oS, b->s, s_bytes);
      CU(cudaMemcpyAsync(d, ctx->h_pack, total, cudaMemcpyHostToDevice, ctx->s_main));
      CU(cudaEventRecord(ctx->ev_staged, ctx->s_main));
      sb.R = d + oR;
      sb.offs = reinterpret_cast<const uint64_t*>(d + oO);
      sb.msgs = d + oM;
      sb.base_off = lo;
      sb.s = d + oS;
      sb.packed = true;
      return POSLO_OK;
    }
  }
  if ((rc = stage(ctx, "R_in", b->R, R_bytes, dev, ctx->s_main, &p))) return rc;
  sb.R = static_cast<const uint8_t*>(p);
  CU(cudaEventRecord(ctx->ev_staged, ctx->s_main));
  if (b->n == 0) {
    uint64_t* z;
    if ((rc = ensure_t(ctx, "offs", 16, &z))) return rc;
    CU(cudaMemsetAsync(z, 0, 16, ctx->s_main));
    sb.offs = z;
    sb.msgs = reinterpret_cast<const uint8_t*>(z);
  } else {
    if ((rc = stage(ctx, "offs", b->offs, (b->n + 1) * 8, dev, ctx->s_main, &p))) return rc;
    sb.offs = static_cast<const uint64_t*>(p);
    if (dev) {
      sb.msgs = b->msgs;
      sb.base_off = 0;
    } else {
      // monotonicity of every offset is checked on the device (k_hash)
      const uint64_t lo = b->offs[0], hi = b->offs[b->n];
      if (hi < lo) return fail(ctx, POSLO_EINVAL, "offsets decrease");
      if ((rc = stage(ctx, "msgs", b->msgs + lo, hi - lo, false, ctx->s_main, &p))) return rc;
      sb.msgs = static_cast<const uint8_t*>(p);
      sb.base_off = lo;
    }
  }
  if ((rc = stage(ctx, "s_in", b->s, s_bytes, dev, ctx->s_main, &p))) return rc;
  sb.s = static_cast<const uint8_t*>(p);
  return POSLO_OK;
}

void make_zpre(const uint8_t vseed[32], uint32_t zpre[10]) {
  uint8_t buf[40] = {'P', 'O', 'S', 'L', 'O', '-', 'Z'};
  memcpy(buf + 7, vseed, 32);
  buf[39] = 0;
  for (int i = 0; i < 10; ++i) zpre[i] = load_be32(buf + 4 * i);
}

// Hash stage shared by AVer, Distill and the inspection call.
int run_hash(poslo_ctx* ctx, const poslo_batch* b, const Staged& sb, uint8_t* e_out, bool weighted, bool with_s,
             uint32_t* z_out, unsigned long long** partial_out, uint32_t* nblocks_out) {
  int rc;
  uint64_t e_first = 0, ne = 0;
  if (b->n) {
    e_first = b->first_index / b->n2;
    ne = (b->first_index + b->n - 1) / b->n2 - e_first + 1;
  }
  uint32_t* seeds;
  if ((rc = run_epoch_seeds(ctx, b->ds, b->ds_nodes, e_first, ne, &seeds))) return rc;
  const int blocks = grid_for(ctx, b->n, kHashThreads, 8);
  unsigned long long* partial;
  if ((rc = ensure_t(ctx, "hash_partial", (size_t)blocks * kPartialWords * 8, &partial))) return rc;
  HashArgs a{};
  a.msgs = sb.msgs;
  a.offs = sb.offs;
  a.base_off = sb.base_off;
  a.n = b->n;
  a.first_index = b->first_index;
  a.e0 = e_first;
  a.n2 = b->n2;
  a.n2_log2 = log2_exact(b->n2);
  a.seeds = seeds;
  a.e_out = e_out;
  a.s = with_s ? sb.s : nullptr;
  a.weighted = weighted ? 1u : 0u;
  make_zpre(ctx->vseed, a.zpre);
  a.z_out = z_out;
  a.partial = partial;
  a.status = ctx->status;
  cudaEvent_t tb, te;
  timer_begin(ctx, "hash", ctx->s_main, &tb, &te);
  launch_hash((int)ctx->inst, (unsigned)blocks, ctx->s_main, a);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  timer_end(ctx, "hash", ctx->s_main, tb, te);
  *partial_out = partial;
  *nblocks_out = (uint32_t)blocks;
  return POSLO_OK;
}

// Window table of Y on the side stream (ordered after the main stream's uploads).
// Window tables of n keys on stream st (k_table_chain, then k_table_fill).
int launch_tables(poslo_ctx* ctx, cudaStream_t st, const uint32_t* enc, const uint32_t* pts, const uint32_t* list,
                  uint32_t n, uint32_t* tables, int use_base, uint8_t* bad_out, uint32_t* const* dst = nullptr) {
  if (n == 0) return POSLO_OK;
  k_table_chain<<<(unsigned)((4ull * n + 127) / 128), 128, 0, st>>>(enc, pts, list, n, tables, dst, ctx->status,
                                                                    use_base, bad_out);
  k_table_fill<<<(unsigned)((4ull * n * kTableWindows + 127) / 128), 128, 0, st>>>(n, tables, dst);
  ctx->launch_count += 2;
  CU(cudaGetLastError());
  return POSLO_OK;
}

// ---- key cache ----
uint32_t* key_slot_table(const poslo_host::KeyCache& C, uint32_t slot) {
  return C.blocks[slot / poslo_host::KeyCache::kBlock] + (size_t)(slot % poslo_host::KeyCache::kBlock) * kTableWords;
}

// Window tables of nd keys (host encodings, 32 bytes each) from the context's key cache:
// tabs[d] is key d's table.  Keys not cached get a slot -- a free one, else the least
// recently used -- and are listed in miss (their index d) and miss_dst (their table) for the
// caller to build.  Returns false, leaving the cache untouched, when the cache is off, holds
// fewer slots than the call has keys, or cannot grow within the memory budget.
bool key_cache_lookup(poslo_ctx* ctx, const uint8_t* Y, uint32_t nd, std::vector<const uint32_t*>& tabs,
                      std::vector<uint32_t>& miss, std::vector<uint32_t*>& miss_dst) {
  poslo_host::KeyCache& C = ctx->keys;
  if (C.capacity == 0 || C.capacity < nd) return false;
  // grow the slot blocks first, so that no key is assigned a slot the cache then cannot hold
  const uint32_t want = std::min(C.capacity, std::max(C.nslots, nd + C.nslots - (uint32_t)C.free_slots.size()));
  while ((size_t)C.blocks.size() * poslo_host::KeyCache::kBlock < want) {
    const size_t bytes = (size_t)poslo_host::KeyCache::kBlock * kTableWords * 4;
    if (ctx->mem_budget && ctx->mem_used + bytes > ctx->mem_budget) return false;
    uint32_t* b = nullptr;
    if (cudaMalloc(&b, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    ctx->mem_used += bytes;
    C.blocks.push_back(b);
  }
  tabs.assign(nd, nullptr);
  miss.clear();
  miss_dst.clear();
  for (uint32_t d = 0; d < nd; ++d) {
    std::array<uint8_t, 32> k;
    memcpy(k.data(), Y + 32 * (size_t)d, 32);
    uint32_t slot;
    auto it = C.slot_of.find(k);
    if (it != C.slot_of.end()) {
      slot = it->second;
      C.lru.splice(C.lru.begin(), C.lru, C.pos[slot]);
      ++C.hits;
    } else {
      ++C.misses;
      if (!C.free_slots.empty()) {
        slot = C.free_slots.back();
        C.free_slots.pop_back();
      } else if (C.nslots < C.capacity && C.nslots < (uint32_t)C.blocks.size() * poslo_host::KeyCache::kBlock) {
        slot = C.nslots++;
        C.key_of.resize(C.nslots);
        C.pos.resize(C.nslots);
      } else {   // evict the least recently used key (never one of this call: nd <= capacity)
        slot = C.lru.back();
        C.lru.pop_back();
        C.slot_of.erase(C.key_of[slot]);
      }
      C.key_of[slot] = k;
      C.slot_of[k] = slot;
      C.lru.push_front(slot);
      C.pos[slot] = C.lru.begin();
      miss.push_back(d);
      miss_dst.push_back(key_slot_table(C, slot));
    }
    tabs[d] = key_slot_table(C, slot);
  }
  return true;
}

// Drops a key from the cache (its table was built from an encoding that does not decode, or
// the call that built it failed).
void key_cache_forget(poslo_ctx* ctx, const uint8_t* Y32) {
  poslo_host::KeyCache& C = ctx->keys;
  std::array<uint8_t, 32> k;
  memcpy(k.data(), Y32, 32);
  auto it = C.slot_of.find(k);
  if (it == C.slot_of.end()) return;
  const uint32_t slot = it->second;
  C.lru.erase(C.pos[slot]);
  C.slot_of.erase(it);
  C.free_slots.push_back(slot);
}

// Until a call has built them, the key cache must not keep the tables of the keys it missed:
// on any early return they are dropped again (armed until the build is known sound).
struct KeyForget {
  poslo_ctx* ctx;
  const uint8_t* Y;                      // the call's key encodings
  const std::vector<uint32_t>* miss;     // indices of the missed keys
  bool armed;
  ~KeyForget() {
    if (armed)
      for (uint32_t k : *miss) key_cache_forget(ctx, Y + 32 * (size_t)k);
  }
};

// The window table of Y, built on the table stream into `into` (a key-cache slot) or, when
// null, into the context's scratch table.
int run_ytable(poslo_ctx* ctx, const uint8_t* Y, uint32_t** table_out, uint32_t* into = nullptr) {
  int rc;
  uint32_t* d_Y;
  if ((rc = ensure_t(ctx, "Y", 32, &d_Y))) return rc;
  uint32_t* tableY = into;
  if (!tableY && (rc = ensure_t(ctx, "tableY", 4 * (size_t)kTableWords, &tableY))) return rc;
  CU(cudaMemcpyAsync(d_Y, Y, 32, cudaMemcpyHostToDevice, ctx->s_main));
  CU(cudaEventRecord(ctx->ev_main, ctx->s_main));
  CU(cudaStreamWaitEvent(ctx->s_table, ctx->ev_main, 0));
  cudaEvent_t tb, te;
  timer_begin(ctx, "table", ctx->s_table, &tb, &te);
  if ((rc = launch_tables(ctx, ctx->s_table, d_Y, nullptr, nullptr, 1, tableY, 0, nullptr))) return rc;
  timer_end(ctx, "table", ctx->s_table, tb, te);
  CU(cudaEventRecord(ctx->ev_table, ctx->s_table));
  *table_out = tableY;
  return POSLO_OK;
}

// Resident decode blocks per SM: below the register-file limit (4) the remaining registers
// host a hash block, so SHA-256 (ALU pipe) runs beside the field arithmetic (IMAD pipe).
#ifndef POSLO_POINTS_BLOCKS
#define POSLO_POINTS_BLOCKS 3
#endif

// The decoding waits for `after` (an event on the main stream) when given, else for all main
// stream work so far.
int run_points(poslo_ctx* ctx, const uint8_t* R, uint64_t count, uint32_t* pts_out, uint8_t* bad_out,
               uint32_t** partial_out, uint32_t* nblocks_out, cudaEvent_t after = nullptr, bool coresident = false) {
  int rc;
  const int blocks = grid_for(ctx, count, kPointThreads, POSLO_POINTS_BLOCKS);
  uint32_t* partial;
  if ((rc = ensure_t(ctx, "point_partial", (size_t)blocks * kPointPartialWords * 4, &partial))) return rc;
  if (!after) {
    CU(cudaEventRecord(ctx->ev_main, ctx->s_main));
    after = ctx->ev_main;
  }
  CU(cudaStreamWaitEvent(ctx->s_points, after, 0));
  uint32_t* work;
  if ((rc = ensure_t(ctx, "point_work", 16, &work))) return rc;
  PointArgs a{};
  a.R = R;
  a.count = count;
  a.partial = partial;
  a.pts_out = pts_out;
  a.bad_out = bad_out;
  a.work = work;
  CU(cudaMemsetAsync(work, 0, 4, ctx->s_points));
  cudaEvent_t tb, te;
  timer_begin(ctx, "points", ctx->s_points, &tb, &te);
  launch_points((unsigned)blocks, ctx->s_points, a, coresident);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  timer_end(ctx, "points", ctx->s_points, tb, te);
  CU(cudaEventRecord(ctx->ev_decoded, ctx->s_points));   // the decoded points alone
  CU(cudaEventRecord(ctx->ev_points, ctx->s_points));    // callers that add work re-record it
  *partial_out = partial;
  *nblocks_out = (uint32_t)blocks;
  return POSLO_OK;
}

// Pippenger plan: the window c comes from the context (poslo_params.msm_window) or from the
// autotuned table for this size class (see poslo_msm_autotune); the default before tuning is
// c = log2(n) - 4 clamped to [8, 16].
MsmPlan msm_plan_c(int c, int sw, int seg_log2 = kMsmSegLog2Min) {
  MsmPlan pl;
  pl.c = c;
  pl.sw = sw;
  const int bits = sw == 4 ? 127 : 256;
  pl.windows = (bits + 1 + c - 1) / c;
  pl.nb = (1u << (c - 1)) + kMsmChunk;
  pl.nchunks = pl.nb / kMsmChunk;
  pl.jbits = c - 4;
  pl.seg_log2 = seg_log2;
  return pl;
}

// Range length 2^lg of the bucket accumulation when it is not tuned: 16 sorted entries,
// doubled while a bucket still averages at least two ranges of the doubled length (so that
// joining the pieces of a bucket stays a short chain) and the accumulation keeps at least
// 1,024 threads per SM.
int msm_seg_default(const MsmPlan& pl, uint64_t n, int sm_count) {
  int lg = kMsmSegLog2Min;
  const uint64_t per_bucket = n >> (pl.c - 1);
  while (lg < kMsmSegLog2Max && (4ull << lg) <= per_bucket &&
         ((uint64_t)pl.windows * n >> (lg + 1)) >= 1024ull * (uint64_t)sm_count)
    ++lg;
  return lg;
}

// A width is balanced when the last window still holds at least 5 bits of the scalar: with
// fewer, its few digit values put a large share of all entries into one or two buckets.
// (127-bit weights: c = 9 and 14 are not; 8-word scalars below 2^253: c = 9, 10, 12, 14.)
bool msm_width_balanced(int c, int sw) {
  const int bits = sw == 4 ? 127 : 253;   // 8-word scalars are usually reduced mod q
  const int windows = (bits + c - 1) / c;
  return bits - (windows - 1) * c >= 5;
}

// The balanced width nearest to c from below (c = 8 is balanced for both scalar widths).
int msm_balanced_width(int c, int sw) {
  while (c > 8 && !msm_width_balanced(c, sw)) --c;
  return c;
}

int log2_floor(uint64_t n) {
  int lg = 0;
  while ((1ull << (lg + 1)) <= std::max<uint64_t>(n, 1)) ++lg;
  return lg;
}

MsmPlan msm_plan(poslo_ctx* ctx, uint64_t n, int sw) {
  int c = (int)ctx->msm_window;
  if (c == 0) {
    const int lg = log2_floor(n);
    auto it = ctx->msm_tuned.find(lg * 16 + sw);
    if (it != ctx->msm_tuned.end()) return msm_plan_c(it->second & 0xff, sw, it->second >> 8);
    c = msm_balanced_width(std::min(16, std::max(8, lg - 4)), sw);
  }
  MsmPlan pl = msm_plan_c(c, sw);
  pl.seg_log2 = msm_seg_default(pl, n, ctx->sm_count);
  return pl;
}

// Pippenger in two halves so the counting sort (which needs only the scalars) can run
// while the points are still being decoded on the other stream.
struct MsmState {
  MsmPlan pl;
  uint64_t n = 0;
  uint32_t *cnt = nullptr, *off = nullptr, *idx = nullptr;
  uint16_t* bkt = nullptr;
};

// Counting sort of (window, entry) pairs by digit; skip_sort entries take no part at all.
int run_msm_sort(poslo_ctx* ctx, cudaStream_t st, const uint32_t* z, int sw, const uint8_t* skip_sort, uint64_t n,
                 MsmState& ms, const MsmPlan* forced = nullptr) {
  int rc;
  ms.pl = forced ? *forced : msm_plan(ctx, n, sw);
  ms.n = n;
  const MsmPlan& pl = ms.pl;
  const size_t nbw = (size_t)pl.windows * pl.nb;
  uint32_t* rank;
  if ((rc = ensure_t(ctx, "msm_cnt", 4 * nbw, &ms.cnt))) return rc;
  if ((rc = ensure_t(ctx, "msm_off", 4 * nbw, &ms.off))) return rc;
  if ((rc = ensure_t(ctx, "msm_rank", 4 * (size_t)pl.windows * std::max<uint64_t>(n, 1), &rank))) return rc;
  if ((rc = ensure_t(ctx, "msm_idx", 4 * (size_t)pl.windows * std::max<uint64_t>(n, 1), &ms.idx))) return rc;
  if ((rc = ensure_t(ctx, "msm_bkt", 2 * (size_t)pl.windows * std::max<uint64_t>(n, 1), &ms.bkt))) return rc;
  cudaEvent_t sb_, se_;
  timer_begin(ctx, "msm_sort", st, &sb_, &se_);
  CU(cudaMemsetAsync(ms.cnt, 0, 4 * nbw, st));
  if (n) {
    const int g = grid_for(ctx, n, kSideThreads, 16);
    k_msm_count<<<g, kSideThreads, 0, st>>>(z, skip_sort, n, pl, ms.cnt, rank);
    k_msm_scan<<<pl.windows, kSideThreads, 0, st>>>(ms.cnt, ms.off, pl);
    k_msm_scatter<<<g, kSideThreads, 0, st>>>(z, skip_sort, n, pl, ms.off, rank, ms.idx, ms.bkt);
    ctx->launch_count += 3;
  }
  CU(cudaGetLastError());
  timer_end(ctx, "msm_sort", st, sb_, se_);
  return POSLO_OK;
}

// Bucket sums (entries flagged in skip_add are left out), window sums and Horner's rule.
int run_msm_finish(poslo_ctx* ctx, cudaStream_t st, const uint32_t* pts, const uint8_t* skip_add, MsmState& ms,
                   uint32_t* out, uint32_t** groups_out = nullptr) {
  int rc;
  const MsmPlan& pl = ms.pl;
  const uint64_t n = ms.n;
  const size_t nbw = (size_t)pl.windows * pl.nb;
  const uint64_t nseg = (std::max<uint64_t>(n, 1) + (1ull << pl.seg_log2) - 1) >> pl.seg_log2;
  uint32_t *buckets, *L, *T, *groups, *segA, *segB;
  if ((rc = ensure_t(ctx, "msm_buckets", 128 * nbw, &buckets))) return rc;
  if ((rc = ensure_t(ctx, "msm_segA", 128 * (size_t)pl.windows * nseg, &segA))) return rc;
  if ((rc = ensure_t(ctx, "msm_segB", 128 * (size_t)pl.windows * nseg, &segB))) return rc;
  if ((rc = ensure_t(ctx, "msm_L", 128 * (size_t)pl.windows * pl.nchunks, &L))) return rc;
  if ((rc = ensure_t(ctx, "msm_T", 128 * (size_t)pl.windows * pl.nchunks, &T))) return rc;
  if ((rc = ensure_t(ctx, "msm_groups", 128 * (size_t)pl.windows * (1 + pl.jbits), &groups))) return rc;
  cudaEvent_t sb_, se_;
  timer_begin(ctx, "msm_bucket", st, &sb_, &se_);
  if (n) {
    const size_t nth = (size_t)pl.windows * nseg;
    k_msm_accum<<<(unsigned)((nth + 127) / 128), 128, 0, st>>>(pts, ms.idx, ms.bkt, ms.off, ms.cnt, n, pl, skip_add,
                                                               buckets, segA, segB);
    ++ctx->launch_count;
  }
  uint32_t* big;   // count, then the list of buckets spanning many ranges
  if ((rc = ensure_t(ctx, "msm_big", 4 * (nbw + 1), &big))) return rc;
  CU(cudaMemsetAsync(big, 0, 4, st));
  k_msm_combine<<<(unsigned)((nbw + 127) / 128), 128, 0, st>>>(ms.off, ms.cnt, std::max<uint64_t>(n, 1), pl, segA,
                                                              segB, buckets, big + 1, big);
  k_msm_combine_big<<<3 * ctx->sm_count, kCombineBigThreads, 0, st>>>(ms.off, ms.cnt, std::max<uint64_t>(n, 1), pl,
                                                                      segA, segB, buckets, big + 1, big);
  ctx->launch_count += 2;
  timer_end(ctx, "msm_bucket", st, sb_, se_);
  timer_begin(ctx, "msm_reduce", st, &sb_, &se_);
  const size_t nch = (size_t)pl.windows * pl.nchunks;
  if (pl.c <= kMsmDirectMaxC) {   // narrow windows: W_w = sum_d d B_d directly (into group 0)
    const unsigned threads = 4u << (pl.c - 1);
    k_msm_direct_groups<<<pl.windows, threads, (size_t)32 * 4 * (threads / 4), st>>>(buckets, pl, groups);
  } else {
    k_msm_chunk<<<(unsigned)((4 * nch + 127) / 128), 128, 0, st>>>(buckets, pl, L, T);
    k_msm_groups<<<pl.windows * (1 + pl.jbits), 512, 0, st>>>(L, T, pl, groups);
  }
  ctx->launch_count += pl.c <= kMsmDirectMaxC ? 1 : 2;
  timer_end(ctx, "msm_reduce", st, sb_, se_);
  if (groups_out) {   // the caller checks window by window (k_msm_window_check)
    *groups_out = groups;
    CU(cudaGetLastError());
    return POSLO_OK;
  }
  timer_begin(ctx, "msm_final", st, &sb_, &se_);
  k_msm_final<<<1, 32, 0, st>>>(groups, pl, out);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  timer_end(ctx, "msm_final", st, sb_, se_);
  return POSLO_OK;
}

// sum_t [z_t] P_t over the stored points, leaving out flagged entries, into out (32 words).
int run_msm(poslo_ctx* ctx, cudaStream_t st, const uint32_t* pts, const uint32_t* z, int sw, const uint8_t* skip,
            uint64_t n, uint32_t* out, const MsmPlan* forced = nullptr) {
  MsmState ms;
  int rc;
  cudaEvent_t tb, te;
  timer_begin(ctx, "msm", st, &tb, &te);
  if ((rc = run_msm_sort(ctx, st, z, sw, skip, n, ms, forced))) return rc;
  if ((rc = run_msm_finish(ctx, st, pts, skip, ms, out))) return rc;
  timer_end(ctx, "msm", st, tb, te);
  return POSLO_OK;
}

int run_finalize(poslo_ctx* ctx, const unsigned long long* hpart, uint32_t nhb, const uint32_t* ppart, uint32_t npb,
                 const uint32_t* R_given, const uint8_t* s_given, const uint32_t* tableY, uint8_t* d_acc,
                 uint32_t* out_words) {
  FinalArgs f{};
  f.hash_partial = hpart;
  f.nhash = nhb;
  f.point_partial = ppart;
  f.npoint = npb;
  f.R_given = R_given;
  f.s_given = s_given;
  f.tableY = tableY;
  f.tableG = ctx->tableG;
  f.accept = d_acc;
  f.out_words = out_words;
  f.status = ctx->status;
  cudaEvent_t tb, te;
  timer_begin(ctx, "finalize", ctx->s_main, &tb, &te);
  k_finalize<<<1, kFinalThreads, 0, ctx->s_main>>>(f);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  timer_end(ctx, "finalize", ctx->s_main, tb, te);
  return POSLO_OK;
}

// Ordered list of flagged entries (first_index + t, ascending) into out (room for cap);
// the full count goes to *d_count (device).
int run_compact(poslo_ctx* ctx, const uint8_t* flags, uint64_t n, uint64_t first_index, uint64_t* out, uint64_t cap,
                uint64_t* d_count) {
  int rc;
  const uint32_t nb = (uint32_t)std::max<uint64_t>(1, (n + kFlagChunk - 1) / kFlagChunk);
  uint32_t* bc;
  uint64_t* bo;
  if ((rc = ensure_t(ctx, "flag_cnt", 4 * (size_t)nb, &bc))) return rc;
  if ((rc = ensure_t(ctx, "flag_off", 8 * (size_t)nb, &bo))) return rc;
  k_flag_count<<<nb, 1024, 0, ctx->s_main>>>(flags, n, bc);
  k_flag_scan<<<1, 1024, 0, ctx->s_main>>>(bc, nb, bo, d_count);
  k_flag_scatter<<<nb, 1024, 0, ctx->s_main>>>(flags, n, first_index, bo, out, cap);
  ctx->launch_count += 3;
  CU(cudaGetLastError());
  return POSLO_OK;
}

// Points stream, after k_points: the unit sum of the decoded points (extended, 32 words),
// optionally its compressed encoding, and the count of undecodable points; then ev_points.
int run_unit_sum(poslo_ctx* ctx, const uint32_t* ppart, uint32_t npb, uint32_t* unitR, uint8_t* enc,
                 uint32_t* pbad) {
  k_sum_encode<<<1, kFinalThreads, 0, ctx->s_points>>>(ppart, npb, unitR, enc, pbad);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  CU(cudaEventRecord(ctx->ev_points, ctx->s_points));
  return POSLO_OK;
}

// Table stream, once hashing is done: [e]Y + [s]G and the malformed-s flag into prep
// (33 words); then ev_prep.  Optionally the unit sum of all s_t for ccd^v as well.
int run_prep(poslo_ctx* ctx, const unsigned long long* hpart, uint32_t nhb, const uint8_t* s_given,
             const uint32_t* tableY, uint32_t* prep, const uint8_t* s_all, uint64_t n, uint8_t* ccd_s,
             cudaStream_t hash_stream = nullptr) {
  CU(cudaEventRecord(ctx->ev_hash, hash_stream ? hash_stream : ctx->s_main));
  CU(cudaStreamWaitEvent(ctx->s_table, ctx->ev_hash, 0));
  PrepArgs pa{};
  pa.hash_partial = hpart;
  pa.nhash = nhb;
  pa.s_given = s_given;
  pa.tableY = tableY;
  pa.tableG = ctx->tableG;
  pa.prep = prep;
  cudaEvent_t tb, te;
  timer_begin(ctx, "prep", ctx->s_table, &tb, &te);
  k_final_prep<<<1, 128, 0, ctx->s_table>>>(pa);
  ++ctx->launch_count;
  timer_end(ctx, "prep", ctx->s_table, tb, te);
  if (ccd_s) {
    int rc;
    const int sblocks = grid_for(ctx, n, kHashThreads, 8);
    unsigned long long* sp;
    if ((rc = ensure_t(ctx, "ccd_spart_fast", (size_t)sblocks * 13 * 8, &sp))) return rc;
    k_sum_scalars<<<sblocks, kHashThreads, 0, ctx->s_table>>>(s_all, n, nullptr, sp);
    k_reduce_scalars<<<1, 256, 0, ctx->s_table>>>(sp, sblocks, ccd_s);
    ctx->launch_count += 2;
  }
  CU(cudaGetLastError());
  CU(cudaEventRecord(ctx->ev_prep, ctx->s_table));
  return POSLO_OK;
}

// Main stream: [8](R - prep) = O and no malformed input -> accept byte.
// Table stream, once hashing is done: the per-window scalar sums E_w, S_w of the MSM plan pl
// and P_w = [E_w] Y + [S_w] G for every window into Pw (32 words each), the malformed-s flag
// into *bad; optionally the unit sum of all s_t for ccd^v; then ev_prep.
int run_prep_windows(poslo_ctx* ctx, const unsigned long long* hpart, uint32_t nhb, const uint32_t* tableY,
                     const uint8_t* e, const uint8_t* s_all, const uint32_t* z, uint64_t n, const MsmPlan& pl,
                     uint32_t* Pw, uint32_t* bad, uint8_t* ccd_s, cudaStream_t hash_stream) {
  int rc;
  CU(cudaEventRecord(ctx->ev_hash, hash_stream));
  CU(cudaStreamWaitEvent(ctx->s_table, ctx->ev_hash, 0));
  const unsigned bx = (unsigned)std::max<int>(1, grid_for(ctx, n, kWindowThreads, 4) / pl.windows);
  unsigned long long* wpart;
  if ((rc = ensure_t(ctx, "win_partial", (size_t)bx * pl.windows * 26 * 8, &wpart))) return rc;
  cudaEvent_t tb, te;
  timer_begin(ctx, "prep", ctx->s_table, &tb, &te);
  k_window_sums<<<dim3(bx, (unsigned)pl.windows), kWindowThreads, 0, ctx->s_table>>>(e, s_all, z, n, pl, wpart);
  k_window_prep<<<(unsigned)pl.windows, kWindowThreads, 0, ctx->s_table>>>(wpart, bx, hpart, nhb, tableY,
                                                                           ctx->tableG, Pw, bad);
  ctx->launch_count += 2;
  timer_end(ctx, "prep", ctx->s_table, tb, te);
  if (ccd_s) {
    const int sblocks = grid_for(ctx, n, kHashThreads, 8);
    unsigned long long* sp;
    if ((rc = ensure_t(ctx, "ccd_spart_fast", (size_t)sblocks * 13 * 8, &sp))) return rc;
    k_sum_scalars<<<sblocks, kHashThreads, 0, ctx->s_table>>>(s_all, n, nullptr, sp);
    k_reduce_scalars<<<1, 256, 0, ctx->s_table>>>(sp, sblocks, ccd_s);
    ctx->launch_count += 2;
  }
  CU(cudaGetLastError());
  CU(cudaEventRecord(ctx->ev_prep, ctx->s_table));
  return POSLO_OK;
}

// Main stream, after the MSM's group sums: the per-window check into d_acc.
int run_window_check(poslo_ctx* ctx, const uint32_t* groups, const MsmPlan& pl, const uint32_t* Pw,
                     const uint32_t* bad, const uint32_t* pbad, uint8_t* d_acc) {
  CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_prep, 0));
  CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_points, 0));
  cudaEvent_t tb, te;
  timer_begin(ctx, "finalize", ctx->s_main, &tb, &te);
  k_msm_window_check<<<1, 32, 0, ctx->s_main>>>(groups, pl, Pw, bad, pbad, ctx->status, d_acc);
  ++ctx->launch_count;
  timer_end(ctx, "finalize", ctx->s_main, tb, te);
  CU(cudaGetLastError());
  return POSLO_OK;
}

int run_check(poslo_ctx* ctx, const uint32_t* prep, const uint32_t* R, const uint32_t* pbad, uint8_t* d_acc) {
  CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_prep, 0));
  CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_points, 0));
  cudaEvent_t tb, te;
  timer_begin(ctx, "finalize", ctx->s_main, &tb, &te);
  k_final_check<<<1, 32, 0, ctx->s_main>>>(prep, R, pbad, ctx->status, d_acc);
  ++ctx->launch_count;
  timer_end(ctx, "finalize", ctx->s_main, tb, te);
  CU(cudaGetLastError());
  return POSLO_OK;
}

}  // namespace

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

int poslo_create(const poslo_params* params, poslo_ctx** out) {
  poslo_ctx* ctx = nullptr;
  if (!out) return POSLO_EINVAL;
  *out = nullptr;
  if (params && params->instantiation != POSLO_INST_SHA256 && params->instantiation != POSLO_INST_AES)
    return POSLO_EINVAL;
  const int device = params ? params->device : 0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= device || device < 0) return POSLO_EDEVICE;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return POSLO_EDEVICE;
  if (prop.major != 10 || prop.minor != 3) return POSLO_EDEVICE;   // built for sm_103a only
  ctx = new poslo_ctx();
  ctx->device = device;
  ctx->sm_count = prop.multiProcessorCount;
  if (params) {
    ctx->msm_window = params->msm_window;
    ctx->inst = params->instantiation;
    ctx->mem_budget = params->mem_budget;
    memcpy(ctx->vseed, params->verifier_seed, 32);
  }
  auto bail = [&](int code) {
    poslo_destroy(ctx);
    return code;
  };
  if (cudaSetDevice(device) != cudaSuccess) return bail(POSLO_EDEVICE);
  if (cudaStreamCreateWithFlags(&ctx->s_main, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->s_table, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->s_points, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->s_copy, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->s_hash, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_copy[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_copy[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_table, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_points, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_decoded, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_main, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_hash, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_prep, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_staged, cudaEventDisableTiming) != cudaSuccess)
    return bail(POSLO_EDEVICE);
  if (cudaMalloc(&ctx->status, 4) != cudaSuccess) return bail(POSLO_ENOMEM);
  // page-locked: the status word, then kSmallHostBytes for small results and records
  if (cudaMallocHost(&ctx->h_status, 256 + kSmallHostBytes) != cudaSuccess) return bail(POSLO_ENOMEM);
  ctx->h_small = reinterpret_cast<uint8_t*>(ctx->h_status) + 256;
  if (cudaMalloc(&ctx->tableG, 4 * (size_t)kTableWords) != cudaSuccess) return bail(POSLO_ENOMEM);
  cudaMemsetAsync(ctx->status, 0, 4, ctx->s_main);
  if (launch_tables(ctx, ctx->s_main, nullptr, nullptr, nullptr, 1, ctx->tableG, 1, nullptr)) return bail(POSLO_EDEVICE);
  ++ctx->launch_count;
  if (cudaStreamSynchronize(ctx->s_main) != cudaSuccess) return bail(POSLO_EDEVICE);
  *out = ctx;
  return POSLO_OK;
}

void poslo_destroy(poslo_ctx* ctx) {
  if (!ctx) return;
  poslo_server_release(ctx);
  cudaSetDevice(ctx->device);
  if (ctx->s_main) cudaStreamSynchronize(ctx->s_main);
  if (ctx->s_table) cudaStreamSynchronize(ctx->s_table);
  if (ctx->s_points) cudaStreamSynchronize(ctx->s_points);
  if (ctx->s_hash) cudaStreamSynchronize(ctx->s_hash);
  if (ctx->s_copy) cudaStreamSynchronize(ctx->s_copy);
  graph_reset(ctx->g_multi);
  graph_reset(ctx->g_distill);
  graph_reset(ctx->g_partial);
  for (uint32_t* b : ctx->keys.blocks) cudaFree(b);
  for (auto& kv : ctx->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  for (auto& p : ctx->pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->tableG) cudaFree(ctx->tableG);
  if (ctx->status) cudaFree(ctx->status);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->h_pack) cudaFreeHost(ctx->h_pack);
  for (poslo_host::StageSet& S : ctx->stage) {
    for (poslo_host::DevBuf* b : {&S.msgs, &S.raw, &S.offs, &S.s, &S.R, &S.meta, &S.regions, &S.status})
      if (b->p) cudaFree(b->p);
    if (S.h) cudaFreeHost(S.h);
  }
  if (ctx->ev_table) cudaEventDestroy(ctx->ev_table);
  if (ctx->ev_points) cudaEventDestroy(ctx->ev_points);
  if (ctx->ev_decoded) cudaEventDestroy(ctx->ev_decoded);
  if (ctx->ev_main) cudaEventDestroy(ctx->ev_main);
  if (ctx->ev_hash) cudaEventDestroy(ctx->ev_hash);
  if (ctx->ev_prep) cudaEventDestroy(ctx->ev_prep);
  if (ctx->ev_staged) cudaEventDestroy(ctx->ev_staged);
  if (ctx->s_main) cudaStreamDestroy(ctx->s_main);
  if (ctx->s_table) cudaStreamDestroy(ctx->s_table);
  if (ctx->s_points) cudaStreamDestroy(ctx->s_points);
  if (ctx->s_copy) cudaStreamDestroy(ctx->s_copy);
  if (ctx->s_hash) cudaStreamDestroy(ctx->s_hash);
  for (cudaEvent_t e : ctx->ev_copy)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

const char* poslo_last_error(const poslo_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

void* poslo_stream(poslo_ctx* ctx) { return ctx ? (void*)ctx->s_main : nullptr; }

int poslo_set_profiling(poslo_ctx* ctx, int enabled) {
  if (!ctx) return POSLO_EINVAL;
  ctx->profiling = enabled != 0;
  return POSLO_OK;
}

int poslo_set_key_cache(poslo_ctx* ctx, uint32_t capacity) {
  if (!ctx) return POSLO_EINVAL;
  poslo_host::KeyCache& C = ctx->keys;
  cudaStreamSynchronize(ctx->s_main);
  cudaStreamSynchronize(ctx->s_table);
  graph_reset(ctx->g_distill);   // it may hold a cached table's address
  for (uint32_t* b : C.blocks) {
    cudaFree(b);
    ctx->mem_used -= (size_t)poslo_host::KeyCache::kBlock * kTableWords * 4;
  }
  const uint64_t hits = C.hits, misses = C.misses;
  C = poslo_host::KeyCache();
  C.capacity = capacity;
  C.hits = hits;
  C.misses = misses;
  return POSLO_OK;
}

int poslo_key_cache_stats(poslo_ctx* ctx, uint64_t* hits, uint64_t* misses) {
  if (!ctx) return POSLO_EINVAL;
  if (hits) *hits = ctx->keys.hits;
  if (misses) *misses = ctx->keys.misses;
  return POSLO_OK;
}

int poslo_set_multi_window_limit(poslo_ctx* ctx, uint64_t max_entries) {
  if (!ctx) return POSLO_EINVAL;
  ctx->multi_window_max = max_entries;
  return POSLO_OK;
}

int poslo_set_graphs(poslo_ctx* ctx, int enabled) {
  if (!ctx) return POSLO_EINVAL;
  ctx->graphs = enabled != 0;
  if (!ctx->graphs) {
    cudaStreamSynchronize(ctx->s_main);
    graph_reset(ctx->g_multi);
    graph_reset(ctx->g_distill);
    graph_reset(ctx->g_partial);
  }
  return POSLO_OK;
}

int poslo_graph_stats(poslo_ctx* ctx, uint64_t* captures, uint64_t* replays) {
  if (!ctx) return POSLO_EINVAL;
  if (captures) *captures = ctx->graph_captures;
  if (replays) *replays = ctx->graph_replays;
  return POSLO_OK;
}

int poslo_kernel_time(poslo_ctx* ctx, const char* name, double* total_ms, uint64_t* launches) {
  if (!ctx || !name) return POSLO_EINVAL;
  timers_collect(ctx);
  if (strcmp(name, "*") == 0) {   // every kernel this context launched, untimed
    if (total_ms) *total_ms = 0;
    if (launches) *launches = ctx->launch_count;
    return POSLO_OK;
  }
  auto it = ctx->timers.find(name);
  if (it == ctx->timers.end()) {
    if (total_ms) *total_ms = 0;
    if (launches) *launches = 0;
    return POSLO_ENOTFOUND;
  }
  if (total_ms) *total_ms = it->second.total_ms;
  if (launches) *launches = it->second.launches;
  return POSLO_OK;
}

void poslo_reset_kernel_times(poslo_ctx* ctx) {
  if (!ctx) return;
  timers_collect(ctx);
  ctx->timers.clear();
}

// ---------------------------------------------------------------------------- signer side

int poslo_keygen_c(poslo_ctx* ctx, const uint8_t y[32], const uint8_t r[32], uint32_t D, uint32_t n2,
                   uint8_t Y_out[32], uint8_t* epoch_R_out) {
  if (!ctx || !y || !r || !Y_out || D > 24 || n2 == 0) return fail(ctx, POSLO_EINVAL, "bad keygen_c arguments");
  int rc;
  const uint64_t n1 = 1ull << D;
  uint8_t *d_in, *d_out;
  if ((rc = ensure_t(ctx, "kg_in", 64, &d_in))) return rc;
  if ((rc = ensure_t(ctx, "kg_out", 32 + 32 * n1, &d_out))) return rc;
  CU(cudaMemcpyAsync(d_in, y, 32, cudaMemcpyHostToDevice, ctx->s_main));
  CU(cudaMemcpyAsync(d_in + 32, r, 32, cudaMemcpyHostToDevice, ctx->s_main));
  k_keygen_y<<<1, 1, 0, ctx->s_main>>>(d_in, ctx->tableG, d_out);
  ++ctx->launch_count;
  k_keygen_c_epochs<<<(unsigned)((n1 + 63) / 64), 64, 0, ctx->s_main>>>(d_in + 32, (uint32_t)n1, n2, ctx->tableG,
                                                                         d_out + 32);
                                                                         ++ctx->launch_count;
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(Y_out, d_out, 32, cudaMemcpyDeviceToHost, ctx->s_main));
  if (epoch_R_out) CU(cudaMemcpyAsync(epoch_R_out, d_out + 32, 32 * n1, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaStreamSynchronize(ctx->s_main));
  return POSLO_OK;
}

int poslo_keygen_f(poslo_ctx* ctx, const uint8_t y[32], const uint8_t* bpv_r, uint32_t v, uint8_t Y_out[32],
                   uint8_t* bpv_R_out) {
  if (!ctx || !y || !Y_out || (v && (!bpv_r || !bpv_R_out))) return fail(ctx, POSLO_EINVAL, "bad keygen_f arguments");
  int rc;
  uint8_t *d_y, *d_r, *d_out;
  if ((rc = ensure_t(ctx, "kg_in", 32, &d_y))) return rc;
  if ((rc = ensure_t(ctx, "kg_bpv", 32 * (size_t)std::max(v, 1u), &d_r))) return rc;
  if ((rc = ensure_t(ctx, "kg_out", 32 + 32 * (size_t)v, &d_out))) return rc;
  CU(cudaMemcpyAsync(d_y, y, 32, cudaMemcpyHostToDevice, ctx->s_main));
  if (v) CU(cudaMemcpyAsync(d_r, bpv_r, 32 * (size_t)v, cudaMemcpyHostToDevice, ctx->s_main));
  k_keygen_y<<<1, 1, 0, ctx->s_main>>>(d_y, ctx->tableG, d_out);
  ++ctx->launch_count;
  if (v) k_keygen_bpv<<<(v + 63) / 64, 64, 0, ctx->s_main>>>(d_r, v, ctx->tableG, d_out + 32);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(Y_out, d_out, 32, cudaMemcpyDeviceToHost, ctx->s_main));
  if (v) CU(cudaMemcpyAsync(bpv_R_out, d_out + 32, 32 * (size_t)v, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaStreamSynchronize(ctx->s_main));
  return POSLO_OK;
}

static int root_ds(const uint8_t root[16], uint32_t D, uint8_t out[24]) {
  memset(out, 0, 24);
  out[0] = (uint8_t)D; out[1] = (uint8_t)(D >> 8); out[2] = (uint8_t)(D >> 16); out[3] = (uint8_t)(D >> 24);
  memcpy(out + 8, root, 16);
  return 0;
}

int poslo_sign_f(poslo_ctx* ctx, const uint8_t y[32], const uint8_t root[16], uint32_t D, uint32_t n2,
                 const uint8_t* bpv_r, const uint8_t* bpv_R, uint32_t v, uint32_t k, const uint16_t* subsets,
                 const uint8_t* msgs, const uint64_t* offs, uint64_t n, uint64_t first_index, uint8_t* s_out,
                 uint8_t* R_out, uint8_t* x_out) {
  if (!ctx || !y || !root || !bpv_r || !bpv_R || !subsets || !offs || !s_out || !R_out || n2 == 0 || v == 0 || D > 40)
    return fail(ctx, POSLO_EINVAL, "bad sign_f arguments");
  if (n == 0) return POSLO_OK;
  if ((first_index + n - 1) / n2 >= (1ull << D)) return fail(ctx, POSLO_EINVAL, "entry index beyond n1*n2");
  for (uint64_t t = 0; t < n; ++t)
    if (offs[t + 1] < offs[t] || offs[t + 1] - offs[t] > 0xffffffffull)
      return fail(ctx, POSLO_EINVAL, "offsets decrease at entry %llu", (unsigned long long)t);
  for (uint64_t t = 0; t < n * k; ++t)
    if (subsets[t] >= v) return fail(ctx, POSLO_EINVAL, "BPV subset index out of range");
  int rc;
  uint8_t ds[24];
  root_ds(root, D, ds);
  const uint64_t e0 = first_index / n2, ne = (first_index + n - 1) / n2 - e0 + 1;
  CU(cudaMemsetAsync(ctx->status, 0, 4, ctx->s_main));
  uint32_t* seeds;
  if ((rc = run_epoch_seeds(ctx, ds, 1, e0, ne, &seeds))) return rc;
  const void* p;
  SignFArgs a{};
  if ((rc = stage(ctx, "offs", offs, (n + 1) * 8, false, ctx->s_main, &p))) return rc;
  a.offs = static_cast<const uint64_t*>(p);
  a.base_off = offs[0];
  if ((rc = stage(ctx, "msgs", msgs + offs[0], offs[n] - offs[0], false, ctx->s_main, &p))) return rc;
  a.msgs = static_cast<const uint8_t*>(p);
  uint8_t* d_y;
  if ((rc = ensure_t(ctx, "sig_y", 32, &d_y))) return rc;
  CU(cudaMemcpyAsync(d_y, y, 32, cudaMemcpyHostToDevice, ctx->s_main));
  if ((rc = stage(ctx, "sig_bpv_r", bpv_r, 32 * (size_t)v, false, ctx->s_main, &p))) return rc;
  a.bpv_r = static_cast<const uint8_t*>(p);
  const uint8_t* d_bpvR;
  if ((rc = stage(ctx, "sig_bpv_R", bpv_R, 32 * (size_t)v, false, ctx->s_main, &p))) return rc;
  d_bpvR = static_cast<const uint8_t*>(p);
  uint32_t* pts;
  if ((rc = ensure_t(ctx, "sig_bpv_pts", 128 * (size_t)v, &pts))) return rc;
  k_decode_table<<<(v + 63) / 64, 64, 0, ctx->s_main>>>(d_bpvR, v, pts, ctx->status);
  ++ctx->launch_count;
  if ((rc = stage(ctx, "sig_subsets", subsets, 2 * n * k, false, ctx->s_main, &p))) return rc;
  a.subsets = static_cast<const uint16_t*>(p);
  uint8_t *d_s, *d_R, *d_x = nullptr;
  if ((rc = ensure_t(ctx, "sig_s", 32 * n, &d_s))) return rc;
  if ((rc = ensure_t(ctx, "sig_R", 32 * n, &d_R))) return rc;
  if (x_out && (rc = ensure_t(ctx, "sig_x", 16 * n, &d_x))) return rc;
  a.n = n;
  a.first_index = first_index;
  a.e0 = e0;
  a.n2 = n2;
  a.seeds = seeds;
  a.y = d_y;
  a.bpv_pts = pts;
  a.v = v;
  a.k = k;
  a.s_out = d_s;
  a.R_out = d_R;
  a.x_out = d_x;
  launch_sign_f((int)ctx->inst, (unsigned)((n + 127) / 128), 128, ctx->s_main, a);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(s_out, d_s, 32 * n, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaMemcpyAsync(R_out, d_R, 32 * n, cudaMemcpyDeviceToHost, ctx->s_main));
  if (x_out) CU(cudaMemcpyAsync(x_out, d_x, 16 * n, cudaMemcpyDeviceToHost, ctx->s_main));
  int st = check_status(ctx);
  if (st == POSLO_OK && (*ctx->h_status & kErrPoint)) return fail(ctx, POSLO_EINVAL, "BPV table point does not decode");
  return st;
}

int poslo_sign_c(poslo_ctx* ctx, const uint8_t y[32], const uint8_t r[32], const uint8_t root[16], uint32_t D,
                 uint32_t n2, const uint8_t* msgs, const uint64_t* offs, uint64_t first_epoch, uint64_t n_epochs,
                 uint8_t* s_out) {
  if (!ctx || !y || !r || !root || !offs || !s_out || n2 == 0 || D > 40)
    return fail(ctx, POSLO_EINVAL, "bad sign_c arguments");
  if (n_epochs == 0) return POSLO_OK;
  if (first_epoch + n_epochs > (1ull << D)) return fail(ctx, POSLO_EINVAL, "epoch beyond n1");
  int rc;
  uint8_t ds[24];
  root_ds(root, D, ds);
  CU(cudaMemsetAsync(ctx->status, 0, 4, ctx->s_main));
  uint32_t* seeds;
  if ((rc = run_epoch_seeds(ctx, ds, 1, first_epoch, n_epochs, &seeds))) return rc;
  const uint64_t n = n_epochs * n2;
  for (uint64_t t = 0; t < n; ++t)
    if (offs[t + 1] < offs[t] || offs[t + 1] - offs[t] > 0xffffffffull)
      return fail(ctx, POSLO_EINVAL, "offsets decrease at entry %llu", (unsigned long long)t);
  const void* p;
  SignCArgs a{};
  if ((rc = stage(ctx, "offs", offs, (n + 1) * 8, false, ctx->s_main, &p))) return rc;
  a.offs = static_cast<const uint64_t*>(p);
  a.base_off = offs[0];
  if ((rc = stage(ctx, "msgs", msgs + offs[0], offs[n] - offs[0], false, ctx->s_main, &p))) return rc;
  a.msgs = static_cast<const uint8_t*>(p);
  uint8_t* d_yr;
  if ((rc = ensure_t(ctx, "sig_yr", 64, &d_yr))) return rc;
  CU(cudaMemcpyAsync(d_yr, y, 32, cudaMemcpyHostToDevice, ctx->s_main));
  CU(cudaMemcpyAsync(d_yr + 32, r, 32, cudaMemcpyHostToDevice, ctx->s_main));
  uint8_t* d_s;
  if ((rc = ensure_t(ctx, "sig_s", 32 * n_epochs, &d_s))) return rc;
  a.n_epochs = n_epochs;
  a.first_epoch = first_epoch;
  a.n2 = n2;
  a.seeds = seeds;
  a.y = d_yr;
  a.r = d_yr + 32;
  a.s_out = d_s;
  launch_sign_c((int)ctx->inst, (unsigned)((n_epochs + 63) / 64), 64, ctx->s_main, a);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(s_out, d_s, 32 * n_epochs, cudaMemcpyDeviceToHost, ctx->s_main));
  return check_status(ctx);
}

int poslo_disclose(poslo_ctx* ctx, const uint8_t root[16], uint32_t D, uint64_t i, uint8_t* ds_out, uint32_t cap_nodes,
                   uint32_t* nodes) {
  if (!ctx || !root || !nodes || D > 40 || i >= (1ull << D)) return fail(ctx, POSLO_EINVAL, "bad disclose arguments");
  // SSO (Fig. 2a) over node positions: merge the top while it sits at the current depth.
  std::vector<std::pair<uint32_t, uint64_t>> stack;
  for (uint64_t k = 0; k <= i; ++k) {
    uint32_t d1 = 0;
    uint64_t i1 = k;
    while (!stack.empty() && stack.back().first == d1) {
      stack.pop_back();
      ++d1;
      i1 >>= 1;
    }
    stack.push_back({d1, i1});
  }
  *nodes = (uint32_t)stack.size();
  if (stack.size() > cap_nodes || !ds_out) return fail(ctx, POSLO_EBUFSMALL, "ds needs %zu nodes", stack.size());
  // seeds: SC(root, D, 0, d, i) on the device, walking from the root
  int rc;
  uint8_t rds[24];
  root_ds(root, D, rds);
  std::vector<DsNode> hroot;
  if ((rc = parse_ds(ctx, rds, 1, hroot))) return rc;
  // node x_d[i] is the ancestor at depth d: compute it as the seed of the leaf range start
  // walked only D-d levels, i.e. an SRet over a shortened tree rooted at the same seed.
  std::vector<uint8_t> out(24 * stack.size());
  for (size_t k = 0; k < stack.size(); ++k) {
    const uint32_t d = stack[k].first;
    const uint64_t idx = stack[k].second;
    DsNode top = hroot[0];
    top.d = D - d;          // a tree of height D-d whose leaves are the depth-d nodes
    uint8_t tmp[24];
    memcpy(tmp, &top.d, 4);
    uint32_t zero = 0;
    memcpy(tmp + 4, &zero, 4);
    memcpy(tmp + 8, root, 16);
    uint32_t* seeds;
    CU(cudaMemsetAsync(ctx->status, 0, 4, ctx->s_main));
    if ((rc = run_epoch_seeds(ctx, tmp, 1, idx, 1, &seeds))) return rc;
    uint32_t w[4];
    CU(cudaMemcpyAsync(w, seeds, 16, cudaMemcpyDeviceToHost, ctx->s_main));
    if ((rc = check_status(ctx))) return rc;
    uint8_t* o = out.data() + 24 * k;
    memcpy(o, &d, 4);
    const uint32_t i32 = (uint32_t)idx;
    memcpy(o + 4, &i32, 4);
    for (int q = 0; q < 4; ++q) {
      o[8 + 4 * q] = (uint8_t)(w[q] >> 24); o[9 + 4 * q] = (uint8_t)(w[q] >> 16);
      o[10 + 4 * q] = (uint8_t)(w[q] >> 8); o[11 + 4 * q] = (uint8_t)w[q];
    }
  }
  memcpy(ds_out, out.data(), out.size());
  return POSLO_OK;
}

// ---------------------------------------------------------------------------- verifier side

int poslo_epoch_seeds(poslo_ctx* ctx, const uint8_t* ds, uint32_t ds_nodes, uint64_t first_epoch, uint64_t n_epochs,
                      uint8_t* x0_out) {
  if (!ctx || !x0_out) return fail(ctx, POSLO_EINVAL, "bad epoch_seeds arguments");
  int rc;
  if ((rc = reset_status(ctx))) return rc;
  uint32_t* seeds;
  if ((rc = run_epoch_seeds(ctx, ds, ds_nodes, first_epoch, n_epochs, &seeds))) return rc;
  std::vector<uint32_t> h(4 * n_epochs);
  if (n_epochs) CU(cudaMemcpyAsync(h.data(), seeds, 16 * n_epochs, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  for (uint64_t k = 0; k < 4 * n_epochs; ++k) {
    x0_out[4 * k] = (uint8_t)(h[k] >> 24); x0_out[4 * k + 1] = (uint8_t)(h[k] >> 16);
    x0_out[4 * k + 2] = (uint8_t)(h[k] >> 8); x0_out[4 * k + 3] = (uint8_t)h[k];
  }
  return POSLO_OK;
}

int poslo_hash_entries(poslo_ctx* ctx, const poslo_batch* batch, uint8_t* e_out) {
  if (!ctx || !e_out) return fail(ctx, POSLO_EINVAL, "bad hash_entries arguments");
  int rc;
  if ((rc = validate_batch(ctx, batch))) return rc;
  if (batch->on_device && (reinterpret_cast<uintptr_t>(e_out) & 15))
    return fail(ctx, POSLO_EINVAL, "device-resident e_out must be 16-byte aligned");
  if ((rc = reset_status(ctx))) return rc;
  Staged sb;
  if ((rc = stage_batch(ctx, batch, sb))) return rc;
  uint8_t* d_e = e_out;
  if (!batch->on_device && (rc = ensure_t(ctx, "e_out", 32 * batch->n, &d_e))) return rc;
  unsigned long long* partial;
  uint32_t nb;
  if ((rc = run_hash(ctx, batch, sb, d_e, false, false, nullptr, &partial, &nb))) return rc;
  if (!batch->on_device && batch->n)
    CU(cudaMemcpyAsync(e_out, d_e, 32 * batch->n, cudaMemcpyDeviceToHost, ctx->s_main));
  return check_status(ctx);
}

int poslo_aver(poslo_ctx* ctx, const poslo_batch* batch, uint32_t agg_mode, uint8_t* accept) {
  if (!ctx || !accept) return fail(ctx, POSLO_EINVAL, "bad aver arguments");
  int rc;
  if ((rc = validate_batch(ctx, batch))) return rc;
  if (batch->n > kMaxCallEntries) return fail(ctx, POSLO_EINVAL, "more than 2^32 - 1 entries in one call");
  const bool F = batch->variant == POSLO_VARIANT_F;
  if (agg_mode == POSLO_AGG_WEIGHTED && !F) return fail(ctx, POSLO_EINVAL, "weighted aggregation needs POSLO-F");
  if (agg_mode > POSLO_AGG_WEIGHTED) return fail(ctx, POSLO_EINVAL, "bad aggregation mode");
  const bool weighted = agg_mode == POSLO_AGG_WEIGHTED;
  if ((rc = reset_status(ctx))) return rc;
  Staged sb;
  if ((rc = stage_batch(ctx, batch, sb))) return rc;
  // the key's window table from the key cache; built (into its slot) only on a miss
  uint32_t* tableY;
  std::vector<const uint32_t*> ktab;
  std::vector<uint32_t> kmiss;
  std::vector<uint32_t*> kdst;
  const bool kcached = key_cache_lookup(ctx, batch->Y, 1, ktab, kmiss, kdst);
  KeyForget kforget{ctx, batch->Y, &kmiss, kcached && !kmiss.empty()};
  if (kcached && kmiss.empty()) {
    tableY = const_cast<uint32_t*>(ktab[0]);
  } else if ((rc = run_ytable(ctx, batch->Y, &tableY, kcached ? kdst[0] : nullptr))) {
    return rc;
  }
  const uint64_t npts = F ? batch->n : batch->R_count;
  uint32_t* pts = nullptr;
  uint8_t* badR = nullptr;
  if (weighted) {
    if ((rc = ensure_t(ctx, "pts", 4 * kPtsWords * std::max<uint64_t>(npts, 1), &pts))) return rc;
    if ((rc = ensure_t(ctx, "badR", std::max<uint64_t>(npts, 1), &badR))) return rc;
  }
  uint32_t *small;   // unit R (32) | weighted R (32) | prep (33) | point bad count (1)
  if ((rc = ensure_t(ctx, "aver_small", 4 * 100, &small))) return rc;
  uint32_t *unitR = small, *Rw = small + 32, *prep = small + 64, *pbad = small + 97;
  uint32_t *ppart, npb;
  if ((rc = run_points(ctx, sb.R, npts, pts, badR, &ppart, &npb, ctx->ev_staged))) return rc;
  if ((rc = run_unit_sum(ctx, ppart, npb, unitR, nullptr, pbad))) return rc;
  uint32_t* z = nullptr;
  if (weighted && (rc = ensure_t(ctx, "z", 16 * std::max<uint64_t>(batch->n, 1), &z))) return rc;
  unsigned long long* hpart;
  uint32_t nhb;
  if ((rc = run_hash(ctx, batch, sb, nullptr, weighted, F, z, &hpart, &nhb))) return rc;
  if ((rc = run_prep(ctx, hpart, nhb, F ? nullptr : sb.s, tableY, prep, nullptr, 0, nullptr))) return rc;
  if (weighted) {
    MsmState ms;
    if ((rc = run_msm_sort(ctx, ctx->s_main, z, 4, nullptr, batch->n, ms))) return rc;
    CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_decoded, 0));
    if ((rc = run_msm_finish(ctx, ctx->s_main, pts, badR, ms, Rw))) return rc;
  }
  uint8_t* d_acc;
  if ((rc = ensure_t(ctx, "accept", 16, &d_acc))) return rc;
  if ((rc = run_check(ctx, prep, weighted ? Rw : unitR, pbad, d_acc))) return rc;
  uint8_t h_acc = 0;
  CU(cudaMemcpyAsync(&h_acc, d_acc, 1, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  kforget.armed = false;   // the key decoded: its table is sound
  *accept = h_acc;
  return POSLO_OK;
}

// Shard partials: the aggregate of poslo_aver up to (not including) its group check, as a
// record other shards of the same log can combine (k_shard.cu).  The uploads come first; the
// rest is a fixed launch sequence that a device-resident batch of the previous call's shape
// replays from a CUDA graph.
int poslo_aver_partial(poslo_ctx* ctx, const poslo_batch* batch, uint32_t agg_mode, poslo_partial* out) {
  if (!ctx || !out) return fail(ctx, POSLO_EINVAL, "bad aver_partial arguments");
  int rc;
  if ((rc = validate_batch(ctx, batch))) return rc;
  if (batch->n > kMaxCallEntries) return fail(ctx, POSLO_EINVAL, "more than 2^32 - 1 entries in one call");
  const bool F = batch->variant == POSLO_VARIANT_F;
  if (agg_mode == POSLO_AGG_WEIGHTED && !F) return fail(ctx, POSLO_EINVAL, "weighted aggregation needs POSLO-F");
  if (agg_mode > POSLO_AGG_WEIGHTED) return fail(ctx, POSLO_EINVAL, "bad aggregation mode");
  const bool weighted = agg_mode == POSLO_AGG_WEIGHTED;
  const uint64_t n = batch->n;
  if ((rc = reset_status(ctx))) return rc;
  Staged sb;
  if ((rc = stage_batch(ctx, batch, sb))) return rc;
  // uploads: the disclosed seeds
  std::vector<DsNode> ds_nodes;
  if ((rc = parse_ds(ctx, batch->ds, batch->ds_nodes, ds_nodes))) return rc;
  DsNode* d_ds;
  if ((rc = ensure_t(ctx, "ds", ds_nodes.size() * sizeof(DsNode), &d_ds))) return rc;
  CU(cudaMemcpyAsync(d_ds, ds_nodes.data(), ds_nodes.size() * sizeof(DsNode), cudaMemcpyHostToDevice, ctx->s_main));
  uint64_t e_first = 0, ne = 0;
  if (n) {
    e_first = batch->first_index / batch->n2;
    ne = (batch->first_index + n - 1) / batch->n2 - e_first + 1;
  }
  // workspace, all of it before any launch (a capture cannot allocate)
  const uint64_t npts = F ? n : batch->R_count;
  uint32_t* pts = nullptr;
  uint8_t* badR = nullptr;
  uint32_t *z = nullptr, *seeds;
  if (weighted) {
    if ((rc = ensure_t(ctx, "pts", 4 * kPtsWords * std::max<uint64_t>(npts, 1), &pts))) return rc;
    if ((rc = ensure_t(ctx, "badR", std::max<uint64_t>(npts, 1), &badR))) return rc;
    if ((rc = ensure_t(ctx, "z", 16 * std::max<uint64_t>(n, 1), &z))) return rc;
  }
  uint32_t* small;   // unit R (32) | weighted R (32) | point bad count (1) | record (kShardWords)
  if ((rc = ensure_t(ctx, "partial_small", 4 * (65 + (size_t)kShardWords), &small))) return rc;
  uint32_t *unitR = small, *Rw = small + 32, *pbad = small + 64, *rec = small + 65;
  if ((rc = ensure_t(ctx, "seeds", std::max<uint64_t>(1, ne) * 16, &seeds))) return rc;
  const uint32_t nhb = (uint32_t)grid_for(ctx, n, kHashThreads, 8);
  unsigned long long* hpart;
  if ((rc = ensure_t(ctx, "hash_partial", (size_t)nhb * kPartialWords * 8, &hpart))) return rc;
  const bool replayable = batch->on_device != 0 || sb.packed;
  ZPre zp;
  make_zpre(ctx->vseed, zp.w);
  HashArgs a{};
  a.msgs = sb.msgs;
  a.offs = sb.offs;
  a.base_off = sb.base_off;
  a.n = n;
  a.first_index = batch->first_index;
  a.e0 = e_first;
  a.n2 = batch->n2;
  a.n2_log2 = log2_exact(batch->n2);
  a.seeds = seeds;
  a.s = F ? sb.s : nullptr;
  a.weighted = weighted ? 1u : 0u;
  for (int q = 0; q < 10; ++q) a.zpre[q] = zp.w[q];
  a.z_in = z;
  a.partial = hpart;
  a.status = ctx->status;
  auto launch = [&]() -> int {
    int rc;
    uint32_t *ppart, npb;
    if ((rc = run_points(ctx, sb.R, npts, pts, badR, &ppart, &npb, replayable ? nullptr : ctx->ev_staged)))
      return rc;
    if ((rc = run_unit_sum(ctx, ppart, npb, unitR, nullptr, pbad))) return rc;
    if (ne) {
      cudaEvent_t b, e;
      timer_begin(ctx, "seeds", ctx->s_main, &b, &e);
      launch_epoch_seeds((int)ctx->inst, (unsigned)((ne + 127) / 128), 128, ctx->s_main, d_ds, (int)ds_nodes.size(),
                         e_first, ne, seeds, ctx->status);
      ++ctx->launch_count;
      CU(cudaGetLastError());
      timer_end(ctx, "seeds", ctx->s_main, b, e);
    }
    cudaEvent_t tb, te;
    if (!weighted) {
      timer_begin(ctx, "hash", ctx->s_main, &tb, &te);
      launch_hash((int)ctx->inst, nhb, ctx->s_main, a);
      ++ctx->launch_count;
      CU(cudaGetLastError());
      timer_end(ctx, "hash", ctx->s_main, tb, te);
    } else {
      // as in Distill: the weights z_t first (they need no message), so the MSM's counting
      // sort runs on the main stream while the messages are hashed on the hashing stream and
      // the points decoded on the points stream
      if (n) {
        k_weights<<<grid_for(ctx, n, kSideThreads, 8), kSideThreads, 0, ctx->s_main>>>(zp, n, batch->first_index, z);
        ++ctx->launch_count;
      }
      CU(cudaEventRecord(ctx->ev_main, ctx->s_main));
      CU(cudaStreamWaitEvent(ctx->s_hash, ctx->ev_main, 0));
      MsmState ms;
      if ((rc = run_msm_sort(ctx, ctx->s_main, z, 4, nullptr, n, ms))) return rc;
      timer_begin(ctx, "hash", ctx->s_hash, &tb, &te);
      launch_hash((int)ctx->inst, nhb, ctx->s_hash, a);
      ++ctx->launch_count;
      CU(cudaGetLastError());
      timer_end(ctx, "hash", ctx->s_hash, tb, te);
      CU(cudaEventRecord(ctx->ev_hash, ctx->s_hash));
      CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_decoded, 0));
      if ((rc = run_msm_finish(ctx, ctx->s_main, pts, badR, ms, Rw))) return rc;
      CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_hash, 0));
    }
    CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_points, 0));
    timer_begin(ctx, "finalize", ctx->s_main, &tb, &te);
    k_partial_out<<<1, kShardThreads, 0, ctx->s_main>>>(hpart, nhb, F ? nullptr : sb.s, weighted ? Rw : unitR, pbad,
                                                        rec);
    ++ctx->launch_count;
    CU(cudaGetLastError());
    timer_end(ctx, "finalize", ctx->s_main, tb, te);
    return POSLO_OK;
  };
  if (replayable) {
    const MsmPlan plan = msm_plan(ctx, n, 4);
    const std::vector<uint64_t> sig = {n, batch->n2, batch->first_index, reinterpret_cast<uint64_t>(sb.msgs),
                                       reinterpret_cast<uint64_t>(sb.offs), reinterpret_cast<uint64_t>(sb.s),
                                       reinterpret_cast<uint64_t>(sb.R), sb.base_off, ds_nodes.size(),
                                       (uint64_t)plan.c, (uint64_t)plan.seg_log2, ctx->inst, agg_mode,
                                       batch->variant, batch->R_count};
    rc = run_replayable(ctx, ctx->g_partial, sig, launch);
  } else {
    rc = launch();
  }
  if (rc != POSLO_OK) return rc;
  uint32_t* h = reinterpret_cast<uint32_t*>(ctx->h_small);   // page-locked: no staging, one sync
  CU(cudaMemcpyAsync(h, rec, 4 * kShardWords, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  memcpy(out->e, h, 32);
  memcpy(out->s, h + 8, 32);
  memcpy(out->R, h + 16, 128);
  out->first_index = batch->first_index;
  out->n = batch->n;
  out->malformed = h[kShardBadWord];
  out->agg_mode = agg_mode;
  return POSLO_OK;
}

// The check of a whole log from its shards' records: sums and [8](R~ - e~ Y - s~ G) = O on the
// device (k_combine_check), with the window table of Y from the key cache.
int poslo_combine_check(poslo_ctx* ctx, const uint8_t Y[32], const poslo_partial* parts, uint32_t n_parts,
                        uint8_t* accept, poslo_partial* total) {
  if (!ctx || !Y || !parts || !accept || n_parts == 0) return fail(ctx, POSLO_EINVAL, "bad combine arguments");
  static_assert(sizeof(poslo_partial) == 4 * kShardWords, "poslo_partial is one 54-word record");
  uint64_t n_all = 0;
  for (uint32_t i = 0; i < n_parts; ++i) {
    if (parts[i].agg_mode != parts[0].agg_mode || parts[i].agg_mode > POSLO_AGG_WEIGHTED)
      return fail(ctx, POSLO_EINVAL, "records of different aggregation modes");
    if (i && parts[i].first_index != parts[i - 1].first_index + parts[i - 1].n)
      return fail(ctx, POSLO_EINVAL, "shard %u does not start where shard %u ends", i, i - 1);
    n_all += parts[i].n;
  }
  int rc;
  if ((rc = reset_status(ctx))) return rc;
  uint32_t* tableY;
  std::vector<const uint32_t*> ktab;
  std::vector<uint32_t> kmiss;
  std::vector<uint32_t*> kdst;
  const bool kcached = key_cache_lookup(ctx, Y, 1, ktab, kmiss, kdst);
  KeyForget kforget{ctx, Y, &kmiss, kcached && !kmiss.empty()};
  const bool built = !(kcached && kmiss.empty());
  if (!built) {
    tableY = const_cast<uint32_t*>(ktab[0]);
  } else if ((rc = run_ytable(ctx, Y, &tableY, kcached ? kdst[0] : nullptr))) {
    return rc;
  }
  uint32_t *d_parts, *d_total;
  uint8_t* d_acc;
  if ((rc = ensure_t(ctx, "combine_parts", sizeof(poslo_partial) * (size_t)n_parts, &d_parts))) return rc;
  if ((rc = ensure_t(ctx, "combine_total", sizeof(poslo_partial), &d_total))) return rc;
  if ((rc = ensure_t(ctx, "accept", 16, &d_acc))) return rc;
  // the records go through the page-locked area when they fit (the copy is then asynchronous)
  const size_t rec_bytes = sizeof(poslo_partial) * (size_t)n_parts;
  const bool via_small = rec_bytes + sizeof(poslo_partial) + 16 <= kSmallHostBytes;
  if (via_small) {
    memcpy(ctx->h_small + sizeof(poslo_partial) + 16, parts, rec_bytes);
    CU(cudaMemcpyAsync(d_parts, ctx->h_small + sizeof(poslo_partial) + 16, rec_bytes, cudaMemcpyHostToDevice,
                       ctx->s_main));
  } else {
    CU(cudaMemcpyAsync(d_parts, parts, rec_bytes, cudaMemcpyHostToDevice, ctx->s_main));
  }
  if (built) CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_table, 0));   // the table this call built
  cudaEvent_t tb, te;
  timer_begin(ctx, "finalize", ctx->s_main, &tb, &te);
  k_combine_check<<<1, kShardThreads, 0, ctx->s_main>>>(d_parts, n_parts, tableY, ctx->tableG, ctx->status, d_total,
                                                        d_acc);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  timer_end(ctx, "finalize", ctx->s_main, tb, te);
  uint32_t* h = reinterpret_cast<uint32_t*>(ctx->h_small);   // total record, then the accept byte
  CU(cudaMemcpyAsync(h, d_total, 4 * kShardWords, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaMemcpyAsync(ctx->h_small + sizeof(poslo_partial), d_acc, 1, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  kforget.armed = false;   // the key decoded: its table is sound
  *accept = ctx->h_small[sizeof(poslo_partial)];
  if (total) {
    memcpy(total->e, h, 32);
    memcpy(total->s, h + 8, 32);
    memcpy(total->R, h + 16, 128);
    total->first_index = parts[0].first_index;
    total->n = n_all;
    total->malformed = h[kShardBadWord];
    total->agg_mode = parts[0].agg_mode;
  }
  return POSLO_OK;
}

// Distill: weighted check of the whole batch first; when it fails (or entries are
// malformed) the segment-tree bisection finds the failing entries, the weighted check of
// the remaining entries confirms them, and per-entry checks of all entries settle the rare
// case where that confirmation fails.
int poslo_distill(poslo_ctx* ctx, const poslo_batch* batch, uint64_t* invalid_idx, uint64_t cap, uint64_t* n_invalid,
                  uint8_t ccd_s[32], uint8_t ccd_R[32]) {
  if (!ctx || !n_invalid) return fail(ctx, POSLO_EINVAL, "bad distill arguments");
  int rc;
  if ((rc = validate_batch(ctx, batch))) return rc;
  if (batch->variant != POSLO_VARIANT_F) return fail(ctx, POSLO_EINVAL, "distill is entry-granular: POSLO-F batches");
  if (batch->n > kMaxCallEntries) return fail(ctx, POSLO_EINVAL, "more than 2^32 - 1 entries in one call");
  const uint64_t n = batch->n;
  const uint64_t n1 = std::max<uint64_t>(n, 1);
  if ((rc = reset_status(ctx))) return rc;
  Staged sb;
  if ((rc = stage_batch(ctx, batch, sb))) return rc;
  // uploads: the key's encoding and the disclosed seeds; the key's window table comes from the
  // key cache (built only when the key is not cached)
  uint32_t *d_Y, *tableY;
  uint32_t** d_ydst;
  if ((rc = ensure_t(ctx, "Y", 32, &d_Y))) return rc;
  if ((rc = ensure_t(ctx, "ydst", 8, &d_ydst))) return rc;
  CU(cudaMemcpyAsync(d_Y, batch->Y, 32, cudaMemcpyHostToDevice, ctx->s_main));
  std::vector<const uint32_t*> ktab;
  std::vector<uint32_t> kmiss;
  std::vector<uint32_t*> kdst;
  const bool kcached = key_cache_lookup(ctx, batch->Y, 1, ktab, kmiss, kdst);
  const bool kbuild = !kcached || !kmiss.empty();
  KeyForget kforget{ctx, batch->Y, &kmiss, kcached && kbuild};
  if (kcached) {
    tableY = const_cast<uint32_t*>(ktab[0]);
    if (kbuild) CU(cudaMemcpyAsync(d_ydst, kdst.data(), 8, cudaMemcpyHostToDevice, ctx->s_main));
  } else if ((rc = ensure_t(ctx, "tableY", 4 * (size_t)kTableWords, &tableY))) {
    return rc;
  }
  std::vector<DsNode> ds_nodes;
  if ((rc = parse_ds(ctx, batch->ds, batch->ds_nodes, ds_nodes))) return rc;
  DsNode* d_ds;
  if ((rc = ensure_t(ctx, "ds", ds_nodes.size() * sizeof(DsNode), &d_ds))) return rc;
  CU(cudaMemcpyAsync(d_ds, ds_nodes.data(), ds_nodes.size() * sizeof(DsNode), cudaMemcpyHostToDevice, ctx->s_main));
  uint64_t e_first = 0, ne = 0;
  if (n) {
    e_first = batch->first_index / batch->n2;
    ne = (batch->first_index + n - 1) / batch->n2 - e_first + 1;
  }
  // workspace
  uint32_t *pts, *z, *small, *seeds;
  uint8_t *badR, *badS, *d_e, *inv, *d_ccd, *d_acc;
  unsigned long long *hpart, *sp;
  const int hblocks = grid_for(ctx, n, kHashThreads, 8);
  const int sblocks = hblocks;
  if ((rc = ensure_t(ctx, "pts", 4 * kPtsWords * n1, &pts))) return rc;
  if ((rc = ensure_t(ctx, "badR", n1, &badR))) return rc;
  if ((rc = ensure_t(ctx, "badS", n1, &badS))) return rc;
  if ((rc = ensure_t(ctx, "z", 16 * n1, &z))) return rc;
  if ((rc = ensure_t(ctx, "e_all", 32 * n1, &d_e))) return rc;
  if ((rc = ensure_t(ctx, "invalid", n1, &inv))) return rc;
  if ((rc = ensure_t(ctx, "distill_small", 4 * 100, &small))) return rc;   // unit R | weighted R | prep | bad count
  if ((rc = ensure_t(ctx, "ccd", 64, &d_ccd))) return rc;
  if ((rc = ensure_t(ctx, "seeds", std::max<uint64_t>(1, ne) * 16, &seeds))) return rc;
  if ((rc = ensure_t(ctx, "hash_partial", (size_t)hblocks * kPartialWords * 8, &hpart))) return rc;
  if ((rc = ensure_t(ctx, "accept", 16, &d_acc))) return rc;
  if ((rc = ensure_t(ctx, "ccd_spart", (size_t)sblocks * 13 * 8, &sp))) return rc;
  uint32_t *unitR = small, *Rw = small + 32, *pbad = small + 97;
  uint32_t* Pw;   // per-window [E_w]Y + [S_w]G (32 words each), then the malformed-s flag
  if ((rc = ensure_t(ctx, "win_P", 4 * (32 * (size_t)kMsmMaxWindows + 1), &Pw))) return rc;
  uint32_t* Pw_bad = Pw + 32 * kMsmMaxWindows;
  // ---- up to the weighted check of the whole batch; a device-resident batch of the previous
  // call's shape replays it from a CUDA graph
  const bool replayable = batch->on_device != 0 || sb.packed;
  auto stage1 = [&]() -> int {
    int rc;
    // window table of Y (table stream), unless cached
    if (kbuild) {
      CU(cudaEventRecord(ctx->ev_main, ctx->s_main));
      CU(cudaStreamWaitEvent(ctx->s_table, ctx->ev_main, 0));
      cudaEvent_t tb, te;
      timer_begin(ctx, "table", ctx->s_table, &tb, &te);
      if ((rc = launch_tables(ctx, ctx->s_table, d_Y, nullptr, nullptr, 1, kcached ? nullptr : tableY, 0, nullptr,
                              kcached ? d_ydst : nullptr)))
        return rc;
      timer_end(ctx, "table", ctx->s_table, tb, te);
      CU(cudaEventRecord(ctx->ev_table, ctx->s_table));
    } else {
      CU(cudaEventRecord(ctx->ev_table, ctx->s_main));
    }
    // decoding (points stream), from the moment the R_t have landed; then the speculative
    // ccd^v of the all-valid case (its R part)
    uint32_t *ppart, npb;
    if ((rc = run_points(ctx, sb.R, n, pts, badR, &ppart, &npb, replayable ? nullptr : ctx->ev_staged))) return rc;
    if ((rc = run_unit_sum(ctx, ppart, npb, unitR, d_ccd + 32, pbad))) return rc;
    // epoch seeds, then the weights z_t alone (they do not depend on the messages) so the
    // MSM's counting sort starts at once; the message hashing (with the per-entry outputs
    // Distill needs) runs on its own stream
    if (ne) {
      cudaEvent_t b, e;
      timer_begin(ctx, "seeds", ctx->s_main, &b, &e);
      launch_epoch_seeds((int)ctx->inst, (unsigned)((ne + 127) / 128), 128, ctx->s_main, d_ds, (int)ds_nodes.size(),
                         e_first, ne, seeds, ctx->status);
      ++ctx->launch_count;
      CU(cudaGetLastError());
      timer_end(ctx, "seeds", ctx->s_main, b, e);
    }
    ZPre zp;
    make_zpre(ctx->vseed, zp.w);
    if (n) {
      k_weights<<<grid_for(ctx, n, kSideThreads, 8), kSideThreads, 0, ctx->s_main>>>(zp, n, batch->first_index, z);
      ++ctx->launch_count;
    }
    CU(cudaEventRecord(ctx->ev_main, ctx->s_main));
    CU(cudaStreamWaitEvent(ctx->s_hash, ctx->ev_main, 0));
    // (measured: hashing beside the decoding, 4.78 ms per 2^20-entry step, beats hashing on the
    // main stream before the sort, 4.88 ms, and beside the bucket accumulation, 4.95 ms)
    cudaStream_t hs = ctx->s_hash;
    HashArgs a{};
    a.msgs = sb.msgs;
    a.offs = sb.offs;
    a.base_off = sb.base_off;
    a.n = n;
    a.first_index = batch->first_index;
    a.e0 = e_first;
    a.n2 = batch->n2;
    a.n2_log2 = log2_exact(batch->n2);
    a.seeds = seeds;
    a.e_out = d_e;
    a.s = sb.s;
    a.weighted = 1;
    for (int q = 0; q < 10; ++q) a.zpre[q] = zp.w[q];
    a.z_in = z;
    a.sbad_out = badS;
    a.partial = hpart;
    a.status = ctx->status;
    MsmState ms;
    if ((rc = run_msm_sort(ctx, ctx->s_main, z, 4, nullptr, n, ms))) return rc;
    {
      cudaEvent_t tb, te;
      timer_begin(ctx, "hash", hs, &tb, &te);
      launch_hash((int)ctx->inst, (unsigned)hblocks, hs, a);
      ++ctx->launch_count;
      CU(cudaGetLastError());
      timer_end(ctx, "hash", hs, tb, te);
    }
    // per-window [E_w]Y + [S_w]G and the s part of ccd^v on the table stream, while the MSM runs
    if ((rc = run_prep_windows(ctx, hpart, (uint32_t)hblocks, tableY, d_e, sb.s, z, n, ms.pl, Pw, Pw_bad, d_ccd,
                               hs)))
      return rc;
    // the MSM needs the decoded points only; the unit sum behind them on the points stream
    // (its encoding is a long inversion chain) is waited for by the check
    CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_decoded, 0));
    // weighted MSM up to its window sums, and the weighted check of the whole batch window by
    // window (it implies the check of the combined equation, and needs no doublings between
    // the windows)
    uint32_t* groups;
    if ((rc = run_msm_finish(ctx, ctx->s_main, pts, badR, ms, nullptr, &groups))) return rc;
    if ((rc = run_window_check(ctx, groups, ms.pl, Pw, Pw_bad, pbad, d_acc))) return rc;
    return POSLO_OK;
  };
  if (replayable) {
    const MsmPlan plan = msm_plan(ctx, n, 4);
    const std::vector<uint64_t> sig = {n, batch->n2, batch->first_index, reinterpret_cast<uint64_t>(sb.msgs),
                                       reinterpret_cast<uint64_t>(sb.offs), reinterpret_cast<uint64_t>(sb.s),
                                       reinterpret_cast<uint64_t>(sb.R), sb.base_off, ds_nodes.size(),
                                       (uint64_t)plan.c, (uint64_t)plan.seg_log2, ctx->inst,
                                       reinterpret_cast<uint64_t>(tableY), kbuild ? 1u : 0u};
    rc = run_replayable(ctx, ctx->g_distill, sig, stage1);
  } else {
    rc = stage1();
  }
  // the decision and the speculative ccd^v of the all-valid case in one round trip
  uint8_t h_acc = 0;
  uint8_t hccd[64];
  if (rc == POSLO_OK) {
    CU(cudaMemcpyAsync(&h_acc, d_acc, 1, cudaMemcpyDeviceToHost, ctx->s_main));
    CU(cudaMemcpyAsync(hccd, d_ccd, 64, cudaMemcpyDeviceToHost, ctx->s_main));
    rc = check_status(ctx);   // synchronises: h_acc and hccd are ready
  }
  if (rc != POSLO_OK) return rc;
  kforget.armed = false;   // the key decoded: its table is sound
  // h_acc covers "no malformed entry and the weighted equation holds": then no entry is
  // invalid and ccd^v is the unit sums of the whole batch, already read
  if (h_acc) {
    *n_invalid = 0;
    if (ccd_s) memcpy(ccd_s, hccd, 32);
    if (ccd_R) memcpy(ccd_R, hccd + 32, 32);
    return POSLO_OK;
  }
  uint64_t* d_idx;
  const uint64_t capn = std::max<uint64_t>(std::min(cap, n), 1);
  if ((rc = ensure_t(ctx, "invalid_idx", 8 * capn + 8, &d_idx))) return rc;
  uint64_t* d_cnt = d_idx + capn;
  uint64_t* fidx;   // local indices of the flagged entries (confirmation, ccd^v), count at fidx[n]
  if ((rc = ensure_t(ctx, "confirm_idx", 8 * (n + 1), &fidx))) return rc;
  uint64_t nf = 0;
  bool confirmed = false;
  if (n <= kDirectCheckMax) {
    // ---- a small batch: every entry's own check (Fig. 4 with |m| = 1) in one launch, the
    // definition itself, instead of the tree, the descent and the confirmation, whose fixed
    // latencies cost more at this size
    DirectCheckArgs a{};
    a.e = d_e;
    a.s = sb.s;
    a.pts = pts;
    a.badR = badR;
    a.badS = badS;
    a.n = n;
    a.tableY = tableY;
    a.tableG = ctx->tableG;
    a.invalid = inv;
    cudaEvent_t tb, te;
    timer_begin(ctx, "direct", ctx->s_main, &tb, &te);
    k_entry_check_group<<<(unsigned)((8 * n + 127) / 128), 128, 0, ctx->s_main>>>(a);
    ++ctx->launch_count;
    CU(cudaGetLastError());
    timer_end(ctx, "direct", ctx->s_main, tb, te);
  } else {
    // ---- localisation: segment-tree bisection over unit aggregates ----
    uint64_t M = 2, L = 1;
    while (M < n) { M <<= 1; ++L; }
    TreeArgs ta{};
    ta.pts = pts;
    ta.e = d_e;
    ta.s = sb.s;
    ta.skip1 = badR;
    ta.skip2 = badS;
    ta.n = n;
    ta.M = M;
    if ((rc = ensure_t(ctx, "tree_pts", 128 * (M - 1), &ta.tree_pts))) return rc;
    if ((rc = ensure_t(ctx, "tree_e", 32 * (M - 1), &ta.tree_e))) return rc;
    if ((rc = ensure_t(ctx, "tree_s", 32 * (M - 1), &ta.tree_s))) return rc;
    cudaEvent_t tb, te;
    timer_begin(ctx, "tree", ctx->s_main, &tb, &te);
    k_tree_leaves<<<(unsigned)((M / 2 + 127) / 128), 128, 0, ctx->s_main>>>(ta);
    ++ctx->launch_count;
    for (uint64_t l = 2; l <= L; ++l) {   // level l from level l - 1 (node (l, k) at M - (M >> (l - 1)) + k)
      const uint64_t count = M >> l;
      k_tree_level<<<(unsigned)((count + 127) / 128), 128, 0, ctx->s_main>>>(ta, M - (M >> (l - 2)),
                                                                             M - (M >> (l - 1)), count);
      ++ctx->launch_count;
    }
    CU(cudaGetLastError());
    timer_end(ctx, "tree", ctx->s_main, tb, te);
    // descent from the root (taken as failing: the weighted check of the batch failed), several
    // levels per step while few nodes fail (k_bisect_step); state on the device, no round trip
    uint64_t* fl;
    uint64_t* cnts;
    int* lvls;
    if ((rc = ensure_t(ctx, "front_lists", 3 * 8 * M, &fl))) return rc;
    if ((rc = ensure_t(ctx, "front_cnt", 3 * 8 + 2 * 4, &cnts))) return rc;
    lvls = reinterpret_cast<int*>(cnts + 3);
    BisectState bst{};
    bst.fail[0] = fl;
    bst.fail[1] = fl + M;
    bst.fail[2] = fl + 2 * M;
    bst.cnt = cnts;
    bst.level = lvls;
    struct {
      uint64_t cnt[3];
      int level[2];
    } init = {{1, 0, 0}, {(int)L, (int)L}};
    static_assert(sizeof(init) == 3 * 8 + 2 * 4, "descent state layout");
    CU(cudaMemsetAsync(fl, 0, 8, ctx->s_main));   // the root's index, 0
    CU(cudaMemcpyAsync(cnts, &init, sizeof(init), cudaMemcpyHostToDevice, ctx->s_main));
    // invalid starts as the malformed entries
    k_flags_or<<<grid_for(ctx, n, 256, 4), 256, 0, ctx->s_main>>>(badR, badS, nullptr, n, inv);
    ++ctx->launch_count;
    // POSLO_BISECT_WAVES waves of resident blocks: a step checks at most as many nodes as the
    // grid has warps
    int bres = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bres, k_bisect_step, 128, 0) != cudaSuccess || bres < 1) bres = 1;
    const int bgrid = ctx->sm_count * bres * POSLO_BISECT_WAVES;
    timer_begin(ctx, "bisect", ctx->s_main, &tb, &te);
    for (int step = 0; step < (int)L; ++step) {
      k_bisect_step<<<bgrid, 128, 0, ctx->s_main>>>(ta, bst, step, tableY, ctx->tableG, inv);
      ++ctx->launch_count;
    }
    CU(cudaGetLastError());
    timer_end(ctx, "bisect", ctx->s_main, tb, te);
    // ---- confirmation: weighted check of every entry not flagged ----
    const int wblocks = grid_for(ctx, n, kHashThreads, 8);
    unsigned long long* wpart;
    if ((rc = ensure_t(ctx, "w_partial", (size_t)wblocks * kPartialWords * 8, &wpart))) return rc;
    k_weighted_sums<<<wblocks, kHashThreads, 0, ctx->s_main>>>(d_e, sb.s, z, inv, nullptr, n, wpart);
    ++ctx->launch_count;
    // sum over the unflagged entries of [z_t]R_t = the whole batch's sum (Horner over the window
    // sums the first weighted check left behind; undecodable points are not in it) minus the
    // flagged entries' with decodable points (an MSM over the flagged entries alone)
    {
      timer_begin(ctx, "confirm", ctx->s_main, &tb, &te);
      const MsmPlan pl1 = msm_plan(ctx, n, 4);
      uint32_t *groups1, *Wc;
      if ((rc = ensure_t(ctx, "msm_groups", 128 * (size_t)pl1.windows * (1 + pl1.jbits), &groups1))) return rc;
      if ((rc = ensure_t(ctx, "confirm_pts", 4 * 96, &Wc))) return rc;
      k_msm_final<<<1, 32, 0, ctx->s_main>>>(groups1, pl1, Wc);
      ++ctx->launch_count;
      if ((rc = run_compact(ctx, inv, n, 0, fidx, n, fidx + n))) return rc;
      CU(cudaMemcpyAsync(&nf, fidx + n, 8, cudaMemcpyDeviceToHost, ctx->s_main));
      CU(cudaStreamSynchronize(ctx->s_main));
      if (nf) {
        uint32_t *gp, *gz;
        uint8_t* gs;
        if ((rc = ensure_t(ctx, "confirm_gpts", 4 * kPtsWords * nf, &gp))) return rc;
        if ((rc = ensure_t(ctx, "confirm_gz", 16 * nf, &gz))) return rc;
        if ((rc = ensure_t(ctx, "confirm_gskip", nf, &gs))) return rc;
        k_gather_flagged<<<(unsigned)((nf + 127) / 128), 128, 0, ctx->s_main>>>(pts, z, badR, fidx, nf, gp, gz, gs);
        ++ctx->launch_count;
        if ((rc = run_msm(ctx, ctx->s_main, gp, gz, 4, gs, nf, Wc + 32))) return rc;
      }
      k_point_diff<<<1, 32, 0, ctx->s_main>>>(Wc, nf ? Wc + 32 : nullptr, Rw);
      ++ctx->launch_count;
      CU(cudaGetLastError());
      timer_end(ctx, "confirm", ctx->s_main, tb, te);
    }
    if ((rc = run_finalize(ctx, wpart, wblocks, nullptr, 0, Rw, nullptr, tableY, d_acc, nullptr))) return rc;
    uint8_t conf = 0;
    CU(cudaMemcpyAsync(&conf, d_acc, 1, cudaMemcpyDeviceToHost, ctx->s_main));
    if ((rc = check_status(ctx))) return rc;
    confirmed = conf != 0;
    if (!confirmed) {
      // errors that cancel inside unit aggregates: settle every entry by its own check
      CheckArgs a{};
      a.e = d_e;
      a.s = sb.s;
      a.R = sb.R;
      a.n = n;
      a.tableY = tableY;
      a.tableG = ctx->tableG;
      a.invalid = inv;
      timer_begin(ctx, "check", ctx->s_main, &tb, &te);
      k_entry_check<<<grid_for(ctx, n, 128, 8), 128, 0, ctx->s_main>>>(a);
      ++ctx->launch_count;
      CU(cudaGetLastError());
      timer_end(ctx, "check", ctx->s_main, tb, te);
    }
  }
  // ordered list of flagged entries and ccd^v over the others; its point is the batch's unit
  // sum (from the first stage) minus the flagged entries' points
  {
    if ((rc = run_compact(ctx, inv, n, batch->first_index, d_idx, std::min(cap, n), d_cnt))) return rc;
    k_sum_scalars<<<sblocks, kHashThreads, 0, ctx->s_main>>>(sb.s, n, inv, sp);
    k_reduce_scalars<<<1, 256, 0, ctx->s_main>>>(sp, sblocks, d_ccd);
    ctx->launch_count += 2;
    // the per-entry checks set the flags (direct localisation, or the fallback after a failed
    // confirmation): list them again; the count stays on the device for k_ccd_points
    if (!confirmed && (rc = run_compact(ctx, inv, n, 0, fidx, n, fidx + n))) return rc;
    k_ccd_points<<<1, 256, 0, ctx->s_main>>>(pts, badR, fidx, fidx + n, unitR, d_ccd + 32);
    ++ctx->launch_count;
    CU(cudaGetLastError());
  }
  uint64_t cnt = 0;
  CU(cudaMemcpyAsync(&cnt, d_cnt, 8, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaMemcpyAsync(hccd, d_ccd, 64, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  const uint64_t got = std::min(cnt, cap);
  if (got && invalid_idx) CU(cudaMemcpy(invalid_idx, d_idx, 8 * got, cudaMemcpyDeviceToHost));
  *n_invalid = cnt;
  if (ccd_s) memcpy(ccd_s, hccd, 32);
  if (ccd_R) memcpy(ccd_R, hccd + 32, 32);
  if (cnt > cap) return fail(ctx, POSLO_EBUFSMALL, "%llu invalid entries, room for %llu", (unsigned long long)cnt,
                             (unsigned long long)cap);
  return POSLO_OK;
}

// Agg: the scalar sum on the main stream beside the decoding and unit sum of the points on
// the points stream; one round trip for both results and the count of undecodable points.
int poslo_agg(poslo_ctx* ctx, const uint8_t* scalars, const uint8_t* points, uint64_t n, uint32_t on_device,
              uint8_t s_out[32], uint8_t R_out[32]) {
  if (!ctx || !s_out || !R_out || (n && (!points || !scalars))) return fail(ctx, POSLO_EINVAL, "bad agg arguments");
  if (n > kMaxCallEntries) return fail(ctx, POSLO_EINVAL, "more than 2^32 - 1 entries in one call");
  if (on_device && n && ((reinterpret_cast<uintptr_t>(points) | reinterpret_cast<uintptr_t>(scalars)) & 15))
    return fail(ctx, POSLO_EINVAL, "device-resident points and scalars must be 16-byte aligned");
  if (n == 0) {   // s~ = 0, R~ = O (encoded y = 1)
    memset(s_out, 0, 32);
    R_out[0] = 1;
    memset(R_out + 1, 0, 31);
    return POSLO_OK;
  }
  int rc;
  if ((rc = reset_status(ctx))) return rc;
  const void *dp, *dsc;
  if ((rc = stage(ctx, "agg_pts_in", points, 32 * n, on_device, ctx->s_main, &dp))) return rc;
  if ((rc = stage(ctx, "agg_sc_in", scalars, 32 * n, on_device, ctx->s_main, &dsc))) return rc;
  uint32_t *ppart, npb;
  if ((rc = run_points(ctx, static_cast<const uint8_t*>(dp), n, nullptr, nullptr, &ppart, &npb))) return rc;
  const int sblocks = grid_for(ctx, n, kHashThreads, 8);
  unsigned long long* sp;
  uint8_t* d_out;   // s~ (32 bytes) | R~ (32 bytes)
  uint32_t* d_bad;
  if ((rc = ensure_t(ctx, "agg_spart", (size_t)sblocks * 13 * 8, &sp))) return rc;
  if ((rc = ensure_t(ctx, "agg_out", 64, &d_out))) return rc;
  if ((rc = ensure_t(ctx, "agg_bad", 16, &d_bad))) return rc;
  k_sum_scalars<<<sblocks, kHashThreads, 0, ctx->s_main>>>(static_cast<const uint8_t*>(dsc), n, nullptr, sp);
  k_reduce_scalars<<<1, 256, 0, ctx->s_main>>>(sp, sblocks, d_out);
  CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_points, 0));
  k_sum_encode<<<1, kFinalThreads, 0, ctx->s_main>>>(ppart, npb, nullptr, d_out + 32, d_bad);
  ctx->launch_count += 3;
  CU(cudaGetLastError());
  uint8_t h[64];
  uint32_t bad = 0;
  CU(cudaMemcpyAsync(h, d_out, 64, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  if (bad) return fail(ctx, POSLO_EINVAL, "%u points do not decode", bad);
  memcpy(s_out, h, 32);
  memcpy(R_out, h + 32, 32);
  return POSLO_OK;
}

int poslo_msm(poslo_ctx* ctx, const uint8_t* points, const uint8_t* scalars, uint64_t n, uint32_t on_device,
              uint8_t out[32]) {
  if (!ctx || !out || (n && (!points || !scalars))) return fail(ctx, POSLO_EINVAL, "bad msm arguments");
  if (n > kMaxCallEntries) return fail(ctx, POSLO_EINVAL, "more than 2^32 - 1 points in one call");
  if (on_device && n && ((reinterpret_cast<uintptr_t>(points) | reinterpret_cast<uintptr_t>(scalars)) & 15))
    return fail(ctx, POSLO_EINVAL, "device-resident points and scalars must be 16-byte aligned");
  int rc;
  if ((rc = reset_status(ctx))) return rc;
  const void *dp, *ds;
  if ((rc = stage(ctx, "msm_pts_in", points, 32 * n, on_device, ctx->s_main, &dp))) return rc;
  if ((rc = stage(ctx, "msm_sc_in", scalars, 32 * n, on_device, ctx->s_main, &ds))) return rc;
  if (n == 0) {
    out[0] = 1;
    memset(out + 1, 0, 31);
    return POSLO_OK;
  }
  uint32_t* pts;
  uint8_t* bad;
  if ((rc = ensure_t(ctx, "pts", 4 * kPtsWords * n, &pts))) return rc;
  if ((rc = ensure_t(ctx, "badR", n, &bad))) return rc;
  uint32_t *ppart, npb;
  if ((rc = run_points(ctx, static_cast<const uint8_t*>(dp), n, pts, bad, &ppart, &npb))) return rc;
  CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_points, 0));
  uint32_t* acc;
  uint8_t* d_out;
  if ((rc = ensure_t(ctx, "msm_acc", 128, &acc))) return rc;
  if ((rc = ensure_t(ctx, "msm_out", 64, &d_out))) return rc;
  if ((rc = run_msm(ctx, ctx->s_main, pts, static_cast<const uint32_t*>(ds), 8, bad, n, acc))) return rc;
  k_encode_ext<<<1, 1, 0, ctx->s_main>>>(acc, d_out);
  ++ctx->launch_count;
  uint32_t *d_bad_cnt;
  if ((rc = ensure_t(ctx, "msm_badcnt", 16, &d_bad_cnt))) return rc;
  k_sum_encode<<<1, kFinalThreads, 0, ctx->s_main>>>(ppart, npb, nullptr, nullptr, d_bad_cnt);
  ++ctx->launch_count;
  uint8_t h[32];
  uint32_t bad_cnt = 0;
  CU(cudaMemcpyAsync(h, d_out, 32, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaMemcpyAsync(&bad_cnt, d_bad_cnt, 4, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  if (bad_cnt) return fail(ctx, POSLO_EINVAL, "%u points do not decode", bad_cnt);
  memcpy(out, h, 32);
  return POSLO_OK;
}

int poslo_msm_autotune(poslo_ctx* ctx, uint64_t n, uint32_t scalar_words, uint32_t* window_out) {
  if (!ctx || n == 0 || n > (1ull << 32) || (scalar_words != 4 && scalar_words != 8))
    return fail(ctx, POSLO_EINVAL, "bad msm_autotune arguments");
  int rc;
  if ((rc = reset_status(ctx))) return rc;
  const int sw = (int)scalar_words;
  const int lg = log2_floor(n);
  uint32_t *pts, *z, *acc;
  if ((rc = ensure_t(ctx, "tune_pts", 4 * kPtsWords * n, &pts))) return rc;
  if ((rc = ensure_t(ctx, "tune_z", 4 * (size_t)sw * n, &z))) return rc;
  if ((rc = ensure_t(ctx, "msm_acc", 128, &acc))) return rc;
  k_msm_tune_fill<<<grid_for(ctx, n, 256, 8), 256, 0, ctx->s_main>>>(pts, z, n, sw);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  int best_c = 0, best_seg = kMsmSegLog2Min;
  float best_ms = 0.f;
  const int c_lo = std::max(8, std::min(16, lg - 8)), c_hi = std::min(16, std::max(8, lg - 1));
  for (int c = c_lo; c <= c_hi && rc == POSLO_OK; ++c) {
    if (!msm_width_balanced(c, sw)) continue;
    // range lengths 2^4 .. 2^8, no longer than an average bucket and leaving at least 512
    // accumulation threads per SM
    const uint64_t per_bucket = n >> (c - 1);
    for (int sl = kMsmSegLog2Min; sl <= kMsmSegLog2Max && rc == POSLO_OK; ++sl) {
      const MsmPlan forced = msm_plan_c(c, sw, sl);
      if (sl > kMsmSegLog2Min &&
          ((1ull << sl) > per_bucket || ((uint64_t)forced.windows * n >> sl) < 512ull * (uint64_t)ctx->sm_count))
        break;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && rc == POSLO_OK; ++rep) {   // the first run grows the buffers
        MsmState st;
        cudaEventRecord(e0, ctx->s_main);
        if ((rc = run_msm_sort(ctx, ctx->s_main, z, sw, nullptr, n, st, &forced))) break;
        if ((rc = run_msm_finish(ctx, ctx->s_main, pts, nullptr, st, acc))) break;
        cudaEventRecord(e1, ctx->s_main);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(ctx, POSLO_EDEVICE, "msm_autotune: %s", "sync failed");
        else cudaEventElapsedTime(&ms, e0, e1);
      }
      if (rc == POSLO_OK && (best_c == 0 || ms < best_ms)) { best_c = c; best_seg = sl; best_ms = ms; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if ((rc = check_status(ctx))) return rc;
  ctx->msm_tuned[lg * 16 + sw] = best_c | (best_seg << 8);
  if (window_out) *window_out = (uint32_t)best_c;
  return POSLO_OK;
}

int poslo_msm_get_plan(poslo_ctx* ctx, uint64_t n, uint32_t scalar_words, uint32_t* window_out,
                       uint32_t* range_log2_out) {
  if (!ctx || (scalar_words != 4 && scalar_words != 8)) return fail(ctx, POSLO_EINVAL, "bad msm_get_plan arguments");
  const MsmPlan pl = msm_plan(ctx, n, (int)scalar_words);
  if (window_out) *window_out = (uint32_t)pl.c;
  if (range_log2_out) *range_log2_out = (uint32_t)pl.seg_log2;
  return POSLO_OK;
}

int poslo_msm_set_plan(poslo_ctx* ctx, uint64_t n, uint32_t scalar_words, uint32_t window, uint32_t range_log2) {
  if (!ctx || (scalar_words != 4 && scalar_words != 8) || window < 8 || window > 16 ||
      range_log2 < (uint32_t)kMsmSegLog2Min || range_log2 > (uint32_t)kMsmSegLog2Max)
    return fail(ctx, POSLO_EINVAL, "bad msm_set_plan arguments");
  ctx->msm_tuned[log2_floor(n) * 16 + (int)scalar_words] = (int)window | ((int)range_log2 << 8);
  return POSLO_OK;
}

// ---------------------------------------------------------------------------- out of core

extern "C" {

int poslo_distill_stream(poslo_ctx* ctx, const poslo_batch* batch, uint64_t chunk_entries, uint8_t* accept,
                         uint64_t* invalid_idx, uint64_t cap, uint64_t* n_invalid) {
  if (!ctx || !accept || !n_invalid || chunk_entries == 0) return fail(ctx, POSLO_EINVAL, "bad distill_stream arguments");
  int rc;
  if ((rc = validate_batch(ctx, batch))) return rc;
  if (batch->variant != POSLO_VARIANT_F) return fail(ctx, POSLO_EINVAL, "streaming Distill is entry-granular: POSLO-F");
  if (batch->on_device) return fail(ctx, POSLO_EINVAL, "streaming takes a batch in host memory");
  const uint64_t n = batch->n;
  const uint64_t nchunks = n ? (n + chunk_entries - 1) / chunk_entries : 0;
  uint64_t max_bytes = 1, max_n = 1;
  for (uint64_t k = 0; k < nchunks; ++k) {   // offsets inside a chunk are checked on the device
    const uint64_t lo = k * chunk_entries, hi = std::min(n, lo + chunk_entries);
    if (batch->offs[hi] < batch->offs[lo]) return fail(ctx, POSLO_EINVAL, "offsets decrease in chunk %llu",
                                                       (unsigned long long)k);
    max_bytes = std::max<uint64_t>(max_bytes, batch->offs[hi] - batch->offs[lo]);
    max_n = std::max(max_n, hi - lo);
  }
  // two sets of staging buffers: messages, offsets (rebased to the chunk), s, R
  uint8_t *msgs[2], *sv[2], *Rv[2];
  uint64_t* offs[2];
  for (int b = 0; b < 2; ++b) {
    const std::string tag = b ? "1" : "0";
    if ((rc = ensure_t(ctx, ("st_msgs" + tag).c_str(), max_bytes, &msgs[b]))) return rc;
    if ((rc = ensure_t(ctx, ("st_offs" + tag).c_str(), 8 * (max_n + 1), &offs[b]))) return rc;
    if ((rc = ensure_t(ctx, ("st_s" + tag).c_str(), 32 * max_n, &sv[b]))) return rc;
    if ((rc = ensure_t(ctx, ("st_R" + tag).c_str(), 32 * max_n, &Rv[b]))) return rc;
  }
  // chunk k's inputs go to set k % 2 on the copy stream; its offsets are rebased there too
  auto issue = [&](uint64_t k) -> int {
    const int b = (int)(k & 1);
    const uint64_t lo = k * chunk_entries, hi = std::min(n, lo + chunk_entries), m = hi - lo;
    const uint64_t base = batch->offs[lo];
    CU(cudaMemcpyAsync(msgs[b], batch->msgs + base, batch->offs[hi] - base, cudaMemcpyHostToDevice, ctx->s_copy));
    CU(cudaMemcpyAsync(offs[b], batch->offs + lo, 8 * (m + 1), cudaMemcpyHostToDevice, ctx->s_copy));
    CU(cudaMemcpyAsync(sv[b], batch->s + 32 * lo, 32 * m, cudaMemcpyHostToDevice, ctx->s_copy));
    CU(cudaMemcpyAsync(Rv[b], batch->R + 32 * lo, 32 * m, cudaMemcpyHostToDevice, ctx->s_copy));
    k_offs_sub<<<(unsigned)((m + 1 + 255) / 256), 256, 0, ctx->s_copy>>>(offs[b], m + 1, base);
    ++ctx->launch_count;
    CU(cudaGetLastError());
    CU(cudaEventRecord(ctx->ev_copy[b], ctx->s_copy));
    return POSLO_OK;
  };
  uint64_t total = 0;
  if (nchunks && (rc = issue(0))) return rc;
  for (uint64_t k = 0; k < nchunks; ++k) {
    const int b = (int)(k & 1);
    const uint64_t lo = k * chunk_entries, hi = std::min(n, lo + chunk_entries);
    // chunk k's verification waits for its copies; chunk k+1's copies start meanwhile (the
    // other set is free: chunk k-1's verification has returned)
    CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_copy[b], 0));
    if (k + 1 < nchunks && (rc = issue(k + 1))) return rc;
    poslo_batch view = *batch;
    view.msgs = msgs[b];
    view.offs = offs[b];
    view.n = hi - lo;
    view.first_index = batch->first_index + lo;
    view.s = sv[b];
    view.R = Rv[b];
    view.R_count = hi - lo;
    view.on_device = 1;
    const uint64_t room = invalid_idx ? (total < cap ? cap - total : 0) : 0;
    uint64_t got = 0;
    rc = poslo_distill(ctx, &view, invalid_idx ? invalid_idx + std::min(total, cap) : nullptr, room, &got, nullptr,
                       nullptr);
    if (rc != POSLO_OK && rc != POSLO_EBUFSMALL) return rc;
    total += got;
  }
  CU(cudaStreamSynchronize(ctx->s_copy));
  *n_invalid = total;
  *accept = total == 0 ? 1 : 0;
  if (total > cap || (total && !invalid_idx))
    return fail(ctx, POSLO_EBUFSMALL, "%llu invalid entries, room for %llu", (unsigned long long)total,
                (unsigned long long)cap);
  return POSLO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------- POSLO-C ccd

namespace {

// 8 little-endian 32-bit limbs to 32 bytes.
void store_le_words(const uint32_t* w, uint8_t* out) {
  for (int k = 0; k < 8; ++k)
    for (int b = 0; b < 4; ++b) out[4 * k + b] = (uint8_t)(w[k] >> (8 * b));
}

// Shared part of C.Distill and SeBVer: checks the batch (whole epochs, per-epoch s~_i and
// R~_i), stages it, starts the key table, and leaves the per-epoch sums e~_i (n1 x 32 bytes,
// limbs little-endian) in *esum.
// The key's window table comes from the key cache; a table this call builds into a new cache
// slot is forgotten again (kforget) unless the caller disarms it once the key has decoded.
int ccd_common(poslo_ctx* ctx, const poslo_batch* batch, uint32_t n_umbrella, Staged& sb, uint64_t& n1,
               uint32_t** tableY, uint8_t** esum, std::vector<uint32_t>& kmiss, KeyForget& kforget) {
  int rc;
  if ((rc = validate_batch(ctx, batch))) return rc;
  if (batch->variant != POSLO_VARIANT_C) return fail(ctx, POSLO_EINVAL, "distillation with ccd is POSLO-C");
  n1 = batch->n / batch->n2;
  if (n1 == 0) return fail(ctx, POSLO_EINVAL, "empty batch");
  if (batch->R_count != n1) return fail(ctx, POSLO_EINVAL, "one R~_i per epoch is required");
  if (n_umbrella == 0 || n1 % n_umbrella) return fail(ctx, POSLO_EINVAL, "n_umbrella must divide n1 = %llu",
                                                      (unsigned long long)n1);
  if ((rc = reset_status(ctx))) return rc;
  if ((rc = stage_batch(ctx, batch, sb, 32 * n1))) return rc;
  std::vector<const uint32_t*> ktab;
  std::vector<uint32_t*> kdst;
  const bool kcached = key_cache_lookup(ctx, batch->Y, 1, ktab, kmiss, kdst);
  kforget.armed = kcached && !kmiss.empty();
  if (kcached && kmiss.empty()) {
    *tableY = const_cast<uint32_t*>(ktab[0]);
    CU(cudaEventRecord(ctx->ev_table, ctx->s_main));   // nothing to wait for
  } else if ((rc = run_ytable(ctx, batch->Y, tableY, kcached ? kdst[0] : nullptr))) {
    return rc;
  }
  uint8_t* d_e;
  if ((rc = ensure_t(ctx, "e_all", 32 * batch->n, &d_e))) return rc;
  if ((rc = ensure_t(ctx, "ccd_esum", 32 * n1, esum))) return rc;
  unsigned long long* hpart;
  uint32_t nhb;
  if ((rc = run_hash(ctx, batch, sb, d_e, false, false, nullptr, &hpart, &nhb))) return rc;
  k_scalar_group_sums<<<(unsigned)n1, kCcdThreads, 0, ctx->s_main>>>(d_e, batch->n2, batch->n, nullptr,
                                                                      reinterpret_cast<uint32_t*>(*esum));
  ++ctx->launch_count;
  CU(cudaGetLastError());
  return POSLO_OK;
}

}  // namespace

extern "C" {

int poslo_distill_c(poslo_ctx* ctx, const poslo_batch* batch, uint32_t n_umbrella, uint8_t* valid,
                    poslo_ccd_c* ccd) {
  if (!ctx || !valid || !ccd || !ccd->s_v || !ccd->R_v || !ccd->umbrellas)
    return fail(ctx, POSLO_EINVAL, "bad distill_c arguments");
  int rc;
  Staged sb;
  uint64_t n1 = 0;
  uint32_t* tableY;
  uint8_t* esum;
  std::vector<uint32_t> kmiss;
  KeyForget kforget{ctx, batch ? batch->Y : nullptr, &kmiss, false};
  if ((rc = ccd_common(ctx, batch, n_umbrella, sb, n1, &tableY, &esum, kmiss, kforget))) return rc;
  const uint64_t g = n1 / n_umbrella;
  uint32_t *pts, *ppart, npb, *words;
  uint8_t *badR, *ok, *inv, *encs;
  uint64_t* d_idx;
  if ((rc = ensure_t(ctx, "ccd_pts", 4 * kPtsWords * n1, &pts))) return rc;
  if ((rc = ensure_t(ctx, "ccd_badR", n1, &badR))) return rc;
  if ((rc = ensure_t(ctx, "ccd_ok", 2 * n1, &ok))) return rc;
  inv = ok + n1;
  if ((rc = ensure_t(ctx, "ccd_words", 32 * (1 + (size_t)n_umbrella), &words))) return rc;
  if ((rc = ensure_t(ctx, "ccd_encs", 32 * (1 + (size_t)n_umbrella), &encs))) return rc;
  const uint64_t capn = std::max<uint64_t>(std::min<uint64_t>(ccd->cap, n1), 1);
  if ((rc = ensure_t(ctx, "ccd_idx", 8 * capn + 8, &d_idx))) return rc;
  uint64_t* d_cnt = d_idx + capn;
  if ((rc = run_points(ctx, sb.R, n1, pts, badR, &ppart, &npb, ctx->ev_staged))) return rc;
  CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_points, 0));
  CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_table, 0));
  // b_i for every epoch, then ccd^v (group 0) and the umbrellas (groups 1..n^u)
  k_check_list<<<(unsigned)((4 * n1 + 127) / 128), 128, 0, ctx->s_main>>>(
      reinterpret_cast<const uint32_t*>(esum), sb.s, pts, badR, (uint32_t)n1, tableY, ctx->tableG, ok);
  k_flip<<<(unsigned)((n1 + 255) / 256), 256, 0, ctx->s_main>>>(ok, n1, inv);
  k_scalar_group_sums<<<1, kCcdThreads, 0, ctx->s_main>>>(sb.s, n1, n1, inv, words);
  k_point_group_sums<<<1, kCcdThreads, 0, ctx->s_main>>>(pts, badR, n1, n1, inv, encs);
  k_scalar_group_sums<<<n_umbrella, kCcdThreads, 0, ctx->s_main>>>(sb.s, g, n1, inv, words + 8);
  k_point_group_sums<<<n_umbrella, kCcdThreads, 0, ctx->s_main>>>(pts, badR, g, n1, inv, encs + 32);
  ctx->launch_count += 6;
  CU(cudaGetLastError());
  const uint64_t first_epoch = batch->first_index / batch->n2;
  if ((rc = run_compact(ctx, inv, n1, first_epoch, d_idx, std::min<uint64_t>(ccd->cap, n1), d_cnt))) return rc;
  std::vector<uint32_t> hw(8 * (1 + (size_t)n_umbrella));
  std::vector<uint8_t> he(32 * (1 + (size_t)n_umbrella));
  uint64_t cnt = 0;
  CU(cudaMemcpyAsync(valid, ok, n1, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaMemcpyAsync(hw.data(), words, 4 * hw.size(), cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaMemcpyAsync(he.data(), encs, he.size(), cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaMemcpyAsync(&cnt, d_cnt, 8, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  kforget.armed = false;   // the key decoded: its table is sound
  store_le_words(hw.data(), ccd->s_v);
  memcpy(ccd->R_v, he.data(), 32);
  for (uint32_t l = 0; l < n_umbrella; ++l) {
    store_le_words(hw.data() + 8 * (1 + (size_t)l), ccd->umbrellas + 64 * (size_t)l);
    memcpy(ccd->umbrellas + 64 * (size_t)l + 32, he.data() + 32 * (1 + (size_t)l), 32);
  }
  const uint64_t got = std::min(cnt, ccd->cap);
  if (got && ccd->invalid) CU(cudaMemcpy(ccd->invalid, d_idx, 8 * got, cudaMemcpyDeviceToHost));
  ccd->n_invalid = cnt;
  if (cnt > ccd->cap) return fail(ctx, POSLO_EBUFSMALL, "%llu invalid epochs, room for %llu",
                                  (unsigned long long)cnt, (unsigned long long)ccd->cap);
  return POSLO_OK;
}

int poslo_sebver_c(poslo_ctx* ctx, const poslo_batch* batch, uint32_t n_umbrella, const poslo_ccd_c* ccd,
                   uint32_t mode, uint8_t* bits) {
  if (!ctx || !ccd || !bits || (mode != POSLO_SEBVER_V && mode != POSLO_SEBVER_U && mode != POSLO_SEBVER_I) ||
      (ccd->n_invalid && !ccd->invalid) || (mode == POSLO_SEBVER_V && (!ccd->s_v || !ccd->R_v)) ||
      (mode == POSLO_SEBVER_U && !ccd->umbrellas))
    return fail(ctx, POSLO_EINVAL, "bad sebver_c arguments");
  int rc;
  Staged sb;
  uint64_t n1 = 0;
  uint32_t* tableY;
  uint8_t* esum;
  std::vector<uint32_t> kmiss;
  KeyForget kforget{ctx, batch ? batch->Y : nullptr, &kmiss, false};
  if ((rc = ccd_common(ctx, batch, n_umbrella, sb, n1, &tableY, &esum, kmiss, kforget))) return rc;
  const uint64_t g = n1 / n_umbrella;
  const uint64_t first_epoch = batch->first_index / batch->n2;
  // the epochs of ccd^i, as positions in the batch
  std::vector<uint8_t> mask(n1, 0);
  std::vector<uint64_t> pos(ccd->n_invalid);
  for (uint64_t k = 0; k < ccd->n_invalid; ++k) {
    const uint64_t i = ccd->invalid[k];
    if (i < first_epoch || i - first_epoch >= n1) return fail(ctx, POSLO_EINVAL, "invalid epoch %llu outside the batch",
                                                              (unsigned long long)i);
    pos[k] = i - first_epoch;
    mask[pos[k]] = 1;
  }
  const uint64_t nchk = mode == POSLO_SEBVER_V ? 1 : (mode == POSLO_SEBVER_U ? n_umbrella : ccd->n_invalid);
  if (nchk == 0) {
    if ((rc = check_status(ctx))) return rc;
    kforget.armed = false;   // the key decoded: its table is sound
    return POSLO_OK;
  }
  uint8_t *d_mask, *s_chk, *R_chk, *bad, *d_bits;
  uint32_t *e_chk, *pts, *ppart, npb;
  uint64_t* d_pos;
  if ((rc = ensure_t(ctx, "seb_mask", n1, &d_mask))) return rc;
  if ((rc = ensure_t(ctx, "seb_pos", 8 * std::max<uint64_t>(ccd->n_invalid, 1), &d_pos))) return rc;
  if ((rc = ensure_t(ctx, "seb_e", 32 * nchk, &e_chk))) return rc;
  if ((rc = ensure_t(ctx, "seb_s", 32 * nchk, &s_chk))) return rc;
  if ((rc = ensure_t(ctx, "seb_R", 32 * nchk, &R_chk))) return rc;
  if ((rc = ensure_t(ctx, "seb_pts", 4 * kPtsWords * nchk, &pts))) return rc;
  if ((rc = ensure_t(ctx, "seb_bad", 2 * nchk, &bad))) return rc;
  d_bits = bad + nchk;
  CU(cudaMemcpyAsync(d_mask, mask.data(), n1, cudaMemcpyHostToDevice, ctx->s_main));
  if (mode == POSLO_SEBVER_V) {
    k_scalar_group_sums<<<1, kCcdThreads, 0, ctx->s_main>>>(esum, n1, n1, d_mask, e_chk);
    CU(cudaMemcpyAsync(s_chk, ccd->s_v, 32, cudaMemcpyHostToDevice, ctx->s_main));
    CU(cudaMemcpyAsync(R_chk, ccd->R_v, 32, cudaMemcpyHostToDevice, ctx->s_main));
    ++ctx->launch_count;
  } else if (mode == POSLO_SEBVER_U) {
    k_scalar_group_sums<<<n_umbrella, kCcdThreads, 0, ctx->s_main>>>(esum, g, n1, d_mask, e_chk);
    ++ctx->launch_count;
    std::vector<uint8_t> hs(32 * nchk), hR(32 * nchk);
    for (uint64_t l = 0; l < nchk; ++l) {
      memcpy(hs.data() + 32 * l, ccd->umbrellas + 64 * l, 32);
      memcpy(hR.data() + 32 * l, ccd->umbrellas + 64 * l + 32, 32);
    }
    CU(cudaMemcpyAsync(s_chk, hs.data(), hs.size(), cudaMemcpyHostToDevice, ctx->s_main));
    CU(cudaMemcpyAsync(R_chk, hR.data(), hR.size(), cudaMemcpyHostToDevice, ctx->s_main));
    CU(cudaStreamSynchronize(ctx->s_main));   // the host staging vectors end here
  } else {
    CU(cudaMemcpyAsync(d_pos, pos.data(), 8 * nchk, cudaMemcpyHostToDevice, ctx->s_main));
    const unsigned gb = (unsigned)((2 * nchk + 255) / 256);
    k_gather32<<<gb, 256, 0, ctx->s_main>>>(esum, d_pos, nchk, reinterpret_cast<uint8_t*>(e_chk));
    k_gather32<<<gb, 256, 0, ctx->s_main>>>(sb.s, d_pos, nchk, s_chk);
    k_gather32<<<gb, 256, 0, ctx->s_main>>>(sb.R, d_pos, nchk, R_chk);
    ctx->launch_count += 3;
    CU(cudaStreamSynchronize(ctx->s_main));   // pos ends here
  }
  CU(cudaGetLastError());
  if ((rc = run_points(ctx, R_chk, nchk, pts, bad, &ppart, &npb))) return rc;
  CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_points, 0));
  CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_table, 0));
  k_check_list<<<(unsigned)((4 * nchk + 127) / 128), 128, 0, ctx->s_main>>>(e_chk, s_chk, pts, bad, (uint32_t)nchk,
                                                                             tableY, ctx->tableG, d_bits);
  ++ctx->launch_count;
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(bits, d_bits, nchk, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  kforget.armed = false;   // the key decoded: its table is sound
  return POSLO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------- multi-device

int poslo_aver_multi(poslo_ctx* ctx, const poslo_multi_batch* mb, uint8_t* accept, uint64_t* invalid_pairs,
                     uint64_t cap, uint64_t* n_invalid) {
  return poslo_host::aver_multi(ctx, mb, nullptr, accept, invalid_pairs, cap, n_invalid);
}

}  // extern "C"

size_t poslo_host::key_table_words() { return kTableWords; }

int poslo_host::build_key_table(poslo_ctx* ctx, const uint8_t Y[32], uint32_t* table_dev) {
  int rc;
  if ((rc = reset_status(ctx))) return rc;
  uint32_t* d_Y;
  uint8_t* d_bad;
  if ((rc = ensure_t(ctx, "reg_Y", 32, &d_Y))) return rc;
  if ((rc = ensure_t(ctx, "reg_bad", 16, &d_bad))) return rc;
  CU(cudaMemcpyAsync(d_Y, Y, 32, cudaMemcpyHostToDevice, ctx->s_main));
  if ((rc = launch_tables(ctx, ctx->s_main, d_Y, nullptr, nullptr, 1, table_dev, 0, d_bad))) return rc;
  uint8_t bad = 1;
  CU(cudaMemcpyAsync(&bad, d_bad, 1, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  if (bad) return fail(ctx, POSLO_EINVAL, "key does not decode");
  return POSLO_OK;
}

namespace {

// Staging errors go to the set (another thread may be using the context meanwhile).
int stage_fail(poslo_host::StageSet& S, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  S.err = buf;
  return code;
}

#define SCU(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return stage_fail(S, POSLO_EDEVICE, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Grows a staging buffer to at least `bytes` (by half again at least); the set's previous
// copies have landed when this runs, and cudaFree waits for the device in any case.
int stage_grow(poslo_host::StageSet& S, poslo_host::DevBuf& b, size_t bytes, void** out) {
  bytes = std::max<size_t>(bytes, 16);
  if (b.cap < bytes) {
    size_t want = std::max(bytes, b.cap + b.cap / 2);
    want = (want + 255) & ~size_t(255);
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    const cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return stage_fail(S, POSLO_ENOMEM, "staging buffer of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    b.cap = want;
  }
  *out = b.p;
  return POSLO_OK;
}

template <class T>
int stage_grow_t(poslo_host::StageSet& S, poslo_host::DevBuf& b, size_t bytes, T** out) {
  void* p;
  const int rc = stage_grow(S, b, bytes, &p);
  *out = static_cast<T*>(p);
  return rc;
}

}  // namespace

int poslo_host::stage_requests(poslo_ctx* ctx, const ReqView* reqs, uint32_t nd, poslo_multi_batch* mb, int set) {
  if (set != 0 && set != 1) return POSLO_EINVAL;
  StageSet& S = ctx->stage[set];
  S.err.clear();
  S.launches = 0;
  int rc;
  // slot: raw offsets of request d at [slot[d], slot[d+1]); start: its first entry in the
  // batch; base: its first message byte in the batch
  std::vector<uint64_t> meta(3 * ((size_t)nd + 1), 0);
  uint64_t* slot = meta.data();
  uint64_t* start = slot + nd + 1;
  uint64_t* base = start + nd + 1;
  for (uint32_t d = 0; d < nd; ++d) {
    const ReqView& r = reqs[d];
    if (r.n && r.offs[r.n] < r.offs[0]) return stage_fail(S, POSLO_EINVAL, "request %u: offsets decrease", d);
    slot[d + 1] = slot[d] + r.n + 1;
    start[d + 1] = start[d] + r.n;
    base[d + 1] = base[d] + (r.n ? r.offs[r.n] - r.offs[0] : 0);
  }
  const uint64_t N = start[nd], M = base[nd];
  uint8_t *msgs, *sv, *Rv;
  uint64_t *raw, *offs, *d_meta;
  uint32_t* d_st;
  if ((rc = stage_grow_t(S, S.msgs, M, &msgs))) return rc;
  if ((rc = stage_grow_t(S, S.raw, 8 * slot[nd], &raw))) return rc;
  if ((rc = stage_grow_t(S, S.offs, 8 * (N + 1), &offs))) return rc;
  if ((rc = stage_grow_t(S, S.s, 32 * N, &sv))) return rc;
  if ((rc = stage_grow_t(S, S.R, 32 * N, &Rv))) return rc;
  if ((rc = stage_grow_t(S, S.meta, 8 * meta.size(), &d_meta))) return rc;
  if ((rc = stage_grow_t(S, S.status, 4, &d_st))) return rc;
  // small requests in mapped page-locked memory: one gather kernel over a table of regions
  // (one launch instead of four copies each); large ones and all others: one copy per array,
  // on the copy engines, which leave the SMs to the verification of other batches
  std::vector<GatherRegion> regions;
  std::vector<uint32_t> copied;
  for (uint32_t d = 0; d < nd; ++d) {
    const ReqView& r = reqs[d];
    if (r.n == 0) continue;
    const uint64_t lo = r.offs[0], len = r.offs[r.n] - lo;
    if (r.d_msgs && r.d_offs && r.d_s && r.d_R && len + 72 * r.n < kGatherMaxRequestBytes) {
      auto add = [&](const uint8_t* src, uint8_t* dst, uint64_t bytes) {
        for (uint64_t o = 0; o < bytes; o += kGatherChunk)
          regions.push_back(GatherRegion{src + o, dst + o, std::min<uint64_t>(kGatherChunk, bytes - o)});
      };
      add(r.d_msgs + lo, msgs + base[d], len);
      add(reinterpret_cast<const uint8_t*>(r.d_offs), reinterpret_cast<uint8_t*>(raw + slot[d]), 8 * (r.n + 1));
      add(r.d_s, sv + 32 * start[d], 32 * r.n);
      add(r.d_R, Rv + 32 * start[d], 32 * r.n);
    } else {
      copied.push_back(d);
    }
  }
  GatherRegion* d_reg = nullptr;
  if (!regions.empty() && (rc = stage_grow_t(S, S.regions, sizeof(GatherRegion) * regions.size(), &d_reg)))
    return rc;
  // the status word and the two tables go up from page-locked memory: a copy from pageable
  // memory would first wait for every copy already queued on the stream
  const size_t meta_bytes = 8 * meta.size(), reg_bytes = sizeof(GatherRegion) * regions.size();
  const size_t h_bytes = 16 + meta_bytes + reg_bytes;
  if (S.h_cap < h_bytes) {
    if (S.h) cudaFreeHost(S.h);
    S.h = nullptr;
    S.h_cap = 0;
    const size_t want = std::max<size_t>(2 * h_bytes, 1 << 16);
    if (cudaMallocHost(&S.h, want) != cudaSuccess) {
      cudaGetLastError();
      return stage_fail(S, POSLO_ENOMEM, "page-locked staging table of %zu bytes", want);
    }
    S.h_cap = want;
  }
  uint32_t* h_st = reinterpret_cast<uint32_t*>(S.h);
  uint8_t* h_meta = S.h + 16;
  uint8_t* h_reg = h_meta + meta_bytes;   // 8-byte aligned, as GatherRegion
  *h_st = 0;
  memcpy(h_meta, meta.data(), meta_bytes);
  if (reg_bytes) memcpy(h_reg, regions.data(), reg_bytes);
  // from here on only the stream's own errors end the staging early.  The copy stream, so
  // that the staging overlaps the verification of the previous batch on s_main; the set's
  // own status word, so that it neither reads nor clears that verification's.
  cudaStream_t st = ctx->s_copy;
  SCU(cudaMemsetAsync(d_st, 0, 4, st));
  for (uint32_t d : copied) {
    const ReqView& r = reqs[d];
    const uint64_t lo = r.offs[0], len = r.offs[r.n] - lo;
    if (len) SCU(cudaMemcpyAsync(msgs + base[d], r.msgs + lo, len, cudaMemcpyHostToDevice, st));
    SCU(cudaMemcpyAsync(raw + slot[d], r.offs, 8 * (r.n + 1), cudaMemcpyHostToDevice, st));
    SCU(cudaMemcpyAsync(sv + 32 * start[d], r.s, 32 * r.n, cudaMemcpyHostToDevice, st));
    SCU(cudaMemcpyAsync(Rv + 32 * start[d], r.R, 32 * r.n, cudaMemcpyHostToDevice, st));
  }
  if (!regions.empty()) {
    SCU(cudaMemcpyAsync(d_reg, h_reg, reg_bytes, cudaMemcpyHostToDevice, st));
    const unsigned grid = (unsigned)std::min<size_t>(regions.size(), (size_t)ctx->sm_count * 8);
    k_stage_gather<<<grid, 256, 0, st>>>(d_reg, (uint32_t)regions.size());
    ++S.launches;
  }
  SCU(cudaMemcpyAsync(d_meta, h_meta, meta_bytes, cudaMemcpyHostToDevice, st));
  SCU(cudaMemsetAsync(offs, 0, 8, st));   // an empty batch still has offs[0] = 0
  if (slot[nd]) {
    k_rebase_offs<<<(unsigned)((slot[nd] + 255) / 256), 256, 0, st>>>(raw, d_meta, d_meta + nd + 1,
                                                                       d_meta + 2 * ((size_t)nd + 1), nd, offs,
                                                                       d_st);
    ++S.launches;
  }
  SCU(cudaMemcpyAsync(h_st, d_st, 4, cudaMemcpyDeviceToHost, st));
  SCU(cudaGetLastError());
  SCU(cudaEventRecord(ctx->ev_copy[set], st));
  mb->msgs = msgs;
  mb->offs = offs;
  mb->s = sv;
  mb->R = Rv;
  mb->on_device = 1;
  return POSLO_OK;
}

#undef SCU

int poslo_host::stage_wait(poslo_ctx* ctx, int set, int issue_rc) {
  if (set != 0 && set != 1) return fail(ctx, POSLO_EINVAL, "staging set must be 0 or 1");
  StageSet& S = ctx->stage[set];
  ctx->launch_count += S.launches;
  // what was issued has to land before the requests' memory may be released, error or not:
  // a staging that stopped part way recorded no event, so the whole copy stream is drained
  if (issue_rc != POSLO_OK) {
    cudaStreamSynchronize(ctx->s_copy);
    cudaGetLastError();
    return fail(ctx, issue_rc, "staging: %s", S.err.c_str());
  }
  CU(cudaEventSynchronize(ctx->ev_copy[set]));
  if (*reinterpret_cast<const uint32_t*>(S.h) & kErrInput)
    return fail(ctx, POSLO_EINVAL, "message offsets decrease (or precede msgs)");
  return POSLO_OK;
}

int poslo_host::aver_multi(poslo_ctx* ctx, const poslo_multi_batch* mb, const uint32_t* const* key_tables,
                           uint8_t* accept, uint64_t* invalid_pairs, uint64_t cap, uint64_t* n_invalid,
                           const std::function<void(const uint8_t* flagged)>* settled) {
  if (!ctx || !mb || !accept || !n_invalid || mb->n_dev == 0 || !mb->Y || !mb->dev_start || !mb->first_index ||
      !mb->n2 || !mb->ds || !mb->ds_off)
    return fail(ctx, POSLO_EINVAL, "bad aver_multi arguments");
  int rc;
  const uint32_t nd = mb->n_dev;
  const uint64_t N = mb->dev_start[nd];
  if (mb->dev_start[0] != 0 || mb->ds_off[0] != 0) return fail(ctx, POSLO_EINVAL, "segment tables must start at 0");
  if (N > kMaxCallEntries) return fail(ctx, POSLO_EINVAL, "more than 2^32 - 1 entries in one call");
  std::vector<uint64_t> e0(nd), seed_off(nd + 1, 0);
  for (uint32_t d = 0; d < nd; ++d) {
    if (mb->dev_start[d + 1] < mb->dev_start[d]) return fail(ctx, POSLO_EINVAL, "dev_start decreases at %u", d);
    if (mb->ds_off[d + 1] <= mb->ds_off[d]) return fail(ctx, POSLO_EINVAL, "device %u has no disclosed seed", d);
    if (mb->n2[d] == 0) return fail(ctx, POSLO_EINVAL, "device %u: n2 = 0", d);
    const uint64_t nd_ = mb->dev_start[d + 1] - mb->dev_start[d];
    uint64_t ne = 0;
    e0[d] = mb->first_index[d] / mb->n2[d];
    if (nd_) ne = (mb->first_index[d] + nd_ - 1) / mb->n2[d] - e0[d] + 1;
    seed_off[d + 1] = seed_off[d] + ne;
  }
  if (N && (!mb->offs || !mb->s || !mb->R)) return fail(ctx, POSLO_EINVAL, "missing batch arrays");
  if (mb->on_device && N && !device_aligned(mb->offs, mb->s, mb->R))
    return fail(ctx, POSLO_EINVAL, "device-resident offs must be 8-byte aligned, s and R 16-byte aligned");
  if ((rc = reset_status(ctx))) return rc;
  // ---- stage the concatenated batch and the segment tables
  poslo_batch view{};
  view.variant = POSLO_VARIANT_F;
  view.n2 = 1;
  view.Y = mb->Y;
  view.msgs = mb->msgs;
  view.offs = mb->offs;
  view.n = N;
  view.s = mb->s;
  view.R = mb->R;
  view.R_count = N;
  view.on_device = mb->on_device;
  Staged sb;
  if ((rc = stage_batch(ctx, &view, sb))) return rc;
  std::vector<DsNode> nodes;
  if ((rc = parse_ds(ctx, mb->ds, mb->ds_off[nd], nodes))) return rc;
  std::vector<uint64_t> meta;   // start | first | seed_off | e0 | devices by size, largest first
  meta.insert(meta.end(), mb->dev_start, mb->dev_start + nd + 1);
  meta.insert(meta.end(), mb->first_index, mb->first_index + nd);
  meta.insert(meta.end(), seed_off.begin(), seed_off.end());
  meta.insert(meta.end(), e0.begin(), e0.end());
  {
    std::vector<uint64_t> order(nd);
    for (uint32_t d = 0; d < nd; ++d) order[d] = d;
    std::stable_sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) {
      return mb->dev_start[a + 1] - mb->dev_start[a] > mb->dev_start[b + 1] - mb->dev_start[b];
    });
    meta.insert(meta.end(), order.begin(), order.end());
    // pieces of the segment sums (devices largest first, a device's pieces together) | the
    // first piece of every device
    std::vector<uint64_t> pfirst(nd);
    for (uint64_t d : order) {
      const uint64_t n_d = mb->dev_start[d + 1] - mb->dev_start[d];
      const uint64_t np = n_d == 0 ? 1 : (n_d + kSegPiece - 1) / kSegPiece;
      pfirst[d] = meta.size() - (5 * (size_t)nd + 2);
      for (uint64_t k = 0; k < np; ++k) meta.push_back(d | (k << 32));
    }
    meta.insert(meta.end(), pfirst.begin(), pfirst.end());
  }
  const uint64_t n_pieces = meta.size() - (6 * (size_t)nd + 2);
  uint64_t* d_meta;
  uint32_t *d_n2, *d_dsoff;
  DsNode* d_nodes;
  uint8_t* d_Y;
  if ((rc = ensure_t(ctx, "m_meta", 8 * meta.size(), &d_meta))) return rc;
  if ((rc = ensure_t(ctx, "m_n2", 4 * (size_t)nd, &d_n2))) return rc;
  if ((rc = ensure_t(ctx, "m_dsoff", 4 * (size_t)(nd + 1), &d_dsoff))) return rc;
  if ((rc = ensure_t(ctx, "m_nodes", sizeof(DsNode) * nodes.size(), &d_nodes))) return rc;
  if ((rc = ensure_t(ctx, "m_Y", 32 * (size_t)nd, &d_Y))) return rc;
  CU(cudaMemcpyAsync(d_meta, meta.data(), 8 * meta.size(), cudaMemcpyHostToDevice, ctx->s_main));
  CU(cudaMemcpyAsync(d_n2, mb->n2, 4 * (size_t)nd, cudaMemcpyHostToDevice, ctx->s_main));
  CU(cudaMemcpyAsync(d_dsoff, mb->ds_off, 4 * (size_t)(nd + 1), cudaMemcpyHostToDevice, ctx->s_main));
  CU(cudaMemcpyAsync(d_nodes, nodes.data(), sizeof(DsNode) * nodes.size(), cudaMemcpyHostToDevice, ctx->s_main));
  CU(cudaMemcpyAsync(d_Y, mb->Y, 32 * (size_t)nd, cudaMemcpyHostToDevice, ctx->s_main));
  // ---- window tables of every device key (built on the table stream from the encodings,
  // unless the caller holds them resident); tabs[d] points at device d's table
  uint8_t* badY;
  const uint32_t** d_tabs;
  uint32_t* tablesY = nullptr;
  if ((rc = ensure_t(ctx, "m_badY", nd, &badY))) return rc;
  if ((rc = ensure_t(ctx, "m_tabs", 8 * (size_t)nd, &d_tabs))) return rc;
  std::vector<const uint32_t*> tabs(nd);
  // without resident tables: the context's key cache, building only the keys it misses (their
  // encodings gathered into m_Ymiss, destinations in m_mdst, decode flags in m_mbad); a
  // cache too small for the call builds every table into m_tablesY
  std::vector<uint32_t> kmiss;
  std::vector<uint32_t*> kdst;
  bool kcached = false;
  uint32_t nbuild = 0;
  uint32_t* d_Ymiss = nullptr;
  uint32_t** d_mdst = nullptr;
  uint8_t* d_mbad = nullptr;
  KeyForget forget{ctx, mb->Y, &kmiss, false};
  if (key_tables) {
    for (uint32_t d = 0; d < nd; ++d) tabs[d] = key_tables[d];
  } else if ((kcached = key_cache_lookup(ctx, mb->Y, nd, tabs, kmiss, kdst))) {
    forget.armed = !kmiss.empty();
    nbuild = (uint32_t)kmiss.size();
    if (nbuild) {
      std::vector<uint8_t> ym(32 * (size_t)nbuild);
      for (uint32_t k = 0; k < nbuild; ++k) memcpy(ym.data() + 32 * (size_t)k, mb->Y + 32 * (size_t)kmiss[k], 32);
      if ((rc = ensure_t(ctx, "m_Ymiss", ym.size(), &d_Ymiss))) return rc;
      if ((rc = ensure_t(ctx, "m_mdst", 8 * (size_t)nbuild, &d_mdst))) return rc;
      if ((rc = ensure_t(ctx, "m_mbad", nbuild, &d_mbad))) return rc;
      CU(cudaMemcpyAsync(d_Ymiss, ym.data(), ym.size(), cudaMemcpyHostToDevice, ctx->s_main));
      CU(cudaMemcpyAsync(d_mdst, kdst.data(), 8 * (size_t)nbuild, cudaMemcpyHostToDevice, ctx->s_main));
    }
  } else {
    if ((rc = ensure_t(ctx, "m_tablesY", 4 * (size_t)kTableWords * nd, &tablesY))) return rc;
    for (uint32_t d = 0; d < nd; ++d) tabs[d] = tablesY + (size_t)d * kTableWords;
  }
  CU(cudaMemcpyAsync(d_tabs, tabs.data(), 8 * (size_t)nd, cudaMemcpyHostToDevice, ctx->s_main));
  const uint64_t* seg_start = d_meta;
  const uint64_t* seg_first = d_meta + nd + 1;
  const uint64_t* seg_seed_off = d_meta + 2 * nd + 1;
  const uint64_t* seg_e0 = d_meta + 3 * nd + 2;
  const uint64_t* seg_order = d_meta + 4 * nd + 2;
  const uint64_t* seg_pieces = d_meta + 5 * nd + 2;
  const uint64_t* seg_pfirst = seg_pieces + n_pieces;
  // ---- workspace of the first stage
  const uint64_t N1 = std::max<uint64_t>(N, 1);
  uint32_t *seeds, *pts, *z, *P1, *segbuf, *tmpart;
  uint8_t *badR, *badS, *d_e, *d_acc, *dev_flag, *eskip;
  const int tmb = grid_for(ctx, (uint64_t)nd * kTableWindows, kPointThreads, 4);
  if ((rc = ensure_t(ctx, "seeds", 16 * std::max<uint64_t>(seed_off[nd], 1), &seeds))) return rc;
  if ((rc = ensure_t(ctx, "pts", 4 * kPtsWords * N1, &pts))) return rc;
  if ((rc = ensure_t(ctx, "badR", N1, &badR))) return rc;
  if ((rc = ensure_t(ctx, "badS", N1, &badS))) return rc;
  if ((rc = ensure_t(ctx, "e_all", 32 * N1, &d_e))) return rc;
  if ((rc = ensure_t(ctx, "z", 16 * N1, &z))) return rc;
  unsigned long long* piece_limbs;
  uint32_t* piece_R;
  if ((rc = ensure_t(ctx, "m_piece_limbs", 8 * kSegLimbWords * n_pieces, &piece_limbs))) return rc;
  if ((rc = ensure_t(ctx, "m_piece_R", 4 * 32 * n_pieces, &piece_R))) return rc;
  if ((rc = ensure_t(ctx, "m_P", 384, &P1))) return rc;
  if ((rc = ensure_t(ctx, "accept", 16, &d_acc))) return rc;
  if ((rc = ensure_t(ctx, "m_devflag", nd, &dev_flag))) return rc;
  if ((rc = ensure_t(ctx, "m_eskip", N1, &eskip))) return rc;
  if ((rc = ensure_t(ctx, "m_seg", (size_t)nd * (32 + 32 + 1) * 4, &segbuf))) return rc;
  if ((rc = ensure_t(ctx, "m_tmpart", (size_t)tmb * kPointPartialWords * 4, &tmpart))) return rc;
  uint32_t *P2 = P1 + 32, *P3 = P1 + 64;
  // batches up to multi_window_max entries (0 by default) check window by window (no Horner
  // over the windows on the critical path); others with the full weights.  Measured: no gain
  // on small batches, whose latency is the decoding's and the key tables' chains, and a loss
  // on served batches with large requests, whose per-device, per-window sums run one block
  // per (device, window) over all of the device's entries
  const MsmPlan plan = msm_plan(ctx, N, 4);
  const bool per_window = N <= ctx->multi_window_max;
  const uint32_t nw = (uint32_t)plan.windows;
  const int tmbw = std::max(1, tmb / (int)nw);
  uint32_t *Wbuf = nullptr, *EWd = nullptr, *tmpw = nullptr;
  if (per_window) {
    if ((rc = ensure_t(ctx, "m_W", 4 * 3 * 32 * (size_t)nw, &Wbuf))) return rc;
    if ((rc = ensure_t(ctx, "m_EWd", 4 * 2 * 8 * (size_t)nw * nd, &EWd))) return rc;
    if ((rc = ensure_t(ctx, "m_tmpw", (size_t)tmbw * nw * kPointPartialWords * 4, &tmpw))) return rc;
  }
  uint32_t *Wall = Wbuf, *Wsub = Wbuf ? Wbuf + 32 * (size_t)nw : nullptr, *P2w = Wbuf ? Wbuf + 64 * (size_t)nw : nullptr;
  uint32_t *Ewd = EWd, *Swd = EWd ? EWd + 8 * (size_t)nw * nd : nullptr;
  SegSums ss;
  ss.Ew = segbuf;
  ss.Sw = ss.Ew + 8 * (size_t)nd;
  ss.Eu = ss.Sw + 8 * (size_t)nd;
  ss.Su = ss.Eu + 8 * (size_t)nd;
  ss.Ru = ss.Su + 8 * (size_t)nd;
  ss.bad = ss.Ru + 32 * (size_t)nd;
  // ---- first stage, up to the combined check: one launch per step over the device segment
  // table, replayed from a CUDA graph when the call has the shape of the previous one
  std::vector<uint64_t> sig = {nd, N, mb->on_device, key_tables ? 1u : 0u, sb.base_off,
                               reinterpret_cast<uint64_t>(sb.msgs), reinterpret_cast<uint64_t>(sb.offs),
                               reinterpret_cast<uint64_t>(sb.s), reinterpret_cast<uint64_t>(sb.R),
                               nodes.size(), (uint64_t)plan.c, (uint64_t)plan.seg_log2, ctx->inst,
                               per_window ? 1u : 0u, kcached ? 1u : 0u, nbuild};
  sig.insert(sig.end(), mb->dev_start, mb->dev_start + nd + 1);
  sig.insert(sig.end(), mb->first_index, mb->first_index + nd);
  sig.insert(sig.end(), mb->n2, mb->n2 + nd);
  sig.insert(sig.end(), mb->ds_off, mb->ds_off + nd + 1);
  auto stage1 = [&]() -> int {
    int rc;
    if (key_tables || (kcached && nbuild == 0)) {
      CU(cudaMemsetAsync(badY, 0, nd, ctx->s_main));
      CU(cudaEventRecord(ctx->ev_table, ctx->s_main));
    } else if (kcached) {
      CU(cudaMemsetAsync(badY, 0, nd, ctx->s_main));
      CU(cudaEventRecord(ctx->ev_main, ctx->s_main));
      CU(cudaStreamWaitEvent(ctx->s_table, ctx->ev_main, 0));
      cudaEvent_t tb, te;
      timer_begin(ctx, "table", ctx->s_table, &tb, &te);
      if ((rc = launch_tables(ctx, ctx->s_table, d_Ymiss, nullptr, nullptr, nbuild, nullptr, 0, d_mbad, d_mdst)))
        return rc;
      timer_end(ctx, "table", ctx->s_table, tb, te);
      CU(cudaEventRecord(ctx->ev_table, ctx->s_table));
    } else {
      CU(cudaEventRecord(ctx->ev_main, ctx->s_main));
      CU(cudaStreamWaitEvent(ctx->s_table, ctx->ev_main, 0));
      cudaEvent_t tb, te;
      timer_begin(ctx, "table", ctx->s_table, &tb, &te);
      if ((rc = launch_tables(ctx, ctx->s_table, reinterpret_cast<const uint32_t*>(d_Y), nullptr, nullptr, nd,
                              tablesY, 0, badY)))
        return rc;
      timer_end(ctx, "table", ctx->s_table, tb, te);
      CU(cudaEventRecord(ctx->ev_table, ctx->s_table));
    }
    // epoch seeds of every device
    if (seed_off[nd]) {
      launch_epoch_seeds_multi((int)ctx->inst, (unsigned)((seed_off[nd] + 127) / 128), 128, ctx->s_main, d_nodes,
                               d_dsoff, seg_seed_off, seg_e0, nd, seeds, ctx->status);
      ++ctx->launch_count;
    }
    // (side stream) decode every R_t, compiled to share the SMs with the hashing
    uint32_t *ppart, npb;
    if ((rc = run_points(ctx, sb.R, N, pts, badR, &ppart, &npb, nullptr, true))) return rc;
    // the weights z_t alone (they depend only on the batch position), so the MSM's counting
    // sort runs beside the decoding; the segmented hashing (per-entry e_t) on its own stream
    ZPre zp;
    make_zpre(ctx->vseed, zp.w);
    if (N) {
      k_weights<<<grid_for(ctx, N, kSideThreads, 8), kSideThreads, 0, ctx->s_main>>>(zp, N, 0, z);
      ++ctx->launch_count;
    }
    CU(cudaEventRecord(ctx->ev_main, ctx->s_main));
    CU(cudaStreamWaitEvent(ctx->s_hash, ctx->ev_main, 0));
    {
      const int blocks = grid_for(ctx, N, kHashThreads, 8);
      unsigned long long* hpart;
      if ((rc = ensure_t(ctx, "hash_partial", (size_t)blocks * kPartialWords * 8, &hpart))) return rc;
      HashArgs a{};
      a.msgs = sb.msgs;
      a.offs = sb.offs;
      a.base_off = sb.base_off;
      a.n = N;
      a.n2 = 1;
      a.n2_log2 = 0xffffffffu;
      a.seeds = seeds;
      a.e_out = d_e;
      a.s = sb.s;
      a.weighted = 1;
      for (int q = 0; q < 10; ++q) a.zpre[q] = zp.w[q];
      a.z_in = z;
      a.sbad_out = badS;
      a.partial = hpart;
      a.status = ctx->status;
      a.n_seg = nd;
      a.seg_start = seg_start;
      a.seg_first = seg_first;
      a.seg_seed_off = seg_seed_off;
      a.seg_e0 = seg_e0;
      a.seg_n2 = d_n2;
      cudaEvent_t tb, te;
      timer_begin(ctx, "hash", ctx->s_hash, &tb, &te);
      launch_hash((int)ctx->inst, (unsigned)blocks, ctx->s_hash, a, true);
      ++ctx->launch_count;
      CU(cudaGetLastError());
      timer_end(ctx, "hash", ctx->s_hash, tb, te);
      CU(cudaEventRecord(ctx->ev_hash, ctx->s_hash));
    }
    MsmState ms;
    if ((rc = run_msm_sort(ctx, ctx->s_main, z, 4, nullptr, N, ms))) return rc;
    CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_points, 0));
    // sum_t z_t R_t (or its window sums), per-device sums, sum_d E_d Y_d, the combined check
    uint32_t* groups = nullptr;
    if ((rc = run_msm_finish(ctx, ctx->s_main, pts, badR, ms, P1, per_window ? &groups : nullptr))) return rc;
    if (per_window) {
      k_msm_windows<<<1, 32, 0, ctx->s_main>>>(groups, ms.pl, Wall);
      ++ctx->launch_count;
    }
    CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_hash, 0));
    {
      cudaEvent_t tb, te;
      timer_begin(ctx, "segment_sums", ctx->s_main, &tb, &te);
      launch_segment_sums((unsigned)n_pieces, ctx->s_main, d_e, sb.s, z, pts, badR, badS, seg_start, seg_pieces,
                          piece_limbs, piece_R, ss);
      ctx->launch_count += 2;
      if (n_pieces > nd) {
        k_segment_combine<<<nd, kSegThreads, 0, ctx->s_main>>>(seg_start, seg_pfirst, piece_limbs, piece_R, nd, ss);
        ++ctx->launch_count;
      }
      if (per_window) {
        k_segment_window_sums<<<nd * nw, kSegThreads, 0, ctx->s_main>>>(d_e, sb.s, z, badR, badS, seg_start,
                                                                        seg_order, nd, ms.pl, Ewd, Swd);
        ++ctx->launch_count;
      }
      timer_end(ctx, "segment_sums", ctx->s_main, tb, te);
    }
    if (per_window) {
      CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_table, 0));
      k_table_msm_windows<<<dim3(tmbw, nw), kPointThreads, 0, ctx->s_main>>>(d_tabs, Ewd, nullptr, nd, tmpw);
      k_window_point_sums<<<nw, kPointThreads, 0, ctx->s_main>>>(tmpw, tmbw, P2w);
      CU(cudaMemsetAsync(d_acc, 1, 1, ctx->s_main));
      k_multi_window_check<<<nw, kFinalThreads, 0, ctx->s_main>>>(Wall, nullptr, P2w, Swd, nullptr, nd,
                                                                 ctx->tableG, d_acc);
      ctx->launch_count += 3;
      CU(cudaGetLastError());
      return POSLO_OK;
    }
    // sum_d E_d Y_d from the key tables
    CU(cudaStreamWaitEvent(ctx->s_main, ctx->ev_table, 0));
    k_table_msm<<<tmb, kPointThreads, 0, ctx->s_main>>>(d_tabs, ss.Ew, nullptr, nd, tmpart);
    k_sum_encode<<<1, kFinalThreads, 0, ctx->s_main>>>(tmpart, tmb, P2, nullptr, nullptr);
    ctx->launch_count += 2;
    k_multi_check<<<1, kFinalThreads, 0, ctx->s_main>>>(P1, nullptr, P2, ss.Sw, nullptr, nd, ctx->tableG, d_acc);
    ++ctx->launch_count;
    CU(cudaGetLastError());
    return POSLO_OK;
  };
  if ((rc = run_replayable(ctx, ctx->g_multi, sig, stage1))) return rc;
  uint8_t all_ok = 0;
  std::vector<uint32_t> bad(nd);
  std::vector<uint8_t> hbadY(nd);
  CU(cudaMemcpyAsync(&all_ok, d_acc, 1, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaMemcpyAsync(bad.data(), ss.bad, 4 * (size_t)nd, cudaMemcpyDeviceToHost, ctx->s_main));
  CU(cudaMemcpyAsync(hbadY.data(), badY, nd, cudaMemcpyDeviceToHost, ctx->s_main));
  std::vector<uint8_t> hmbad(nbuild);
  if (nbuild) CU(cudaMemcpyAsync(hmbad.data(), d_mbad, nbuild, cudaMemcpyDeviceToHost, ctx->s_main));
  if ((rc = check_status(ctx))) return rc;
  for (uint32_t k = 0; k < nbuild; ++k)
    if (hmbad[k]) hbadY[kmiss[k]] = 1;
  for (uint32_t d = 0; d < nd; ++d)
    if (hbadY[d]) return fail(ctx, POSLO_EINVAL, "public key of device %u does not decode", d);
  forget.armed = false;   // the built tables are sound
  uint64_t total_bad = 0;
  for (uint32_t d = 0; d < nd; ++d) total_bad += bad[d];
  std::vector<uint8_t> flag(nd, 0);
  if (!(all_ok && total_bad == 0)) {
    // ---- localisation across devices: unit check per device, then confirm the rest together
    k_device_unit_check<<<(unsigned)((4ull * nd + 127) / 128), 128, 0, ctx->s_main>>>(d_tabs, ss, nd, ctx->tableG,
                                                                                     dev_flag);
    // the weighted sum over the devices not flagged = P1 minus the flagged devices' part,
    // an MSM over their entries only
    k_device_to_entries<<<nd, 256, 0, ctx->s_main>>>(dev_flag, seg_start, badR, eskip, 1);
    ctx->launch_count += 2;
    if (per_window) {
      // the same plan, so the flagged part's windows line up with the whole batch's
      MsmState ms2;
      uint32_t* groups2;
      if ((rc = run_msm_sort(ctx, ctx->s_main, z, 4, eskip, N, ms2))) return rc;
      if ((rc = run_msm_finish(ctx, ctx->s_main, pts, eskip, ms2, nullptr, &groups2))) return rc;
      k_msm_windows<<<1, 32, 0, ctx->s_main>>>(groups2, ms2.pl, Wsub);
      k_table_msm_windows<<<dim3(tmbw, nw), kPointThreads, 0, ctx->s_main>>>(d_tabs, Ewd, dev_flag, nd, tmpw);
      k_window_point_sums<<<nw, kPointThreads, 0, ctx->s_main>>>(tmpw, tmbw, P2w);
      CU(cudaMemsetAsync(d_acc, 1, 1, ctx->s_main));
      k_multi_window_check<<<nw, kFinalThreads, 0, ctx->s_main>>>(Wall, Wsub, P2w, Swd, dev_flag, nd, ctx->tableG,
                                                                 d_acc);
      ctx->launch_count += 4;
    } else {
      if ((rc = run_msm(ctx, ctx->s_main, pts, z, 4, eskip, N, P3))) return rc;
      k_table_msm<<<tmb, kPointThreads, 0, ctx->s_main>>>(d_tabs, ss.Ew, dev_flag, nd, tmpart);
      k_sum_encode<<<1, kFinalThreads, 0, ctx->s_main>>>(tmpart, tmb, P2, nullptr, nullptr);
      ctx->launch_count += 2;
      k_multi_check<<<1, kFinalThreads, 0, ctx->s_main>>>(P1, P3, P2, ss.Sw, dev_flag, nd, ctx->tableG, d_acc);
      ++ctx->launch_count;
    }
    uint8_t confirmed = 0;
    CU(cudaMemcpyAsync(&confirmed, d_acc, 1, cudaMemcpyDeviceToHost, ctx->s_main));
    CU(cudaMemcpyAsync(flag.data(), dev_flag, nd, cudaMemcpyDeviceToHost, ctx->s_main));
    if ((rc = check_status(ctx))) return rc;
    if (!confirmed) std::fill(flag.begin(), flag.end(), 1);   // cancelling errors: settle every device
  }
  if (settled) (*settled)(flag.data());
  // ---- localise inside the flagged devices: the single-entry check of every entry of every
  // flagged device in one launch, with the key tables built above
  std::vector<uint32_t> fl;
  std::vector<uint64_t> fst(1, 0);
  for (uint32_t d = 0; d < nd; ++d) {
    accept[d] = 1;
    if (flag[d]) {
      fl.push_back(d);
      fst.push_back(fst.back() + (mb->dev_start[d + 1] - mb->dev_start[d]));
    }
  }
  const uint32_t nfl = (uint32_t)fl.size();
  uint64_t cnt = 0;
  if (nfl) {
    uint32_t* d_fl;
    uint64_t *d_fst, *d_idx;
    uint8_t *inv, *d_any;
    const uint64_t capn = std::max<uint64_t>(std::min(cap, N), 1);
    if ((rc = ensure_t(ctx, "m_fl", 4 * (size_t)nfl, &d_fl))) return rc;
    if ((rc = ensure_t(ctx, "m_fst", 8 * (size_t)(nfl + 1), &d_fst))) return rc;
    if ((rc = ensure_t(ctx, "m_inv", N1, &inv))) return rc;
    if ((rc = ensure_t(ctx, "m_any", nfl, &d_any))) return rc;
    if ((rc = ensure_t(ctx, "m_idx", 8 * capn + 8, &d_idx))) return rc;
    uint64_t* d_cnt = d_idx + capn;
    CU(cudaMemcpyAsync(d_fl, fl.data(), 4 * (size_t)nfl, cudaMemcpyHostToDevice, ctx->s_main));
    CU(cudaMemcpyAsync(d_fst, fst.data(), 8 * (size_t)(nfl + 1), cudaMemcpyHostToDevice, ctx->s_main));
    CU(cudaMemsetAsync(inv, 0, N1, ctx->s_main));
    cudaEvent_t tb, te;
    timer_begin(ctx, "localise", ctx->s_main, &tb, &te);
    MultiCheckArgs ca{};
    ca.pts = pts;
    ca.e = d_e;
    ca.s = sb.s;
    ca.badR = badR;
    ca.badS = badS;
    ca.seg_start = seg_start;
    ca.fl = d_fl;
    ca.fstart = d_fst;
    ca.nfl = nfl;
    ca.tabs = d_tabs;
    ca.tableG = ctx->tableG;
    ca.inv = inv;
    if (fst[nfl] && fst[nfl] <= kMultiGroupCheckMax)
      k_multi_entry_check_group<<<(unsigned)((8 * fst[nfl] + 127) / 128), 128, 0, ctx->s_main>>>(ca);
    else if (fst[nfl])
      k_multi_entry_check<<<grid_for(ctx, fst[nfl], 128, 8), 128, 0, ctx->s_main>>>(ca);
    k_segment_any<<<nfl, 256, 0, ctx->s_main>>>(inv, seg_start, d_fl, d_any);
    ctx->launch_count += 2;
    CU(cudaGetLastError());
    if ((rc = run_compact(ctx, inv, N, 0, d_idx, std::min(cap, N), d_cnt))) return rc;
    timer_end(ctx, "localise", ctx->s_main, tb, te);
    std::vector<uint8_t> any(nfl);
    CU(cudaMemcpyAsync(&cnt, d_cnt, 8, cudaMemcpyDeviceToHost, ctx->s_main));
    CU(cudaMemcpyAsync(any.data(), d_any, nfl, cudaMemcpyDeviceToHost, ctx->s_main));
    if ((rc = check_status(ctx))) return rc;
    for (uint32_t k = 0; k < nfl; ++k)
      if (any[k]) accept[fl[k]] = 0;
    const uint64_t got = std::min(cnt, cap);
    if (got && invalid_pairs) {
      std::vector<uint64_t> g(got);
      CU(cudaMemcpy(g.data(), d_idx, 8 * got, cudaMemcpyDeviceToHost));
      // global positions ascend, and so do devices: walk the device table once
      uint32_t d = 0;
      for (uint64_t q = 0; q < got; ++q) {
        while (mb->dev_start[d + 1] <= g[q]) ++d;
        invalid_pairs[2 * q] = d;
        invalid_pairs[2 * q + 1] = mb->first_index[d] + (g[q] - mb->dev_start[d]);
      }
    }
  }
  *n_invalid = cnt;
  if (cnt > cap) return fail(ctx, POSLO_EBUFSMALL, "%llu invalid entries, room for %llu", (unsigned long long)cnt,
                             (unsigned long long)cap);
  return POSLO_OK;
}

extern "C" {

}  // extern "C"
