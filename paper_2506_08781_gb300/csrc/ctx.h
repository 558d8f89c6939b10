// Host-side state of a libposlo context (shared by the C-ABI translation units).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstddef>
#include <functional>
#include <array>
#include <list>
#include <map>
#include <string>
#include <vector>

#include "../../include/poslo.h"

namespace poslo_host {

constexpr size_t kSmallHostBytes = 4096;   // page-locked scratch of a context for small transfers

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

// One staging set of a serving worker: the device buffers its next batch is copied into and
// a page-locked area for the small tables that go up with it.  A staging thread fills a set
// while the worker's own thread verifies from the other, so a set keeps its buffers, its
// launch count and its error apart from the context's workspace map and fields.
struct StageSet {
  DevBuf msgs, raw, offs, s, R, meta, regions, status;
  uint8_t* h = nullptr;   // page-locked: status word (16 bytes), offsets table, gather regions
  size_t h_cap = 0;
  uint64_t launches = 0;
  std::string err;
};

struct KernelTimer {
  double total_ms = 0;
  uint64_t launches = 0;
};

struct Server;   // continuous-batching service (serve.cu)

// Window tables of recently used public keys, kept on the device so that a later call with
// the same key skips the 252-doubling table chain.  Slots live in blocks of kBlock keys that
// never move; least recently used keys are evicted.
struct KeyCache {
  static constexpr uint32_t kBlock = 256;
  uint32_t capacity = 4096;                          // keys (0: no cache)
  std::vector<uint32_t*> blocks;                     // kBlock tables each
  std::map<std::array<uint8_t, 32>, uint32_t> slot_of;
  std::vector<std::array<uint8_t, 32>> key_of;       // slot -> key
  std::list<uint32_t> lru;                           // slots in use, most recent first
  std::vector<std::list<uint32_t>::iterator> pos;    // slot -> its place in lru
  std::vector<uint32_t> free_slots;
  uint32_t nslots = 0;                               // slots handed out so far
  uint64_t hits = 0, misses = 0;
};

// A captured launch sequence (CUDA graph) and the shape of the call it was captured from.
// A call whose shape equals the previous call's is captured; later calls of that shape
// replay it, as long as no workspace buffer has been reallocated since (alloc_gen).
struct GraphSlot {
  std::vector<uint64_t> sig;        // shape of the captured call
  std::vector<uint64_t> last_sig;   // shape of the previous call
  uint64_t gen = 0;                 // ctx->alloc_gen at capture
  uint64_t launches = 0;            // kernels in the graph
  cudaGraphExec_t exec = nullptr;
};

}  // namespace poslo_host

struct poslo_ctx {
  int device = 0;
  int sm_count = 0;
  uint32_t msm_window = 0;
  uint32_t inst = 0;              // POSLO_INST_SHA256 or POSLO_INST_AES
  uint64_t mem_budget = 0;
  uint64_t mem_used = 0;
  uint8_t vseed[32] = {0};
  cudaStream_t s_main = nullptr, s_table = nullptr, s_points = nullptr;
  cudaStream_t s_copy = nullptr;                 // host-to-device copies of the next chunk
  cudaStream_t s_hash = nullptr;                 // message hashing of Distill
  cudaEvent_t ev_copy[2] = {nullptr, nullptr};   // chunk k's inputs have landed in set k % 2
  cudaEvent_t ev_table = nullptr, ev_points = nullptr, ev_main = nullptr, ev_hash = nullptr, ev_prep = nullptr;
  cudaEvent_t ev_decoded = nullptr;   // points stream, right after the decoding (before its sums)
  cudaEvent_t ev_staged = nullptr;   // main stream, right after a batch's R_t have been staged
  std::map<std::string, poslo_host::DevBuf> bufs;
  uint32_t* tableG = nullptr;     // fixed-window table of G (64 KiB)
  uint32_t* status = nullptr;     // device status word
  uint32_t* h_status = nullptr;   // pinned mirror
  uint8_t* h_small = nullptr;     // pinned, kSmallHostBytes: small results and shard records
  poslo_host::StageSet stage[2];  // serving staging sets (filled by a worker's staging thread)
  uint8_t* h_pack = nullptr;      // page-locked packing of small host batches
  size_t h_pack_cap = 0;
  std::string err;
  bool profiling = false;
  uint64_t launch_count = 0;      // kernels launched by this context
  std::map<std::string, poslo_host::KernelTimer> timers;
  std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> event_pool;
  std::map<int, int> msm_tuned;   // (log2 n) * 16 + scalar words -> best window c | range log2 << 8
  poslo_host::Server* server = nullptr;
  uint64_t multi_window_max = 0;  // multi-device batches up to this size check per window (off)
  bool graphs = true;             // replay repeated call shapes from CUDA graphs
  bool capturing = false;         // a stream capture is open on s_main
  uint64_t alloc_gen = 0;         // counts workspace (re)allocations
  uint64_t graph_captures = 0, graph_replays = 0;
  poslo_host::GraphSlot g_multi;  // poslo_aver_multi up to its combined check
  poslo_host::GraphSlot g_distill;   // poslo_distill up to its weighted check
  poslo_host::GraphSlot g_partial;   // poslo_aver_partial up to its record
  poslo_host::KeyCache keys;         // window tables of recently used keys
};

// Stops and frees the context's service, if one runs (serve.cu).
void poslo_server_release(poslo_ctx* ctx);

namespace poslo_host {
// poslo_aver_multi with the devices' window tables given (device pointers, one per device,
// host array); with key_tables = nullptr the tables are built from the keys (poslo.cu).
// When settled is given, it is called once the devices that need no entry-level localisation
// are known (flagged[d] = 0: device d is accepted, its result is final), before the
// localisation of the others runs; a service publishes those results early.
int aver_multi(poslo_ctx* ctx, const poslo_multi_batch* mb, const uint32_t* const* key_tables, uint8_t* accept,
               uint64_t* invalid_pairs, uint64_t cap, uint64_t* n_invalid,
               const std::function<void(const uint8_t* flagged)>* settled = nullptr);
// Decodes Y and writes its window table (kTableWords words) to table_dev; EINVAL if Y does
// not decode.  Synchronous.
int build_key_table(poslo_ctx* ctx, const uint8_t Y[32], uint32_t* table_dev);
// 32-bit words of one window table.
size_t key_table_words();
// One request's inputs in host memory: entry t's message is msgs[offs[t] .. offs[t+1]).
struct ReqView {
  const uint8_t* msgs;
  const uint64_t* offs;   // n+1, absolute into msgs
  uint64_t n;
  const uint8_t* s;
  const uint8_t* R;
  // When all four arrays are page-locked host memory mapped into the device's address space,
  // their device addresses (the staging then reads them with one gather kernel instead of a
  // copy per array); null otherwise.
  const uint8_t* d_msgs = nullptr;
  const uint64_t* d_offs = nullptr;
  const uint8_t* d_s = nullptr;
  const uint8_t* d_R = nullptr;
};
// Issues the copies of the requests' inputs into device staging set `set` (0 or 1) of ctx
// (the messages back to back, offsets rebased on the device) and points mb's msgs, offs, s, R
// at them (mb->on_device = 1).  Nothing waits: the copies and the gather run on ctx's copy
// stream and end with ctx->ev_copy[set], so a worker stages its next batch while the current
// one is verified on the main stream.  It touches only ctx->stage[set], s_copy and
// ev_copy[set], so it may run on another thread than the one using the rest of ctx.  The
// requests' host memory must stay valid, and the set unused, until stage_wait(ctx, set, rc)
// has returned.
int stage_requests(poslo_ctx* ctx, const ReqView* reqs, uint32_t nd, poslo_multi_batch* mb, int set);
// On the context's own thread: waits for staging set `set` to land and returns the staging's
// status (issue_rc from stage_requests, else EINVAL if a request's offsets fell below its
// first), with its message in the context's error.
int stage_wait(poslo_ctx* ctx, int set, int issue_rc);
}  // namespace poslo_host
