// Serving: continuous batching of verification requests from many IoT devices over keys
// registered once and kept by the service.  Not in the paper (it verifies one signer's log
// at a time); built on the multi-device path.
//
// Requests are copied at submission (or lent in page-locked memory) and admitted against a
// device-memory budget (EBUSY when it would be exceeded).  W worker threads, each with its
// own internal context (streams and workspace), take the oldest pending requests up to a
// batch size and verify them as one multi-device batch.  While no worker is idle, a worker
// also takes its next batch before verifying the current one and stages it into its second
// set of device buffers on its copy stream, so the copies of one batch overlap the
// verification of the previous one on the same worker.  A request that arrives while the
// workers are busy joins the next batch.  Each request's result (accept bit and invalid
// indices) is by definition independent of the batch it was verified in.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <future>
#include <memory>
#include <mutex>
#include <system_error>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/poslo.h"
#include "ctx.h"

namespace poslo_host {

struct Req {
  uint64_t ticket = 0;
  uint32_t key_id = 0, n2 = 1;
  uint64_t first_index = 0, n = 0;
  std::vector<uint8_t> msgs, s, R, ds;
  std::vector<uint64_t> offs;   // n+1, rebased to start at 0
  ReqView view{};               // where the inputs are: the vectors above, or the caller's (borrowed)
  uint64_t charge = 0;          // bytes of the budget held until the result is read
  int state = 0;                // 0 pending, 1 running, 2 done
  int rc = POSLO_OK;
  uint8_t accept = 0;
  std::vector<uint64_t> invalid;
  std::chrono::steady_clock::time_point t_submit, t_done;
};

// One served batch on the service's clock (ns since poslo_serve_start).
struct BatchRecord {
  uint32_t worker = 0, requests = 0;
  uint64_t entries = 0;
  uint64_t t_take = 0, t_staged = 0, t_verify = 0, t_checked = 0, t_done = 0;
};

struct Server {
  poslo_ctx* owner = nullptr;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  std::vector<BatchRecord> timeline;   // drained by poslo_serve_timeline (bounded)
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  std::vector<std::array<uint8_t, 32>> keys;
  // Resident window tables of the registered keys, kKeysPerBlock keys per device allocation;
  // blocks never move, so workers read them while new keys are added.
  static constexpr uint32_t kKeysPerBlock = 256;
  std::vector<uint32_t*> table_blocks;
  std::mutex reg_mu;   // serialises key registration (it uses the owner context's stream)
  std::vector<std::thread> workers;
  std::vector<poslo_ctx*> wctx;
  bool stop = false;
  uint64_t next_ticket = 1;
  uint64_t budget = 0, used = 0;
  uint32_t max_dev = 4096;
  uint64_t max_entries = 1ull << 22;
  uint64_t batches = 0, batched_requests = 0;
  uint32_t idle = 0;   // workers waiting for requests with no batch in hand
  uint64_t pending_entries = 0;   // entries of the pending requests
};

namespace {

// Device bytes a request occupies while it is verified: its inputs and the per-entry
// workspace of the multi-device path (decoded points, e, z, flags, MSM sort and segments).
uint64_t request_charge(uint64_t n, uint64_t msg_bytes) { return msg_bytes + n * 640 + 4096; }

// The device address of page-locked host memory mapped into the device's address space, or
// null (pageable or unknown memory, which is staged by copies instead).
const void* mapped_address(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

uint64_t since(const Server* S) {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - S->t0)
      .count();
}

constexpr size_t kMaxTimeline = 1u << 20;   // records kept between two reads
constexpr uint64_t kMinShare = 1u << 16;     // entries: below this a batch is not split further

// A batch taken by a worker: its requests, the multi-device description of them and the
// staging set its inputs are copied into.
struct TakenBatch {
  std::vector<Req*> batch;
  BatchRecord rec;
  int set = 0, rc = POSLO_OK;
  uint64_t total = 0;
  std::vector<uint8_t> Y, ds;
  std::vector<uint64_t> start, first;
  std::vector<uint32_t> n2, ds_off;
  std::vector<const uint32_t*> tabs;
  std::vector<ReqView> views;
  poslo_multi_batch mb{};
};

// Describes the batch and issues the copies of its inputs into staging set `set` (nothing
// waits for them here).
std::unique_ptr<TakenBatch> issue_staging(Server* S, poslo_ctx* w, uint32_t worker, std::vector<Req*>&& batch,
                                          int set) {
  cudaSetDevice(w->device);   // also on a staging thread
  auto B = std::make_unique<TakenBatch>();
  B->batch = std::move(batch);
  B->set = set;
  B->rec.worker = worker;
  B->rec.t_take = since(S);
  const uint32_t nd = (uint32_t)B->batch.size();
  B->Y.resize(32 * (size_t)nd);
  B->start.assign(nd + 1, 0);
  B->first.resize(nd);
  B->n2.resize(nd);
  B->ds_off.assign(nd + 1, 0);
  B->tabs.resize(nd);
  B->views.resize(nd);
  {
    std::lock_guard<std::mutex> lock(S->mu);
    const size_t words = key_table_words();
    for (uint32_t d = 0; d < nd; ++d) {
      const uint32_t k = B->batch[d]->key_id;
      memcpy(B->Y.data() + 32 * (size_t)d, S->keys[k].data(), 32);
      B->tabs[d] = S->table_blocks[k / Server::kKeysPerBlock] + (size_t)(k % Server::kKeysPerBlock) * words;
    }
  }
  for (uint32_t d = 0; d < nd; ++d) {
    Req* r = B->batch[d];
    B->views[d] = r->view;
    B->total += r->n;
    B->start[d + 1] = B->start[d] + r->n;
    B->first[d] = r->first_index;
    B->n2[d] = r->n2;
    B->ds.insert(B->ds.end(), r->ds.begin(), r->ds.end());
    B->ds_off[d + 1] = B->ds_off[d] + (uint32_t)(r->ds.size() / 24);
  }
  poslo_multi_batch& mb = B->mb;
  mb.n_dev = nd;
  mb.Y = B->Y.data();
  mb.dev_start = B->start.data();
  mb.first_index = B->first.data();
  mb.n2 = B->n2.data();
  mb.ds = B->ds.data();
  mb.ds_off = B->ds_off.data();
  // each request's inputs go straight from its own buffers into the worker's device staging
  B->rc = stage_requests(w, B->views.data(), nd, &mb, set);
  B->rec.t_staged = since(S);
  B->rec.requests = nd;
  B->rec.entries = B->total;
  return B;
}

// Waits for the batch's inputs, verifies it and publishes every request's result.
void run_batch(Server* S, poslo_ctx* w, TakenBatch& B) {
  std::vector<Req*>& batch = B.batch;
  BatchRecord& rec = B.rec;
  const uint32_t nd = (uint32_t)batch.size();
  const uint64_t total = B.total;
  poslo_multi_batch& mb = B.mb;
  // what was issued lands before anything else, even when issuing failed part way
  int rc = stage_wait(w, B.set, B.rc);
  rec.t_verify = since(S);
  std::vector<uint8_t> acc(nd);
  std::vector<uint64_t> pairs(2 * std::max<uint64_t>(total, 1));
  uint64_t cnt = 0;
  // requests whose device passes the device-level checks are final before the entry-level
  // localisation of the others: publish them at once (a reader may then release them, so
  // they are not touched again here)
  std::vector<uint8_t> published(nd, 0);
  const std::function<void(const uint8_t*)> settled = [&](const uint8_t* flagged) {
    {
      std::lock_guard<std::mutex> lock(S->mu);
      const auto now = std::chrono::steady_clock::now();
      for (uint32_t d = 0; d < nd; ++d) {
        if (flagged[d]) continue;
        Req* r = batch[d];
        r->rc = POSLO_OK;
        r->accept = 1;
        r->invalid.clear();
        r->state = 2;
        r->t_done = now;
        std::vector<uint8_t>().swap(r->msgs);
        std::vector<uint8_t>().swap(r->s);
        std::vector<uint8_t>().swap(r->R);
        std::vector<uint64_t>().swap(r->offs);
        r->view = ReqView{};
        published[d] = 1;
      }
    }
    S->cv_done.notify_all();
  };
  if (rc == POSLO_OK) rc = aver_multi(w, &mb, B.tabs.data(), acc.data(), pairs.data(), total, &cnt, &settled);
  rec.t_checked = since(S);
  std::vector<int> rcs(nd, rc);
  std::vector<std::vector<uint64_t>> inv(nd);
  if (rc == POSLO_OK) {
    for (uint64_t k = 0; k < cnt; ++k) inv[pairs[2 * k]].push_back(pairs[2 * k + 1]);
  } else if (nd > 1) {
    // one malformed request must not fail the others: verify each on its own
    for (uint32_t d = 0; d < nd; ++d) {
      if (published[d]) continue;
      poslo_batch b{};
      Req* r = batch[d];
      b.variant = POSLO_VARIANT_F;
      b.n2 = r->n2;
      static const uint8_t kNone[32] = {0};
      b.Y = B.Y.data() + 32 * (size_t)d;
      b.msgs = r->view.msgs ? r->view.msgs : kNone;
      b.offs = r->view.offs;
      b.n = r->n;
      b.first_index = r->first_index;
      b.s = r->view.s ? r->view.s : kNone;
      b.R = r->view.R ? r->view.R : kNone;
      b.R_count = r->n;
      b.ds = r->ds.data();
      b.ds_nodes = (uint32_t)(r->ds.size() / 24);
      std::vector<uint64_t> idx(std::max<uint64_t>(r->n, 1));
      uint64_t k = 0;
      rcs[d] = poslo_distill(w, &b, idx.data(), r->n, &k, nullptr, nullptr);
      acc[d] = (rcs[d] == POSLO_OK && k == 0) ? 1 : 0;
      inv[d].assign(idx.begin(), idx.begin() + (rcs[d] == POSLO_OK ? k : 0));
    }
  }
  std::lock_guard<std::mutex> lock(S->mu);
  for (uint32_t d = 0; d < nd; ++d) {
    if (published[d]) continue;
    Req* r = batch[d];
    r->rc = rcs[d];
    r->accept = rcs[d] == POSLO_OK ? acc[d] : 0;
    r->invalid = std::move(inv[d]);
    r->state = 2;
    r->t_done = std::chrono::steady_clock::now();
    // the inputs are no longer needed; the budget is released when the result is read
    std::vector<uint8_t>().swap(r->msgs);
    std::vector<uint8_t>().swap(r->s);
    std::vector<uint8_t>().swap(r->R);
    std::vector<uint64_t>().swap(r->offs);
    r->view = ReqView{};
  }
  S->batches += 1;
  S->batched_requests += nd;
  rec.t_done = since(S);
  if (S->timeline.size() < kMaxTimeline) S->timeline.push_back(rec);
}

void worker_loop(Server* S, poslo_ctx* w, uint32_t worker) {
  cudaSetDevice(w->device);
  std::unique_ptr<TakenBatch> cur;   // staged, not yet verified
  int set = 0;
  for (;;) {
    std::vector<Req*> batch;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      if (!cur) {
        ++S->idle;
        S->cv_work.wait(lock, [&] { return S->stop || !S->pending.empty(); });
        --S->idle;
        if (S->stop && S->pending.empty()) return;
      }
      // with a batch in hand, take the next one only while no worker is idle: an idle worker
      // verifies it at once, this one only after its current batch
      if (!cur || S->idle == 0) {
        // when fewer entries wait than the workers' next batches hold, an even share each, so
        // that the last batches of a burst end together rather than one after another
        const uint64_t W = S->wctx.size();
        uint64_t cap = S->max_entries;
        if (S->pending_entries < W * cap) cap = std::max<uint64_t>((S->pending_entries + W - 1) / W, kMinShare);
        uint64_t ent = 0;
        while (!S->pending.empty() && batch.size() < S->max_dev) {
          Req* r = S->pending.front();
          if (!batch.empty() && ent + r->n > cap) break;
          S->pending.pop_front();
          S->pending_entries -= r->n;
          r->state = 1;
          batch.push_back(r);
          ent += r->n;
        }
      }
    }
    // the next batch's copies are issued on a staging thread (the calls take milliseconds for
    // hundreds of requests) and run while the current batch is verified on this one
    std::unique_ptr<TakenBatch> next;
    if (!batch.empty()) {
      if (cur) {
        std::future<std::unique_ptr<TakenBatch>> issue;
        try {
          // a copy of the list: a launch that fails may already have taken its arguments
          issue = std::async(std::launch::async, issue_staging, S, w, worker, std::vector<Req*>(batch), set);
        } catch (const std::system_error&) {   // no thread to be had: issue it here
          issue = std::async(std::launch::deferred, issue_staging, S, w, worker, std::move(batch), set);
        }
        run_batch(S, w, *cur);
        S->cv_done.notify_all();
        cur.reset();
        next = issue.get();
      } else {
        next = issue_staging(S, w, worker, std::move(batch), set);
      }
      set ^= 1;
    }
    if (cur) {
      run_batch(S, w, *cur);
      S->cv_done.notify_all();
    }
    cur = std::move(next);
  }
}

}  // namespace
}  // namespace poslo_host

using poslo_host::Req;
using poslo_host::Server;

void poslo_server_release(poslo_ctx* ctx) {
  if (!ctx || !ctx->server) return;
  Server* S = ctx->server;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (poslo_ctx* w : S->wctx) poslo_destroy(w);
  cudaSetDevice(ctx->device);
  for (uint32_t* b : S->table_blocks) cudaFree(b);
  delete S;
  ctx->server = nullptr;
}

extern "C" {

int poslo_serve_start(poslo_ctx* ctx, uint32_t workers, uint32_t max_batch_devices, uint64_t max_batch_entries) {
  if (!ctx || workers == 0 || workers > 8 || max_batch_devices == 0 || max_batch_entries == 0) return POSLO_EINVAL;
  if (ctx->server) return POSLO_EBUSY;
  Server* S = new Server();
  S->owner = ctx;
  S->budget = ctx->mem_budget;
  S->max_dev = max_batch_devices;
  S->max_entries = max_batch_entries;
  for (uint32_t k = 0; k < workers; ++k) {
    poslo_params p{};
    p.device = ctx->device;
    p.msm_window = ctx->msm_window;
    p.instantiation = ctx->inst;
    p.mem_budget = 0;
    memcpy(p.verifier_seed, ctx->vseed, 32);
    p.verifier_seed[31] ^= (uint8_t)(k + 1);   // independent weights per worker
    poslo_ctx* w = nullptr;
    const int rc = poslo_create(&p, &w);
    if (rc != POSLO_OK) {
      for (poslo_ctx* c : S->wctx) poslo_destroy(c);
      delete S;
      return rc;
    }
    // served batches rarely repeat a shape: no graph captures on the workers' contexts (which
    // also keeps every capture away from the staging threads' allocations)
    w->graphs = false;
    S->wctx.push_back(w);
  }
  for (uint32_t k = 0; k < (uint32_t)S->wctx.size(); ++k)
    S->workers.emplace_back(poslo_host::worker_loop, S, S->wctx[k], k);
  ctx->server = S;
  return POSLO_OK;
}

int poslo_serve_stop(poslo_ctx* ctx) {
  if (!ctx || !ctx->server) return POSLO_EINVAL;
  poslo_server_release(ctx);
  return POSLO_OK;
}

int poslo_register_key(poslo_ctx* ctx, const uint8_t Y[32], uint32_t* key_id) {
  if (!ctx || !ctx->server || !Y || !key_id) return POSLO_EINVAL;
  Server* S = ctx->server;
  std::lock_guard<std::mutex> reg(S->reg_mu);
  uint32_t id;
  uint32_t* block = nullptr;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    id = (uint32_t)S->keys.size();
    if (id / Server::kKeysPerBlock < S->table_blocks.size()) block = S->table_blocks[id / Server::kKeysPerBlock];
  }
  const size_t words = poslo_host::key_table_words();
  if (!block) {
    cudaSetDevice(ctx->device);
    if (cudaMalloc(&block, 4 * words * Server::kKeysPerBlock) != cudaSuccess) return POSLO_ENOMEM;
    std::lock_guard<std::mutex> lock(S->mu);
    S->table_blocks.push_back(block);
  }
  // decode Y once and keep its window table resident (EINVAL if Y does not decode)
  const int rc = poslo_host::build_key_table(ctx, Y, block + (size_t)(id % Server::kKeysPerBlock) * words);
  if (rc != POSLO_OK) return rc;
  std::array<uint8_t, 32> k;
  memcpy(k.data(), Y, 32);
  std::lock_guard<std::mutex> lock(S->mu);
  S->keys.push_back(k);
  *key_id = id;
  return POSLO_OK;
}

int poslo_submit(poslo_ctx* ctx, const poslo_request* q, uint64_t* ticket) {
  if (!ctx || !ctx->server || !q || !ticket) return POSLO_EINVAL;
  const auto t_submit = std::chrono::steady_clock::now();
  Server* S = ctx->server;
  if (q->n2 == 0 || !q->ds || q->ds_nodes == 0 || (q->n && (!q->offs || !q->s || !q->R || !q->msgs)))
    return POSLO_EINVAL;
  for (uint64_t t = 0; t < q->n; ++t)
    if (q->offs[t + 1] < q->offs[t]) return POSLO_EINVAL;
  auto r = std::make_unique<Req>();
  r->t_submit = t_submit;
  r->key_id = q->key_id;
  r->n2 = q->n2;
  r->first_index = q->first_index;
  r->n = q->n;
  const uint64_t lo = q->n ? q->offs[0] : 0, hi = q->n ? q->offs[q->n] : 0;
  r->charge = poslo_host::request_charge(q->n, hi - lo);
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (q->key_id >= S->keys.size()) return POSLO_ENOTFOUND;
    if (S->budget && S->used + r->charge > S->budget) return POSLO_EBUSY;
    S->used += r->charge;   // reserve before copying
  }
  if (q->flags & POSLO_REQ_BORROW) {
    // the caller keeps the inputs until the result is read; the offsets stay absolute
    r->view = poslo_host::ReqView{q->msgs, q->offs, q->n, q->s, q->R};
    if (q->n == 0) {
      r->offs.assign(1, 0);
      r->view.offs = r->offs.data();
    } else {
      // page-locked buffers the device can read are staged by a gather kernel
      const void *dm = poslo_host::mapped_address(q->msgs + lo), *d_o = poslo_host::mapped_address(q->offs),
                 *d_s = poslo_host::mapped_address(q->s), *d_R = poslo_host::mapped_address(q->R);
      if (dm && d_o && d_s && d_R) {
        r->view.d_msgs = static_cast<const uint8_t*>(dm) - lo;
        r->view.d_offs = static_cast<const uint64_t*>(d_o);
        r->view.d_s = static_cast<const uint8_t*>(d_s);
        r->view.d_R = static_cast<const uint8_t*>(d_R);
      }
    }
  } else {
    r->msgs.assign(q->msgs ? q->msgs + lo : nullptr, q->msgs ? q->msgs + hi : nullptr);
    r->offs.resize(q->n + 1);
    for (uint64_t t = 0; t <= q->n; ++t) r->offs[t] = q->n ? q->offs[t] - lo : 0;
    r->s.assign(q->s, q->s + 32 * q->n);
    r->R.assign(q->R, q->R + 32 * q->n);
    r->view = poslo_host::ReqView{r->msgs.data(), r->offs.data(), q->n, r->s.data(), r->R.data()};
  }
  r->ds.assign(q->ds, q->ds + 24 * (size_t)q->ds_nodes);
  {
    std::lock_guard<std::mutex> lock(S->mu);
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    S->pending.push_back(r.get());
    S->pending_entries += r->n;
    S->reqs.emplace(r->ticket, std::move(r));
  }
  S->cv_work.notify_one();
  return POSLO_OK;
}

int poslo_poll(poslo_ctx* ctx, uint64_t ticket, uint32_t wait_ms, uint8_t* accept, uint64_t* invalid_idx,
               uint64_t cap, uint64_t* n_invalid, uint64_t* latency_ns) {
  if (!ctx || !ctx->server || !accept || !n_invalid) return POSLO_EINVAL;
  Server* S = ctx->server;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return POSLO_ENOTFOUND;
  Req* r = it->second.get();
  if (r->state != 2 && wait_ms)
    S->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return r->state == 2; });
  if (r->state != 2) return POSLO_PENDING;
  *accept = r->accept;
  *n_invalid = r->invalid.size();
  if (latency_ns)
    *latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(r->t_done - r->t_submit).count();
  if (invalid_idx)
    for (uint64_t k = 0; k < std::min<uint64_t>(cap, r->invalid.size()); ++k) invalid_idx[k] = r->invalid[k];
  const int rc = r->rc != POSLO_OK ? r->rc : (r->invalid.size() > cap ? POSLO_EBUFSMALL : POSLO_OK);
  if (rc != POSLO_EBUFSMALL) {
    S->used -= r->charge;
    S->reqs.erase(it);
  }
  return rc;
}

int poslo_serve_stats(poslo_ctx* ctx, uint64_t* batches, uint64_t* requests, uint64_t* bytes_in_use) {
  if (!ctx || !ctx->server) return POSLO_EINVAL;
  Server* S = ctx->server;
  std::lock_guard<std::mutex> lock(S->mu);
  if (batches) *batches = S->batches;
  if (requests) *requests = S->batched_requests;
  if (bytes_in_use) *bytes_in_use = S->used;
  return POSLO_OK;
}

int poslo_serve_timeline(poslo_ctx* ctx, poslo_batch_record* out, uint64_t cap, uint64_t* n) {
  if (!ctx || !ctx->server || !n || (cap && !out)) return POSLO_EINVAL;
  Server* S = ctx->server;
  std::lock_guard<std::mutex> lock(S->mu);
  const uint64_t k = std::min<uint64_t>(cap, S->timeline.size());
  for (uint64_t i = 0; i < k; ++i) {
    const poslo_host::BatchRecord& r = S->timeline[i];
    out[i].worker = r.worker;
    out[i].requests = r.requests;
    out[i].entries = r.entries;
    out[i].t_take_ns = r.t_take;
    out[i].t_staged_ns = r.t_staged;
    out[i].t_verify_ns = r.t_verify;
    out[i].t_checked_ns = r.t_checked;
    out[i].t_done_ns = r.t_done;
  }
  *n = k;
  S->timeline.erase(S->timeline.begin(), S->timeline.begin() + (ptrdiff_t)k);
  return POSLO_OK;
}

}  // extern "C"
