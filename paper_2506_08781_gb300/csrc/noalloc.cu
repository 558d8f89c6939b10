// poslo_hash_entries_noalloc: the per-entry hashing of poslo_hash_entries for callers that
// cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: a host process whose device memory
// is owned by another allocator that has reserved it all (a framework's caching allocator
// or a fixed pool sized at start-up), or a service that forbids any allocation after its
// initialisation so that its memory footprint stays fixed.  They can still pass device
// buffers for their inputs and outputs.  This entry point needs no context (creating one
// allocates) and keeps all of its scratch memory in one file-scope device array.
//
// Scratch layout inside g_scratch (fixed maximum sizes):
//   status word                    256 bytes (one 32-bit word used)
//   disclosed-seed nodes           kMaxDsNodes * 24 bytes
//   epoch seeds x_0[i]             kMaxEpochs * 16 bytes
//   per-block hash partials        kMaxBlocks * kPartialWords * 8 bytes
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/poslo.h"
#include "common.cuh"

using namespace poslo;

namespace {

constexpr uint32_t kMaxDsNodes = 64;
constexpr uint64_t kMaxEpochs = 1ull << 16;
constexpr int kMaxBlocks = 2048;

constexpr size_t kOffStatus = 0;
constexpr size_t kOffDs = 256;
constexpr size_t kOffSeeds = kOffDs + ((kMaxDsNodes * sizeof(DsNode) + 255) / 256) * 256;
constexpr size_t kOffPartial = kOffSeeds + kMaxEpochs * 16;
constexpr size_t kScratchBytes = kOffPartial + (size_t)kMaxBlocks * kPartialWords * 8;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) uint8_t g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint8_t* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (set up once per device).
int scratch_address(int device, uint8_t** out) {
  if (device < 0 || device >= kMaxDevices) return POSLO_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return POSLO_EDEVICE;
    g_scratch_ptr[device] = static_cast<uint8_t*>(p);
  }
  *out = g_scratch_ptr[device];
  return POSLO_OK;
}

uint32_t be32(const uint8_t* b) {
  return ((uint32_t)b[0] << 24) | ((uint32_t)b[1] << 16) | ((uint32_t)b[2] << 8) | b[3];
}

}  // namespace

extern "C" int poslo_hash_entries_noalloc(const poslo_batch* batch, uint8_t* e_out, void* stream) {
  if (!batch || !e_out) return POSLO_EINVAL;
  const poslo_batch& b = *batch;
  if (!b.on_device) return POSLO_EINVAL;                  // device buffers only: no staging copies
  if (b.variant != POSLO_VARIANT_C && b.variant != POSLO_VARIANT_F) return POSLO_EINVAL;
  if (b.n2 == 0 || (b.n && (!b.msgs || !b.offs))) return POSLO_EINVAL;
  // a POSLO-C batch is whole epochs, as poslo_hash_entries requires (Y, s and R are not read)
  if (b.variant == POSLO_VARIANT_C && (b.n % b.n2 || b.first_index % b.n2)) return POSLO_EINVAL;
  // offsets are read as 8-byte words, e_t written as 16-byte vectors
  if ((reinterpret_cast<uintptr_t>(b.offs) & 7) || (reinterpret_cast<uintptr_t>(e_out) & 15)) return POSLO_EINVAL;
  if (!b.ds || b.ds_nodes == 0 || b.ds_nodes > kMaxDsNodes) return POSLO_EINVAL;
  uint64_t e0 = 0, ne = 0;
  if (b.n) {
    e0 = b.first_index / b.n2;
    ne = (b.first_index + b.n - 1) / b.n2 - e0 + 1;
  }
  if (ne > kMaxEpochs) return POSLO_EINVAL;                // the batch spans too many epochs
  if (b.n == 0) return POSLO_OK;                           // nothing to hash, no device work
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return POSLO_EDEVICE;
  uint8_t* scratch;
  int rc = scratch_address(device, &scratch);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* status = reinterpret_cast<uint32_t*>(scratch + kOffStatus);
  DsNode* d_ds = reinterpret_cast<DsNode*>(scratch + kOffDs);
  uint32_t* seeds = reinterpret_cast<uint32_t*>(scratch + kOffSeeds);
  unsigned long long* partial = reinterpret_cast<unsigned long long*>(scratch + kOffPartial);

  DsNode h[kMaxDsNodes];
  for (uint32_t k = 0; k < b.ds_nodes; ++k) {
    const uint8_t* p = b.ds + 24 * (size_t)k;
    memcpy(&h[k].d, p, 4);
    memcpy(&h[k].i, p + 4, 4);
    if (h[k].d > 40) return POSLO_EINVAL;
    for (int w = 0; w < 4; ++w) h[k].seed[w] = be32(p + 8 + 4 * w);
  }
  // the array keeps the previous call's contents: clear the status word first
  if (cudaMemsetAsync(status, 0, 4, st) != cudaSuccess) return POSLO_EDEVICE;
  if (cudaMemcpyAsync(d_ds, h, b.ds_nodes * sizeof(DsNode), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return POSLO_EDEVICE;
  if (ne) {
    launch_epoch_seeds(kInstSha, (unsigned)((ne + 127) / 128), 128, st, d_ds, (int)b.ds_nodes, e0, ne, seeds, status);
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return POSLO_EDEVICE;
  const uint64_t need = (b.n + kHashThreads - 1) / kHashThreads;
  const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, std::min(kMaxBlocks, sms * 8)));
  HashArgs a{};
  a.msgs = b.msgs;
  a.offs = b.offs;
  a.base_off = 0;
  a.n = b.n;
  a.first_index = b.first_index;
  a.e0 = e0;
  a.n2 = b.n2;
  a.n2_log2 = 0xffffffffu;
  if ((b.n2 & (b.n2 - 1)) == 0) {
    uint32_t l = 0;
    while ((1u << l) < b.n2) ++l;
    a.n2_log2 = l;
  }
  a.seeds = seeds;
  a.e_out = e_out;
  a.partial = partial;
  a.status = status;
  launch_hash(kInstSha, (unsigned)blocks, st, a);
  if (cudaGetLastError() != cudaSuccess) return POSLO_EDEVICE;
  uint32_t h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return POSLO_EDEVICE;
  if (cudaStreamSynchronize(st) != cudaSuccess) return POSLO_EDEVICE;
  if (h_status & (kErrSeed | kErrInput)) return POSLO_EINVAL;
  return POSLO_OK;
}
