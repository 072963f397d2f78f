// segmented_noalloc.cu - the batched segmented sort for callers that cannot
// allocate device memory.
//
// darm_segmented_sort keeps its block tables, segment slots and work counter
// in device buffers it allocates (and caches a CUDA graph per layout).  Some
// callers cannot let a library allocate: an application whose allocator owns
// every byte of the GPU, or a latency-critical loop that cannot afford the
// device-wide synchronisation cudaMalloc/cudaFree imply.  This variant keeps
// that scratch in one fixed array compiled into the library instead: the
// tables of each launch are copied into it on the caller's stream right
// before the launch, so the call allocates no device memory at all.
//
// The array lives in every GPU that loads the library, for the life of the
// process.  All calls share it and it keeps the last call's contents, so two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it; calls on one stream are ordered and safe.  The
// tables are copied from host memory the call reuses and frees, so the call
// refuses a stream that is capturing a graph (DARM_ERR_INVALID_ARG).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "batch.h"
#include "darm.h"
#include "darm_internal.h"

namespace darm {
namespace {

// Scratch for one launch: its work counter, segment slots and block table.
constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;  // 1 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DARM_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      fprintf(stderr, "darm: scratch address lookup failed: %s\n", cudaGetErrorString(e));
      return DARM_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DARM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace darm

using namespace darm;

extern "C" int darm_segmented_sort_noalloc(uint32_t* keys, uint32_t* vals,
                                           const uint64_t* seg_offsets, const uint32_t* seg_len,
                                           uint32_t num_segs, int dir, int variant,
                                           const uint8_t* seg_desc, void* stream) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (dir != DARM_ASC && dir != DARM_DESC) return DARM_ERR_INVALID_ARG;
  if (variant < DARM_DIVERGENT || variant > DARM_AUTO) return DARM_ERR_INVALID_ARG;
  if (num_segs == 0) return DARM_OK;
  if (!keys || !seg_offsets || !seg_len) return DARM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(keys) & 15u) != 0) return DARM_ERR_INVALID_ARG;
  if (vals && (reinterpret_cast<uintptr_t>(vals) & 15u) != 0) return DARM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Each launch's tables are copied from host memory that this call reuses
  // and frees, so a graph captured from this call would replay copies of
  // freed memory: refuse a capturing stream before enqueueing anything.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    fprintf(stderr, "darm_segmented_sort_noalloc: the stream is capturing a graph; call it "
                    "outside stream capture\n");
    return DARM_ERR_INVALID_ARG;
  }
  std::vector<BatchSeg> segs;
  int rc = segmented_parse(seg_offsets, seg_len, num_segs, dir, seg_desc, segs);
  if (rc != DARM_OK) return rc;
  if (segs.empty()) return DARM_OK;

  void* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != DARM_OK) return rc;
  unsigned char* base = static_cast<unsigned char*>(scratch);

  const bool has_vals = vals != nullptr;
  int cmax = 0;
  for (const BatchSeg& sg : segs) cmax = std::max(cmax, sg.c);
  const Tuning tn = batch_tuning(KEY_U32, has_vals, cmax);
  BatchTables bt;
  rc = batch_append(bt, KEY_U32, has_vals, tn, variant, segs, 0, 0);
  for (int p = tn.t + 1; p <= cmax && rc == DARM_OK; ++p)
    rc = batch_append(bt, KEY_U32, has_vals, tn, variant, segs, p, 0);
  if (rc != DARM_OK) return rc;

  // singletons (capacity 1): their table goes through the scratch too
  std::vector<uint64_t> sbase;
  std::vector<uint32_t> sld;
  for (const BatchSeg& sg : segs)
    if (sg.c == 0) {
      sbase.push_back(sg.base);
      sld.push_back((sg.len ? 1u : 0u) | (sg.desc ? 2u : 0u));
    }

  // Check every launch fits before enqueueing anything.
  const size_t L = bt.launches.size();
  std::vector<size_t> nblk(L), nslot(L);
  for (size_t i = 0; i < L; ++i) {
    const size_t bend = (i + 1 < L) ? bt.block_off[i + 1] : bt.blocks.size();
    nblk[i] = bend - bt.block_off[i];
    // slots of a launch: from its phase's first slot to that phase's end
    size_t send = bt.slots.size();
    for (size_t j = i + 1; j < L; ++j)
      if (bt.slot_off[j] != bt.slot_off[i]) {
        send = bt.slot_off[j];
        break;
      }
    nslot[i] = send - bt.slot_off[i];
    const size_t need = 256 + align256(nslot[i] * sizeof(SegSlot)) + nblk[i] * sizeof(SegBlock);
    if (need > kNoAllocScratchBytes) {
      fprintf(stderr,
              "darm_segmented_sort_noalloc: one launch needs %zu bytes of scratch, more than "
              "the %zu-byte maximum (use darm_segmented_sort, or split the segments)\n",
              need, kNoAllocScratchBytes);
      return DARM_ERR_INVALID_ARG;
    }
  }
  const size_t single_need = align256(sbase.size() * 8) + sld.size() * 4;
  if (single_need > kNoAllocScratchBytes) {
    fprintf(stderr, "darm_segmented_sort_noalloc: %zu capacity-1 segments exceed the scratch\n",
            sbase.size());
    return DARM_ERR_INVALID_ARG;
  }

  std::vector<unsigned char> staging;
  for (size_t i = 0; i < L; ++i) {
    // layout in the scratch: [counter (zeroed) | slots | blocks]
    const size_t slot_bytes = nslot[i] * sizeof(SegSlot);
    const size_t off_slots = 256;
    const size_t off_blocks = off_slots + align256(slot_bytes);
    const size_t total = off_blocks + nblk[i] * sizeof(SegBlock);
    staging.assign(total, 0);
    if (slot_bytes)
      std::memcpy(staging.data() + off_slots, bt.slots.data() + bt.slot_off[i], slot_bytes);
    if (nblk[i])
      std::memcpy(staging.data() + off_blocks, bt.blocks.data() + bt.block_off[i],
                  nblk[i] * sizeof(SegBlock));
    // pageable source: the runtime stages it before returning, so `staging`
    // can be reused; the copy runs after the previous launch on `s`
    if (cudaMemcpyAsync(base, staging.data(), total, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return DARM_ERR_CUDA;
    std::vector<Launch> one(1, bt.launches[i]);
    Launch& Lh = one[0];
    Lh.P.slots = reinterpret_cast<SegSlot*>(base + off_slots);
    Lh.P.blocks = reinterpret_cast<SegBlock*>(base + off_blocks);
    const bool persistent =
        std::find(bt.persistent.begin(), bt.persistent.end(), int(i)) != bt.persistent.end();
    Lh.P.work_counter = persistent ? reinterpret_cast<unsigned int*>(base) : nullptr;
    rc = launch_plan(one, KEY_U32, keys, vals, s);
    if (rc != DARM_OK) return rc;
  }
  if (!sbase.empty()) {
    const size_t off_ld = align256(sbase.size() * 8);
    staging.assign(off_ld + sld.size() * 4, 0);
    std::memcpy(staging.data(), sbase.data(), sbase.size() * 8);
    std::memcpy(staging.data() + off_ld, sld.data(), sld.size() * 4);
    if (cudaMemcpyAsync(base, staging.data(), staging.size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return DARM_ERR_CUDA;
    if (launch_singletons(keys, vals, reinterpret_cast<const uint64_t*>(base),
                          reinterpret_cast<const uint32_t*>(base + off_ld), uint32_t(sbase.size()),
                          s) != cudaSuccess)
      return DARM_ERR_CUDA;
    g_ctx.launches.fetch_add(1, std::memory_order_relaxed);
  }
  return DARM_OK;
}
