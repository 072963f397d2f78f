// darm_internal.h - state and helpers shared by the library's translation
// units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "batch.h"
#include "plan.h"

namespace darm {

// Everything that identifies a compiled whole-array plan.
using PlanKey = std::tuple<int, int, int, int, uint32_t, uint32_t, int, int, int, int, int, int>;

struct Context {
  bool inited = false;
  int device = -1;
  int sms = 0;
  size_t smem_limit = 0;
  int* d_status = nullptr;           // device status word
  cudaStream_t host_stream = nullptr;  // stream of host-buffer sorts
  cudaStream_t host_copy_stream = nullptr;  // their chunked host->device copies
  cudaStream_t host_stream2 = nullptr;      // tile passes of the second half
  cudaEvent_t host_join_ev = nullptr;       // ... joined back into host_stream
  cudaEvent_t host_chunk_ev[8] = {};        // one per chunk copied
  cudaStream_t split_stream = nullptr;  // second half of a split whole-array sort
  cudaEvent_t split_fork_ev = nullptr;  // caller's stream -> split_stream
  cudaEvent_t split_join_ev = nullptr;  // split_stream -> caller's stream
  void* ws = nullptr;                // workspace of host-buffer sorts
  size_t ws_bytes = 0;
  std::mutex mu;       // plans, tuning table, init/finalize
  std::mutex host_mu;  // host-buffer workspace
  std::atomic<uint64_t> launches{0};
  std::map<std::tuple<int, int, int>, Tuning> tuned;  // (key kind, has vals, log2 n)
  std::map<PlanKey, std::vector<Launch>> plans;
};

extern Context g_ctx;

const void* kernel_fn(KeyKind kk, bool has_vals, int loge, int variant);
const void* fixed_kernel_fn(KeyKind kk, bool has_vals, int loge, int logt, int variant, bool merge);
// Enqueue every launch of `plan` on `stream`; `count` adds them to the
// library's launch counter (off while capturing a graph, whose replays are
// counted instead).
int launch_plan(const std::vector<Launch>& plan, KeyKind kk, void* keys, uint32_t* vals,
                cudaStream_t stream, bool count = true);
// The same for the launches [first, last) of a plan.
int launch_range(const Launch* first, const Launch* last, KeyKind kk, void* keys, uint32_t* vals,
                 cudaStream_t stream, bool count = true);
Tuning tuning_for(KeyKind kk, bool has_vals, int m);
const std::vector<Launch>* cached_plan(KeyKind kk, bool has_vals, int m, int variant,
                                       uint32_t map_in, uint32_t map_out);
int sort_device(KeyKind kk, bool f32, void* keys, uint32_t* vals, size_t n, int dir, int variant,
                cudaStream_t stream);
void segmented_release_all();

// Validate a segment layout (host arrays) and list its non-empty segments.
int segmented_parse(const uint64_t* seg_offsets, const uint32_t* seg_len, uint32_t num_segs, int dir,
                    const uint8_t* seg_desc, std::vector<BatchSeg>& segs);

// Capacity-1 segments: write the sentinel into the empty ones.  base[i] is
// the element offset, len_desc[i] bit 0 = real length 1, bit 1 = descending.
// Returns the status of this launch alone.
cudaError_t launch_singletons(uint32_t* keys, uint32_t* vals, const uint64_t* base,
                              const uint32_t* len_desc, uint32_t n, cudaStream_t s);

// PCM's merge-split kernels (pcm.cu) and the odd-even bucket kernels
// (oddeven.cu), for the shared-memory limit set at init.
void for_each_pcm_kernel(void (*fn)(const void*, void*), void* ctx);
void for_each_oddeven_kernel(void (*fn)(const void*, void*), void* ctx);

}  // namespace darm
