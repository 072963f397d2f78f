// segmented.cu - batched sort of independent power-of-two segments.
//
// The paper's bitonic workload sorts an input bucket by bucket, one bucket
// per thread block (Section VI-A, "Bitonic Sort (BIT)").  Here thousands of
// independent segments of uneven capacity are sorted by one launch sequence:
//
//   1. one persistent tile launch: CTAs take entries of a block table in
//      order from a global counter.  The table lists the tiles of segments
//      larger than a tile first (longest processing time first), then blocks
//      that each pack 2^(t - c) whole segments of capacity 2^c < T.  A block
//      runs the tile schedule only up to its segments' last stage.  The first
//      load writes the sentinel past each segment's real length and
//      complements the keys of descending segments;
//   2. segments larger than a tile continue with window and merge passes,
//      one launch per pass over all segments still in that stage;
//   3. segments of capacity 2..8 are sorted in registers by one thread each;
//      capacity-1 segments only receive their sentinel when empty.
//
// The segments are dealt into two groups of about equal padded size, each
// with its own sequence; the two sequences are captured once per layout as
// one CUDA graph on two streams and replayed on later calls with the same
// segments, pointers, direction and variant.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "darm.h"
#include "darm_internal.h"
#include "kernel_table.h"
#include "plan.h"
#include "batch.h"
#include "tile_kernel.cuh"

namespace darm {

namespace {

// Capacity-1 segments: sorted by definition; an empty one gets its sentinel.
__global__ void seg_singletons_kernel(uint32_t* keys, uint32_t* vals, const uint64_t* base,
                                      const uint32_t* len_desc, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t ld = len_desc[i];
  if ((ld & 1u) == 0u) {  // real length 0
    keys[base[i]] = (ld & 2u) ? 0u : 0xFFFFFFFFu;
    if (vals) vals[base[i]] = 0xFFFFFFFFu;
  }
}

}  // namespace

cudaError_t launch_singletons(uint32_t* keys, uint32_t* vals, const uint64_t* base,
                              const uint32_t* len_desc, uint32_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  void* args[] = {&keys, &vals, &base, &len_desc, &n};
  // the status of this launch alone (no sticky error of earlier work)
  return cudaLaunchKernel(reinterpret_cast<const void*>(&seg_singletons_kernel),
                          dim3((n + 255) / 256), dim3(256), args, 0, s);
}

namespace {

struct SegPlan {
  std::vector<Launch> launches;
  SegSlot* d_slots = nullptr;
  SegBlock* d_blocks = nullptr;
  unsigned int* d_counter = nullptr;
  uint64_t* d_single_base = nullptr;
  uint32_t* d_single_ld = nullptr;
  uint32_t n_single = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernel_nodes = 0;

  ~SegPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (d_slots) cudaFree(d_slots);
    if (d_blocks) cudaFree(d_blocks);
    if (d_counter) cudaFree(d_counter);
    if (d_single_base) cudaFree(d_single_base);
    if (d_single_ld) cudaFree(d_single_ld);
  }
};

std::mutex g_seg_mu;
std::map<std::vector<uint64_t>, std::unique_ptr<SegPlan>> g_seg_plans;

int log2u(uint64_t v) {
  int m = 0;
  while ((uint64_t(1) << m) < v) ++m;
  return m;
}

// Build the launch list, device tables and graph for one layout.
int build_seg_plan(SegPlan& sp, uint32_t* keys, uint32_t* vals, const std::vector<BatchSeg>& segs,
                   int variant, const Tuning& tn) {
  const bool has_vals = vals != nullptr;
  const KeyKind kk = KEY_U32;
  // Two groups of segments of about equal padded size (largest first, each
  // to the lighter group), each with its own launch sequence: the graph
  // runs the two sequences on two streams, so that one group's passes fill
  // the other's launch ramps and tails and its HBM-bound passes run beside
  // the other's ALU-bound tile pass.  Segments are independent, so the
  // result is each segment's own network.
  std::vector<BatchSeg> group[2];
  {
    std::vector<const BatchSeg*> order;
    for (const BatchSeg& s : segs)
      if (s.c >= 1) order.push_back(&s);
    std::stable_sort(order.begin(), order.end(),
                     [](const BatchSeg* a, const BatchSeg* b) { return a->c > b->c; });
    uint64_t load[2] = {0, 0};
    for (const BatchSeg* s : order) {
      const int g = (load[1] < load[0]) ? 1 : 0;
      group[g].push_back(*s);
      load[g] += uint64_t(1) << s->c;
    }
  }
  BatchTables bt;
  size_t second = 0;  // first launch of group 1
  int rc = DARM_OK;
  for (int g = 0; g < 2 && rc == DARM_OK; ++g) {
    if (g == 1) second = bt.launches.size();
    int cmax = 0;
    for (const BatchSeg& s : group[g]) cmax = std::max(cmax, s.c);
    if (group[g].empty()) continue;
    rc = batch_append(bt, kk, has_vals, tn, variant, group[g], 0, 0);
    for (int p = tn.t + 1; p <= cmax && rc == DARM_OK; ++p)
      rc = batch_append(bt, kk, has_vals, tn, variant, group[g], p, 0);
  }
  if (rc != DARM_OK) return rc;

  // singletons
  std::vector<uint64_t> sbase;
  std::vector<uint32_t> sld;
  for (const BatchSeg& s : segs)
    if (s.c == 0) {
      sbase.push_back(s.base);
      sld.push_back((s.len ? 1u : 0u) | (s.desc ? 2u : 0u));
    }

  // upload
  if (!bt.slots.empty()) {
    if (cudaMalloc(&sp.d_slots, bt.slots.size() * sizeof(SegSlot)) != cudaSuccess) return DARM_ERR_OOM;
    cudaMemcpy(sp.d_slots, bt.slots.data(), bt.slots.size() * sizeof(SegSlot), cudaMemcpyHostToDevice);
  }
  if (!bt.blocks.empty()) {
    if (cudaMalloc(&sp.d_blocks, bt.blocks.size() * sizeof(SegBlock)) != cudaSuccess) return DARM_ERR_OOM;
    cudaMemcpy(sp.d_blocks, bt.blocks.data(), bt.blocks.size() * sizeof(SegBlock),
               cudaMemcpyHostToDevice);
  }
  const size_t ncounters = std::max<size_t>(1, bt.persistent.size());
  if (cudaMalloc(&sp.d_counter, ncounters * sizeof(unsigned int)) != cudaSuccess) return DARM_ERR_OOM;
  if (!sbase.empty()) {
    sp.n_single = uint32_t(sbase.size());
    cudaMalloc(&sp.d_single_base, sbase.size() * sizeof(uint64_t));
    cudaMalloc(&sp.d_single_ld, sld.size() * sizeof(uint32_t));
    cudaMemcpy(sp.d_single_base, sbase.data(), sbase.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(sp.d_single_ld, sld.data(), sld.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  }
  if (cudaGetLastError() != cudaSuccess) return DARM_ERR_CUDA;
  batch_bind(bt, sp.d_blocks, sp.d_slots, sp.d_counter);
  sp.launches = bt.launches;

  // capture: group 0 on cs, group 1 on cs2 (forked from cs after the
  // counters are zeroed, joined back before the singletons)
  cudaStream_t cs, cs2;
  cudaEvent_t fork_ev, join_ev;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return DARM_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return DARM_ERR_CUDA;
  }
  if (cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(cs);
    cudaStreamDestroy(cs2);
    return DARM_ERR_CUDA;
  }
  cudaMemsetAsync(sp.d_counter, 0, ncounters * sizeof(unsigned int), cs);
  const Launch* L0 = sp.launches.data();
  if (second > 0 && second < sp.launches.size()) {
    cudaEventRecord(fork_ev, cs);
    cudaStreamWaitEvent(cs2, fork_ev, 0);
    rc = launch_range(L0, L0 + second, kk, keys, vals, cs, /*count=*/false);
    if (rc == DARM_OK)
      rc = launch_range(L0 + second, L0 + sp.launches.size(), kk, keys, vals, cs2, false);
    cudaEventRecord(join_ev, cs2);
    cudaStreamWaitEvent(cs, join_ev, 0);
  } else {
    rc = launch_plan(sp.launches, kk, keys, vals, cs, /*count=*/false);
  }
  if (rc == DARM_OK && sp.n_single) {
    if (launch_singletons(keys, vals, sp.d_single_base, sp.d_single_ld, sp.n_single, cs) !=
        cudaSuccess)
      rc = DARM_ERR_CUDA;
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  cudaStreamDestroy(cs2);
  cudaEventDestroy(fork_ev);
  cudaEventDestroy(join_ev);
  if (rc != DARM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ec != cudaSuccess || !graph) return DARM_ERR_CUDA;
  sp.graph = graph;
  if (cudaGraphInstantiate(&sp.exec, graph, 0) != cudaSuccess) return DARM_ERR_CUDA;
  sp.kernel_nodes = int(sp.launches.size()) + (sp.n_single ? 1 : 0);
  return DARM_OK;
}

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 0x100000001B3ull;
  }
  return h;
}

// Every field of a tuning that changes a batch's launches.
uint64_t tuning_key(const Tuning& tn) {
  uint64_t k = 0;
  for (int v : {tn.t, tn.e1, tn.e2, tn.c2, tn.w2, tn.tma, tn.shfl, tn.em, tn.var[0], tn.var[1],
                tn.var[2]})
    k = k * 64 + uint64_t(v & 63);
  return k;
}

}  // namespace

int segmented_parse(const uint64_t* seg_offsets, const uint32_t* seg_len, uint32_t num_segs, int dir,
                    const uint8_t* seg_desc, std::vector<BatchSeg>& segs) {
  segs.clear();
  segs.reserve(num_segs);
  for (uint32_t s = 0; s < num_segs; ++s) {
    const uint64_t a = seg_offsets[s], b = seg_offsets[s + 1];
    if (b < a) return DARM_ERR_INVALID_ARG;
    const uint64_t cap = b - a;
    if (cap == 0) continue;
    if ((cap & (cap - 1)) != 0) return DARM_ERR_NOT_POW2;
    if (cap > (uint64_t(1) << 31)) return DARM_ERR_INVALID_ARG;
    if ((a & (std::min<uint64_t>(cap, 4) - 1)) != 0) return DARM_ERR_INVALID_ARG;
    if (seg_len[s] > cap) return DARM_ERR_INVALID_ARG;
    BatchSeg si;
    si.base = a;
    si.len = seg_len[s];
    si.c = log2u(cap);
    si.desc = seg_desc ? (seg_desc[s] != 0) : (dir == DARM_DESC);
    segs.push_back(si);
  }
  return DARM_OK;
}

void segmented_release_all() {
  std::lock_guard<std::mutex> lk(g_seg_mu);
  if (!g_seg_plans.empty()) cudaDeviceSynchronize();
  g_seg_plans.clear();
}

}  // namespace darm

using namespace darm;

extern "C" int darm_segmented_sort(uint32_t* keys, uint32_t* vals, const uint64_t* seg_offsets,
                                   const uint32_t* seg_len, uint32_t num_segs, int dir,
                                   int variant, const uint8_t* seg_desc, void* stream) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (dir != DARM_ASC && dir != DARM_DESC) return DARM_ERR_INVALID_ARG;
  if (variant < DARM_DIVERGENT || variant > DARM_AUTO) return DARM_ERR_INVALID_ARG;
  if (num_segs == 0) return DARM_OK;
  if (!keys || !seg_offsets || !seg_len) return DARM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(keys) & 15u) != 0) return DARM_ERR_INVALID_ARG;
  if (vals && (reinterpret_cast<uintptr_t>(vals) & 15u) != 0) return DARM_ERR_INVALID_ARG;

  std::vector<BatchSeg> segs;
  const int prc = segmented_parse(seg_offsets, seg_len, num_segs, dir, seg_desc, segs);
  if (prc != DARM_OK) return prc;
  if (segs.empty()) return DARM_OK;

  // layout key: pointers, direction, variant, the tuning the batch runs with
  // and a hash of the arrays
  uint64_t h = 0xCBF29CE484222325ull;
  h = fnv1a(h, seg_offsets, sizeof(uint64_t) * (size_t(num_segs) + 1));
  h = fnv1a(h, seg_len, sizeof(uint32_t) * num_segs);
  if (seg_desc) h = fnv1a(h, seg_desc, num_segs);
  int cmax = 0;
  for (const BatchSeg& sg : segs) cmax = std::max(cmax, sg.c);
  const Tuning tn = batch_tuning(KEY_U32, vals != nullptr, cmax);
  std::vector<uint64_t> key = {h,
                               uint64_t(num_segs),
                               reinterpret_cast<uint64_t>(keys),
                               reinterpret_cast<uint64_t>(vals),
                               uint64_t(dir),
                               uint64_t(variant),
                               uint64_t(seg_desc != nullptr),
                               tuning_key(tn)};

  std::lock_guard<std::mutex> lk(g_seg_mu);
  auto it = g_seg_plans.find(key);
  if (it == g_seg_plans.end()) {
    auto sp = std::make_unique<SegPlan>();
    const int rc = build_seg_plan(*sp, keys, vals, segs, variant, tn);
    if (rc != DARM_OK) return rc;
    it = g_seg_plans.emplace(key, std::move(sp)).first;
  }
  SegPlan& sp = *it->second;
  if (cudaGraphLaunch(sp.exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return DARM_ERR_CUDA;
  g_ctx.launches.fetch_add(uint64_t(sp.kernel_nodes), std::memory_order_relaxed);
  return DARM_OK;
}

// Autotuner for batches: times whole batched sorts of the caller's layout for
// each candidate tuning (tile size, register windows per window pass,
// elements per thread in window passes), then the divergent or melded form
// per pass kind, and keeps the fastest as the batch tuning.
extern "C" int darm_autotune_segmented(uint32_t* keys, uint32_t* vals, const uint64_t* seg_offsets,
                                       const uint32_t* seg_len, uint32_t num_segs,
                                       const char* db_path) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (!keys || !seg_offsets || !seg_len || num_segs == 0) return DARM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(keys) & 15u) != 0) return DARM_ERR_INVALID_ARG;
  if (vals && (reinterpret_cast<uintptr_t>(vals) & 15u) != 0) return DARM_ERR_INVALID_ARG;
  std::vector<BatchSeg> segs;
  int rc = segmented_parse(seg_offsets, seg_len, num_segs, DARM_ASC, nullptr, segs);
  if (rc != DARM_OK) return rc;
  if (segs.empty()) return DARM_ERR_INVALID_ARG;
  const bool hv = vals != nullptr;
  int cmax = 0;
  for (const BatchSeg& sg : segs) cmax = std::max(cmax, sg.c);

  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return DARM_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // best of three replays of the batch's graph (after one warm-up); < 0 if
  // the tuning cannot run this layout
  auto time_tuning = [&](const Tuning& tn0) -> float {
    Tuning tn = tn0;
    if (!fit_tuning(tn, KEY_U32, hv, std::max(cmax, tn.t), g_ctx.smem_limit)) return -1.f;
    SegPlan sp;
    if (build_seg_plan(sp, keys, vals, segs, DARM_AUTO, tn) != DARM_OK) {
      cudaGetLastError();
      return -1.f;
    }
    float best = -1.f;
    for (int r = 0; r < 4; ++r) {
      cudaEventRecord(e0, s);
      if (cudaGraphLaunch(sp.exec, s) != cudaSuccess) return -1.f;
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && (best < 0.f || ms < best)) best = ms;
    }
    return best;
  };

  const Tuning base = default_tuning(KEY_U32, hv);
  Tuning best = base;
  float best_ms = -1.f;
  // merge passes: the table-driven tile kernel (0) or the bulk-copy merge
  // with its staging buffers (1 for key-value, 2 for keys)
  const int tma_on = hv ? 1 : 2;
  for (int t = base.t - 1; t <= base.t + 1; ++t)
    for (int e2 = 3; e2 <= 5; ++e2)
      for (int w2 = 1; w2 <= 2; ++w2)
      for (int tma : {0, tma_on}) {
        Tuning tn = base;
        tn.t = t;
        tn.e2 = e2;
        tn.w2 = w2;
        tn.tma = tma;
        tn.var[0] = tn.var[1] = tn.var[2] = kMelded;
        const float ms = time_tuning(tn);
        if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
          best_ms = ms;
          best = tn;
        }
      }
  // merges on tiles half the tile pass's (the window passes take the bit
  // between)
  if (best_ms >= 0.f && best.t - 1 >= best.e1) {
    Tuning tn = best;
    tn.tm = best.t - 1;
    const float ms = time_tuning(tn);
    if (ms >= 0.f && ms < best_ms) {
      best_ms = ms;
      best = tn;
    }
  }
  // the divergent or melded form per pass kind (tile, window, merge)
  if (best_ms >= 0.f) {
    const Tuning shape = best;
    for (int combo = 0; combo < 8; ++combo) {
      Tuning tn = shape;
      for (int k = 0; k < 3; ++k) tn.var[k] = ((combo >> k) & 1) ? kDivergent : kMelded;
      if (combo == 0) continue;  // all melded: timed above
      const float ms = time_tuning(tn);
      if (ms >= 0.f && ms < best_ms) {
        best_ms = ms;
        best = tn;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (cudaGetLastError() != cudaSuccess) return DARM_ERR_CUDA;
  if (best_ms < 0.f) return DARM_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(g_ctx.mu);
    g_ctx.tuned[std::make_tuple(int(KEY_U32), int(hv), 0)] = best;
  }
  segmented_release_all();  // graphs built under the previous tuning
  if (db_path) {
    FILE* f = fopen(db_path, "a");
    if (!f) return DARM_ERR_INVALID_ARG;
    fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %.6f %d %d %d\n", int(KEY_U32), int(hv), 0,
            best.t, best.e1, best.e2, best.c2, best.w2, best.tma, best.var[0], best.var[1],
            best.var[2], double(best_ms), best.shfl, best.em, best.tm);
    fclose(f);
  }
  return DARM_OK;
}
