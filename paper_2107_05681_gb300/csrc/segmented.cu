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
// The whole sequence is captured once per layout as a CUDA graph and replayed
// on later calls with the same segments, pointers, direction and variant.
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

// Index of the round after which a tile-schedule block whose segments have
// capacity 2^c is complete (the bottom window of stage c).
int rounds_through(int c, int e) {
  int n = 1;
  for (int p = e + 1; p <= c; ++p) n += (p + e - 1) / e;
  return n;
}

int occupancy_grid(const void* fn, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * std::max(1, g_ctx.sms);
}

struct SegInfo {
  uint32_t idx;
  uint64_t base;
  uint32_t len;
  int c;
  bool desc;
};

// Build the launch list, device tables and graph for one layout.
int build_seg_plan(SegPlan& sp, uint32_t* keys, uint32_t* vals, const std::vector<SegInfo>& segs,
                   int variant) {
  const bool has_vals = vals != nullptr;
  const KeyKind kk = KEY_U32;
  Tuning tn = tuning_for(kk, has_vals, 0);
  int cmax = 0;
  for (const SegInfo& s : segs) cmax = std::max(cmax, s.c);
  if (!fit_tuning(tn, kk, has_vals, std::max(cmax, tn.t), g_ctx.smem_limit)) return DARM_ERR_INVALID_ARG;
  const int t = tn.t, e = tn.e1;
  const size_t tile_smem = size_t(elem_bytes(kk, has_vals)) * smem_words(1u << t);

  // --- tables -------------------------------------------------------------
  std::vector<SegSlot> slots;
  std::vector<SegBlock> blocks;
  std::vector<const SegInfo*> order;
  for (const SegInfo& s : segs)
    if (s.c >= e) order.push_back(&s);
  std::stable_sort(order.begin(), order.end(),
                   [](const SegInfo* a, const SegInfo* b) { return a->c > b->c; });
  std::vector<uint32_t> slot_of(segs.size(), 0xFFFFFFFFu);
  auto add_slot = [&](const SegInfo& s) {
    SegSlot sl{};
    sl.base = s.base;
    sl.len = s.len;
    sl.flags = s.desc ? kSlotDesc : 0u;
    slots.push_back(sl);
    return uint32_t(slots.size() - 1);
  };

  // tile pass blocks, longest first
  const int nr_full = rounds_through(t, e);
  size_t i = 0;
  while (i < order.size()) {
    const int c = order[i]->c;
    if (c >= t) {
      const SegInfo& s = *order[i];
      const uint32_t sl = add_slot(s);
      slot_of[&s - &segs[0]] = sl;
      for (uint32_t b = 0; b < (1u << (c - t)); ++b) {
        SegBlock B{};
        B.first_slot = sl;
        B.blk_in_seg = b;
        B.log2cap = uint8_t(c);
        B.nrounds = uint8_t(nr_full);
        B.final_pass = (c == t) ? 1 : 0;
        B.fill = 1;
        blocks.push_back(B);
      }
      ++i;
    } else {
      // pack 2^(t-c) segments of this class per block
      const uint32_t per = 1u << (t - c);
      const uint32_t first = uint32_t(slots.size());
      uint32_t taken = 0;
      while (i < order.size() && order[i]->c == c && taken < per) {
        add_slot(*order[i]);
        ++taken;
        ++i;
      }
      for (; taken < per; ++taken) {
        SegSlot empty{};
        empty.flags = kSlotEmpty;
        slots.push_back(empty);
      }
      SegBlock B{};
      B.first_slot = first;
      B.blk_in_seg = 0;
      B.log2cap = uint8_t(c);
      B.nrounds = uint8_t(rounds_through(c, e));
      B.final_pass = 1;
      B.fill = 1;
      blocks.push_back(B);
    }
  }
  const uint32_t tile_blocks = uint32_t(blocks.size());

  // tiny segments (capacity 2..2^(e-1)): one thread per segment, Phase A only
  struct TinyLaunch {
    int c;
    uint32_t first_block, nblocks;
  };
  std::vector<TinyLaunch> tiny;
  const int tiny_threads_log2 = 7;
  for (int c = e - 1; c >= 1; --c) {
    std::vector<const SegInfo*> cls;
    for (const SegInfo& s : segs)
      if (s.c == c) cls.push_back(&s);
    if (cls.empty()) continue;
    const uint32_t per = 1u << tiny_threads_log2;
    TinyLaunch tl{c, uint32_t(blocks.size()), 0};
    for (size_t j = 0; j < cls.size(); j += per) {
      const uint32_t first = uint32_t(slots.size());
      for (size_t q = 0; q < per; ++q) {
        if (j + q < cls.size()) {
          add_slot(*cls[j + q]);
        } else {
          SegSlot empty{};
          empty.flags = kSlotEmpty;
          slots.push_back(empty);
        }
      }
      SegBlock B{};
      B.first_slot = first;
      B.log2cap = uint8_t(c);
      B.nrounds = 1;
      B.final_pass = 1;
      B.fill = 1;
      blocks.push_back(B);
      ++tl.nblocks;
    }
    tiny.push_back(tl);
  }

  // passes for segments larger than a tile
  struct BigLaunch {
    Launch L;
    uint32_t first_block, nblocks;
  };
  std::vector<BigLaunch> big;
  for (int p = t + 1; p <= cmax; ++p) {
    std::vector<const SegInfo*> act;
    for (const SegInfo* s : order)
      if (s->c >= p) act.push_back(s);
    if (act.empty()) break;
    // window passes: one plan_array stage gives the shapes; copy them
    std::vector<Launch> shape;
    plan_array(shape, kk, has_vals, p, tn, variant, 0, 0, g_ctx.smem_limit);
    // the launches of stage p are the ones after the stage p-1 merge pass:
    // take every window pass with rounds at stage p, and the final merge
    for (const Launch& L0 : shape) {
      if (L0.kind == PASS_TILE) continue;
      if (L0.P.rounds[0].p != p) continue;
      BigLaunch bl;
      bl.L = L0;
      bl.first_block = uint32_t(blocks.size());
      const uint32_t bsize_log2 = L0.P.b;
      for (const SegInfo* s : act) {
        const uint32_t sl = slot_of[s - &segs[0]];
        for (uint32_t b = 0; b < (1u << (s->c - bsize_log2)); ++b) {
          SegBlock B{};
          B.first_slot = sl;
          B.blk_in_seg = b;
          B.log2cap = uint8_t(s->c);
          B.nrounds = uint8_t(L0.P.nrounds);
          B.final_pass = (L0.kind == PASS_MERGE && s->c == p) ? 1 : 0;
          B.fill = 0;
          blocks.push_back(B);
        }
      }
      bl.nblocks = uint32_t(blocks.size()) - bl.first_block;
      big.push_back(bl);
    }
  }

  // singletons
  std::vector<uint64_t> sbase;
  std::vector<uint32_t> sld;
  for (const SegInfo& s : segs)
    if (s.c == 0) {
      sbase.push_back(s.base);
      sld.push_back((s.len ? 1u : 0u) | (s.desc ? 2u : 0u));
    }

  // --- upload ---------------------------------------------------------------
  if (!slots.empty()) {
    if (cudaMalloc(&sp.d_slots, slots.size() * sizeof(SegSlot)) != cudaSuccess) return DARM_ERR_OOM;
    cudaMemcpy(sp.d_slots, slots.data(), slots.size() * sizeof(SegSlot), cudaMemcpyHostToDevice);
  }
  if (!blocks.empty()) {
    if (cudaMalloc(&sp.d_blocks, blocks.size() * sizeof(SegBlock)) != cudaSuccess) return DARM_ERR_OOM;
    cudaMemcpy(sp.d_blocks, blocks.data(), blocks.size() * sizeof(SegBlock), cudaMemcpyHostToDevice);
  }
  if (cudaMalloc(&sp.d_counter, sizeof(unsigned int)) != cudaSuccess) return DARM_ERR_OOM;
  if (!sbase.empty()) {
    sp.n_single = uint32_t(sbase.size());
    cudaMalloc(&sp.d_single_base, sbase.size() * sizeof(uint64_t));
    cudaMalloc(&sp.d_single_ld, sld.size() * sizeof(uint32_t));
    cudaMemcpy(sp.d_single_base, sbase.data(), sbase.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(sp.d_single_ld, sld.data(), sld.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
  }
  if (cudaGetLastError() != cudaSuccess) return DARM_ERR_CUDA;

  // --- launches -------------------------------------------------------------
  sp.launches.clear();
  if (tile_blocks > 0) {
    Launch L{};
    L.kind = PASS_TILE;
    L.loge = e;
    L.variant = (variant == DARM_AUTO) ? tn.var[PASS_TILE] : variant;
    L.threads = 1u << (t - e);
    L.smem = tile_smem;
    L.P.b = L.P.c = L.P.w0 = uint32_t(t);
    L.P.s = 0;
    L.P.log2cap = uint32_t(t);
    std::vector<Round> rs = tile_rounds(t, e);
    L.P.nrounds = uint32_t(rs.size());
    for (size_t r = 0; r < rs.size(); ++r) L.P.rounds[r] = rs[r];
    L.P.blocks = sp.d_blocks;
    L.P.slots = sp.d_slots;
    L.fixed = fixed_kernel_fn(kk, has_vals, e, t, L.variant, false) != nullptr;
    if (L.fixed) {
      const void* fn = fixed_kernel_fn(kk, has_vals, e, t, L.variant, false);
      L.P.work_counter = sp.d_counter;
      L.P.nblocks = tile_blocks;
      L.grid = uint32_t(std::min<int>(int(tile_blocks), occupancy_grid(fn, int(L.threads), L.smem)));
    } else {
      L.grid = tile_blocks;
    }
    sp.launches.push_back(L);
  }
  for (const TinyLaunch& tl : tiny) {
    Launch L{};
    L.kind = PASS_TILE;
    L.fixed = false;
    L.loge = tl.c;
    L.variant = (variant == DARM_AUTO) ? tn.var[PASS_TILE] : variant;
    L.threads = 1u << tiny_threads_log2;
    L.grid = tl.nblocks;
    L.smem = 0;
    L.P.b = L.P.c = L.P.w0 = uint32_t(tl.c + tiny_threads_log2);
    L.P.s = 0;
    L.P.log2cap = uint32_t(tl.c);
    std::vector<Round> rs = tile_rounds(tl.c, tl.c);
    L.P.nrounds = 1;
    L.P.rounds[0] = rs[0];
    L.P.blocks = sp.d_blocks + tl.first_block;
    L.P.slots = sp.d_slots;
    sp.launches.push_back(L);
  }
  for (const BigLaunch& bl : big) {
    Launch L = bl.L;
    L.grid = bl.nblocks;
    L.P.blocks = sp.d_blocks + bl.first_block;
    L.P.slots = sp.d_slots;
    L.P.log2cap = 0;
    L.P.map_in = L.P.map_out = 0;
    sp.launches.push_back(L);
  }

  // --- capture --------------------------------------------------------------
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return DARM_ERR_CUDA;
  int rc = DARM_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return DARM_ERR_CUDA;
  }
  cudaMemsetAsync(sp.d_counter, 0, sizeof(unsigned int), cs);
  rc = launch_plan(sp.launches, kk, keys, vals, cs, /*count=*/false);
  if (rc == DARM_OK && sp.n_single) {
    seg_singletons_kernel<<<(sp.n_single + 255) / 256, 256, 0, cs>>>(keys, vals, sp.d_single_base,
                                                                       sp.d_single_ld, sp.n_single);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
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

}  // namespace

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

  std::vector<SegInfo> segs;
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
    SegInfo si;
    si.idx = s;
    si.base = a;
    si.len = seg_len[s];
    si.c = log2u(cap);
    si.desc = seg_desc ? (seg_desc[s] != 0) : (dir == DARM_DESC);
    segs.push_back(si);
  }
  if (segs.empty()) return DARM_OK;

  // layout key: pointers, direction, variant and a hash of the arrays
  uint64_t h = 0xCBF29CE484222325ull;
  h = fnv1a(h, seg_offsets, sizeof(uint64_t) * (size_t(num_segs) + 1));
  h = fnv1a(h, seg_len, sizeof(uint32_t) * num_segs);
  if (seg_desc) h = fnv1a(h, seg_desc, num_segs);
  const Tuning tn = tuning_for(KEY_U32, vals != nullptr, 0);
  std::vector<uint64_t> key = {h,
                               uint64_t(num_segs),
                               reinterpret_cast<uint64_t>(keys),
                               reinterpret_cast<uint64_t>(vals),
                               uint64_t(dir),
                               uint64_t(variant),
                               uint64_t(seg_desc != nullptr),
                               uint64_t(tn.t * 1000 + tn.e1 * 100 + tn.e2 * 10 + tn.w2)};

  std::lock_guard<std::mutex> lk(g_seg_mu);
  auto it = g_seg_plans.find(key);
  if (it == g_seg_plans.end()) {
    auto sp = std::make_unique<SegPlan>();
    const int rc = build_seg_plan(*sp, keys, vals, segs, variant);
    if (rc != DARM_OK) return rc;
    it = g_seg_plans.emplace(key, std::move(sp)).first;
  }
  SegPlan& sp = *it->second;
  if (cudaGraphLaunch(sp.exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return DARM_ERR_CUDA;
  g_ctx.launches.fetch_add(uint64_t(sp.kernel_nodes), std::memory_order_relaxed);
  return DARM_OK;
}
