// batch.cu - block tables and launch lists for batches of segments (batch.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "batch.h"
#include "darm.h"
#include "darm_internal.h"
#include "kernel_table.h"
#include "tile_shfl_kernel.cuh"

namespace darm {

namespace {

// Round count of the tile schedule through stage 2^c (its bottom window).
int rounds_through(int c, int e) {
  int n = 1;
  for (int p = e + 1; p <= c; ++p) n += (p + e - 1) / e;
  return n;
}

int occupancy_grid(const void* fn, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm * std::max(1, g_ctx.sms);
}

constexpr int kTinyThreadsLog2 = 7;
constexpr uint32_t kPaddingThreads = 256;

}  // namespace

Tuning batch_tuning(KeyKind kk, bool has_vals, int cmax) {
  Tuning tn = tuning_for(kk, has_vals, 0);
  bool tuned;
  {
    std::lock_guard<std::mutex> lk(g_ctx.mu);
    tuned = g_ctx.tuned.count(std::make_tuple(int(kk), int(has_vals), 0)) != 0;
  }
  // Untuned 32-bit key-value batches take 8 Ki-pair tiles (10,000 segments
  // of up to 2^16 pairs: 4.92 -> 4.52 ms against 4 Ki-pair tiles, when the
  // merge passes ran the table-driven tile kernel).
  if (!tuned && kk == KEY_U32 && has_vals) tn.t = 13;
  if (!tuned) tn.tm = 0;  // one tile size unless a batch tuning asks for a smaller merge tile
  // tma: staging buffers of the bulk-copy merge, which reads each tile's
  // place from the block table (0: the table-driven tile kernel; no
  // swizzled in-place form for batches)
  if (kk != KEY_U32)
    tn.tma = 0;
  else if (!tuned)
    tn.tma = has_vals ? 1 : 2;
  else
    tn.tma = std::min(tn.tma, 2);
  fit_tuning(tn, kk, has_vals, std::max(cmax, tn.t), g_ctx.smem_limit);
  return tn;
}

int batch_append(BatchTables& bt, KeyKind kk, bool has_vals, const Tuning& tn, int variant,
                 const std::vector<BatchSeg>& segs, int phase, uint32_t map_in) {
  const int t = tn.t, e = tn.e1;
  const size_t slot0 = bt.slots.size();
  const size_t block0 = bt.blocks.size();
  auto add_slot = [&](const BatchSeg& s) {
    SegSlot sl{};
    sl.base = s.base;
    sl.len = s.len;
    sl.flags = s.desc ? kSlotDesc : 0u;
    bt.slots.push_back(sl);
    return uint32_t(bt.slots.size() - slot0 - 1);
  };
  auto add_empty = [&]() {
    SegSlot sl{};
    sl.flags = kSlotEmpty;
    bt.slots.push_back(sl);
  };
  auto pick = [&](PassKind k) { return (variant == DARM_AUTO) ? tn.var[k] : variant; };

  if (phase == 0) {
    // the tile pass with shuffle stages, where one is built for this shape
    const bool shfl = (tn.shfl & 1) != 0 && kk == KEY_U32 &&
                      tile_shfl_seg_kernel_u32(has_vals, e, t, 1).fn != nullptr;
    auto rounds_to = [&](int c) { return shfl ? shfl_rounds_through(c, t, e) : rounds_through(c, e); };
    std::vector<const BatchSeg*> order;
    for (const BatchSeg& s : segs)
      if (s.c >= e) order.push_back(&s);
    std::stable_sort(order.begin(), order.end(),
                     [](const BatchSeg* a, const BatchSeg* b) { return a->c > b->c; });
    // tile blocks, longest segments first.  A block of a segment longer
    // than the tile that lies wholly beyond the segment's real length holds
    // only sentinels: every compare-exchange of the tile's stages meets two
    // equal keys and equal payloads and, swaps being strict, moves nothing,
    // so the block's tile-pass result is the sentinel at every position.
    // Such blocks go to a launch of their own that only writes that result
    // (a tile launch with no rounds).
    const int nr_full = rounds_to(t);
    std::vector<SegBlock> padding;
    size_t i = 0;
    while (i < order.size()) {
      const int c = order[i]->c;
      if (c >= t) {
        const uint32_t sl = add_slot(*order[i]);
        for (uint32_t b = 0; b < (1u << (c - t)); ++b) {
          SegBlock B{};
          B.first_slot = sl;
          B.blk_in_seg = b;
          B.log2cap = uint8_t(c);
          B.nrounds = uint8_t(nr_full);
          B.final_pass = (c == t) ? 1 : 0;
          B.fill = 1;
          if (c > t && (uint64_t(b) << t) >= order[i]->len) {
            B.nrounds = 0;
            padding.push_back(B);
          } else {
            bt.blocks.push_back(B);
          }
        }
        ++i;
      } else {
        const uint32_t per = 1u << (t - c);
        const uint32_t first = uint32_t(bt.slots.size() - slot0);
        uint32_t taken = 0;
        while (i < order.size() && order[i]->c == c && taken < per) {
          add_slot(*order[i]);
          ++taken;
          ++i;
        }
        for (; taken < per; ++taken) add_empty();
        SegBlock B{};
        B.first_slot = first;
        B.log2cap = uint8_t(c);
        B.nrounds = uint8_t(rounds_to(c));
        B.final_pass = 1;
        B.fill = 1;
        bt.blocks.push_back(B);
      }
    }
    const uint32_t tile_blocks = uint32_t(bt.blocks.size() - block0);
    if (tile_blocks > 0) {
      Launch L{};
      L.kind = PASS_TILE;
      L.loge = e;
      L.variant = pick(PASS_TILE);
      L.threads = 1u << (t - e);
      L.smem = size_t(elem_bytes(kk, has_vals)) * smem_words(1u << t);
      L.P.b = L.P.c = L.P.w0 = uint32_t(t);
      L.P.log2cap = uint32_t(t);
      L.P.map_in = map_in;
      const std::vector<Round> rs = shfl ? tile_rounds_shfl(t, e) : tile_rounds(t, e);
      L.P.nrounds = uint32_t(rs.size());
      for (size_t r = 0; r < rs.size(); ++r) L.P.rounds[r] = rs[r];
      const void* fn = shfl ? tile_shfl_seg_kernel_u32(has_vals, e, t, L.variant).fn
                            : fixed_kernel_fn(kk, has_vals, e, t, L.variant, false);
      L.fixed = fn != nullptr;
      L.shfl = shfl;
      if (L.fixed) {
        L.P.nblocks = tile_blocks;
        L.grid = uint32_t(std::min<int>(int(tile_blocks), occupancy_grid(fn, int(L.threads), L.smem)));
        bt.persistent.push_back(int(bt.launches.size()));
      } else {
        L.grid = tile_blocks;
      }
      bt.launches.push_back(L);
      bt.block_off.push_back(block0);
      bt.slot_off.push_back(slot0);
    }
    if (!padding.empty()) {
      Launch L{};
      L.kind = PASS_TILE;
      L.fixed = false;
      L.variant = pick(PASS_TILE);
      L.threads = kPaddingThreads;
      L.grid = uint32_t(padding.size());
      L.P.b = L.P.c = L.P.w0 = uint32_t(t);
      L.P.log2cap = uint32_t(t);
      L.P.map_in = map_in;
      L.P.nrounds = 0;  // no network: the launch writes the sentinel result
      bt.block_off.push_back(bt.blocks.size());
      bt.slot_off.push_back(slot0);
      bt.blocks.insert(bt.blocks.end(), padding.begin(), padding.end());
      bt.launches.push_back(L);
    }
    // capacities 2 .. 2^(e-1): one thread sorts a whole segment in registers
    for (int c = e - 1; c >= 1; --c) {
      std::vector<const BatchSeg*> cls;
      for (const BatchSeg& s : segs)
        if (s.c == c) cls.push_back(&s);
      if (cls.empty()) continue;
      const size_t bfirst = bt.blocks.size();
      const uint32_t per = 1u << kTinyThreadsLog2;
      for (size_t j = 0; j < cls.size(); j += per) {
        const uint32_t first = uint32_t(bt.slots.size() - slot0);
        for (size_t q = 0; q < per; ++q) {
          if (j + q < cls.size())
            add_slot(*cls[j + q]);
          else
            add_empty();
        }
        SegBlock B{};
        B.first_slot = first;
        B.log2cap = uint8_t(c);
        B.nrounds = 1;
        B.final_pass = 1;
        B.fill = 1;
        bt.blocks.push_back(B);
      }
      Launch L{};
      L.kind = PASS_TILE;
      L.fixed = false;
      L.loge = c;
      L.variant = pick(PASS_TILE);
      L.threads = 1u << kTinyThreadsLog2;
      L.grid = uint32_t(bt.blocks.size() - bfirst);
      L.P.b = L.P.c = L.P.w0 = uint32_t(c + kTinyThreadsLog2);
      L.P.log2cap = uint32_t(c);
      L.P.map_in = map_in;
      L.P.nrounds = 1;
      L.P.rounds[0] = tile_rounds(c, c)[0];
      bt.launches.push_back(L);
      bt.block_off.push_back(bfirst);
      bt.slot_off.push_back(slot0);
    }
    return DARM_OK;
  }

  // stage p > t for every segment still in it
  const int p = phase;
  std::vector<const BatchSeg*> act;
  for (const BatchSeg& s : segs)
    if (s.c >= p) act.push_back(&s);
  if (act.empty()) return DARM_OK;
  std::vector<uint32_t> sl(act.size());
  for (size_t j = 0; j < act.size(); ++j) sl[j] = add_slot(*act[j]);
  std::vector<Launch> shape;
  Tuning tp = tn;
  tp.tma = 0;  // the whole-array shapes; merges are given the bulk-copy kernel below
  if (!plan_array(shape, kk, has_vals, p, tp, variant, 0, 0, g_ctx.smem_limit))
    return DARM_ERR_INVALID_ARG;
  // Stage p's comparators stay inside aligned blocks of 2^p elements.  One
  // that starts at or beyond a segment's real length held only sentinels
  // after the tile pass (whose padding-only blocks store them) and keeps
  // them through every stage below the one whose block reaches the length:
  // its compare-exchanges meet equal elements and, the swaps being strict,
  // move nothing.  A block of a pass of stage p inside such a 2^p block is
  // left out of the launch, unless the pass is the segment's last (which
  // also maps the keys back for output).  A pass block's elements share
  // their index bits >= p (its own bits, the window bits and the bits
  // between them all lie below p), so the block's first element decides.
  for (const Launch& L0 : shape) {
    if (L0.kind == PASS_TILE || L0.P.rounds[0].p != p) continue;
    const size_t bfirst = bt.blocks.size();
    const uint32_t nmid = L0.P.w0 - L0.P.c;
    for (size_t j = 0; j < act.size(); ++j) {
      const bool final_pass = (L0.kind == PASS_MERGE && act[j]->c == p);
      for (uint32_t b = 0; b < (1u << (act[j]->c - int(L0.P.b))); ++b) {
        const uint64_t g0 = (uint64_t(b & ((1u << nmid) - 1u)) << L0.P.c) |
                            (uint64_t(b >> nmid) << (L0.P.w0 + L0.P.s));
        if (!final_pass && ((g0 >> p) << p) >= act[j]->len) continue;
        SegBlock B{};
        B.first_slot = sl[j];
        B.blk_in_seg = b;
        B.log2cap = uint8_t(act[j]->c);
        B.nrounds = uint8_t(L0.P.nrounds);
        B.final_pass = final_pass ? 1 : 0;
        B.fill = 0;
        bt.blocks.push_back(B);
      }
    }
    if (bt.blocks.size() == bfirst) continue;  // every block of the pass is padding
    Launch L = L0;
    // the window kernels with compile-time shapes address whole arrays only
    L.win2 = false;
    L.win2t = false;
    L.win1 = false;
    L.tma = 0;
    L.mshfl = false;
    L.grid = uint32_t(bt.blocks.size() - bfirst);
    size_t tma_smem = 0;
    if (L0.kind == PASS_MERGE && kk == KEY_U32 && (tn.tma == 1 || tn.tma == 2)) {
      // merge blocks are whole tiles of one segment: the persistent
      // bulk-copy merge streams them in, finding each in the table
      const KernelEntry te =
          tma_merge_kernel_u32(has_vals, L0.loge, int(L0.P.b), tn.tma, L.variant, &tma_smem);
      if (te.fn != nullptr && tma_smem <= g_ctx.smem_limit && int(L.threads) == te.max_threads) {
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, te.fn, int(L.threads), tma_smem) !=
                cudaSuccess ||
            per_sm < 1) {
          cudaGetLastError();
          per_sm = 1;
        }
        L.tma = tn.tma;
        L.smem = tma_smem;
        L.P.nblocks = L.grid;
        L.grid = std::min<uint32_t>(L.grid, uint32_t(std::max(1, g_ctx.sms) * per_sm));
      }
    }
    L.P.log2cap = 0;
    L.P.map_in = map_in;
    L.P.map_out = 0;
    bt.launches.push_back(L);
    bt.block_off.push_back(bfirst);
    bt.slot_off.push_back(slot0);
  }
  return DARM_OK;
}

void batch_bind(BatchTables& bt, SegBlock* d_blocks, SegSlot* d_slots, unsigned int* d_counters) {
  for (size_t i = 0; i < bt.launches.size(); ++i) {
    Launch& L = bt.launches[i];
    L.P.blocks = d_blocks + bt.block_off[i];
    L.P.slots = d_slots + bt.slot_off[i];
    L.P.work_counter = nullptr;
  }
  for (size_t k = 0; k < bt.persistent.size(); ++k)
    bt.launches[size_t(bt.persistent[k])].P.work_counter = d_counters + k;
}

}  // namespace darm
