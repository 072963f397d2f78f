// batch.h - launch lists and block tables for batches of independent
// power-of-two segments (used by the segmented sort and the serving loop).
//
// A batch is sorted phase by phase:
//   phase 0      the tile pass of every segment (capacity >= 2): segments
//                larger than a tile get one block per tile, smaller ones are
//                packed 2^(t - c) per block, capacities 2..2^(e-1) are sorted
//                in registers by one thread each;
//   phase p > t  stage 2^p of every segment of capacity >= 2^p: its window
//                passes and its merge pass.
// The first phase writes sentinels past each real length and complements the
// keys of descending segments; the phase that completes a segment undoes the
// key maps.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "plan.h"

namespace darm {

struct BatchSeg {
  uint64_t base;  // first element
  uint32_t len;   // real elements
  int c;          // log2 capacity
  bool desc;
};

struct BatchTables {
  std::vector<SegSlot> slots;
  std::vector<SegBlock> blocks;
  std::vector<Launch> launches;
  // per launch: index of its first block / slot in the tables
  std::vector<size_t> block_off, slot_off;
  // launches that take blocks from a global counter (one counter each, in
  // this order); the caller zeroes the counters before the launches run
  std::vector<int> persistent;
};

// Append the launches of `phase` for `segs` to bt.  map_in is applied to
// every key on its first load (kMapF32 for float keys); descending segments
// add the complement.  Returns a darm_status.
int batch_append(BatchTables& bt, KeyKind kk, bool has_vals, const Tuning& tn, int variant,
                 const std::vector<BatchSeg>& segs, int phase, uint32_t map_in);

// Point every launch at the uploaded tables and counters.
void batch_bind(BatchTables& bt, SegBlock* d_blocks, SegSlot* d_slots, unsigned int* d_counters);

// The tile size and elements per thread a batch of these segments uses.
Tuning batch_tuning(KeyKind kk, bool has_vals, int cmax);

}  // namespace darm
