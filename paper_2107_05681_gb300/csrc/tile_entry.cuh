// tile_entry.cuh - kernel-table entries of the compile-time-schedule tile and
// merge kernels; each tile_u32_*.cu file instantiates one group of shapes so
// that the groups compile in parallel.
#pragma once

#include "kernel_table.h"
#include "tile_kernel.cuh"

namespace darm {

template <typename K, bool V, int LOGE, int LOGT, int VAR, bool MERGE>
KernelEntry tile_entry() {
  constexpr int MT = 1 << (LOGT - LOGE);  // one tile per CTA
  return KernelEntry{
      reinterpret_cast<const void*>(&darm_tile_kernel<K, V, LOGE, LOGT, VAR, MERGE, MT>), MT};
}

template <typename K, bool V, int LOGE, int LOGT>
KernelEntry tile_pick(int var, bool merge) {
  if (merge) return var ? tile_entry<K, V, LOGE, LOGT, 1, true>() : tile_entry<K, V, LOGE, LOGT, 0, true>();
  return var ? tile_entry<K, V, LOGE, LOGT, 1, false>() : tile_entry<K, V, LOGE, LOGT, 0, false>();
}

// The groups (defined in tile_u32_keys16.cu, tile_u32_keys32.cu,
// tile_u32_pairs.cu); nullptr entries for shapes a group does not hold.
KernelEntry tile_kernel_u32_keys16(int logt, int var, bool merge);
KernelEntry tile_kernel_u32_keys32(int logt, int var, bool merge);
KernelEntry tile_kernel_u32_pairs(int loge, int logt, int var, bool merge);

}  // namespace darm
