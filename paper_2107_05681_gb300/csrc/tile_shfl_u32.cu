// tile_shfl_u32.cu - instantiations of the tile pass with shuffle stages
// (tile_shfl_kernel.cuh) for uint32_t keys, and the schedule the planner
// checks them against.
#include "kernel_table.h"
#include "tile_shfl_kernel.cuh"

namespace darm {
namespace {

template <bool V, int LOGE, int LOGT, bool SEG = false>
KernelEntry shfl_entry(int var) {
  constexpr int MT = 1 << (LOGT - LOGE);
  if (var)
    return KernelEntry{reinterpret_cast<const void*>(
                           &darm_tile_shfl_kernel<uint32_t, V, LOGE, LOGT, 1, MT, SEG>),
                       MT};
  return KernelEntry{reinterpret_cast<const void*>(
                         &darm_tile_shfl_kernel<uint32_t, V, LOGE, LOGT, 0, MT, SEG>),
                     MT};
}

template <int LOGE, int LOGT>
int copy_schedule(SRound* out, int cap) {
  using S = ShflSchedule<LOGT, LOGE>;
  for (int i = 0; i < S::count && i < cap; ++i) out[i] = S::value.r[i];
  return S::count;
}

}  // namespace

KernelEntry tile_shfl_kernel_u32(bool has_vals, int loge, int logt, int var) {
  if (!has_vals && loge == 5 && logt == 15) return shfl_entry<false, 5, 15>(var);
  if (!has_vals && loge == 5 && logt == 14) return shfl_entry<false, 5, 14>(var);
  if (!has_vals && loge == 5 && logt == 13) return shfl_entry<false, 5, 13>(var);
  if (!has_vals && loge == 4 && logt == 12) return shfl_entry<false, 4, 12>(var);
  if (has_vals && loge == 4 && logt == 12) return shfl_entry<true, 4, 12>(var);
  if (has_vals && loge == 4 && logt == 13) return shfl_entry<true, 4, 13>(var);
  return KernelEntry{nullptr, 0};
}

// Batched segments (block tables, persistent launch): the shapes the batch
// tunings use.
KernelEntry tile_shfl_seg_kernel_u32(bool has_vals, int loge, int logt, int var) {
  if (has_vals && loge == 4 && logt == 13) return shfl_entry<true, 4, 13, true>(var);
  if (has_vals && loge == 4 && logt == 12) return shfl_entry<true, 4, 12, true>(var);
  if (!has_vals && loge == 5 && logt == 14) return shfl_entry<false, 5, 14, true>(var);
  return KernelEntry{nullptr, 0};
}

int shfl_schedule_rounds(int logt, int loge, SRound* out, int cap) {
  if (loge == 5 && logt == 15) return copy_schedule<5, 15>(out, cap);
  if (loge == 5 && logt == 14) return copy_schedule<5, 14>(out, cap);
  if (loge == 5 && logt == 13) return copy_schedule<5, 13>(out, cap);
  if (loge == 4 && logt == 12) return copy_schedule<4, 12>(out, cap);
  if (loge == 4 && logt == 13) return copy_schedule<4, 13>(out, cap);
  return -1;
}

void for_each_tile_shfl_kernel_u32(void (*fn)(const void*, void*), void* ctx) {
  for (int var = 0; var < 2; ++var) {
    fn(tile_shfl_kernel_u32(false, 5, 15, var).fn, ctx);
    fn(tile_shfl_kernel_u32(false, 5, 14, var).fn, ctx);
    fn(tile_shfl_kernel_u32(false, 5, 13, var).fn, ctx);
    fn(tile_shfl_kernel_u32(false, 4, 12, var).fn, ctx);
    fn(tile_shfl_seg_kernel_u32(true, 4, 13, var).fn, ctx);
    fn(tile_shfl_seg_kernel_u32(true, 4, 12, var).fn, ctx);
    fn(tile_shfl_seg_kernel_u32(false, 5, 14, var).fn, ctx);
    fn(tile_shfl_kernel_u32(true, 4, 12, var).fn, ctx);
    fn(tile_shfl_kernel_u32(true, 4, 13, var).fn, ctx);
  }
}

}  // namespace darm
