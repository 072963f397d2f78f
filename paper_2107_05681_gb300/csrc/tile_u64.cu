// tile_u64.cu - compile-time-schedule tile and merge kernels for uint64_t keys.
#include "kernel_table.h"
#include "tile_kernel.cuh"

namespace darm {
namespace {

template <bool V, int LOGE, int LOGT, int VAR, bool MERGE>
KernelEntry tentry() {
  constexpr int MT = 1 << (LOGT - LOGE);  // one tile per CTA
  static_assert((1 << (LOGT - LOGE)) <= MT, "tile too large for the block size");
  return KernelEntry{
      reinterpret_cast<const void*>(&darm_tile_kernel<uint64_t, V, LOGE, LOGT, VAR, MERGE, MT>), MT};
}

template <bool V, int LOGE, int LOGT>
KernelEntry tpick(int var, bool merge) {
  if (merge) return var ? tentry<V, LOGE, LOGT, 1, true>() : tentry<V, LOGE, LOGT, 0, true>();
  return var ? tentry<V, LOGE, LOGT, 1, false>() : tentry<V, LOGE, LOGT, 0, false>();
}

struct Combo {
  bool v;
  int loge, logt;
};
constexpr Combo kCombos[] = {{false, 4, 12}, {false, 4, 13}, {true, 3, 12}};

}  // namespace

KernelEntry tile_kernel_u64(bool has_vals, int loge, int logt, int var, bool merge) {
  if (!has_vals && loge == 4 && logt == 12) return tpick<false, 4, 12>(var, merge);
  if (!has_vals && loge == 4 && logt == 13) return tpick<false, 4, 13>(var, merge);
  if (has_vals && loge == 3 && logt == 12) return tpick<true, 3, 12>(var, merge);
  return KernelEntry{nullptr, 0};
}

void for_each_tile_kernel_u64(void (*fn)(const void*, void*), void* ctx) {
  for (const Combo& c : kCombos)
    for (int var = 0; var < 2; ++var)
      for (int merge = 0; merge < 2; ++merge) {
        KernelEntry e = tile_kernel_u64(c.v, c.loge, c.logt, var, merge != 0);
        if (e.fn) fn(e.fn, ctx);
      }
}

}  // namespace darm
