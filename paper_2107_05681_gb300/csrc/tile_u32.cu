// tile_u32.cu - table of the compile-time-schedule tile and merge kernels for
// uint32_t keys (instantiated in tile_u32_keys16.cu, tile_u32_keys32.cu and
// tile_u32_pairs.cu) and the schedules the planner checks them against.
#include "tile_entry.cuh"

namespace darm {
namespace {

struct Combo {
  bool v;
  int loge, logt;
};
constexpr Combo kCombos[] = {{false, 4, 12}, {false, 4, 13}, {false, 4, 14}, {true, 4, 12},
                             {true, 4, 13}, {false, 5, 14}, {false, 5, 13}};

}  // namespace

KernelEntry tile_kernel_u32(bool has_vals, int loge, int logt, int var, bool merge) {
  if (has_vals) return tile_kernel_u32_pairs(loge, logt, var, merge);
  if (loge == 4) return tile_kernel_u32_keys16(logt, var, merge);
  if (loge == 5) return tile_kernel_u32_keys32(logt, var, merge);
  return KernelEntry{nullptr, 0};
}

void for_each_tile_kernel_u32(void (*fn)(const void*, void*), void* ctx) {
  for (const Combo& c : kCombos)
    for (int var = 0; var < 2; ++var)
      for (int merge = 0; merge < 2; ++merge) {
        KernelEntry e = tile_kernel_u32(c.v, c.loge, c.logt, var, merge != 0);
        if (e.fn) fn(e.fn, ctx);
      }
}

// The compile-time schedules, exported so that the planner can check them
// against its own round lists.
int fixed_schedule_rounds(int logt, int loge, bool merge, SRound* out, int cap) {
  auto copy = [&](const auto& sch, int n) {
    for (int i = 0; i < n && i < cap; ++i) out[i] = sch.r[i];
    return n;
  };
  if (loge == 4 && logt == 12)
    return merge ? copy(Schedule<12, 4, true>::value, Schedule<12, 4, true>::count)
                 : copy(Schedule<12, 4, false>::value, Schedule<12, 4, false>::count);
  if (loge == 4 && logt == 13)
    return merge ? copy(Schedule<13, 4, true>::value, Schedule<13, 4, true>::count)
                 : copy(Schedule<13, 4, false>::value, Schedule<13, 4, false>::count);
  if (loge == 4 && logt == 14)
    return merge ? copy(Schedule<14, 4, true>::value, Schedule<14, 4, true>::count)
                 : copy(Schedule<14, 4, false>::value, Schedule<14, 4, false>::count);
  if (loge == 5 && logt == 13)
    return merge ? copy(Schedule<13, 5, true>::value, Schedule<13, 5, true>::count)
                 : copy(Schedule<13, 5, false>::value, Schedule<13, 5, false>::count);
  if (loge == 5 && logt == 14)
    return merge ? copy(Schedule<14, 5, true>::value, Schedule<14, 5, true>::count)
                 : copy(Schedule<14, 5, false>::value, Schedule<14, 5, false>::count);
  if (loge == 3 && logt == 12)
    return merge ? copy(Schedule<12, 3, true>::value, Schedule<12, 3, true>::count)
                 : copy(Schedule<12, 3, false>::value, Schedule<12, 3, false>::count);
  return -1;
}

}  // namespace darm
