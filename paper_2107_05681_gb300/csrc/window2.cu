// window2.cu - instantiations of the two-window pass kernel.
#include "kernel_table.h"
#include "window2_kernel.cuh"

namespace darm {
namespace {

template <typename K, bool V, int LOGE, int C>
KernelEntry wentry(int var) {
  constexpr int MT = 1 << (C + LOGE);
  if (var)
    return KernelEntry{reinterpret_cast<const void*>(&darm_window2_kernel<K, V, LOGE, C, 1, MT>), MT};
  return KernelEntry{reinterpret_cast<const void*>(&darm_window2_kernel<K, V, LOGE, C, 0, MT>), MT};
}

}  // namespace

KernelEntry window2_kernel_u32(bool has_vals, int loge, int c, int var) {
  if (has_vals && loge == 4 && c == 4) return wentry<uint32_t, true, 4, 4>(var);
  if (has_vals && loge == 4 && c == 5) return wentry<uint32_t, true, 4, 5>(var);
  if (!has_vals && loge == 5 && c == 4) return wentry<uint32_t, false, 5, 4>(var);
  if (!has_vals && loge == 4 && c == 5) return wentry<uint32_t, false, 4, 5>(var);
  return KernelEntry{nullptr, 0};
}

KernelEntry window2_kernel_u64(bool has_vals, int loge, int c, int var) {
  if (has_vals && loge == 3 && c == 5) return wentry<uint64_t, true, 3, 5>(var);
  if (!has_vals && loge == 4 && c == 4) return wentry<uint64_t, false, 4, 4>(var);
  return KernelEntry{nullptr, 0};
}

void for_each_window2_kernel(void (*fn)(const void*, void*), void* ctx) {
  for (int var = 0; var < 2; ++var) {
    fn(window2_kernel_u32(true, 4, 4, var).fn, ctx);
    fn(window2_kernel_u32(true, 4, 5, var).fn, ctx);
    fn(window2_kernel_u32(false, 5, 4, var).fn, ctx);
    fn(window2_kernel_u32(false, 4, 5, var).fn, ctx);
    fn(window2_kernel_u64(true, 3, 5, var).fn, ctx);
    fn(window2_kernel_u64(false, 4, 4, var).fn, ctx);
  }
}

}  // namespace darm
