// kernels_u64.cu - instantiations of the pass kernel for uint64_t keys.
#include "kernel_table.h"
#include "pass_kernel.cuh"

namespace darm {
namespace {

template <bool V, int LOGE, int VAR>
KernelEntry entry() {
  constexpr int MT = max_threads_for<uint64_t, V, LOGE>();
  return KernelEntry{reinterpret_cast<const void*>(&darm_pass_kernel<uint64_t, V, LOGE, VAR, MT>), MT};
}

template <bool V, int VAR>
KernelEntry by_loge(int loge) {
  switch (loge) {
    case 1: return entry<V, 1, VAR>();
    case 2: return entry<V, 2, VAR>();
    case 3: return entry<V, 3, VAR>();
    case 4: return entry<V, 4, VAR>();
    case 5: return entry<V, 5, VAR>();
    default: return KernelEntry{nullptr, 0};
  }
}

}  // namespace

KernelEntry kernel_u64(bool has_vals, int loge, int var) {
  if (has_vals) return var ? by_loge<true, 1>(loge) : by_loge<true, 0>(loge);
  return var ? by_loge<false, 1>(loge) : by_loge<false, 0>(loge);
}

void for_each_kernel_u64(void (*fn)(const void*, void*), void* ctx) {
  for (int v = 0; v < 2; ++v)
    for (int var = 0; var < 2; ++var)
      for (int loge = 1; loge <= 5; ++loge) {
        KernelEntry e = kernel_u64(v != 0, loge, var);
        if (e.fn) fn(e.fn, ctx);
      }
}

}  // namespace darm
