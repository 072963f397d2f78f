// window2.cu - instantiations of the one- and two-window pass kernels
// (window1_kernel.cuh, window2_kernel.cuh) and of the two-window pass that
// streams its blocks through shared memory with TMA (window2_tma.cuh).
#include "kernel_table.h"
#include "window1_kernel.cuh"
#include "window2_kernel.cuh"
#include "window2_tma.cuh"

namespace darm {
namespace {

template <typename K, bool V, int LOGE, int C>
KernelEntry wentry(int var) {
  constexpr int MT = 1 << (C + LOGE);
  if (var)
    return KernelEntry{reinterpret_cast<const void*>(&darm_window2_kernel<K, V, LOGE, C, 1, MT>), MT};
  return KernelEntry{reinterpret_cast<const void*>(&darm_window2_kernel<K, V, LOGE, C, 0, MT>), MT};
}

template <typename K, bool V, int LOGE, int C>
KernelEntry w1entry() {
  constexpr int MT = 1 << C;
  return KernelEntry{reinterpret_cast<const void*>(&darm_window1_kernel<K, V, LOGE, C, MT>), MT};
}

}  // namespace

KernelEntry window1_kernel(bool u64, bool has_vals, int loge, int c) {
  if (c != 8) return KernelEntry{nullptr, 0};
  if (!u64 && has_vals && loge == 4) return w1entry<uint32_t, true, 4, 8>();
  if (!u64 && !has_vals && loge == 5) return w1entry<uint32_t, false, 5, 8>();
  if (!u64 && !has_vals && loge == 4) return w1entry<uint32_t, false, 4, 8>();
  if (u64 && has_vals && loge == 3) return w1entry<uint64_t, true, 3, 8>();
  if (u64 && !has_vals && loge == 4) return w1entry<uint64_t, false, 4, 8>();
  return KernelEntry{nullptr, 0};
}

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

KernelEntry window2_tma_kernel_u32(bool has_vals, size_t* smem_bytes) {
  if (has_vals) {
    if (smem_bytes) *smem_bytes = W2t<true>::kBytes;
    return KernelEntry{reinterpret_cast<const void*>(&darm_window2_tma_kernel<true>), W2t<true>::kThreads};
  }
  if (smem_bytes) *smem_bytes = W2t<false>::kBytes;
  return KernelEntry{reinterpret_cast<const void*>(&darm_window2_tma_kernel<false>), W2t<false>::kThreads};
}

void for_each_window2_kernel(void (*fn)(const void*, void*), void* ctx) {
  fn(window2_tma_kernel_u32(false, nullptr).fn, ctx);
  fn(window2_tma_kernel_u32(true, nullptr).fn, ctx);
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
