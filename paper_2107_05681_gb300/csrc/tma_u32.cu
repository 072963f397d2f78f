// tma_u32.cu - instantiations of the bulk-copy-prefetching merge passes for
// uint32_t keys: dense staging buffers (tma_merge.cuh, 1 or 2 buffers) and
// the in-place swizzled form with bulk tensor stores (tma_merge_swz.cuh,
// "3 buffers": keys alone, or keys with a payload in two buffer halves).
#include "kernel_table.h"
#include "tma_merge.cuh"
#include "tma_merge_swz.cuh"

namespace darm {
namespace {

template <bool V, int LOGE, int LOGT, int NS, bool SH = false>
KernelEntry mentry(int var, size_t* smem_bytes) {
  constexpr int MT = 1 << (LOGT - LOGE);
  if (smem_bytes) *smem_bytes = TmaMergeSmem<uint32_t, V, LOGT, NS>::kBytes;
  if (var)
    return KernelEntry{reinterpret_cast<const void*>(
                           &darm_merge_tma_kernel<uint32_t, V, LOGE, LOGT, NS, 1, MT, SH>),
                       MT};
  return KernelEntry{reinterpret_cast<const void*>(
                         &darm_merge_tma_kernel<uint32_t, V, LOGE, LOGT, NS, 0, MT, SH>),
                     MT};
}

template <int LOGT>
KernelEntry swz_entry(size_t* smem_bytes) {
  if (smem_bytes) *smem_bytes = SwzMergeSmem<LOGT>::kBytes;
  return KernelEntry{reinterpret_cast<const void*>(&darm_merge_swz_kernel<LOGT>), 1 << (LOGT - 5)};
}

template <int LOGT, int NB = kSwzBuffers>
KernelEntry swz_kv_entry(size_t* smem_bytes) {
  if (smem_bytes) *smem_bytes = SwzKvSmem<LOGT, NB>::kBytes;
  return KernelEntry{reinterpret_cast<const void*>(&darm_merge_swz_kv_kernel<LOGT, NB>),
                     1 << (LOGT - 4)};
}

template <bool V, int LOGE, int LOGT>
KernelEntry mpick(int ns, int var, size_t* smem_bytes) {
  if (ns == 1) return mentry<V, LOGE, LOGT, 1>(var, smem_bytes);
  if (ns == 2) return mentry<V, LOGE, LOGT, 2>(var, smem_bytes);
  return KernelEntry{nullptr, 0};
}

}  // namespace

KernelEntry tma_merge_shfl_kernel_u32(int loge, int logt, int ns, int var, size_t* smem_bytes) {
  if (loge == 5 && logt == 14 && ns == 2) return mentry<false, 5, 14, 2, true>(var, smem_bytes);
  if (loge == 5 && logt == 13 && ns == 2) return mentry<false, 5, 13, 2, true>(var, smem_bytes);
  return KernelEntry{nullptr, 0};
}

KernelEntry tma_merge_kernel_u32(bool has_vals, int loge, int logt, int ns, int var,
                                 size_t* smem_bytes) {
  if (ns == 4) {  // in place, two buffers per CTA (more CTAs per SM)
    if (has_vals && loge == 4 && logt == 12) return swz_kv_entry<12, 2>(smem_bytes);
    return KernelEntry{nullptr, 0};
  }
  if (ns == 3) {  // one form: the direction is uniform per tile
    if (!has_vals && loge == 5 && logt == 14) return swz_entry<14>(smem_bytes);
    if (!has_vals && loge == 5 && logt == 13) return swz_entry<13>(smem_bytes);
    if (has_vals && loge == 4 && logt == 12) return swz_kv_entry<12>(smem_bytes);
    if (has_vals && loge == 4 && logt == 13) return swz_kv_entry<13>(smem_bytes);
    return KernelEntry{nullptr, 0};
  }
  if (has_vals && loge == 4 && logt == 12) return mpick<true, 4, 12>(ns, var, smem_bytes);
  if (has_vals && loge == 4 && logt == 13) return mpick<true, 4, 13>(ns, var, smem_bytes);
  if (!has_vals && loge == 5 && logt == 13) return mpick<false, 5, 13>(ns, var, smem_bytes);
  if (!has_vals && loge == 5 && logt == 14) return mpick<false, 5, 14>(ns, var, smem_bytes);
  if (!has_vals && loge == 4 && logt == 14) return mpick<false, 4, 14>(ns, var, smem_bytes);
  return KernelEntry{nullptr, 0};
}

namespace {

// One warp waits on an mbarrier that nothing ever completes, with the bounded
// wait of the bulk-copy passes: the wait must give up and latch the timeout.
__global__ void darm_bounded_wait_check_kernel(int* status) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = smem_addr(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (!mbar_wait_bounded(b, 0u) && threadIdx.x == 0) atomicOr(status, int(kStatusTimeout));
}

}  // namespace

cudaError_t launch_bounded_wait_check(int* status, cudaStream_t s) {
  void* args[] = {&status};
  return cudaLaunchKernel(reinterpret_cast<const void*>(&darm_bounded_wait_check_kernel), dim3(1),
                          dim3(32), args, 0, s);
}

void for_each_tma_kernel_u32(void (*fn)(const void*, void*), void* ctx) {
  for (int var = 0; var < 2; ++var)
    for (int ns = 1; ns <= 2; ++ns) {
      fn(tma_merge_kernel_u32(true, 4, 12, ns, var, nullptr).fn, ctx);
      fn(tma_merge_kernel_u32(true, 4, 13, ns, var, nullptr).fn, ctx);
      fn(tma_merge_kernel_u32(false, 5, 13, ns, var, nullptr).fn, ctx);
      fn(tma_merge_kernel_u32(false, 5, 14, ns, var, nullptr).fn, ctx);
      fn(tma_merge_kernel_u32(false, 4, 14, ns, var, nullptr).fn, ctx);
    }
  fn(tma_merge_kernel_u32(false, 5, 14, 3, 0, nullptr).fn, ctx);
  fn(tma_merge_kernel_u32(false, 5, 13, 3, 0, nullptr).fn, ctx);
  fn(tma_merge_kernel_u32(true, 4, 12, 3, 0, nullptr).fn, ctx);
  fn(tma_merge_kernel_u32(true, 4, 13, 3, 0, nullptr).fn, ctx);
  fn(tma_merge_kernel_u32(true, 4, 12, 4, 0, nullptr).fn, ctx);
  for (int var = 0; var < 2; ++var) {
    fn(tma_merge_shfl_kernel_u32(5, 14, 2, var, nullptr).fn, ctx);
    fn(tma_merge_shfl_kernel_u32(5, 13, 2, var, nullptr).fn, ctx);
  }
}

}  // namespace darm
