// kernel_table.h - host-side lookup of the compiled pass-kernel
// instantiations (one per key type, payload flag, elements per thread and
// variant).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace darm {

struct KernelEntry {
  const void* fn;   // __global__ function address, or nullptr if not built
  int max_threads;  // block size the instantiation was compiled for
};

// loge: log2 elements per thread (1..5); var: 0 divergent, 1 melded.
KernelEntry kernel_u32(bool has_vals, int loge, int var);
KernelEntry kernel_u64(bool has_vals, int loge, int var);

// Tile / merge kernels with a compile-time schedule for one tile size
// (tile_kernel.cuh); {nullptr, 0} when that combination is not built.
KernelEntry tile_kernel_u32(bool has_vals, int loge, int logt, int var, bool merge);
KernelEntry tile_kernel_u64(bool has_vals, int loge, int logt, int var, bool merge);

// Tile passes whose stages 2E .. 32E run across lanes with shuffles
// (tile_shfl_kernel.cuh), whole arrays only; {nullptr, 0} when not built.
KernelEntry tile_shfl_kernel_u32(bool has_vals, int loge, int logt, int var);
// The same pass for batched segments (block tables, persistent launch).
KernelEntry tile_shfl_seg_kernel_u32(bool has_vals, int loge, int logt, int var);

// Persistent merge kernels that prefetch tiles with bulk copies
// (tma_merge.cuh); smem_bytes receives the dynamic shared memory they need.
KernelEntry tma_merge_kernel_u32(bool has_vals, int loge, int logt, int ns, int var,
                                 size_t* smem_bytes);
// The same merge in two rounds, its lower layers across lanes by shuffles
// (keys only).
KernelEntry tma_merge_shfl_kernel_u32(int loge, int logt, int ns, int var, size_t* smem_bytes);

// Two-window passes with a compile-time shape (window2_kernel.cuh): E =
// 2^loge, c low consecutive-element bits.
KernelEntry window2_kernel_u32(bool has_vals, int loge, int c, int var);
// One-window passes with a compile-time shape (window1_kernel.cuh): 2^c
// threads, E = 2^loge; nullptr where none was built.
KernelEntry window1_kernel(bool u64, bool has_vals, int loge, int c);
KernelEntry window2_kernel_u64(bool has_vals, int loge, int c, int var);
// The two-window pass of 32-bit keys, 16 consecutive elements per block
// (window2_tma.cuh): keys alone with 32 per thread, or with a payload with 16
// pairs per thread; persistent, blocks streamed through three shared-memory
// buffers by TMA tensor copies.
KernelEntry window2_tma_kernel_u32(bool has_vals, size_t* smem_bytes);

// Call fn(kernel address, ctx) for every instantiation (used to configure
// shared-memory limits once per device).
void for_each_kernel_u32(void (*fn)(const void*, void*), void* ctx);
void for_each_kernel_u64(void (*fn)(const void*, void*), void* ctx);
void for_each_tile_kernel_u32(void (*fn)(const void*, void*), void* ctx);
void for_each_tile_kernel_u64(void (*fn)(const void*, void*), void* ctx);
// Enqueue the bounded-wait check (tma_u32.cu): one warp waits on an
// mbarrier nothing completes and latches the timeout status in `status`.
cudaError_t launch_bounded_wait_check(int* status, cudaStream_t s);
void for_each_tma_kernel_u32(void (*fn)(const void*, void*), void* ctx);
void for_each_tile_shfl_kernel_u32(void (*fn)(const void*, void*), void* ctx);
void for_each_window2_kernel(void (*fn)(const void*, void*), void* ctx);

}  // namespace darm
