// oddeven.cu - Batcher's odd-even merge sort network on one thread block, in
// a divergent and a melded form.
//
// The paper's PCM benchmark (Section VI-A) is a parallel sort built on
// Batcher's odd-even merge sort; like the bitonic kernel of Fig. 1 it runs a
// fixed comparator network whose two sides (here: the lower and the upper
// element of a compare-exchange) are near-identical instruction sequences
// that diverge within a warp on thread-index bits.  This kernel sorts up to
// 4096 uint32 keys (with an optional uint32 payload) in shared memory; a
// grid of such blocks sorts an array bucket by bucket, the way the paper's
// benchmarks sort their 2^26-element input (one bucket per thread block).
//
// Network (ascending, strict swaps): for p = 1, 2, 4, ... < n and
// k = p, p/2, ..., 1, element x is
//   - the lower end of a comparator (x, x + k) when k == p and bit p of x is
//     clear, or when k < p, bit k of x is set and x + k stays inside x's
//     block of 2p elements;
//   - the upper end of (x - k, x) when k == p and bit p of x is set, or when
//     k < p, bit k of x is clear and x - k stays inside the block;
//   - idle otherwise.
// Every thread updates the elements it owns: the lower end keeps the
// smaller key, the upper end the larger, both decided by the one predicate
// key[upper] < key[lower], so equal keys never move.  The bucket lives in
// two shared-memory buffers: each layer reads one and writes the other, so
// one barrier separates layers.
//
// Divergent form: one branch per role, each with its own partner load and
// compare.  Melded form (the paper's region-region meld, Algorithm 2): the
// two roles' loads are unified, the compares aligned by selecting their
// operands, so the warp runs one copy of the body; idle elements skip it.
#include <cuda_runtime.h>

#include <cstdint>

#include "darm.h"
#include "darm_internal.h"

namespace darm {
namespace {

constexpr uint32_t kOddEvenMax = 4096;
constexpr uint32_t kOddEvenThreads = 1024;
constexpr int kPerThread = kOddEvenMax / kOddEvenThreads;

// Block b sorts keys[b*n .. (b+1)*n) (and the same payload range).
template <bool V, int VAR>
__global__ void __launch_bounds__(kOddEvenThreads, 1)
    darm_oddeven_block_kernel(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t n) {
  keys += size_t(blockIdx.x) * n;
  if (V) vals += size_t(blockIdx.x) * n;
  // dynamic: two key buffers of n words, then (with a payload) two payload
  // buffers
  extern __shared__ __align__(16) uint32_t oe_smem[];
  uint32_t* sk2[2] = {oe_smem, oe_smem + n};
  uint32_t* sv2[2] = {oe_smem + 2 * n, oe_smem + 3 * n};
  const uint32_t tid = threadIdx.x;
  const uint32_t nt = blockDim.x;
  for (uint32_t x = tid; x < n; x += nt) {
    sk2[0][x] = keys[x];
    if (V) sv2[0][x] = vals[x];
  }
  __syncthreads();
  uint32_t cur = 0;  // buffer holding the bucket before this layer
  for (uint32_t p = 1; p < n; p <<= 1) {
    for (uint32_t k = p; k >= 1; k >>= 1) {
      const uint32_t* sk = cur ? sk2[1] : sk2[0];
      const uint32_t* sv = cur ? sv2[1] : sv2[0];
      uint32_t* dk = cur ? sk2[0] : sk2[1];
      uint32_t* dv = cur ? sv2[0] : sv2[1];
#pragma unroll
      for (int r = 0; r < kPerThread; ++r) {
        const uint32_t x = tid + uint32_t(r) * nt;
        if (x >= n) break;
        const uint32_t q = x & (2 * p - 1);  // position inside the block of 2p
        bool lower, upper;
        if (k == p) {
          lower = (x & p) == 0;
          upper = !lower;
        } else {
          lower = (x & k) != 0 && q + k < 2 * p;
          upper = (x & k) == 0 && q >= k;
        }
        uint32_t key = sk[x];
        uint32_t val = V ? sv[x] : 0u;
        if (VAR == 0) {
          if (lower) {
            const uint32_t b = sk[x + k];
            if (b < key) {
              key = b;
              if (V) val = sv[x + k];
            }
          } else if (upper) {
            const uint32_t a = sk[x - k];
            if (key < a) {
              key = a;
              if (V) val = sv[x - k];
            }
          }
        } else {
          if (lower || upper) {
            const uint32_t partner = lower ? x + k : x - k;
            const uint32_t b = sk[partner];
            const uint32_t lhs = lower ? b : key;  // key[upper]
            const uint32_t rhs = lower ? key : b;  // key[lower]
            if (lhs < rhs) {
              key = b;
              if (V) val = sv[partner];
            }
          }
        }
        dk[x] = key;
        if (V) dv[x] = val;
      }
      cur ^= 1u;
      __syncthreads();
    }
  }
  for (uint32_t x = tid; x < n; x += nt) {
    keys[x] = (cur ? sk2[1] : sk2[0])[x];
    if (V) vals[x] = (cur ? sv2[1] : sv2[0])[x];
  }
}

}  // namespace

void for_each_oddeven_kernel(void (*fn)(const void*, void*), void* ctx) {
  fn(reinterpret_cast<const void*>(&darm_oddeven_block_kernel<false, 0>), ctx);
  fn(reinterpret_cast<const void*>(&darm_oddeven_block_kernel<false, 1>), ctx);
  fn(reinterpret_cast<const void*>(&darm_oddeven_block_kernel<true, 0>), ctx);
  fn(reinterpret_cast<const void*>(&darm_oddeven_block_kernel<true, 1>), ctx);
}

}  // namespace darm

using namespace darm;

extern "C" int darm_oddeven_sort_buckets(uint32_t* keys, uint32_t* vals, size_t n,
                                         size_t bucket, int variant, void* stream) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (variant < DARM_DIVERGENT || variant > DARM_AUTO) return DARM_ERR_INVALID_ARG;
  if (n == 0) return DARM_OK;
  if (bucket == 0 || (bucket & (bucket - 1)) != 0) return DARM_ERR_NOT_POW2;
  if (bucket > kOddEvenMax || n % bucket != 0 || !keys) return DARM_ERR_INVALID_ARG;
  if (n / bucket > size_t(0x7FFFFFFF)) return DARM_ERR_INVALID_ARG;
  if (bucket == 1) return DARM_OK;
  const uint32_t threads = uint32_t(bucket < kOddEvenThreads ? bucket : kOddEvenThreads);
  const dim3 grid(uint32_t(n / bucket));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool melded = variant != DARM_DIVERGENT;
  const uint32_t nb = uint32_t(bucket);
  const size_t smem = size_t(vals ? 4 : 2) * nb * sizeof(uint32_t);
  if (vals) {
    if (melded)
      darm_oddeven_block_kernel<true, 1><<<grid, threads, smem, s>>>(keys, vals, nb);
    else
      darm_oddeven_block_kernel<true, 0><<<grid, threads, smem, s>>>(keys, vals, nb);
  } else {
    if (melded)
      darm_oddeven_block_kernel<false, 1><<<grid, threads, smem, s>>>(keys, nullptr, nb);
    else
      darm_oddeven_block_kernel<false, 0><<<grid, threads, smem, s>>>(keys, nullptr, nb);
  }
  if (cudaGetLastError() != cudaSuccess) return DARM_ERR_CUDA;
  g_ctx.launches.fetch_add(1, std::memory_order_relaxed);
  return DARM_OK;
}

extern "C" int darm_oddeven_sort_block(uint32_t* keys, uint32_t* vals, size_t n, int variant,
                                       void* stream) {
  if (n <= 1) return g_ctx.inited ? DARM_OK : DARM_ERR_NOT_INIT;
  if ((n & (n - 1)) != 0) return g_ctx.inited ? DARM_ERR_NOT_POW2 : DARM_ERR_NOT_INIT;
  return darm_oddeven_sort_buckets(keys, vals, n, n, variant, stream);
}
