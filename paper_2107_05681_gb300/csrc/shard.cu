// shard.cu - the bitonic network of one array split into G shards, as three
// building blocks a multi-process driver composes (one shard per process):
//
//   darm_bitonic_sort_shard   stages k = 2 .. N of the whole array's network
//                             on this shard (N = shard length), every
//                             comparator taking its direction from the
//                             element's index in the whole array;
//   darm_bitonic_exchange     one layer j >= N of a stage k > N: element i
//                             of shard r meets element i of shard
//                             r ^ (j / N), the pair ordered by bit k of its
//                             index (uniform over the shard, the final stage
//                             ascending); the peer's copy arrives in a buffer
//                             of this device (the driver moves it);
//   darm_bitonic_merge_shard  the layers j = N/2 .. 1 of a stage k > N on
//                             this shard.
// Run as: sort_shard; then for every stage k = 2N .. G N: the exchange layers
// j = k/2 .. N, then merge_shard.  Every comparator is the whole array's
// (Fig. 1), so the concatenated shards equal the one-array sort bit for bit.
//
// Between the first and the last call the keys stay in the network's
// internal form (float keys as totalOrder words, descending sorts
// complemented): darm_bitonic_sort_shard applies the key map on its first
// load and keeps it; darm_bitonic_merge_shard of the final stage undoes it.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "darm.h"
#include "darm_internal.h"
#include "plan.h"

namespace darm {
namespace {

int log2_of(size_t n) {
  int m = 0;
  while ((size_t(1) << m) < n) ++m;
  return m;
}

bool pow2(size_t n) { return n != 0 && (n & (n - 1)) == 0; }

// Shared argument checks; fills the key kind, map and sizes.
int shard_args(const void* keys, const uint32_t* vals, size_t n, int dtype, size_t shard,
               size_t nshards, int dir, KeyKind* kk, uint32_t* map, int* m, int* M) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (dtype < DARM_U32 || dtype > DARM_U64 || (dir != DARM_ASC && dir != DARM_DESC))
    return DARM_ERR_INVALID_ARG;
  if (!pow2(n) || n < 2 || !pow2(nshards)) return DARM_ERR_NOT_POW2;
  if (shard >= nshards || n * nshards > (size_t(1) << 31) || !keys) return DARM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(keys) & 15u) != 0) return DARM_ERR_INVALID_ARG;
  if (vals && (reinterpret_cast<uintptr_t>(vals) & 15u) != 0) return DARM_ERR_INVALID_ARG;
  *kk = dtype == DARM_U64 ? KEY_U64 : KEY_U32;
  *map = (dtype == DARM_F32 ? kMapF32 : 0u) | (dir == DARM_DESC ? kMapComplement : 0u);
  *m = log2_of(n);
  *M = log2_of(n * nshards);
  return DARM_OK;
}

template <typename K, bool V>
__global__ void __launch_bounds__(256) darm_exchange_kernel(K* __restrict__ keys,
                                                            uint32_t* __restrict__ vals,
                                                            const K* __restrict__ pk,
                                                            const uint32_t* __restrict__ pv,
                                                            size_t n, bool keep_lower, bool asc) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const K a = keys[i];
    const K b = pk[i];
    const K lower = keep_lower ? a : b;  // key at the lower index of the pair
    const K upper = keep_lower ? b : a;
    const bool swap = asc ? (upper < lower) : (upper > lower);
    if (swap) {
      keys[i] = b;
      if (V) vals[i] = pv[i];
    }
  }
}

}  // namespace
}  // namespace darm

using namespace darm;

extern "C" int darm_bitonic_sort_shard(void* keys, uint32_t* vals, size_t n, int dtype,
                                       size_t shard, size_t nshards, int dir, int variant,
                                       void* stream) {
  KeyKind kk;
  uint32_t map;
  int m, M;
  int rc = shard_args(keys, vals, n, dtype, shard, nshards, dir, &kk, &map, &m, &M);
  if (rc != DARM_OK) return rc;
  if (variant < DARM_DIVERGENT || variant > DARM_AUTO) return DARM_ERR_INVALID_ARG;
  const bool hv = vals != nullptr;
  std::vector<Launch> plan;
  // one shard alone is a whole array: undo the key map at the end
  if (!plan_array(plan, kk, hv, m, tuning_for(kk, hv, m), variant, map,
                  nshards == 1 ? map : 0u, g_ctx.smem_limit))
    return DARM_ERR_INVALID_ARG;
  for (Launch& L : plan) {
    L.P.log2cap = uint32_t(M);
    L.P.dir_base = uint32_t(shard * n);
  }
  return launch_plan(plan, kk, keys, vals, static_cast<cudaStream_t>(stream));
}

extern "C" int darm_bitonic_exchange(void* keys, uint32_t* vals, const void* peer_keys,
                                     const uint32_t* peer_vals, size_t n, int dtype, size_t shard,
                                     size_t nshards, int log2k, int log2j, int dir, void* stream) {
  KeyKind kk;
  uint32_t map;
  int m, M;
  int rc = shard_args(keys, vals, n, dtype, shard, nshards, dir, &kk, &map, &m, &M);
  if (rc != DARM_OK) return rc;
  if (log2j < m || log2k <= log2j || log2k > M || !peer_keys || (vals && !peer_vals))
    return DARM_ERR_INVALID_ARG;
  const size_t peer = shard ^ ((size_t(1) << log2j) >> m);
  if (peer >= nshards) return DARM_ERR_INVALID_ARG;
  const bool keep_lower = shard < peer;
  // bit k of every element's index in the whole array is bit (log2k - m) of
  // the shard number; the final stage (k = the whole array) is ascending.
  // Keys are in the internal form, where every comparator is ascending-
  // or descending by this bit only.
  const bool asc = (log2k == M) || (((shard << m) >> log2k) & 1u) == 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned grid = unsigned(std::min<size_t>((n + 255) / 256, size_t(g_ctx.sms) * 8));
  if (kk == KEY_U64) {
    auto* k = static_cast<uint64_t*>(keys);
    auto* p = static_cast<const uint64_t*>(peer_keys);
    if (vals)
      darm_exchange_kernel<uint64_t, true><<<grid, 256, 0, s>>>(k, vals, p, peer_vals, n, keep_lower, asc);
    else
      darm_exchange_kernel<uint64_t, false><<<grid, 256, 0, s>>>(k, nullptr, p, nullptr, n, keep_lower, asc);
  } else {
    auto* k = static_cast<uint32_t*>(keys);
    auto* p = static_cast<const uint32_t*>(peer_keys);
    if (vals)
      darm_exchange_kernel<uint32_t, true><<<grid, 256, 0, s>>>(k, vals, p, peer_vals, n, keep_lower, asc);
    else
      darm_exchange_kernel<uint32_t, false><<<grid, 256, 0, s>>>(k, nullptr, p, nullptr, n, keep_lower, asc);
  }
  if (cudaPeekAtLastError() != cudaSuccess) return DARM_ERR_CUDA;
  g_ctx.launches.fetch_add(1, std::memory_order_relaxed);
  return DARM_OK;
}

extern "C" int darm_bitonic_merge_shard(void* keys, uint32_t* vals, size_t n, int dtype,
                                        size_t shard, size_t nshards, int log2k, int dir,
                                        int variant, void* stream) {
  KeyKind kk;
  uint32_t map;
  int m, M;
  int rc = shard_args(keys, vals, n, dtype, shard, nshards, dir, &kk, &map, &m, &M);
  if (rc != DARM_OK) return rc;
  if (variant < DARM_DIVERGENT || variant > DARM_AUTO || log2k <= m || log2k > M)
    return DARM_ERR_INVALID_ARG;
  const bool hv = vals != nullptr;
  // the layers below bit m of a stage above it: the launches of the final
  // stage of a shard-sized plan (window passes over bits m-1 .. t, then the
  // merge), with that stage's direction bit moved to k
  std::vector<Launch> plan;
  if (!plan_array(plan, kk, hv, m, tuning_for(kk, hv, m), variant, 0u,
                  log2k == M ? map : 0u, g_ctx.smem_limit))
    return DARM_ERR_INVALID_ARG;
  size_t first = plan.size();
  while (first > 0 && plan[first - 1].kind != PASS_TILE && int(plan[first - 1].P.rounds[0].p) == m)
    --first;
  if (first == plan.size() || first == 0) return DARM_ERR_INVALID_ARG;  // shard within one tile
  std::vector<Launch> tail(plan.begin() + first, plan.end());
  for (Launch& L : tail) {
    for (uint32_t r = 0; r < L.P.nrounds; ++r) {
      L.P.rounds[r].p = uint8_t(log2k);
      L.P.rounds[r].lanediv = 0;  // bit k lies above every block: one direction per block
    }
    L.P.log2cap = uint32_t(M);
    L.P.dir_base = uint32_t(shard * n);
  }
  return launch_plan(tail, kk, keys, vals, static_cast<cudaStream_t>(stream));
}
