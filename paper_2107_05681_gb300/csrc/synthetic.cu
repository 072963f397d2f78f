// synthetic.cu - the paper's synthetic divergent kernels SB1-SB4 and their
// -R variants (Section VI-A), in a divergent and a melded form.
//
// Two nested loops; the inner loop holds a divergent region whose paths work
// on different words of the thread's shared-memory slice.  SB1: a two-way
// diamond, SB4: a three-way if-else-if-else; in SB1/SB4 every path computes
// the same function, in SB1-R/SB4-R each path its own.  Thread t of a block
// owns s[q*256 + t], q = 0..3 (column-major: the 32 lanes of a warp hit 32
// banks).  Per iteration `it` and inner step j:
//   SB1:  c = (t ^ j ^ it) & 1  -> path 0 on words (j, j+1) when c == 1,
//         path 1 on (j+2, j+3) otherwise
//   SB4:  c = (t + j + it) % 3  -> path c on words (j+c, j+c+1)
// (word indices mod 4); the path then runs `rounds` times
//   v = g_path(v, w),  g_0 = 3v + w,  g_1 = 5v ^ w,  g_2 = 7v - w  (-R)
//   v = 3v + w                                                      (SB1, SB4)
// on v = s[a], w = s[b] and stores v back to s[a].
//   SB2:  the SB1 paths, each an if-then region guarded by the data
//         (s[b] & 1) around the rounds (paired regions B2 / B3);
//   SB3:  the SB1 paths with two if-then regions each: the SB2 one, then,
//         if (s[a] & 2), rounds of s[b] = g2(s[b], s[a]) (regions C2 / C3
//         and C6 / C5), g2 = 3v + w, or in SB3-R path 0: 7v - w.
// The path condition
// alternates between neighbouring lanes, so every warp takes every path.
//
// Divergent form: one branch per path with its own loads, loop and store.
// Melded form (region-region meld, Algorithm 2): the word indices (and the
// -R multiplier) are selected by the path, one load pair, one loop and one
// store run for all paths; in the -R variants the paths' unaligned
// operations (add / xor / sub) are computed side by side and the path's
// result is selected.
#include <cuda_runtime.h>

#include <cstdint>

#include "darm.h"
#include "darm_internal.h"

namespace darm {
namespace {

constexpr int kSbThreads = 256;

template <int PATH, bool SAME>
__device__ __forceinline__ uint32_t sb_round(uint32_t v, uint32_t w) {
  if (SAME || PATH == 0) return 3u * v + w;
  if (PATH == 1) return (5u * v) ^ w;
  return 7u * v - w;
}

// one path of the divergent form: words (a, b) of the thread's slice
template <int PATH, bool SAME>
__device__ __forceinline__ void sb_path(uint32_t* s, uint32_t t, uint32_t a, uint32_t b,
                                        int rounds) {
  uint32_t v = s[a * kSbThreads + t];
  const uint32_t w = s[b * kSbThreads + t];
  for (int r = 0; r < rounds; ++r) v = sb_round<PATH, SAME>(v, w);
  s[a * kSbThreads + t] = v;
}

// SB2 / SB3: the path's if-then regions (divergent form)
template <int PATH, bool SAME, bool TWO_REGIONS>
__device__ __forceinline__ void sb_regions(uint32_t* s, uint32_t t, uint32_t a, uint32_t b,
                                           int rounds) {
  const uint32_t w = s[b * kSbThreads + t];
  if (w & 1u) {  // region B2 / B3 (C2 / C3)
    uint32_t v = s[a * kSbThreads + t];
    for (int r = 0; r < rounds; ++r) v = sb_round<PATH, SAME>(v, w);
    s[a * kSbThreads + t] = v;
  }
  if (TWO_REGIONS) {
    const uint32_t x = s[a * kSbThreads + t];
    if (x & 2u) {  // region C6 / C5
      uint32_t u = s[b * kSbThreads + t];
      for (int r = 0; r < rounds; ++r) u = (SAME || PATH == 1) ? 3u * u + x : 7u * u - x;
      s[b * kSbThreads + t] = u;
    }
  }
}

template <int PATTERN, int VAR>
__global__ void __launch_bounds__(kSbThreads) darm_sb_kernel(uint32_t* data, int iters, int rounds) {
  constexpr int BASE = PATTERN % 100;
  constexpr bool THREE = (BASE == 4);
  constexpr bool REGIONS = (BASE == 2 || BASE == 3);
  constexpr bool TWO_REGIONS = (BASE == 3);
  constexpr bool SAME = (PATTERN < 100);
  __shared__ uint32_t s[4 * kSbThreads];
  const uint32_t t = threadIdx.x;
  uint32_t* d = data + size_t(blockIdx.x) * (4 * kSbThreads);
#pragma unroll
  for (int q = 0; q < 4; ++q) s[q * kSbThreads + t] = d[q * kSbThreads + t];
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j) {
      uint32_t c;  // path index
      if (THREE) {
        c = (t + j + uint32_t(it)) % 3u;
      } else {
        c = ((t ^ j ^ uint32_t(it)) & 1u) ? 0u : 1u;
      }
      if (REGIONS) {
        if (VAR == 0) {
          if (c == 0)
            sb_regions<0, SAME, TWO_REGIONS>(s, t, j & 3u, (j + 1) & 3u, rounds);
          else
            sb_regions<1, SAME, TWO_REGIONS>(s, t, (j + 2) & 3u, (j + 3) & 3u, rounds);
        } else {
          // the paths' regions melded pairwise: selected words and, in the
          // -R variants, selected multipliers and operations
          const uint32_t a = c == 0 ? (j & 3u) : ((j + 2) & 3u);
          const uint32_t b = (a + 1) & 3u;
          const uint32_t w = s[b * kSbThreads + t];
          if (w & 1u) {
            uint32_t v = s[a * kSbThreads + t];
            if (SAME) {
              for (int r = 0; r < rounds; ++r) v = 3u * v + w;
            } else {
              const uint32_t mul = c == 0 ? 3u : 5u;
              for (int r = 0; r < rounds; ++r) {
                const uint32_t m = mul * v;
                v = c == 0 ? m + w : m ^ w;
              }
            }
            s[a * kSbThreads + t] = v;
          }
          if (TWO_REGIONS) {
            const uint32_t x = s[a * kSbThreads + t];
            if (x & 2u) {
              uint32_t u = s[b * kSbThreads + t];
              if (SAME) {
                for (int r = 0; r < rounds; ++r) u = 3u * u + x;
              } else {
                const uint32_t mul = c == 0 ? 7u : 3u;
                for (int r = 0; r < rounds; ++r) {
                  const uint32_t m = mul * u;
                  u = c == 0 ? m - x : m + x;
                }
              }
              s[b * kSbThreads + t] = u;
            }
          }
        }
      } else if (VAR == 0) {
        if (THREE) {
          if (c == 0)
            sb_path<0, SAME>(s, t, j & 3u, (j + 1) & 3u, rounds);
          else if (c == 1)
            sb_path<1, SAME>(s, t, (j + 1) & 3u, (j + 2) & 3u, rounds);
          else
            sb_path<2, SAME>(s, t, (j + 2) & 3u, (j + 3) & 3u, rounds);
        } else {
          if (c == 0)
            sb_path<0, SAME>(s, t, j & 3u, (j + 1) & 3u, rounds);
          else
            sb_path<1, SAME>(s, t, (j + 2) & 3u, (j + 3) & 3u, rounds);
        }
      } else {
        const uint32_t a = THREE ? ((j + c) & 3u) : (c == 0 ? (j & 3u) : ((j + 2) & 3u));
        const uint32_t b = (a + 1) & 3u;
        uint32_t v = s[a * kSbThreads + t];
        const uint32_t w = s[b * kSbThreads + t];
        if (SAME) {
          for (int r = 0; r < rounds; ++r) v = 3u * v + w;
        } else {
          const uint32_t mul = c == 0 ? 3u : (c == 1 ? 5u : 7u);
          for (int r = 0; r < rounds; ++r) {
            const uint32_t m = mul * v;
            const uint32_t r0 = m + w, r1 = m ^ w;
            v = c == 0 ? r0 : r1;
            if (THREE) v = c == 2 ? m - w : v;
          }
        }
        s[a * kSbThreads + t] = v;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) d[q * kSbThreads + t] = s[q * kSbThreads + t];
}

template <int PATTERN>
void sb_launch(bool melded, uint32_t* data, uint32_t nblocks, int iters, int rounds,
               cudaStream_t s) {
  if (melded)
    darm_sb_kernel<PATTERN, 1><<<nblocks, kSbThreads, 0, s>>>(data, iters, rounds);
  else
    darm_sb_kernel<PATTERN, 0><<<nblocks, kSbThreads, 0, s>>>(data, iters, rounds);
}

}  // namespace
}  // namespace darm

using namespace darm;

extern "C" int darm_sb_run(int pattern, uint32_t* data, size_t nblocks, int iters, int rounds,
                           int variant, void* stream) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (variant < DARM_DIVERGENT || variant > DARM_AUTO) return DARM_ERR_INVALID_ARG;
  const int base = pattern % 100;
  if (base < 1 || base > 4 || (pattern != base && pattern != base + 100)) return DARM_ERR_INVALID_ARG;
  if (iters < 0 || rounds < 0 || nblocks > size_t(0x7FFFFFFF)) return DARM_ERR_INVALID_ARG;
  if (nblocks == 0) return DARM_OK;
  if (!data) return DARM_ERR_INVALID_ARG;
  const bool melded = variant != DARM_DIVERGENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t nb = uint32_t(nblocks);
  switch (pattern) {
    case 1: sb_launch<1>(melded, data, nb, iters, rounds, s); break;
    case 2: sb_launch<2>(melded, data, nb, iters, rounds, s); break;
    case 3: sb_launch<3>(melded, data, nb, iters, rounds, s); break;
    case 4: sb_launch<4>(melded, data, nb, iters, rounds, s); break;
    case 101: sb_launch<101>(melded, data, nb, iters, rounds, s); break;
    case 102: sb_launch<102>(melded, data, nb, iters, rounds, s); break;
    case 103: sb_launch<103>(melded, data, nb, iters, rounds, s); break;
    default: sb_launch<104>(melded, data, nb, iters, rounds, s); break;
  }
  if (cudaGetLastError() != cudaSuccess) return DARM_ERR_CUDA;
  g_ctx.launches.fetch_add(1, std::memory_order_relaxed);
  return DARM_OK;
}
