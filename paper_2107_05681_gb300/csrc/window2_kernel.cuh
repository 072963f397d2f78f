// window2_kernel.cuh - window pass with two register windows and one
// shared-memory exchange, its shape fixed at compile time.
//
// A window pass runs layers j >= T of one stage k on blocks of
// 2^(C + 2*LOGE) elements: the C low index bits (consecutive elements, for
// coalesced HBM access) and the 2*LOGE layer bits w0 .. w0+2*LOGE-1.  Round 0
// loads each thread's E elements of the top window straight from HBM, runs
// its layers (all LOGE of them) in registers and writes them to shared
// memory; round 1 reads the bottom window, runs the remaining `cnt` layers
// and stores to HBM.  Only w0, k and cnt are run-time values, so every
// shared-memory offset is an immediate.  Bit k lies above the window: the
// direction is uniform per block, so both forms keep Fig. 1's branch.
#pragma once

#include <type_traits>

#include "tile_kernel.cuh"

namespace darm {

template <typename K, bool V, int LOGE, int C, int VAR, int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT >= 1024) ? 1 : 1024 / MAXT) darm_window2_kernel(const __grid_constant__ PassParams P) {
  constexpr int E = 1 << LOGE;
  constexpr int B = C + 2 * LOGE;  // log2 block elements
  constexpr int PAD = TilePad<K, V, LOGE>::value;  // pad words per 32 elements
  constexpr uint32_t SW = smem_words(1u << B);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* sk = reinterpret_cast<K*>(smem_raw);
  uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + sizeof(K) * SW);

  K* __restrict__ gk = reinterpret_cast<K*>(P.keys);
  uint32_t* __restrict__ gv = P.vals;
  const uint32_t tid = threadIdx.x;
  const uint32_t w0 = P.w0;
  const uint32_t blk = blockIdx.x;
  const uint32_t nmid = w0 - uint32_t(C);
  const uint32_t gblk = ((blk & ((1u << nmid) - 1u)) << C) | ((blk >> nmid) << (w0 + 2 * LOGE));
  const uint32_t capmask = (1u << P.log2cap) - 1u;
  const uint32_t p = P.rounds[0].p;
  const int cnt1 = P.rounds[1].cnt;
  const bool asc = (((gblk | P.dir_base) & (1u << p) & capmask) == 0u);

  K kr[E];
  uint32_t vr[E];
#pragma unroll
  for (int r = 0; r < E; ++r) vr[r] = 0;

  // round 0: window = local bits C+LOGE .. C+2*LOGE-1 (layer bits
  // w0+LOGE ..), lanes on the low bits
  {
    constexpr int A = C + LOGE;
    const uint32_t tl = (tid & ((1u << A) - 1u)) | ((tid >> A) << (A + LOGE));
    const uint32_t g_t = (tl & ((1u << C) - 1u)) | ((tl >> C) << w0) | gblk;
    const uint32_t sh = w0 + uint32_t(LOGE);  // register r sits at g_t + (r << sh)
    const uint32_t s_base = Interleave<K, V>::value ? phys8(tl) : physp<PAD>(tl);
    auto body = [&](auto asc_c) {
      constexpr bool ASC = decltype(asc_c)::value;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const uint32_t g = g_t + (uint32_t(r) << sh);
        kr[r] = gk[g];
        if (V) vr[r] = gv[g];
      }
      window_side<K, V, LOGE, ASC>(kr, vr, LOGE);
      s_store<K, V, LOGE, A, false, false, PAD>(kr, vr, false, gk, gv, 0u, sk, sv, s_base, 0u, K(0));
    };
    if (asc)
      body(std::true_type{});
    else
      body(std::false_type{});
  }
  __syncthreads();
  // round 1: window = local bits C .. C+LOGE-1 (layer bits w0 ..)
  {
    constexpr int A = C;
    const uint32_t tl = (tid & ((1u << A) - 1u)) | ((tid >> A) << (A + LOGE));
    const uint32_t g_t = (tl & ((1u << C) - 1u)) | ((tl >> C) << w0) | gblk;
    const uint32_t s_base = Interleave<K, V>::value ? phys8(tl) : physp<PAD>(tl);
    auto body = [&](auto asc_c) {
      constexpr bool ASC = decltype(asc_c)::value;
      s_load<K, V, LOGE, A, false, PAD>(kr, vr, false, gk, gv, 0u, sk, sv, s_base, 0u, K(0));
      window_side<K, V, LOGE, ASC>(kr, vr, cnt1);
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const uint32_t g = g_t + (uint32_t(r) << w0);
        gk[g] = kr[r];
        if (V) gv[g] = vr[r];
      }
    };
    if (asc)
      body(std::true_type{});
    else
      body(std::false_type{});
  }
}

}  // namespace darm
