// window1_kernel.cuh - window pass with one register window, its shape
// fixed at compile time.
//
// A one-window pass runs up to LOGE layers j >= T of one stage k on blocks
// of 2^(C + LOGE) elements: the C low index bits (2^C consecutive elements,
// one per thread, for coalesced HBM access) and the LOGE layer bits
// w0 .. w0+LOGE-1 (a thread's E registers).  Each thread loads its E
// elements straight from HBM, runs the top `cnt` layers of its window in
// registers and stores them back: no shared memory, no barrier.  Bit k lies
// above the window, so the direction is uniform per block and both forms
// keep Fig. 1's branch.
#pragma once

#include <type_traits>

#include "tile_kernel.cuh"

namespace darm {

// Up to 128 registers a thread: each thread keeps E independent loads in
// flight, so fewer resident warps still cover HBM latency.
template <typename K, bool V, int LOGE, int C, int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT >= 512) ? 1 : 512 / MAXT) darm_window1_kernel(const __grid_constant__ PassParams P) {
  constexpr int E = 1 << LOGE;
  K* __restrict__ gk = reinterpret_cast<K*>(P.keys);
  uint32_t* __restrict__ gv = P.vals;
  const uint32_t w0 = P.w0;
  const uint32_t blk = blockIdx.x;
  const uint32_t nmid = w0 - uint32_t(C);
  const uint32_t gblk = ((blk & ((1u << nmid) - 1u)) << C) | ((blk >> nmid) << (w0 + LOGE));
  const uint32_t capmask = (1u << P.log2cap) - 1u;
  const uint32_t p = P.rounds[0].p;
  const int cnt = P.rounds[0].cnt;
  const bool asc = (((gblk | P.dir_base) & (1u << p) & capmask) == 0u);
  const uint32_t g_t = threadIdx.x | gblk;  // register r sits at g_t + (r << w0)

  K kr[E];
  uint32_t vr[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const uint32_t g = g_t + (uint32_t(r) << w0);
    kr[r] = gk[g];
    vr[r] = V ? gv[g] : 0u;
  }
  if (asc)
    window_side<K, V, LOGE, true>(kr, vr, cnt);
  else
    window_side<K, V, LOGE, false>(kr, vr, cnt);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const uint32_t g = g_t + (uint32_t(r) << w0);
    gk[g] = kr[r];
    if (V) gv[g] = vr[r];
  }
}

}  // namespace darm
