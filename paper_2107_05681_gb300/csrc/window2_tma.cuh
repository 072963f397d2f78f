// window2_tma.cuh - two-window pass of 32-bit keys (alone, or with a 32-bit
// payload) that streams its blocks through shared memory with TMA tensor
// copies and works on them in place.
//
// A two-window pass runs up to 2e layers j >= T of one stage k (layer bits
// w0 .. w0+2e-1) on blocks of 16 x 2^(2e) elements: 16 consecutive elements
// (local bits 0..3) at each position of the two windows (local bits
// 4..3+e: layer bits w0..w0+e-1, local bits 4+e..3+2e: the top window).
// Keys alone: e = 5, 32 keys per thread, 512 threads; with a payload: e = 4,
// 16 pairs per thread, 256 threads, keys and payloads in two halves of each
// block buffer (two tensor maps, same box).  The plain
// two-window kernel (window2_kernel.cuh) loads each thread's 32 keys
// straight from HBM into registers, exchanges them once through shared
// memory and stores them from registers; at two CTAs per SM it stalls on
// those loads and stores (about 94 us per pass on 2^26 keys against 75 us
// for a one-window pass).  Here, as in the in-place merge
// (tma_merge_swz.cuh):
//   - a 5-D tensor map views the array as (16 consecutive elements, the
//     bits between them and the windows, bottom window, top window, the bits
//     above), so one box of 16 x 1 x 2^e x 2^e x 1 is one block, dense in
//     shared memory in local-index order (no swizzle);
//   - persistent CTAs keep three block buffers: blocks stream in two ahead,
//     both rounds read and write the thread's own 2^e elements in place,
//     and one thread hands the finished block to a bulk tensor store;
//   - round 0 (registers on the top window) puts 32 consecutive words on a
//     warp's lanes.  In round 1 (registers on the bottom window) a warp's two
//     half-warps sit 2^(4+e) words apart, on the same 16 banks; so lanes 16..31
//     hold their registers in pair-swapped order (register r holds bottom
//     window position r ^ 1), which moves them to the other 16 banks.  That
//     swap reverses which register of a pair holds the lower index only in
//     the layer of the window's lowest bit: there those lanes exchange the
//     roles of min and max (keys alone: two selects per pair; with a
//     payload: the strict swap test reads the pair's operands in the other
//     order).
// The direction (bit k of the index) lies above the block: uniform per
// block, so the two forms are the same code.  Waits are bounded as in the
// merge kernels.
#pragma once

#include "tma_merge_swz.cuh"

namespace darm {

// Block shape of the TMA two-window pass: V = with a payload.
template <bool V>
struct W2t {
  static constexpr int kLogE = V ? 4 : 5;                  // window bits e
  static constexpr int kLog2Block = 4 + 2 * kLogE;         // 16 consecutive x 2 windows
  static constexpr int kThreads = 1 << (kLog2Block - kLogE);
  static constexpr uint32_t kHalf = 4u << kLog2Block;      // keys (or payloads) of a block
  static constexpr uint32_t kSet = V ? 2 * kHalf : kHalf;  // one block buffer
  static constexpr size_t kBytes = 1024 + size_t(kSwzBuffers) * kSet + 8 * kSwzBuffers;
};

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* tm, int c1, int c4,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(tm), "r"(0), "r"(c1), "r"(0), "r"(0), "r"(c4), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_store_5d(const CUtensorMap* tm, int c1, int c4, uint32_t src) {
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(tm),
      "r"(0), "r"(c1), "r"(0), "r"(0), "r"(c4), "r"(src)
      : "memory");
}

// One two-window pass over P.nblocks blocks (block b: mid bits b mod 2^(w0-4)
// between the consecutive elements and the windows, high bits b >> (w0-4)).
// Round 0 runs the top window's e layers, round 1 the top P.rounds[1].cnt
// layers of the bottom window.  `tmv` maps the payload (V only).
template <bool V>
__global__ void __launch_bounds__(W2t<V>::kThreads, V ? 2 : 1)
    darm_window2_tma_kernel(const __grid_constant__ PassParams P, const __grid_constant__ CUtensorMap tmk,
                            const __grid_constant__ CUtensorMap tmv) {
  using K = uint32_t;
  using S = W2t<V>;
  constexpr int LOGE = S::kLogE;
  constexpr int E = 1 << LOGE;
  constexpr int A0 = 4 + LOGE;  // round 0 window bits A0 .. A0+e-1
  extern __shared__ __align__(1024) unsigned char w2t_smem[];
  const uint32_t sraw = smem_addr(w2t_smem);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  unsigned char* sbuf = w2t_smem + (sbase - sraw);
  const uint32_t bar0 = sbase + uint32_t(kSwzBuffers) * S::kSet;
  const uint32_t tid = threadIdx.x;
  const uint32_t nblocks = P.nblocks;
  const uint32_t w0 = P.w0;
  const uint32_t nmid = w0 - 4u;
  const uint32_t midmask = (1u << nmid) - 1u;
  const uint32_t capmask = (1u << P.log2cap) - 1u;
  const uint32_t p = P.rounds[0].p;
  const int cnt1 = P.rounds[1].cnt;

  auto issue_load = [&](uint32_t blk, int b) {  // thread 0
    const uint32_t bar = bar0 + 8u * uint32_t(b);
    const uint32_t d = sbase + uint32_t(b) * S::kSet;
    mbar_expect_tx(bar, S::kSet);
    tma_load_5d(d, &tmk, int(blk & midmask), int(blk >> nmid), bar);
    if (V) tma_load_5d(d + S::kHalf, &tmv, int(blk & midmask), int(blk >> nmid), bar);
  };
  auto issue_store = [&](uint32_t blk, int b) {  // thread 0
    const uint32_t d = sbase + uint32_t(b) * S::kSet;
    tma_store_5d(&tmk, int(blk & midmask), int(blk >> nmid), d);
    if (V) tma_store_5d(&tmv, int(blk & midmask), int(blk >> nmid), d + S::kHalf);
    bulk_commit();
  };

  uint32_t blk = blockIdx.x;
  if (blk >= nblocks) return;
  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmk) : "memory");
    if (V) asm volatile("prefetch.tensormap [%0];" ::"l"(&tmv) : "memory");
#pragma unroll
    for (int b = 0; b < kSwzBuffers; ++b) mbar_init(bar0 + 8u * uint32_t(b), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t pending = 0;
#pragma unroll
  for (int b = 0; b < kSwzBuffers; ++b) {
    const uint32_t bl = blk + uint32_t(b) * gridDim.x;
    if (bl < nblocks) {
      if (tid == 0) issue_load(bl, b);
      pending |= 1u << b;
    }
  }

  // round 1: lanes on local bits 0..3 and A0..; lanes 16..31 of a warp hold
  // bottom-window position r ^ 1 in register r
  const uint32_t tw0 = (tid >> 4) & 1u;
  const uint32_t base1 = (tid & 15u) | ((tid >> 4) << A0);
  const uint32_t even1 = base1 + (tw0 << 4);  // register r even: base1 + ((r + tw0) << 4)
  const uint32_t odd1 = base1 - (tw0 << 4);   // register r odd:  base1 + ((r - tw0) << 4)

  K kr[E];
  uint32_t vr[E];
#pragma unroll
  for (int r = 0; r < E; ++r) vr[r] = 0;

  uint32_t phase = 0;
  int b = 0;
  bool first = true;
  for (; blk < nblocks; blk += gridDim.x) {
    const uint32_t bar = bar0 + 8u * uint32_t(b);
    if (!mbar_wait_bounded(bar, (phase >> b) & 1u)) {
      if (tid == 0 && P.status != nullptr) atomicOr(P.status, int(kStatusTimeout));
#pragma unroll
      for (int q = 0; q < kSwzBuffers; ++q)
        if ((pending >> q) & 1u) mbar_wait_bounded(bar0 + 8u * uint32_t(q), (phase >> q) & 1u);
      if (tid == 0) bulk_wait_all();
      return;
    }
    phase ^= 1u << b;
    pending &= ~(1u << b);
    K* sk = reinterpret_cast<K*>(sbuf + size_t(b) * S::kSet);
    uint32_t* sv = reinterpret_cast<uint32_t*>(sbuf + size_t(b) * S::kSet + S::kHalf);
    const uint32_t gblk = ((blk & midmask) << 4) | ((blk >> nmid) << (w0 + 2u * LOGE));
    const bool asc = (((gblk | P.dir_base) & (1u << p) & capmask) == 0u);

    // round 0: the top window's e layers
#pragma unroll
    for (int r = 0; r < E; ++r) {
      kr[r] = sk[tid + (uint32_t(r) << A0)];
      if (V) vr[r] = sv[tid + (uint32_t(r) << A0)];
    }
    if (asc)
      window_side<K, V, LOGE, true, !V>(kr, vr, LOGE);
    else
      window_side<K, V, LOGE, false, !V>(kr, vr, LOGE);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      sk[tid + (uint32_t(r) << A0)] = kr[r];
      if (V) sv[tid + (uint32_t(r) << A0)] = vr[r];
    }
    __syncthreads();
    {
      const uint32_t nb = blk + uint32_t(kSwzBuffers - 1) * gridDim.x;
      const int pb = (b == 0) ? kSwzBuffers - 1 : b - 1;
      if (!first && nb < nblocks) {
        if (tid == 0) {
          bulk_wait_read_all();
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue_load(nb, pb);
        }
        pending |= 1u << pb;
      }
    }
    // round 1: the bottom window's top cnt1 layers
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const uint32_t w = ((r & 1) ? odd1 : even1) + (uint32_t(r) << 4);
      kr[r] = sk[w];
      if (V) vr[r] = sv[w];
    }
    auto round1 = [&](auto asc_c) {
      constexpr bool ASC = decltype(asc_c)::value;
      window_side<K, V, LOGE, ASC, !V>(kr, vr, cnt1 < LOGE - 1 ? cnt1 : LOGE - 1);
      if (cnt1 == LOGE) {
        // layer of the window's lowest bit: pair (r, r + 1); in lanes
        // 16..31 register r + 1 holds the lower index
        const bool flip = tw0 != 0u;
#pragma unroll
        for (int r = 0; r < E; r += 2) {
          if constexpr (V) {
            ce_kv_flip<ASC>(kr[r], kr[r + 1], vr[r], vr[r + 1], flip);
          } else {
            const bool keep_lo_first = ASC != flip;
            const K lo = kmin(kr[r], kr[r + 1]);
            const K hi = kmax(kr[r], kr[r + 1]);
            kr[r] = keep_lo_first ? lo : hi;
            kr[r + 1] = keep_lo_first ? hi : lo;
          }
        }
      }
    };
    if (asc)
      round1(std::true_type{});
    else
      round1(std::false_type{});
    if (P.map_out != 0u) {
#pragma unroll
      for (int r = 0; r < E; ++r) kr[r] = key_out<K>(kr[r], P.map_out);
    }
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const uint32_t w = ((r & 1) ? odd1 : even1) + (uint32_t(r) << 4);
      sk[w] = kr[r];
      if (V) sv[w] = vr[r];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) issue_store(blk, b);
    first = false;
    b = (b + 1 == kSwzBuffers) ? 0 : b + 1;
  }
  if (tid == 0) bulk_wait_all();
}

}  // namespace darm
