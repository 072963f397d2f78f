// tma_merge_swz.cuh - merge pass of 32-bit keys (no payload) that works on
// its tiles in place, in swizzled shared memory, and writes them back with
// bulk tensor stores.
//
// The merge pass of a stage k > T runs layers T/2 .. 1 on every tile of
// T = 2^LOGT keys, 32 keys per thread, in three rounds: window bits
// LOGT-5 .. LOGT-1 (LOGT-10 layers), bits 5 .. 9 (5 layers) and bits 0 .. 4
// (5 layers).  The plain bulk-copy merge (tma_merge.cuh) keeps dense staging
// buffers plus one padded work buffer and stores the last round straight
// from registers; on 2^26 keys that last round took 2.5x as long as the
// middle one, its warps stalled behind their own global stores.  Here:
//   - tiles arrive by TMA tensor copies (boxes of 256 rows x 128 bytes) in
//     the 128-byte swizzled layout: 16-byte chunk c of 128-byte row w of the
//     buffer holds the tile's chunk c ^ (w mod 8);
//   - every round reads and writes the thread's own 32 keys in place, so a
//     tile needs no second buffer; in the swizzled layout all three rounds
//     are free of bank conflicts (rounds 0 and 1: a warp's 32 lanes cover
//     one row; round 2: eight consecutive threads read eight different
//     chunk columns with 16-byte loads);
//   - after the last round one thread hands the tile to the TMA engine as a
//     bulk tensor store and the warps go on to the next tile; the buffer is
//     refilled (the tile three steps ahead) once the store has read it.
// Three tile buffers (192 KiB for T = 2^14) give two tiles of prefetch.
// Every mbarrier wait is bounded (about one second); when one runs out the
// kernel latches DARM_ERR_TIMEOUT, waits (bounded) for its loads in flight
// and for its stores, and returns.
#pragma once

#include <cuda.h>

#include "tma_merge.cuh"

namespace darm {

constexpr int kSwzBuffers = 3;

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(tm), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tm, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(tm),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// The stores issued so far by this thread have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// The stores issued so far by this thread are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int LOGT>
struct SwzMergeSmem {
  static constexpr uint32_t kTileBytes = 4u << LOGT;
  static constexpr size_t kAlign = 1024;  // the 128-byte swizzle repeats every 1024 bytes
  static constexpr size_t kBytes = kAlign + size_t(kSwzBuffers) * kTileBytes + 8 * kSwzBuffers;
};

// Rows of a tile and rows per TMA box (the box height is at most 256).
template <int LOGT>
struct SwzRows {
  static constexpr uint32_t kRows = 1u << (LOGT - 5);
  static constexpr uint32_t kBox = kRows < 256u ? kRows : 256u;
  static constexpr int kBoxes = int(kRows / kBox);
};

// One merge pass over P.nblocks tiles; `tmap` maps the array as rows of 32
// keys (128 bytes) with boxes of SwzRows<LOGT>::kBox rows and the 128-byte
// swizzle.  The stage's direction is uniform per tile (bit p of the tile's
// index), so the two forms are the same code.
template <int LOGT>
__global__ void __launch_bounds__(1 << (LOGT - 5), (LOGT <= 13) ? 2 : 1)
    darm_merge_swz_kernel(const __grid_constant__ PassParams P, const __grid_constant__ CUtensorMap tmap) {
  static_assert(LOGT >= 13 && LOGT <= 14, "round 0 addressing needs window bits >= 8; 32 keys a thread");
  using K = uint32_t;
  constexpr int E = 32;
  constexpr int A0 = LOGT - 5;  // round 0 window bits A0 .. LOGT-1
  constexpr uint32_t kTileB = SwzMergeSmem<LOGT>::kTileBytes;
  using RW = SwzRows<LOGT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t sraw = smem_addr(smem_raw);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  unsigned char* sbuf = smem_raw + (sbase - sraw);
  const uint32_t bar0 = sbase + uint32_t(kSwzBuffers) * kTileB;
  const uint32_t tid = threadIdx.x;
  const uint32_t ntiles = P.nblocks;
  const uint32_t capmask = (1u << P.log2cap) - 1u;
  const uint32_t p = P.rounds[0].p;
  const CUtensorMap* tm = &tmap;

  auto issue_load = [&](uint32_t tl, int b) {  // thread 0
    const uint32_t bar = bar0 + 8u * uint32_t(b);
    mbar_expect_tx(bar, kTileB);
    const uint32_t d = sbase + uint32_t(b) * kTileB;
#pragma unroll
    for (int h = 0; h < RW::kBoxes; ++h)
      tma_load_2d(d + uint32_t(h) * RW::kBox * 128u, tm, 0, int(tl * RW::kRows + uint32_t(h) * RW::kBox), bar);
  };
  auto issue_store = [&](uint32_t tl, int b) {  // thread 0
    const uint32_t d = sbase + uint32_t(b) * kTileB;
#pragma unroll
    for (int h = 0; h < RW::kBoxes; ++h)
      tma_store_2d(tm, 0, int(tl * RW::kRows + uint32_t(h) * RW::kBox), d + uint32_t(h) * RW::kBox * 128u);
    bulk_commit();
  };

  uint32_t tile = blockIdx.x;
  if (tile >= ntiles) return;
  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(tm) : "memory");
#pragma unroll
    for (int b = 0; b < kSwzBuffers; ++b) mbar_init(bar0 + 8u * uint32_t(b), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // Every thread keeps the same account of which buffers have a load in
  // flight (bit b of `pending`) and of each barrier's phase (bit b of
  // `phase`), so that a timed-out wait can drain them.
  uint32_t pending = 0;
#pragma unroll
  for (int b = 0; b < kSwzBuffers; ++b) {
    const uint32_t tl = tile + uint32_t(b) * gridDim.x;
    if (tl < ntiles) {
      if (tid == 0) issue_load(tl, b);
      pending |= 1u << b;
    }
  }

  // Swizzled word offsets.  Round 0: element tid | r << A0 lies in row
  // (tid >> 5) | (r << (A0 - 5)), whose low three bits are those of tid >> 5.
  const uint32_t a0 = tid ^ (((tid >> 5) & 7u) << 2);
  // Round 1: element lane | r << 5 | warp << 10 lies in row r | warp << 5.
  const uint32_t a1 = (tid >> 5) << 10;
  const uint32_t lane = tid & 31u;
  // Round 2: the thread's 32 keys are row tid; chunk q sits at q ^ (tid & 7).
  const uint32_t a2 = tid << 5;
  const uint32_t t7 = tid & 7u;

  K kr[E];
  uint32_t vr[E];  // unused (no payload); window_side's signature
#pragma unroll
  for (int r = 0; r < E; ++r) vr[r] = 0;

  uint32_t phase = 0;
  int b = 0;
  bool first = true;
  for (; tile < ntiles; tile += gridDim.x) {
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
    K* sk = reinterpret_cast<K*>(sbuf + size_t(b) * kTileB);
    const bool asc = ((((tile << LOGT) | P.dir_base) & (1u << p) & capmask) == 0u);

    // round 0: layers LOGT-1 .. 10
#pragma unroll
    for (int r = 0; r < E; ++r) kr[r] = sk[a0 + (uint32_t(r) << A0)];
    if (asc)
      window_side<K, false, 5, true, true>(kr, vr, LOGT - 10);
    else
      window_side<K, false, 5, false, true>(kr, vr, LOGT - 10);
#pragma unroll
    for (int r = 0; r < E; ++r) sk[a0 + (uint32_t(r) << A0)] = kr[r];
    __syncthreads();
    // Every thread has left the previous tile's buffer (its store was issued
    // before this barrier): once the store has read it, load the tile
    // kSwzBuffers - 1 steps ahead into it.
    {
      const uint32_t nt = tile + uint32_t(kSwzBuffers - 1) * gridDim.x;
      const int pb = (b == 0) ? kSwzBuffers - 1 : b - 1;
      if (!first && nt < ntiles) {
        if (tid == 0) {
          bulk_wait_read_all();
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue_load(nt, pb);
        }
        pending |= 1u << pb;
      }
    }
    // round 1: layers 9 .. 5
#pragma unroll
    for (int r = 0; r < E; ++r) kr[r] = sk[a1 + (uint32_t(r) << 5) + (lane ^ (uint32_t(r & 7) << 2))];
    if (asc)
      window_side<K, false, 5, true, true>(kr, vr, 5);
    else
      window_side<K, false, 5, false, true>(kr, vr, 5);
#pragma unroll
    for (int r = 0; r < E; ++r) sk[a1 + (uint32_t(r) << 5) + (lane ^ (uint32_t(r & 7) << 2))] = kr[r];
    __syncthreads();
    // round 2: layers 4 .. 0, then the key map of the sort's last pass
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint4 w = *reinterpret_cast<const uint4*>(sk + a2 + ((uint32_t(q) ^ t7) << 2));
      kr[4 * q] = w.x;
      kr[4 * q + 1] = w.y;
      kr[4 * q + 2] = w.z;
      kr[4 * q + 3] = w.w;
    }
    if (asc)
      window_side<K, false, 5, true, true>(kr, vr, 5);
    else
      window_side<K, false, 5, false, true>(kr, vr, 5);
    if (P.map_out != 0u) {
#pragma unroll
      for (int r = 0; r < E; ++r) kr[r] = key_out<K>(kr[r], P.map_out);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<uint4*>(sk + a2 + ((uint32_t(q) ^ t7) << 2)) =
          make_uint4(kr[4 * q], kr[4 * q + 1], kr[4 * q + 2], kr[4 * q + 3]);
    // make this thread's writes visible to the bulk store
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) issue_store(tile, b);
    first = false;
    b = (b + 1 == kSwzBuffers) ? 0 : b + 1;
  }
  if (tid == 0) bulk_wait_all();
}

}  // namespace darm
