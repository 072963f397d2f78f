// tma_merge_swz.cuh - merge passes of 32-bit keys that work on their tiles
// in place, in swizzled shared memory, and write them back with bulk tensor
// stores: keys alone (32 per thread, first kernel) and keys with a 32-bit
// payload (16 pairs per thread, second kernel, below).
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
  extern __shared__ __align__(1024) unsigned char swz_smem[];
  const uint32_t sraw = smem_addr(swz_smem);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  unsigned char* sbuf = swz_smem + (sbase - sraw);
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

// ---------------------------------------------------------------------------
// Key-value merge in place: 32-bit keys with a 32-bit payload, 16 pairs per
// thread, tiles of 2^12 or 2^13 pairs.  Keys and payloads arrive in two
// swizzled buffers (two tensor maps, same box); the rounds follow the
// compile-time merge schedule (windows at bits 8 and above, at bit 4 and at
// bit 0):
//   - a window at bit A >= 8: a warp's lanes cover one 128-byte row;
//   - the window at bit 4: the two half-warps of a warp sit 8 rows apart, on
//     the same banks, so lanes 16..31 hold window position r ^ 1 in
//     register r (the other 16 banks), and exchange the roles of their pair
//     in the window's lowest layer;
//   - the window at bit 0: each thread's 16 consecutive pairs are four
//     16-byte chunks of keys and four of payloads, eight consecutive threads
//     on eight different chunk columns.
// The compare-exchange is Fig. 1's strict swap of (key, payload) by key.
namespace darm {

template <int LOGT, int NB = kSwzBuffers>
struct SwzKvSmem {
  static constexpr uint32_t kHalf = 4u << LOGT;  // keys (or payloads) of one tile
  static constexpr uint32_t kSet = 2 * kHalf;
  static constexpr size_t kBytes = 1024 + size_t(NB) * kSet + 8 * NB;
};

// One pair of the window's lowest layer where the lane may hold the pair in
// swapped order (`flip`: register a holds the higher index).
template <bool ASC>
__device__ __forceinline__ void ce_kv_flip(uint32_t& a, uint32_t& b, uint32_t& va, uint32_t& vb,
                                           bool flip) {
  const uint32_t lo = flip ? b : a;  // key at the lower index
  const uint32_t up = flip ? a : b;
  cswap<uint32_t, true>(ASC ? (up < lo) : (up > lo), a, b, va, vb);
}

// NB tile buffers per CTA: three (two CTAs per SM for 2^12-pair tiles), or
// two (three CTAs per SM).
template <int LOGT, int NB = kSwzBuffers>
__global__ void __launch_bounds__(1 << (LOGT - 4), (LOGT <= 12) ? (NB == 2 ? 3 : 2) : 1)
    darm_merge_swz_kv_kernel(const __grid_constant__ PassParams P, const __grid_constant__ CUtensorMap tmk,
                             const __grid_constant__ CUtensorMap tmv) {
  static_assert(LOGT == 12 || LOGT == 13, "tiles of 2^12 or 2^13 pairs");
  using K = uint32_t;
  constexpr int LOGE = 4;
  constexpr int E = 1 << LOGE;
  using SK = SwzKvSmem<LOGT, NB>;  // a tile's keys (or payloads): one box of 2^(LOGT-5) <= 256 rows
  extern __shared__ __align__(1024) unsigned char swz_smem[];
  const uint32_t sraw = smem_addr(swz_smem);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  unsigned char* sbuf = swz_smem + (sbase - sraw);
  const uint32_t bar0 = sbase + uint32_t(NB) * SK::kSet;
  const uint32_t tid = threadIdx.x;
  const uint32_t ntiles = P.nblocks;
  const uint32_t p = P.rounds[0].p;

  // tile tl: first pair (a multiple of 32), direction index, capacity mask,
  // key map of its last store (whole arrays or a segment's tile)
  struct TileAt {
    size_t start;
    uint32_t dir_idx, capmask, mout;
  };
  auto tile_at = [&](uint32_t tl) -> TileAt {
    if (P.blocks == nullptr)
      return TileAt{size_t(tl) << LOGT, (tl << LOGT) | P.dir_base, (1u << P.log2cap) - 1u, P.map_out};
    const SegBlock B = P.blocks[tl];
    const SegSlot S = P.slots[B.first_slot];
    const uint32_t f = P.map_in | ((S.flags & kSlotDesc) ? kMapComplement : 0u);
    return TileAt{size_t(S.base) + (size_t(B.blk_in_seg) << LOGT), B.blk_in_seg << LOGT,
                  (1u << B.log2cap) - 1u, B.final_pass ? f : 0u};
  };
  auto issue_load = [&](uint32_t tl, int b) {  // thread 0
    const uint32_t bar = bar0 + 8u * uint32_t(b);
    const int row = int(tile_at(tl).start >> 5);
    const uint32_t d = sbase + uint32_t(b) * SK::kSet;
    mbar_expect_tx(bar, SK::kSet);
    tma_load_2d(d, &tmk, 0, row, bar);
    tma_load_2d(d + SK::kHalf, &tmv, 0, row, bar);
  };
  auto issue_store = [&](size_t start, int b) {  // thread 0
    const int row = int(start >> 5);
    const uint32_t d = sbase + uint32_t(b) * SK::kSet;
    tma_store_2d(&tmk, 0, row, d);
    tma_store_2d(&tmv, 0, row, d + SK::kHalf);
    bulk_commit();
  };

  uint32_t tile = blockIdx.x;
  if (tile >= ntiles) return;
  if (tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmk) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&tmv) : "memory");
#pragma unroll
    for (int b = 0; b < NB; ++b) mbar_init(bar0 + 8u * uint32_t(b), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t pending = 0;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const uint32_t tl = tile + uint32_t(b) * gridDim.x;
    if (tl < ntiles) {
      if (tid == 0) issue_load(tl, b);
      pending |= 1u << b;
    }
  }

  const uint32_t lane = tid & 31u;
  const bool flip = (lane >> 4) != 0u;  // window at bit 4: pair-swapped lanes
  const uint32_t t7 = (tid >> 1) & 7u;  // window at bit 0: row tid/2's swizzle

  K kr[E];
  uint32_t vr[E];
  using SCHED = Schedule<LOGT, LOGE, true>;
  constexpr int NR = SCHED::count;

  uint32_t phase = 0;
  int b = 0;
  bool first = true;
  for (; tile < ntiles; tile += gridDim.x) {
    const uint32_t bar = bar0 + 8u * uint32_t(b);
    if (!mbar_wait_bounded(bar, (phase >> b) & 1u)) {
      if (tid == 0 && P.status != nullptr) atomicOr(P.status, int(kStatusTimeout));
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if ((pending >> q) & 1u) mbar_wait_bounded(bar0 + 8u * uint32_t(q), (phase >> q) & 1u);
      if (tid == 0) bulk_wait_all();
      return;
    }
    phase ^= 1u << b;
    pending &= ~(1u << b);
    const TileAt at = tile_at(tile);
    K* sk = reinterpret_cast<K*>(sbuf + size_t(b) * SK::kSet);
    uint32_t* sv = reinterpret_cast<uint32_t*>(sbuf + size_t(b) * SK::kSet + SK::kHalf);
    const bool asc = ((at.dir_idx & (1u << p) & at.capmask) == 0u);

    static_for<0, NR>([&](auto I) {
      constexpr int IDX = decltype(I)::value;
      constexpr SRound R = SCHED::value.r[IDX];
      constexpr int A = R.a;
      constexpr int CNT = R.cnt;
      constexpr bool LAST = (IDX + 1 == NR);
      static_assert(A == 0 || A == 4 || A >= 8, "window positions the swizzled addressing covers");
      auto body = [&](auto asc_c) {
        constexpr bool ASC = decltype(asc_c)::value;
        if constexpr (A >= 8) {
          const uint32_t tl = (tid & ((1u << A) - 1u)) | ((tid >> A) << (A + LOGE));
          const uint32_t w0 = tl ^ (((tl >> 5) & 7u) << 2);  // register r: w0 + (r << A)
#pragma unroll
          for (int r = 0; r < E; ++r) {
            kr[r] = sk[w0 + (uint32_t(r) << A)];
            vr[r] = sv[w0 + (uint32_t(r) << A)];
          }
          window_side<K, true, LOGE, ASC>(kr, vr, CNT);
#pragma unroll
          for (int r = 0; r < E; ++r) {
            sk[w0 + (uint32_t(r) << A)] = kr[r];
            sv[w0 + (uint32_t(r) << A)] = vr[r];
          }
        } else if constexpr (A == 4) {
          // register r holds window position r ^ flip: local index
          // tl | ((r ^ flip) << 4), in row (r >> 1) | ((tid >> 4) << 3)
          const uint32_t tl = (tid & 15u) | ((tid >> 4) << 8);
          const uint32_t be = tl | (uint32_t(flip) << 4);   // r even
          const uint32_t bo = tl | (uint32_t(!flip) << 4);  // r odd
          uint32_t w[E];
#pragma unroll
          for (int r = 0; r < E; ++r)
            w[r] = (((r & 1) ? bo : be) ^ (uint32_t((r >> 1) & 7) << 2)) + (uint32_t(r >> 1) << 5);
#pragma unroll
          for (int r = 0; r < E; ++r) {
            kr[r] = sk[w[r]];
            vr[r] = sv[w[r]];
          }
          window_side<K, true, LOGE, ASC>(kr, vr, CNT < 3 ? CNT : 3);
          if constexpr (CNT == 4) {
#pragma unroll
            for (int r = 0; r < E; r += 2) ce_kv_flip<ASC>(kr[r], kr[r + 1], vr[r], vr[r + 1], flip);
          }
#pragma unroll
          for (int r = 0; r < E; ++r) {
            sk[w[r]] = kr[r];
            sv[w[r]] = vr[r];
          }
        } else {
          // 16 consecutive pairs: row tid / 2, chunks 4 (tid & 1) .. +3
          const uint32_t row = (tid >> 1) << 5;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t c = ((((tid & 1u) << 2) | uint32_t(q)) ^ t7) << 2;
            const uint4 k4 = *reinterpret_cast<const uint4*>(sk + row + c);
            const uint4 v4 = *reinterpret_cast<const uint4*>(sv + row + c);
            kr[4 * q] = k4.x;
            kr[4 * q + 1] = k4.y;
            kr[4 * q + 2] = k4.z;
            kr[4 * q + 3] = k4.w;
            vr[4 * q] = v4.x;
            vr[4 * q + 1] = v4.y;
            vr[4 * q + 2] = v4.z;
            vr[4 * q + 3] = v4.w;
          }
          window_side<K, true, LOGE, ASC>(kr, vr, CNT);
          if (LAST && at.mout != 0u) {
#pragma unroll
            for (int r = 0; r < E; ++r) kr[r] = key_out<K>(kr[r], at.mout);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t c = ((((tid & 1u) << 2) | uint32_t(q)) ^ t7) << 2;
            *reinterpret_cast<uint4*>(sk + row + c) =
                make_uint4(kr[4 * q], kr[4 * q + 1], kr[4 * q + 2], kr[4 * q + 3]);
            *reinterpret_cast<uint4*>(sv + row + c) =
                make_uint4(vr[4 * q], vr[4 * q + 1], vr[4 * q + 2], vr[4 * q + 3]);
          }
        }
      };
      if (asc)
        body(std::true_type{});
      else
        body(std::false_type{});
      if constexpr (LAST) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if constexpr (IDX == 0) {
        // the previous tile's buffers: once its stores have read them, load
        // the tile NB - 1 steps ahead of this one into them
        const uint32_t nt = tile + uint32_t(NB - 1) * gridDim.x;
        const int pb = (b == 0) ? NB - 1 : b - 1;
        if (!first && nt < ntiles) {
          if (tid == 0) {
            bulk_wait_read_all();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_load(nt, pb);
          }
          pending |= 1u << pb;
        }
      }
    });
    if (tid == 0) issue_store(at.start, b);
    first = false;
    b = (b + 1 == NB) ? 0 : b + 1;
  }
  if (tid == 0) bulk_wait_all();
}

}  // namespace darm
