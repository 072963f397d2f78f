// tma_merge.cuh - persistent merge pass that prefetches tiles with the
// bulk-copy (TMA) engine.
//
// A merge pass of stage k > T runs layers T/2 .. 1 on every tile of T
// elements.  The plain merge kernel loads a tile, processes it and stores it,
// so an SM alternates between waiting on HBM and working on shared memory.
// Here one CTA per SM (or a few) walks over tiles
// (tile = blockIdx.x + i * gridDim.x) with NS dense staging buffers:
//   - one thread issues cp.async.bulk copies of a tile's keys (and payload)
//     into a free staging buffer, completing on that buffer's mbarrier;
//   - round 0 reads the staged tile (dense, the window's lanes are
//     consecutive elements), runs its layers and writes the padded work
//     buffer; the staging buffer is then free and the copy of the tile NS
//     steps ahead is issued at once, so NS tiles stream in while rounds
//     1 .. n-1 run;
//   - the last round stores straight from registers to HBM, in 256-bit
//     stores where the address allows.
// Waits on an mbarrier are bounded (about one second of %globaltimer); if one
// runs out the kernel latches DARM_ERR_TIMEOUT in the status word, waits
// (bounded again) for the copies it still has in flight and returns instead
// of hanging.
#pragma once

#include <type_traits>

#include "tile_kernel.cuh"

namespace darm {

constexpr uint32_t kStatusTimeout = 7u;  // == DARM_ERR_TIMEOUT

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of the barrier for at most ~1 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > 1000000000ull) return false;
  }
}

template <typename K, bool V, int LOGT, int NS>
struct TmaMergeSmem {
  static constexpr uint32_t kTile = 1u << LOGT;
  static constexpr size_t kStageK = size_t(kTile) * sizeof(K);
  static constexpr size_t kStageV = V ? size_t(kTile) * 4 : 0;
  static constexpr size_t kStage = kStageK + kStageV;  // one staging buffer
  static constexpr size_t kWork = size_t(sizeof(K) + (V ? 4 : 0)) * smem_words(kTile);
  static constexpr size_t kWorkOff = NS * kStage;
  static constexpr size_t kBarOff = (kWorkOff + kWork + 15) / 16 * 16;
  static constexpr size_t kBytes = kBarOff + 8 * NS;
};

// Block size MAXT = threads of one tile; small tiles ask for 64 registers so
// that several CTAs share an SM.
// SH (keys only): two rounds instead of three.  Round 0 runs the top LOGE
// layers from the staging buffer into the work buffer as usual; round 1 loads
// each thread's E consecutive keys, runs the layers whose partner is in
// another lane of the warp with __shfl_xor_sync (partner strides E .. 16E)
// and the layers below E in registers, and stores to HBM.  The direction is
// uniform per tile, so no lane diverges.
template <typename K, int LOGE, uint32_t MASK>
__device__ __forceinline__ void merge_shfl_layer(K (&kr)[1 << LOGE], uint32_t lm, bool asc) {
  const bool keep_min = ((threadIdx.x & lm) == 0u) == asc;
#pragma unroll
  for (int r = 0; r < (1 << LOGE); ++r) {
    const K y = __shfl_xor_sync(MASK, kr[r], lm);
    const K lo = kmin(kr[r], y);
    const K hi = kmax(kr[r], y);
    kr[r] = keep_min ? lo : hi;
  }
}

template <typename K, bool V, int LOGE, int LOGT, int NS, int VAR, int MAXT, bool SH = false>
__global__ void __launch_bounds__(MAXT, (MAXT <= 256) ? 4 : 1) darm_merge_tma_kernel(const __grid_constant__ PassParams P) {
  static_assert(!SH || (!V && MAXT >= 32 && LOGT - LOGE >= LOGE && LOGT - 2 * LOGE <= 5),
                "two-round merge: keys only, the lane bits cover what the two windows leave");
  static_assert(NS >= 1 && NS <= 4, "one to four staging buffers");
  constexpr int E = 1 << LOGE;
  using L = TmaMergeSmem<K, V, LOGT, NS>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* sk = reinterpret_cast<K*>(smem_raw + L::kWorkOff);
  uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + L::kWorkOff + sizeof(K) * smem_words(L::kTile));
  const uint32_t bar0 = smem_addr(smem_raw + L::kBarOff);

  K* __restrict__ gk = reinterpret_cast<K*>(P.keys);
  uint32_t* __restrict__ gv = P.vals;
  const uint32_t tid = threadIdx.x;
  const uint32_t ntiles = P.nblocks;
  const uint32_t p = P.rounds[0].p;
  constexpr uint32_t kBytes = uint32_t(L::kStage);

  // Tile `tl` of this launch: its first element in the arrays, the index
  // its comparator directions are taken from, the capacity mask of the
  // sequence it belongs to and the key map its last store undoes.  Whole
  // arrays: tile tl of the array.  Batches: entry tl of the block table, a
  // tile of one segment (merge blocks never pack several segments).
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
  // copy tile `tl` into staging buffer `b` (thread 0 only)
  auto issue = [&](uint32_t tl, int b) {
    const uint32_t bar = bar0 + 8u * uint32_t(b);
    unsigned char* st = smem_raw + size_t(b) * L::kStage;
    const size_t start = tile_at(tl).start;
    mbar_expect_tx(bar, kBytes);
    bulk_g2s(smem_addr(st), gk + start, uint32_t(L::kStageK), bar);
    if (V) bulk_g2s(smem_addr(st + L::kStageK), gv + start, uint32_t(L::kStageV), bar);
  };

  uint32_t tile = blockIdx.x;
  if (tile >= ntiles) return;
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < NS; ++b) mbar_init(bar0 + 8u * uint32_t(b), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // Every thread keeps the same account of which buffers have a copy in
  // flight (bit b of `pending`) and of each barrier's phase (bit b of
  // `phase`), so that a timed-out wait can drain them.
  uint32_t pending = 0;
#pragma unroll
  for (int b = 0; b < NS; ++b) {
    const uint32_t tl = tile + uint32_t(b) * gridDim.x;
    if (tl < ntiles) {
      if (tid == 0) issue(tl, b);
      pending |= 1u << b;
    }
  }

  using SCHED = Schedule<LOGT, LOGE, true>;
  constexpr int NR = SCHED::count;
  K kr[E];
  uint32_t vr[E];
#pragma unroll
  for (int r = 0; r < E; ++r) vr[r] = 0;

  uint32_t phase = 0;
  int b = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    const uint32_t bar = bar0 + 8u * uint32_t(b);
    if (!mbar_wait_bounded(bar, (phase >> b) & 1u)) {
      if (tid == 0 && P.status != nullptr) atomicOr(P.status, int(kStatusTimeout));
      // give every copy in flight a last bounded chance to land before leaving
#pragma unroll
      for (int q = 0; q < NS; ++q)
        if ((pending >> q) & 1u) mbar_wait_bounded(bar0 + 8u * uint32_t(q), (phase >> q) & 1u);
      return;
    }
    phase ^= 1u << b;
    pending &= ~(1u << b);
    const K* stage_k = reinterpret_cast<const K*>(smem_raw + size_t(b) * L::kStage);
    const uint32_t* stage_v = reinterpret_cast<const uint32_t*>(smem_raw + size_t(b) * L::kStage + L::kStageK);
    const TileAt at = tile_at(tile);
    K* const tk = gk + at.start;
    uint32_t* const tv = V ? gv + at.start : nullptr;
    const bool asc = ((at.dir_idx & (1u << p) & at.capmask) == 0u);
    const uint32_t next = tile + uint32_t(NS) * gridDim.x;

    if constexpr (SH) {
      constexpr int A0 = LOGT - LOGE;  // round 0: window bits A0 .. LOGT-1
      {
        const uint32_t tl = (tid & ((1u << A0) - 1u)) | ((tid >> A0) << (A0 + LOGE));
        auto body = [&](auto asc_c) {
          constexpr bool ASC = decltype(asc_c)::value;
#pragma unroll
          for (int r = 0; r < E; ++r) kr[r] = stage_k[tl | (uint32_t(r) << A0)];
          window_side<K, V, LOGE, ASC, true>(kr, vr, LOGE);
          s_store<K, V, LOGE, A0, false, true>(kr, vr, false, tk, tv, 0u, sk, sv, phys(tl), 0u, K(0));
        };
        if (asc)
          body(std::true_type{});
        else
          body(std::false_type{});
      }
      __syncthreads();
      if (next < ntiles) {
        if (tid == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue(next, b);
        }
        pending |= 1u << b;
      }
      {
        // round 1: E consecutive keys per thread; lane bits are index bits
        // LOGE .. LOGE+4
        const uint32_t tl = tid << LOGE;
        s_load<K, V, LOGE, 0, false>(kr, vr, false, tk, tv, 0u, sk, sv, phys(tl), 0u, K(0));
#pragma unroll
        for (int q = A0 - 1; q >= LOGE; --q)
          merge_shfl_layer<K, LOGE, 0xFFFFFFFFu>(kr, 1u << (q - LOGE), asc);
        if (asc)
          window_side<K, V, LOGE, true, true>(kr, vr, LOGE);
        else
          window_side<K, V, LOGE, false, true>(kr, vr, LOGE);
        s_store<K, V, LOGE, 0, false, true>(kr, vr, true, tk, tv, tl, sk, sv, 0u, at.mout, K(0));
      }
      __syncthreads();
      b = (b + 1 == NS) ? 0 : b + 1;
      continue;
    }
    static_for<0, NR>([&](auto I) {
      constexpr int IDX = decltype(I)::value;
      constexpr SRound R = SCHED::value.r[IDX];
      constexpr int A = R.a;
      constexpr bool LAST = (IDX + 1 == NR);
      const uint32_t tl = (tid & ((1u << A) - 1u)) | ((tid >> A) << (A + LOGE));
      const uint32_t g_full = tl;  // relative to the tile's first element
      const uint32_t s_base = Interleave<K, V>::value ? phys8(tl) : phys(tl);
      const uint32_t mout = LAST ? at.mout : 0u;
      if constexpr (IDX == 0) {
        // from the dense staging buffer into the padded work buffer
        auto body = [&](auto asc_c) {
          constexpr bool ASC = decltype(asc_c)::value;
#pragma unroll
          for (int r = 0; r < E; ++r) {
            const uint32_t l = tl | (uint32_t(r) << A);
            kr[r] = stage_k[l];
            if (V) vr[r] = stage_v[l];
          }
          window_side<K, V, LOGE, ASC, true>(kr, vr, R.cnt);
          s_store<K, V, LOGE, A, false, true>(kr, vr, LAST, tk, tv, g_full, sk, sv, s_base, mout, K(0));
        };
        if (asc)
          body(std::true_type{});
        else
          body(std::false_type{});
        __syncthreads();
        // the staging buffer is free: stream the tile NS steps ahead in
        // behind the remaining rounds
        if (next < ntiles) {
          if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(next, b);
          }
          pending |= 1u << b;
        }
      } else {
        if (asc) {
          s_load<K, V, LOGE, A, false>(kr, vr, false, tk, tv, g_full, sk, sv, s_base, 0u, K(0));
          window_side<K, V, LOGE, true, true>(kr, vr, R.cnt);
          s_store<K, V, LOGE, A, false, true>(kr, vr, LAST, tk, tv, g_full, sk, sv, s_base, mout, K(0));
        } else {
          s_load<K, V, LOGE, A, true>(kr, vr, false, tk, tv, g_full, sk, sv, s_base, 0u, K(0));
          window_side<K, V, LOGE, false, true>(kr, vr, R.cnt);
          s_store<K, V, LOGE, A, true, true>(kr, vr, LAST, tk, tv, g_full, sk, sv, s_base, mout, K(0));
        }
        __syncthreads();
      }
    });
    b = (b + 1 == NS) ? 0 : b + 1;
  }
}

}  // namespace darm
