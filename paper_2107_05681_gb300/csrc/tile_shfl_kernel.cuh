// tile_shfl_kernel.cuh - tile pass whose stages with partner strides E .. 16E
// run across the lanes of a warp with __shfl_xor_sync instead of through
// shared memory.
//
// Every thread loads E = 2^LOGE consecutive elements of its tile from HBM and
// sorts stages k = 2 .. E in registers (Phase A, as in the plain tile pass).
// The 32 lanes of a warp then hold 32E consecutive elements: lane bit b is
// index bit LOGE + b.  Stages k = 2E .. 2^(LOGE+S), S = min(5, LOGT - LOGE),
// run without shared memory: for each such stage the layers whose partner
// i ^ j sits in another lane (E <= j < 32E) exchange keys (and payloads) with
// __shfl_xor_sync - the lane of the lower index keeps the smaller key of the
// pair when the stage's block is ascending, the larger when descending, both
// lanes deciding on the one strict predicate key[upper] < key[lower] (or >)
// - and the layers j < E run in registers.  Only then is the tile written to
// shared memory, and the stages k > 2^(LOGE+S) run the plain tile pass's
// register windows through shared memory (tile_kernel.cuh).
//
// Divergence.  The direction of stage k is index bit k, a lane bit for
// E < k < 32E: the lanes of one warp go different ways, as in Fig. 1 for
// k < 32.  A warp-level intrinsic is never part of a melded region (Section
// IV-C: melding subgraphs that hold one can deadlock), so in both forms every
// lane executes the shuffles outside the direction branch.  The divergent
// form branches on the direction around each group of compare-exchanges
// (one copy per direction); the melded form complements a descending
// thread's keys for the stage (~x reverses unsigned order) and runs the
// ascending copy only.
//
// Whole arrays (one CTA per tile) and batched segments (a persistent launch
// over a block table, as the plain tile pass).
#pragma once

#include "tile_kernel.cuh"

namespace darm {

__host__ __device__ constexpr int shfl_stages(int t, int e) { return s_min(5, t - e); }

// The window rounds that follow the shuffle stages: stages LOGE+S+1 .. LOGT,
// after a first round (Phase A + shuffle stages) that loads from HBM.
__host__ __device__ constexpr int shfl_tile_round_count(int t, int e) {
  int n = 1;
  for (int p = e + shfl_stages(t, e) + 1; p <= t; ++p) n += (p + e - 1) / e;
  return n;
}

template <int T, int E>
__host__ __device__ constexpr SSchedule<shfl_tile_round_count(T, E)> make_shfl_tile_schedule() {
  SSchedule<shfl_tile_round_count(T, E)> s{};
  int n = 0;
  const int last_shfl = E + shfl_stages(T, E);
  s.r[n++] = SRound{RK_PHASE_A, last_shfl, 0, E, LOC_GLOBAL, (T == last_shfl) ? LOC_GLOBAL : LOC_SMEM,
                    (T > E) ? 1 : 0};
  for (int p = last_shfl + 1; p <= T; ++p) {
    const int nw = (p + E - 1) / E;
    for (int i = nw - 1; i >= 0; --i) {
      const int lo = i * E;
      const int hi = s_min((i + 1) * E, p) - 1;
      const int a = hi - E + 1;
      s.r[n++] = SRound{RK_WINDOW, p, a, hi - lo + 1, LOC_SMEM, LOC_SMEM, s_lanediv(p, a, E, T)};
    }
  }
  s.r[n - 1].dst = LOC_GLOBAL;
  return s;
}

template <int T, int E>
struct ShflSchedule {
  static constexpr SSchedule<shfl_tile_round_count(T, E)> value = make_shfl_tile_schedule<T, E>();
  static constexpr int count = shfl_tile_round_count(T, E);
};

// Compare-exchange of register values x (this lane) against y (the partner
// lane's) for a group of G registers; `lower`: this lane holds the lower
// index of every pair of the layer.  ASC: the lower index ends with the
// smaller key.  Keys only: min / max; with a payload the strict predicate on
// (key[lower], key[upper]) decides whether both lanes take the partner's
// element.
template <typename K, bool V, bool ASC, int G>
__device__ __forceinline__ void shfl_ce_side(K* x, uint32_t* v, const K* y, const uint32_t* vy,
                                             bool lower) {
#pragma unroll
  for (int i = 0; i < G; ++i) {
    if constexpr (!V) {
      const K lo = kmin(x[i], y[i]);
      const K hi = kmax(x[i], y[i]);
      x[i] = (lower == ASC) ? lo : hi;
    } else {
      const K kl = lower ? x[i] : y[i];  // key at the lower index
      const K ku = lower ? y[i] : x[i];  // key at the upper index
      const bool s = ASC ? (ku < kl) : (ku > kl);
      x[i] = s ? y[i] : x[i];
      v[i] = s ? vy[i] : v[i];
    }
  }
}

// One layer whose partner is lane ^ LM: shuffles for every register (all
// lanes, outside the direction branch), then the compare-exchanges.
template <typename K, bool V, int LOGE, int VAR, uint32_t MASK>
__device__ __forceinline__ void shfl_layer(K (&kr)[1 << LOGE], uint32_t (&vr)[1 << LOGE],
                                           uint32_t lm, bool asc, bool lanediv) {
  constexpr int E = 1 << LOGE;
  constexpr int G = (E < 8) ? E : 8;  // registers per shuffle group
  const bool lower = (threadIdx.x & lm) == 0u;
#pragma unroll
  for (int g = 0; g < E; g += G) {
    K y[G];
    uint32_t vy[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      y[i] = __shfl_xor_sync(MASK, kr[g + i], lm);
      vy[i] = V ? __shfl_xor_sync(MASK, vr[g + i], lm) : 0u;
    }
    if (VAR == kDivergent || !lanediv) {
      if (asc)
        shfl_ce_side<K, V, true, G>(kr + g, vr + g, y, vy, lower);
      else
        shfl_ce_side<K, V, false, G>(kr + g, vr + g, y, vy, lower);
    } else {
      // melded: the keys of a descending thread are complemented for the
      // whole stage, so one ascending copy serves both directions
      shfl_ce_side<K, V, true, G>(kr + g, vr + g, y, vy, lower);
    }
  }
}

// Rounds of the schedule through stage 2^c (a segment of capacity 2^c stops
// there): the first round holds every stage up to 2^(LOGE+S).
__host__ __device__ constexpr int shfl_rounds_through(int c, int t, int e) {
  int n = 1;
  for (int p = e + shfl_stages(t, e) + 1; p <= c; ++p) n += (p + e - 1) / e;
  return n;
}

// One tile of the pass.  `bidx` is the block number, or the entry of the
// segmented block table (segments padded with sentinels, small segments
// packed into one tile, as in tile_kernel.cuh's tile_block).
template <typename K, bool V, int LOGE, int LOGT, int VAR, uint32_t MASK, bool SEG>
__device__ __forceinline__ void tile_block_shfl(const PassParams& P, uint32_t bidx, K* sk,
                                                uint32_t* sv) {
  constexpr int E = 1 << LOGE;
  constexpr int S = shfl_stages(LOGT, LOGE);
  constexpr int PADT = TilePad<K, V, LOGE>::value;
  K* __restrict__ gk = reinterpret_cast<K*>(P.keys);
  uint32_t* __restrict__ gv = P.vals;
  const uint32_t tid = threadIdx.x;

  uint32_t blk = bidx;
  uint32_t log2cap = P.log2cap;
  uint32_t nrounds = P.nrounds;
  bool final_pass = true;
  bool fill = false;
  const SegSlot* slots = nullptr;
  if (SEG && P.blocks != nullptr) {
    const SegBlock B = P.blocks[bidx];
    blk = B.blk_in_seg;
    log2cap = B.log2cap;
    nrounds = B.nrounds;
    final_pass = B.final_pass != 0;
    fill = B.fill != 0;
    slots = P.slots + B.first_slot;
  }
  const uint32_t gblk = blk << LOGT;
  const uint32_t capmask = (1u << log2cap) - 1u;

  K kr[E];
  uint32_t vr[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    if (SEG) kr[r] = K(0);  // threads of an unused slot shuffle these
    vr[r] = 0;
  }

  using SCHED = ShflSchedule<LOGT, LOGE>;
  constexpr int NR = SCHED::count;
  bool done = false;
  static_for<0, NR>([&](auto I) {
    constexpr int IDX = decltype(I)::value;
    constexpr SRound R = SCHED::value.r[IDX];
    constexpr int A = R.a;
    if (SEG && done) return;
    // whole arrays run every round: `last` is a compile-time constant there
    const bool last = SEG ? (uint32_t(IDX) + 1 == nrounds) : (IDX + 1 == NR);
    const bool from_global = (R.src == LOC_GLOBAL);
    const bool to_global = last || (R.dst == LOC_GLOBAL);
    const uint32_t tl = (tid & ((1u << A) - 1u)) | ((tid >> A) << (A + LOGE));
    const uint32_t g_full = tl | gblk;
    const uint32_t s_base = Interleave<K, V>::value ? phys8(tl) : physp<PADT>(tl);
    uint32_t min_ = 0, mout = 0, g_t = g_full;
    K* bk = gk;
    uint32_t* bv = gv;
    uint32_t seg_len = 0xFFFFFFFFu;
    bool skip = false;  // unused slot of a packed block: touch no memory
    if (SEG && slots != nullptr && (from_global || to_global)) {
      const SegSlot Sl = slots[g_full >> log2cap];
      bk = gk + Sl.base;
      if (V) bv = gv + Sl.base;
      seg_len = Sl.len;
      skip = (Sl.flags & kSlotEmpty) != 0;
      const uint32_t f = P.map_in | ((Sl.flags & kSlotDesc) ? kMapComplement : 0u);
      if (IDX == 0 && from_global && fill) min_ = f;
      if (last && final_pass) mout = f;
      g_t = g_full & capmask;
    } else {
      if (IDX == 0 && from_global) min_ = P.map_in;
      if (last) mout = P.map_out;
    }
    const uint32_t g_dir = (g_full | P.dir_base) & capmask;
    const bool do_store = !(to_global && skip);
    if constexpr (R.kind == RK_PHASE_A) {
      if (!skip)
        s_load<K, V, LOGE, 0, false, PADT>(kr, vr, true, bk, bv, g_t, sk, sv, s_base, min_, K(0));
      if (SEG && fill) {
        bool collide = false;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const uint32_t pos = g_t + uint32_t(r);
          if (pos >= seg_len) {
            kr[r] = ~K(0);
            if (V) vr[r] = 0xFFFFFFFFu;
          } else if (V && kr[r] == ~K(0)) {
            collide = true;
          }
        }
        if (collide && !skip && P.status != nullptr) atomicOr(P.status, int(kStatusSentinelCollision));
      }
      phase_a_small<K, V, LOGE>(kr, vr, log2cap);
      if (uint32_t(LOGE) <= log2cap) {
        const bool asc = ((g_dir & uint32_t(E)) == 0u);
        if (VAR == kDivergent) {
          if (asc)
            window_side<K, V, LOGE, true>(kr, vr, LOGE);
          else
            window_side<K, V, LOGE, false>(kr, vr, LOGE);
        } else {
          const K m = asc ? K(0) : ~K(0);
#pragma unroll
          for (int r = 0; r < E; ++r) kr[r] ^= m;
          window_side<K, V, LOGE, true>(kr, vr, LOGE);
#pragma unroll
          for (int r = 0; r < E; ++r) kr[r] ^= m;
        }
      }
      // stages 2E .. 2^(LOGE+S): lane layers by shuffles, then registers.
      // The condition is uniform per block (one capacity per block), so
      // every lane of a warp takes part in every shuffle.
      static_for<1, S + 1>([&](auto SI) {
        constexpr int P_ = LOGE + decltype(SI)::value;
        if (uint32_t(P_) > log2cap) return;
        const bool asc = ((g_dir & (1u << P_)) == 0u);
        constexpr bool LANEDIV = (P_ - LOGE) < 5;  // bit P_ is a lane bit
        const K m = (VAR == kMelded && LANEDIV && !asc) ? ~K(0) : K(0);
        if (VAR == kMelded && LANEDIV) {
#pragma unroll
          for (int r = 0; r < E; ++r) kr[r] ^= m;
        }
        static_for<0, P_ - LOGE>([&](auto QI) {
          constexpr int Q = P_ - 1 - decltype(QI)::value;  // layer bit, high to low
          shfl_layer<K, V, LOGE, VAR, MASK>(kr, vr, 1u << (Q - LOGE), asc, LANEDIV);
        });
        if (VAR == kDivergent || !LANEDIV) {
          if (asc)
            window_side<K, V, LOGE, true>(kr, vr, LOGE);
          else
            window_side<K, V, LOGE, false>(kr, vr, LOGE);
        } else {
          window_side<K, V, LOGE, true>(kr, vr, LOGE);
#pragma unroll
          for (int r = 0; r < E; ++r) kr[r] ^= m;
        }
      });
      if (do_store)
        s_store<K, V, LOGE, 0, false, false, PADT>(kr, vr, to_global, bk, bv, g_t, sk, sv, s_base,
                                                   mout, K(0));
    } else {
      const bool asc = ((g_dir & (1u << R.p)) == 0u);
      if (VAR == kDivergent || !R.lanediv) {
        if (asc) {
          s_load<K, V, LOGE, A, false, PADT>(kr, vr, false, bk, bv, g_t, sk, sv, s_base, 0u, K(0));
          window_side<K, V, LOGE, true>(kr, vr, R.cnt);
          if (do_store)
            s_store<K, V, LOGE, A, false, false, PADT>(kr, vr, to_global, bk, bv, g_t, sk, sv,
                                                       s_base, mout, K(0));
        } else {
          s_load<K, V, LOGE, A, true, PADT>(kr, vr, false, bk, bv, g_t, sk, sv, s_base, 0u, K(0));
          window_side<K, V, LOGE, false>(kr, vr, R.cnt);
          if (do_store)
            s_store<K, V, LOGE, A, true, false, PADT>(kr, vr, to_global, bk, bv, g_t, sk, sv,
                                                      s_base, mout, K(0));
        }
      } else {
        const K m = asc ? K(0) : ~K(0);
        s_load<K, V, LOGE, A, false, PADT>(kr, vr, false, bk, bv, g_t, sk, sv, s_base, 0u, m);
        window_side<K, V, LOGE, true>(kr, vr, R.cnt);
        if (do_store)
          s_store<K, V, LOGE, A, false, false, PADT>(kr, vr, to_global, bk, bv, g_t, sk, sv, s_base,
                                                     mout, m);
      }
    }
    if (to_global) {
      done = true;
    } else {
      __syncthreads();
    }
  });
  (void)done;
}

// SEG: the launch may address segments through a block table and take
// blocks persistently (batched sorts); without it, whole arrays only (the
// table logic compiled out, which spares registers).
template <typename K, bool V, int LOGE, int LOGT, int VAR, int MAXT, bool SEG = false>
__global__ void __launch_bounds__(MAXT, tile_min_blocks(MAXT))
    darm_tile_shfl_kernel(const __grid_constant__ PassParams P) {
  constexpr int S = shfl_stages(LOGT, LOGE);
  constexpr int LANES = (MAXT < 32) ? MAXT : 32;
  constexpr uint32_t MASK = (LANES == 32) ? 0xFFFFFFFFu : ((1u << LANES) - 1u);
  static_assert(MAXT == (1 << (LOGT - LOGE)), "one tile per CTA");
  static_assert((1 << S) <= LANES, "shuffle stages stay inside a warp");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* sk = reinterpret_cast<K*>(smem_raw);
  uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + sizeof(K) * smem_words(1u << LOGT));
  if (!SEG || P.work_counter == nullptr) {
    tile_block_shfl<K, V, LOGE, LOGT, VAR, MASK, SEG>(P, blockIdx.x, sk, sv);
    return;
  }
  // persistent: blocks of the table (longest segments first) are taken in
  // order from a global counter as CTAs become free
  __shared__ uint32_t s_next;
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(P.work_counter, 1u);
    __syncthreads();
    const uint32_t b = s_next;
    __syncthreads();
    if (b >= P.nblocks) break;
    tile_block_shfl<K, V, LOGE, LOGT, VAR, MASK, SEG>(P, b, sk, sv);
  }
}

}  // namespace darm
