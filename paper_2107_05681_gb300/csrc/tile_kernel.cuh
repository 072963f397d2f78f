// tile_kernel.cuh - tile and merge passes with their round schedule fixed
// at compile time.
//
// Same network, rounds and direction handling as darm_pass_kernel
// (pass_kernel.cuh), specialised for one tile size T = 2^LOGT and
// E = 2^LOGE elements per thread: every window position, layer count and
// direction bit is a template constant, so shared-memory and global offsets
// of every register are immediates and the round loop disappears.
//   MERGE = false  tile pass: stages k = 2 .. T (Phase A in registers for
//                  k <= E, then register windows through shared memory);
//   MERGE = true   merge pass of one stage k > T (runtime p): layers
//                  j = T/2 .. 1 inside the tile, direction uniform per block.
#pragma once

#include "pass_kernel.cuh"

namespace darm {

struct SRound {
  int kind;     // RK_PHASE_A or RK_WINDOW
  int p;        // stage bit (tile pass; merge passes take p at run time)
  int a;        // window position
  int cnt;      // layers (top `cnt` window bits)
  int src, dst; // Loc
  int lanediv;  // direction can differ between lanes of a warp
};

template <int N>
struct SSchedule {
  SRound r[N];
};

__host__ __device__ constexpr int s_min(int x, int y) { return x < y ? x : y; }

// Lane j of a round with window a..a+e-1 sits at local bit (j < a ? j : j + e).
__host__ __device__ constexpr int s_lanediv(int p, int a, int e, int t) {
  if (p >= t) return 0;
  const int lanes = s_min(5, t - e);
  for (int j = 0; j < lanes; ++j)
    if (((j < a) ? j : j + e) == p) return 1;
  return 0;
}

__host__ __device__ constexpr int tile_round_count(int t, int e) {
  int n = 1;
  for (int p = e + 1; p <= t; ++p) n += (p + e - 1) / e;
  return n;
}

template <int T, int E>
__host__ __device__ constexpr SSchedule<tile_round_count(T, E)> make_tile_schedule() {
  SSchedule<tile_round_count(T, E)> s{};
  int n = 0;
  s.r[n++] = SRound{RK_PHASE_A, E, 0, E, LOC_GLOBAL, (T == E) ? LOC_GLOBAL : LOC_SMEM,
                    (T > E) ? 1 : 0};
  for (int p = E + 1; p <= T; ++p) {
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

__host__ __device__ constexpr int merge_round_count(int t, int e) { return (t + e - 1) / e; }

template <int T, int E>
__host__ __device__ constexpr SSchedule<merge_round_count(T, E)> make_merge_schedule() {
  SSchedule<merge_round_count(T, E)> s{};
  int n = 0;
  const int nw = (T + E - 1) / E;
  for (int i = nw - 1; i >= 0; --i) {
    const int lo = i * E;
    const int hi = s_min((i + 1) * E, T) - 1;
    s.r[n++] = SRound{RK_WINDOW, 0, hi - E + 1, hi - lo + 1, LOC_SMEM, LOC_SMEM, 0};
  }
  s.r[0].src = LOC_GLOBAL;
  s.r[n - 1].dst = LOC_GLOBAL;
  return s;
}

template <int T, int E, bool MERGE>
struct Schedule;
template <int T, int E>
struct Schedule<T, E, false> {
  static constexpr SSchedule<tile_round_count(T, E)> value = make_tile_schedule<T, E>();
  static constexpr int count = tile_round_count(T, E);
};
template <int T, int E>
struct Schedule<T, E, true> {
  static constexpr SSchedule<merge_round_count(T, E)> value = make_merge_schedule<T, E>();
  static constexpr int count = merge_round_count(T, E);
};

template <int I>
struct IC {
  static constexpr int value = I;
};

template <int I, int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(IC<I>{});
    static_for<I + 1, N>(f);
  }
}

// 256-bit global stores (sm_100 and later): a thread that owns eight or
// more consecutive 32-bit words writes them as whole 32-byte sectors, so no
// sector of a warp's store is written in two halves by two instructions.
// The address must be 32-byte aligned; callers fall back to 128-bit stores
// otherwise.
__device__ __forceinline__ bool aligned32(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 31u) == 0;
}

__device__ __forceinline__ void st_global_v8(void* p, const uint32_t (&w)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]),
               "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
               : "memory");
}

// Key-value tiles with 32-bit keys keep each (key, payload) pair together in
// one 8-byte shared-memory slot, so one 64-bit access moves both.  Pair l
// lives at slot phys8(l) = l + 2 * (l / 16): two pad slots after every 16
// pairs keep the bottom window's 16-byte accesses and the lanes of the
// higher windows on distinct banks.  phys8 is additive over disjoint bits,
// like phys.
template <typename K, bool V>
struct Interleave {
  static constexpr bool value = V && sizeof(K) == 4;
};
__host__ __device__ constexpr uint32_t phys8_c(uint32_t l) { return l + ((l >> 4) << 1); }

// Pad words per 32 elements of the tile kernels' own shared memory.  Tiles
// of 32-bit keys without payload and 32 keys per thread pad one word per 32
// keys: local bit b >= 5 then moves an index by 2^(b-5) banks, so the lanes
// of every round (local bits 0..a-1 and a+5..9 for a window at bit a) fall
// on 32 distinct banks, including the rounds whose window starts at bits
// 1..4, where four pad words per 32 keys leave 2- to 4-way conflicts.  The
// price is that the bottom-window rounds (window at bit 0) move words one at
// a time instead of in 16-byte vectors (same wavefronts, more instructions).
// Other shapes keep four pad words (16-byte aligned rows).
template <typename K, bool V, int LOGE>
struct TilePad {
  static constexpr int value = (!V && sizeof(K) == 4 && LOGE == 5) ? 1 : 4;
};
template <int PAD>
__host__ __device__ constexpr uint32_t physp(uint32_t l) { return l + (l >> 5) * uint32_t(PAD); }

// Static-offset element access: register r of a round with window A sits at
// local index tl | (r << A); phys() is additive over disjoint bits, so its
// shared-memory word is phys(tl) + phys(r << A), a compile-time offset.
template <typename K, bool V, int LOGE, int A, bool REV, int PAD = 4>
__device__ __forceinline__ void s_load(K (&kr)[1 << LOGE], uint32_t (&vr)[1 << LOGE], bool from_global,
                                       const K* __restrict__ gk, const uint32_t* __restrict__ gv,
                                       uint32_t g_t, const K* sk, const uint32_t* sv,
                                       uint32_t s_base, uint32_t mapf, K m) {
  constexpr int E = 1 << LOGE;
  constexpr int KPV = 16 / sizeof(K);
  if (from_global) {
    if constexpr (A == 0 && E >= KPV) {
#pragma unroll
      for (int q0 = 0; q0 < E / KPV; ++q0) {
        const int q = REV ? (E / KPV - 1 - q0) : q0;
        const uint4 w = *reinterpret_cast<const uint4*>(gk + g_t + q * KPV);
        const K* wk = reinterpret_cast<const K*>(&w);
#pragma unroll
        for (int u = 0; u < KPV; ++u) kr[q * KPV + u] = key_in<K>(wk[u], mapf) ^ m;
      }
      if constexpr (V && E >= 4) {
#pragma unroll
        for (int q0 = 0; q0 < E / 4; ++q0) {
          const int q = REV ? (E / 4 - 1 - q0) : q0;
          const uint4 w = *reinterpret_cast<const uint4*>(gv + g_t + q * 4);
          vr[q * 4 + 0] = w.x;
          vr[q * 4 + 1] = w.y;
          vr[q * 4 + 2] = w.z;
          vr[q * 4 + 3] = w.w;
        }
      } else if constexpr (V) {
#pragma unroll
        for (int r = 0; r < E; ++r) vr[r] = gv[g_t + r];
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        kr[r] = key_in<K>(gk[g_t + (uint32_t(r) << A)], mapf) ^ m;
        if (V) vr[r] = gv[g_t + (uint32_t(r) << A)];
      }
    }
  } else if constexpr (Interleave<K, V>::value) {
    const uint2* s2 = reinterpret_cast<const uint2*>(sk);
    if constexpr (A == 0) {
#pragma unroll
      for (int q0 = 0; q0 < E / 2; ++q0) {
        const int q = REV ? (E / 2 - 1 - q0) : q0;
        const uint4 w = *reinterpret_cast<const uint4*>(s2 + s_base + phys8_c(uint32_t(2 * q)));
        kr[2 * q] = K(w.x) ^ m;
        vr[2 * q] = w.y;
        kr[2 * q + 1] = K(w.z) ^ m;
        vr[2 * q + 1] = w.w;
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint2 w = s2[s_base + phys8_c(uint32_t(r) << A)];
        kr[r] = K(w.x) ^ m;
        vr[r] = w.y;
      }
    }
  } else {
    if constexpr (PAD == 4 && A == 0 && E >= KPV) {
#pragma unroll
      for (int q0 = 0; q0 < E / KPV; ++q0) {
        const int q = REV ? (E / KPV - 1 - q0) : q0;
        const uint4 w = *reinterpret_cast<const uint4*>(sk + s_base + q * KPV);
        const K* wk = reinterpret_cast<const K*>(&w);
#pragma unroll
        for (int u = 0; u < KPV; ++u) kr[q * KPV + u] = wk[u] ^ m;
      }
      if constexpr (V && E >= 4) {
#pragma unroll
        for (int q0 = 0; q0 < E / 4; ++q0) {
          const int q = REV ? (E / 4 - 1 - q0) : q0;
          const uint4 w = *reinterpret_cast<const uint4*>(sv + s_base + q * 4);
          vr[q * 4 + 0] = w.x;
          vr[q * 4 + 1] = w.y;
          vr[q * 4 + 2] = w.z;
          vr[q * 4 + 3] = w.w;
        }
      } else if constexpr (V) {
#pragma unroll
        for (int r = 0; r < E; ++r) vr[r] = sv[s_base + r];
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint32_t off = physp<PAD>(uint32_t(r << A));
        kr[r] = sk[s_base + off] ^ m;
        if (V) vr[r] = sv[s_base + off];
      }
    }
  }
}

template <typename K, bool V, int LOGE, int A, bool REV, bool WIDE = false, int PAD = 4>
__device__ __forceinline__ void s_store(const K (&kr)[1 << LOGE], const uint32_t (&vr)[1 << LOGE],
                                        bool to_global, K* __restrict__ gk, uint32_t* __restrict__ gv,
                                        uint32_t g_t, K* sk, uint32_t* sv, uint32_t s_base,
                                        uint32_t mapf, K m) {
  constexpr int E = 1 << LOGE;
  constexpr int KPV = 16 / sizeof(K);
  if (to_global) {
    if constexpr (WIDE && A == 0 && sizeof(K) == 4 && E >= 8) {
      if (aligned32(gk + g_t) && (!V || aligned32(gv + g_t))) {
#pragma unroll
        for (int q0 = 0; q0 < E / 8; ++q0) {
          const int q = REV ? (E / 8 - 1 - q0) : q0;
          uint32_t w[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) w[u] = uint32_t(key_out<K>(kr[q * 8 + u] ^ m, mapf));
          st_global_v8(gk + g_t + q * 8, w);
          if constexpr (V) {
#pragma unroll
            for (int u = 0; u < 8; ++u) w[u] = vr[q * 8 + u];
            st_global_v8(gv + g_t + q * 8, w);
          }
        }
        return;
      }
    }
    if constexpr (A == 0 && E >= KPV) {
#pragma unroll
      for (int q0 = 0; q0 < E / KPV; ++q0) {
        const int q = REV ? (E / KPV - 1 - q0) : q0;
        uint4 w;
        K* wk = reinterpret_cast<K*>(&w);
#pragma unroll
        for (int u = 0; u < KPV; ++u) wk[u] = key_out<K>(kr[q * KPV + u] ^ m, mapf);
        *reinterpret_cast<uint4*>(gk + g_t + q * KPV) = w;
      }
      if constexpr (V && E >= 4) {
#pragma unroll
        for (int q0 = 0; q0 < E / 4; ++q0) {
          const int q = REV ? (E / 4 - 1 - q0) : q0;
          uint4 w;
          w.x = vr[q * 4 + 0];
          w.y = vr[q * 4 + 1];
          w.z = vr[q * 4 + 2];
          w.w = vr[q * 4 + 3];
          *reinterpret_cast<uint4*>(gv + g_t + q * 4) = w;
        }
      } else if constexpr (V) {
#pragma unroll
        for (int r = 0; r < E; ++r) gv[g_t + r] = vr[r];
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        gk[g_t + (uint32_t(r) << A)] = key_out<K>(kr[r] ^ m, mapf);
        if (V) gv[g_t + (uint32_t(r) << A)] = vr[r];
      }
    }
  } else if constexpr (Interleave<K, V>::value) {
    uint2* s2 = reinterpret_cast<uint2*>(sk);
    if constexpr (A == 0) {
#pragma unroll
      for (int q0 = 0; q0 < E / 2; ++q0) {
        const int q = REV ? (E / 2 - 1 - q0) : q0;
        uint4 w;
        w.x = uint32_t(kr[2 * q] ^ m);
        w.y = vr[2 * q];
        w.z = uint32_t(kr[2 * q + 1] ^ m);
        w.w = vr[2 * q + 1];
        *reinterpret_cast<uint4*>(s2 + s_base + phys8_c(uint32_t(2 * q))) = w;
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        s2[s_base + phys8_c(uint32_t(r) << A)] = make_uint2(uint32_t(kr[r] ^ m), vr[r]);
      }
    }
  } else {
    if constexpr (PAD == 4 && A == 0 && E >= KPV) {
#pragma unroll
      for (int q0 = 0; q0 < E / KPV; ++q0) {
        const int q = REV ? (E / KPV - 1 - q0) : q0;
        uint4 w;
        K* wk = reinterpret_cast<K*>(&w);
#pragma unroll
        for (int u = 0; u < KPV; ++u) wk[u] = kr[q * KPV + u] ^ m;
        *reinterpret_cast<uint4*>(sk + s_base + q * KPV) = w;
      }
      if constexpr (V && E >= 4) {
#pragma unroll
        for (int q0 = 0; q0 < E / 4; ++q0) {
          const int q = REV ? (E / 4 - 1 - q0) : q0;
          uint4 w;
          w.x = vr[q * 4 + 0];
          w.y = vr[q * 4 + 1];
          w.z = vr[q * 4 + 2];
          w.w = vr[q * 4 + 3];
          *reinterpret_cast<uint4*>(sv + s_base + q * 4) = w;
        }
      } else if constexpr (V) {
#pragma unroll
        for (int r = 0; r < E; ++r) sv[s_base + r] = vr[r];
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint32_t off = physp<PAD>(uint32_t(r << A));
        sk[s_base + off] = kr[r] ^ m;
        if (V) sv[s_base + off] = vr[r];
      }
    }
  }
}

// One block of a tile or merge pass.  `bidx` is the block number, or the
// entry of the segmented block table.
template <typename K, bool V, int LOGE, int LOGT, int VAR, bool MERGE>
__device__ __forceinline__ void tile_block(const PassParams& P, uint32_t bidx, K* sk, uint32_t* sv) {
  constexpr int E = 1 << LOGE;
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
  if (P.blocks != nullptr) {
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
  const uint32_t merge_p = P.rounds[0].p;

  K kr[E];
  uint32_t vr[E];
#pragma unroll
  for (int r = 0; r < E; ++r) vr[r] = 0;

  using SCHED = Schedule<LOGT, LOGE, MERGE>;
  constexpr int NR = SCHED::count;

  bool done = false;
  static_for<0, NR>([&](auto I) {
    constexpr SRound R = SCHED::value.r[decltype(I)::value];
    constexpr int A = R.a;
    if (done) return;
    const uint32_t rd = uint32_t(decltype(I)::value);
    const bool last = (rd + 1 == nrounds);
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
    if (slots != nullptr && (from_global || to_global)) {
      const SegSlot S = slots[g_full >> log2cap];
      bk = gk + S.base;
      if (V) bv = gv + S.base;
      seg_len = S.len;
      skip = (S.flags & kSlotEmpty) != 0;
      const uint32_t f = P.map_in | ((S.flags & kSlotDesc) ? kMapComplement : 0u);
      if (rd == 0 && from_global && fill) min_ = f;
      if (last && final_pass) mout = f;
      g_t = g_full & capmask;
    } else {
      if (rd == 0 && from_global) min_ = P.map_in;
      if (last) mout = P.map_out;
    }
    const uint32_t g_dir = (g_full | P.dir_base) & capmask;
    const bool do_store = !(to_global && skip);

    if constexpr (R.kind == RK_PHASE_A) {
      if (!skip) s_load<K, V, LOGE, 0, false, PADT>(kr, vr, true, bk, bv, g_t, sk, sv, s_base, min_, K(0));
      if (fill) {
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
        if (collide && !skip && P.status != nullptr)
          atomicOr(P.status, int(kStatusSentinelCollision));
      }
      phase_a_small<K, V, LOGE>(kr, vr, log2cap);
      if (uint32_t(LOGE) <= log2cap) {
        const bool asc = ((g_dir & uint32_t(E) & capmask) == 0u);
        if (VAR == kDivergent || !R.lanediv) {
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
      if (do_store)
        s_store<K, V, LOGE, 0, false, false, PADT>(kr, vr, to_global, bk, bv, g_t, sk, sv, s_base, mout, K(0));
    } else {
      const uint32_t p = MERGE ? merge_p : uint32_t(R.p);
      const bool asc = ((g_dir & (1u << p) & capmask) == 0u);
      if (VAR == kDivergent || !R.lanediv) {
        // Fig. 1: one full copy of the body per direction
        if (asc) {
          s_load<K, V, LOGE, A, false, PADT>(kr, vr, from_global, bk, bv, g_t, sk, sv, s_base, min_, K(0));
          window_side<K, V, LOGE, true>(kr, vr, R.cnt);
          if (do_store)
            s_store<K, V, LOGE, A, false, false, PADT>(kr, vr, to_global, bk, bv, g_t, sk, sv, s_base, mout, K(0));
        } else {
          s_load<K, V, LOGE, A, true, PADT>(kr, vr, from_global, bk, bv, g_t, sk, sv, s_base, min_, K(0));
          window_side<K, V, LOGE, false>(kr, vr, R.cnt);
          if (do_store)
            s_store<K, V, LOGE, A, true, false, PADT>(kr, vr, to_global, bk, bv, g_t, sk, sv, s_base, mout, K(0));
        }
      } else {
        // melded: one copy; the descending side's keys enter complemented
        const K m = asc ? K(0) : ~K(0);
        s_load<K, V, LOGE, A, false, PADT>(kr, vr, from_global, bk, bv, g_t, sk, sv, s_base, min_, m);
        window_side<K, V, LOGE, true>(kr, vr, R.cnt);
        if (do_store)
          s_store<K, V, LOGE, A, false, false, PADT>(kr, vr, to_global, bk, bv, g_t, sk, sv, s_base, mout, m);
      }
    }
    if (to_global) {
      done = true;
    } else {
      __syncthreads();
    }
  });
}

// Resident CTAs asked of the compiler for a tile kernel of MAXT threads: 64
// registers per thread, so that 2048 threads share an SM.  (Allowing a
// 256-thread tile 80 registers removed most of its spills but left three
// CTAs per SM, and batched segmented sorts ran 9 % slower.)
constexpr int tile_min_blocks(int maxt) {
  return maxt >= 1024 ? 1 : (maxt >= 512 ? 2 : (maxt >= 256 ? 4 : 8));
}

template <typename K, bool V, int LOGE, int LOGT, int VAR, bool MERGE, int MAXT>
__global__ void __launch_bounds__(MAXT, tile_min_blocks(MAXT)) darm_tile_kernel(const __grid_constant__ PassParams P) {
  constexpr uint32_t SW = smem_words(1u << LOGT);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* sk = reinterpret_cast<K*>(smem_raw);
  uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + sizeof(K) * SW);
  if (P.work_counter == nullptr) {
    tile_block<K, V, LOGE, LOGT, VAR, MERGE>(P, blockIdx.x, sk, sv);
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
    tile_block<K, V, LOGE, LOGT, VAR, MERGE>(P, b, sk, sv);
  }
}

}  // namespace darm
