// pass_kernel.cuh - the one CUDA kernel every stage of the bitonic network
// runs in, in its divergent and melded forms.
//
// Network (DARM paper, Fig. 1 / Section III): for k = 2, 4, ..., cap and
// j = k/2, ..., 1, each index i whose partner l = i ^ j lies above it runs
// a compare-exchange on (key[i], key[l]); the block of size k that i belongs
// to is ascending when bit k of i is clear.  Ascending swaps when
// key[l] < key[i], descending when key[l] > key[i] (strict).
//
// A launch ("pass") owns blocks of 2^b elements.  A block's local index l
// maps to the index g within its array (or segment) by a bit map: the low c
// local bits are the low c bits of g, the next s local bits land at g-bits
// w0 .. w0+s-1, and the block number fills every other g-bit.  A pass is a
// list of rounds.  In a round every thread holds E = 2^LOGE elements in
// registers whose local indices differ exactly in the window bits
// a .. a+LOGE-1; the round loads them (from HBM or from the block's copy in
// shared memory), runs up to LOGE layers of one stage k in registers, and
// stores them back to the same place.  Because a thread writes back exactly
// what it read, one barrier per round separates rounds.
//
// Direction.  Descending sorts complement the keys on the first load and
// on the last store (a descending comparator on x is an ascending one on
// ~x), so the kernel only evaluates Fig. 1's ascending test
// ((g & k) == 0), masked by the segment capacity so that the final stage of
// a segment is ascending.  Within a window round the direction bit k lies
// above the window, so it is constant for a thread over the whole round:
//   - it varies between lanes of a warp exactly when bit k falls on a lane
//     bit (the small stages inside a tile, like Fig. 1's k < 32);
//   - DIVERGENT wraps the whole round body (loads, compares, swaps,
//     stores) in Fig. 1's if/else, one full copy per direction;
//   - MELDED is that region after DARM's region-region meld (Section IV-G):
//     the loads and stores of both sides are aligned into one copy, the two
//     compares (< and >) stay unaligned, and a select on the direction picks
//     the swap condition (Algorithm 2, SetOperands), so the warp reconverges
//     before the swap.
// Stages whose direction bit is inside the thread's registers (k < E) have
// a compile-time direction per register pair and no branch in either form.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace darm {

constexpr int kMaxRounds = 64;
constexpr int kDivergent = 0;
constexpr int kMelded = 1;

enum RoundKind : uint8_t {
  RK_PHASE_A = 0,  // register sort of E consecutive elements, stages k <= E
  RK_WINDOW = 1    // layers of one stage k on the window bits a..a+LOGE-1
};
enum Loc : uint8_t { LOC_GLOBAL = 0, LOC_SMEM = 1 };

struct Round {
  uint8_t kind;  // RoundKind
  uint8_t p;     // stage k = 2^p (window rounds)
  uint8_t a;     // lowest local bit of the register window
  uint8_t cnt;   // layers run: window bits a+LOGE-1 down to a+LOGE-cnt
  uint8_t src;   // Loc the round loads from
  uint8_t dst;   // Loc the round stores to
  uint8_t pad0, pad1;
};

// Key transforms applied on the first load / undone on the last store.
constexpr uint32_t kMapF32 = 1u;         // IEEE totalOrder bit map
constexpr uint32_t kMapComplement = 2u;  // descending: x -> ~x

// Segmented passes resolve each block through a table.  A segment of
// capacity cap = 2^log2cap starts at element `base` of the key/payload
// arrays and holds `len` real elements; the rest is sentinel padding.
struct SegSlot {
  uint64_t base;   // first element of the segment
  uint32_t len;    // real elements (positions >= len get the sentinel)
  uint32_t desc;   // 1: this segment sorts descending
};
// One entry per launched block.  A block either covers part of one segment
// (blk_in_seg numbers the blocks of that segment) or, when the segment is
// smaller than the block, 2^(b - log2cap) whole segments stored in
// consecutive slots.
struct SegBlock {
  uint32_t first_slot;
  uint32_t blk_in_seg;
  uint8_t log2cap;
  uint8_t nrounds;     // rounds this block runs (small segments stop early)
  uint8_t final_pass;  // this pass completes the segment: undo key maps
  uint8_t fill;        // first load writes sentinels beyond len
};

constexpr uint32_t kStatusSentinelCollision = 8u;  // == DARM_ERR_SENTINEL_COLLISION

struct PassParams {
  void* keys;          // device keys (uint32 or uint64)
  uint32_t* vals;      // device payload or nullptr
  uint32_t b;          // log2 elements per block
  uint32_t c, w0, s;   // block bit map (see header)
  uint32_t log2cap;    // single array: log2 of its length
  uint32_t map_in;     // kMap* flags applied when round 0 loads from HBM
  uint32_t map_out;    // kMap* flags undone when the last round stores to HBM
  uint32_t nrounds;
  const SegBlock* blocks;  // segmented passes: per-block table, else nullptr
  const SegSlot* slots;
  int* status;             // device status word (sentinel collisions)
  Round rounds[kMaxRounds];
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

// Shared-memory address swizzle: fold the higher index bits onto the five
// bank bits with XOR.  It is linear over GF(2), so
// swz(x | y) == swz(x) ^ swz(y) for disjoint x, y, and a bijection on any
// power-of-two range.
__device__ __forceinline__ uint32_t swz(uint32_t x) {
  return x ^ (((x >> 5) ^ (x >> 10) ^ (x >> 15)) & 31u);
}

template <typename K>
__device__ __forceinline__ K key_in(K x, uint32_t f);
template <typename K>
__device__ __forceinline__ K key_out(K x, uint32_t f);

template <>
__device__ __forceinline__ uint32_t key_in<uint32_t>(uint32_t x, uint32_t f) {
  if (f & kMapF32) x = (x & 0x80000000u) ? ~x : (x | 0x80000000u);
  if (f & kMapComplement) x = ~x;
  return x;
}
template <>
__device__ __forceinline__ uint32_t key_out<uint32_t>(uint32_t x, uint32_t f) {
  if (f & kMapComplement) x = ~x;
  if (f & kMapF32) x = (x & 0x80000000u) ? (x & 0x7FFFFFFFu) : ~x;
  return x;
}
template <>
__device__ __forceinline__ uint64_t key_in<uint64_t>(uint64_t x, uint32_t f) {
  return (f & kMapComplement) ? ~x : x;
}
template <>
__device__ __forceinline__ uint64_t key_out<uint64_t>(uint64_t x, uint32_t f) {
  return (f & kMapComplement) ? ~x : x;
}

// Conditional swap of two (key, payload) elements by selects.
template <typename K, bool V>
__device__ __forceinline__ void cswap(bool s, K& a, K& b, uint32_t& va, uint32_t& vb) {
  const K ta = s ? b : a;
  const K tb = s ? a : b;
  a = ta;
  b = tb;
  if (V) {
    const uint32_t ua = s ? vb : va;
    const uint32_t ub = s ? va : vb;
    va = ua;
    vb = ub;
  }
}

// The two sides of Fig. 1's direction branch.
template <typename K, bool V, bool ASC>
__device__ __forceinline__ void ce_side(K& a, K& b, uint32_t& va, uint32_t& vb) {
  cswap<K, V>(ASC ? (b < a) : (b > a), a, b, va, vb);
}

// The melded compare-exchange: both compares execute (the unaligned
// instructions of the two sides) and a select on the direction picks the
// swap condition.
template <typename K, bool V>
__device__ __forceinline__ void ce_melded(bool asc, K& a, K& b, uint32_t& va, uint32_t& vb) {
  const bool lt = b < a;
  const bool gt = b > a;
  cswap<K, V>(asc ? lt : gt, a, b, va, vb);
}

// ---------------------------------------------------------------------------
// per-round element access
// ---------------------------------------------------------------------------

struct RoundAddr {
  uint32_t g_t;  // index-in-array bits contributed by the thread and block
  uint32_t s_t;  // swizzled shared-memory index of the thread part
  uint32_t a;    // window position
  uint32_t c, w0;
};

__device__ __forceinline__ uint32_t gmap(uint32_t l, uint32_t c, uint32_t w0) {
  return (l & ((1u << c) - 1u)) | ((l >> c) << w0);
}

template <int LOGE>
__device__ __forceinline__ uint32_t reg_g(const RoundAddr& A, int r) {
  return gmap(uint32_t(r) << A.a, A.c, A.w0);
}
template <int LOGE>
__device__ __forceinline__ uint32_t reg_s(const RoundAddr& A, int r) {
  return swz(uint32_t(r) << A.a);
}

// Load the thread's E elements for a round.  REV loads in the opposite
// register order (used by the descending side of the divergent form so that
// the compiler cannot hoist the two sides' identical leading loads out of
// the branch, which would be a partial meld of exactly the code compared).
template <typename K, bool V, int LOGE, bool REV>
__device__ __forceinline__ void load_elems(K (&kr)[1 << LOGE], uint32_t (&vr)[1 << LOGE],
                                           uint8_t src, bool vec, const RoundAddr& A,
                                           const K* __restrict__ gk,
                                           const uint32_t* __restrict__ gv,
                                           const K* sk, const uint32_t* sv, uint32_t mapf) {
  constexpr int E = 1 << LOGE;
  if (src == LOC_GLOBAL) {
    if (vec) {
      // the window is the low LOGE bits of g: E consecutive elements
      constexpr int KPV = 16 / sizeof(K);  // keys per 16-byte vector
      if constexpr (E >= KPV) {
#pragma unroll
        for (int q0 = 0; q0 < E / KPV; ++q0) {
          const int q = REV ? (E / KPV - 1 - q0) : q0;
          const uint4 w = *reinterpret_cast<const uint4*>(gk + A.g_t + q * KPV);
          const K* wk = reinterpret_cast<const K*>(&w);
#pragma unroll
          for (int u = 0; u < KPV; ++u) kr[q * KPV + u] = key_in<K>(wk[u], mapf);
        }
      } else {
#pragma unroll
        for (int r0 = 0; r0 < E; ++r0) {
          const int r = REV ? (E - 1 - r0) : r0;
          kr[r] = key_in<K>(gk[A.g_t + r], mapf);
        }
      }
      if (V) {
        if constexpr (E >= 4) {
#pragma unroll
          for (int q0 = 0; q0 < E / 4; ++q0) {
            const int q = REV ? (E / 4 - 1 - q0) : q0;
            const uint4 w = *reinterpret_cast<const uint4*>(gv + A.g_t + q * 4);
            vr[q * 4 + 0] = w.x;
            vr[q * 4 + 1] = w.y;
            vr[q * 4 + 2] = w.z;
            vr[q * 4 + 3] = w.w;
          }
        } else {
#pragma unroll
          for (int r0 = 0; r0 < E; ++r0) {
            const int r = REV ? (E - 1 - r0) : r0;
            vr[r] = gv[A.g_t + r];
          }
        }
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint32_t g = A.g_t + reg_g<LOGE>(A, r);
        kr[r] = key_in<K>(gk[g], mapf);
        if (V) vr[r] = gv[g];
      }
    }
  } else {
#pragma unroll
    for (int r0 = 0; r0 < E; ++r0) {
      const int r = REV ? (E - 1 - r0) : r0;
      const uint32_t si = A.s_t ^ reg_s<LOGE>(A, r);
      kr[r] = sk[si];
      if (V) vr[r] = sv[si];
    }
  }
}

template <typename K, bool V, int LOGE, bool REV>
__device__ __forceinline__ void store_elems(const K (&kr)[1 << LOGE], const uint32_t (&vr)[1 << LOGE],
                                            uint8_t dst, bool vec, const RoundAddr& A,
                                            K* __restrict__ gk, uint32_t* __restrict__ gv,
                                            K* sk, uint32_t* sv, uint32_t mapf) {
  constexpr int E = 1 << LOGE;
  if (dst == LOC_GLOBAL) {
    if (vec) {
      constexpr int KPV = 16 / sizeof(K);
      if constexpr (E >= KPV) {
#pragma unroll
        for (int q0 = 0; q0 < E / KPV; ++q0) {
          const int q = REV ? (E / KPV - 1 - q0) : q0;
          uint4 w;
          K* wk = reinterpret_cast<K*>(&w);
#pragma unroll
          for (int u = 0; u < KPV; ++u) wk[u] = key_out<K>(kr[q * KPV + u], mapf);
          *reinterpret_cast<uint4*>(gk + A.g_t + q * KPV) = w;
        }
      } else {
#pragma unroll
        for (int r0 = 0; r0 < E; ++r0) {
          const int r = REV ? (E - 1 - r0) : r0;
          gk[A.g_t + r] = key_out<K>(kr[r], mapf);
        }
      }
      if (V) {
        if constexpr (E >= 4) {
#pragma unroll
          for (int q0 = 0; q0 < E / 4; ++q0) {
            const int q = REV ? (E / 4 - 1 - q0) : q0;
            uint4 w;
            w.x = vr[q * 4 + 0];
            w.y = vr[q * 4 + 1];
            w.z = vr[q * 4 + 2];
            w.w = vr[q * 4 + 3];
            *reinterpret_cast<uint4*>(gv + A.g_t + q * 4) = w;
          }
        } else {
#pragma unroll
          for (int r0 = 0; r0 < E; ++r0) {
            const int r = REV ? (E - 1 - r0) : r0;
            gv[A.g_t + r] = vr[r];
          }
        }
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint32_t g = A.g_t + reg_g<LOGE>(A, r);
        gk[g] = key_out<K>(kr[r], mapf);
        if (V) gv[g] = vr[r];
      }
    }
  } else {
#pragma unroll
    for (int r0 = 0; r0 < E; ++r0) {
      const int r = REV ? (E - 1 - r0) : r0;
      const uint32_t si = A.s_t ^ reg_s<LOGE>(A, r);
      sk[si] = kr[r];
      if (V) sv[si] = vr[r];
    }
  }
}

// ---------------------------------------------------------------------------
// register layers
// ---------------------------------------------------------------------------

// Layers of one stage on the window: register bit q pairs r with r | 2^q.
// Window bit LOGE-1 is the highest; `cnt` layers run from the top down.
template <typename K, bool V, int LOGE, bool ASC>
__device__ __forceinline__ void window_side(K (&kr)[1 << LOGE], uint32_t (&vr)[1 << LOGE], int cnt) {
  constexpr int E = 1 << LOGE;
#pragma unroll
  for (int i = 0; i < LOGE; ++i) {
    if (i < cnt) {
      const int q = LOGE - 1 - i;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        if ((r >> q) & 1) continue;
        ce_side<K, V, ASC>(kr[r], kr[r | (1 << q)], vr[r], vr[r | (1 << q)]);
      }
    }
  }
}

template <typename K, bool V, int LOGE>
__device__ __forceinline__ void window_melded(bool asc, K (&kr)[1 << LOGE], uint32_t (&vr)[1 << LOGE],
                                              int cnt) {
  constexpr int E = 1 << LOGE;
#pragma unroll
  for (int i = 0; i < LOGE; ++i) {
    if (i < cnt) {
      const int q = LOGE - 1 - i;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        if ((r >> q) & 1) continue;
        ce_melded<K, V>(asc, kr[r], kr[r | (1 << q)], vr[r], vr[r | (1 << q)]);
      }
    }
  }
}

// Stages k = 2 .. E/2 on E consecutive elements: the direction bit lies in
// the register index, so each pair's direction is a compile-time constant
// (stage k == cap, the final stage of a tiny segment, is ascending).
template <typename K, bool V, int LOGE>
__device__ __forceinline__ void phase_a_small(K (&kr)[1 << LOGE], uint32_t (&vr)[1 << LOGE],
                                              uint32_t log2cap) {
  constexpr int E = 1 << LOGE;
#pragma unroll
  for (int p = 1; p < LOGE; ++p) {
    if (uint32_t(p) <= log2cap) {
      const bool final_stage = (uint32_t(p) == log2cap);
#pragma unroll
      for (int q = p - 1; q >= 0; --q) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
          if ((r >> q) & 1) continue;
          const bool asc_pair = ((r >> p) & 1) == 0;
          if (asc_pair)
            ce_side<K, V, true>(kr[r], kr[r | (1 << q)], vr[r], vr[r | (1 << q)]);
          else if (final_stage)
            ce_side<K, V, true>(kr[r], kr[r | (1 << q)], vr[r], vr[r | (1 << q)]);
          else
            ce_side<K, V, false>(kr[r], kr[r | (1 << q)], vr[r], vr[r | (1 << q)]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

// Sentinel for padded positions, in the (possibly complemented) key space
// the network runs in: always the largest key.
template <typename K>
__device__ __forceinline__ K key_max() { return ~K(0); }

template <typename K, bool V, int LOGE, int VAR, int MAXT>
__global__ void __launch_bounds__(MAXT) darm_pass_kernel(const __grid_constant__ PassParams P) {
  constexpr int E = 1 << LOGE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* sk = reinterpret_cast<K*>(smem_raw);
  uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + (size_t(sizeof(K)) << P.b));

  K* __restrict__ gk = reinterpret_cast<K*>(P.keys);
  uint32_t* __restrict__ gv = P.vals;
  const uint32_t tid = threadIdx.x;

  uint32_t blk = blockIdx.x;
  uint32_t log2cap = P.log2cap;
  uint32_t nrounds = P.nrounds;
  bool final_pass = true;
  bool fill = false;
  const SegSlot* slots = nullptr;
  if (P.blocks != nullptr) {
    const SegBlock B = P.blocks[blockIdx.x];
    blk = B.blk_in_seg;
    log2cap = B.log2cap;
    nrounds = B.nrounds;
    final_pass = B.final_pass != 0;
    fill = B.fill != 0;
    slots = P.slots + B.first_slot;
  }

  const uint32_t nmid = P.w0 - P.c;
  const uint32_t gblk = ((blk & ((1u << nmid) - 1u)) << P.c) | ((blk >> nmid) << (P.w0 + P.s));
  const uint32_t capmask = (1u << log2cap) - 1u;

  K kr[E];
  uint32_t vr[E];
#pragma unroll
  for (int r = 0; r < E; ++r) vr[r] = 0;

  for (uint32_t rd = 0; rd < nrounds; ++rd) {
    const Round R = P.rounds[rd];
    const bool last = (rd + 1 == nrounds);
    const uint8_t src = R.src;
    const uint8_t dst = last ? uint8_t(LOC_GLOBAL) : R.dst;
    RoundAddr A;
    A.a = R.a;
    A.c = P.c;
    A.w0 = P.w0;
    const uint32_t tl = (tid & ((1u << R.a) - 1u)) | ((tid >> R.a) << (R.a + LOGE));
    const uint32_t g_full = gmap(tl, P.c, P.w0) | gblk;  // index within the segment(s)
    A.s_t = swz(tl);
    const bool vec = (R.a == 0) && (P.c >= uint32_t(LOGE));
    uint32_t min_ = 0, mout = 0;
    K* bk = gk;
    uint32_t* bv = gv;
    uint32_t seg_len = 0xFFFFFFFFu;
    if (slots != nullptr && (src == LOC_GLOBAL || dst == LOC_GLOBAL)) {
      // all E elements of this thread lie in one segment (E <= cap)
      const SegSlot S = slots[g_full >> log2cap];
      bk = gk + S.base;
      if (V) bv = gv + S.base;
      seg_len = S.len;
      const uint32_t f = P.map_in | (S.desc ? kMapComplement : 0u);
      if (rd == 0 && src == LOC_GLOBAL) min_ = f;
      if (last && final_pass) mout = f;
      A.g_t = g_full & capmask;
    } else {
      A.g_t = g_full;
      if (rd == 0 && src == LOC_GLOBAL) min_ = P.map_in;
      if (last) mout = P.map_out;
    }
    // direction bits are read from the index within the segment
    const uint32_t g_dir = g_full & capmask;

    if (R.kind == RK_PHASE_A) {
      load_elems<K, V, LOGE, false>(kr, vr, src, vec, A, bk, bv, sk, sv, min_);
      if (fill) {
        // segment padding: positions at or beyond the real length take the
        // largest key; a real key equal to it is a collision when a payload
        // rides along (its place among the padding is then ambiguous)
        bool collide = false;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const uint32_t pos = A.g_t + uint32_t(r);
          if (pos >= seg_len) {
            kr[r] = key_max<K>();
            if (V) vr[r] = 0xFFFFFFFFu;
          } else if (V && kr[r] == key_max<K>()) {
            collide = true;
          }
        }
        if (collide && P.status != nullptr) atomicOr(P.status, int(kStatusSentinelCollision));
      }
      phase_a_small<K, V, LOGE>(kr, vr, log2cap);
      if (uint32_t(LOGE) <= log2cap) {
        // stage k = E: the direction bit is the lowest thread bit
        const bool asc = ((g_dir & uint32_t(E) & capmask) == 0u);
        if (VAR == kDivergent) {
          if (asc)
            window_side<K, V, LOGE, true>(kr, vr, LOGE);
          else
            window_side<K, V, LOGE, false>(kr, vr, LOGE);
        } else {
          window_melded<K, V, LOGE>(asc, kr, vr, LOGE);
        }
      }
      store_elems<K, V, LOGE, false>(kr, vr, dst, vec, A, bk, bv, sk, sv, mout);
    } else {
      const bool asc = ((g_dir & (1u << R.p) & capmask) == 0u);
      const int cnt = R.cnt;
      if (VAR == kDivergent) {
        if (asc) {
          load_elems<K, V, LOGE, false>(kr, vr, src, vec, A, bk, bv, sk, sv, min_);
          window_side<K, V, LOGE, true>(kr, vr, cnt);
          store_elems<K, V, LOGE, false>(kr, vr, dst, vec, A, bk, bv, sk, sv, mout);
        } else {
          load_elems<K, V, LOGE, true>(kr, vr, src, vec, A, bk, bv, sk, sv, min_);
          window_side<K, V, LOGE, false>(kr, vr, cnt);
          store_elems<K, V, LOGE, true>(kr, vr, dst, vec, A, bk, bv, sk, sv, mout);
        }
      } else {
        load_elems<K, V, LOGE, false>(kr, vr, src, vec, A, bk, bv, sk, sv, min_);
        window_melded<K, V, LOGE>(asc, kr, vr, cnt);
        store_elems<K, V, LOGE, false>(kr, vr, dst, vec, A, bk, bv, sk, sv, mout);
      }
    }
    if (dst == LOC_SMEM) __syncthreads();
  }
}

// Largest block size a (K, V, E) instantiation is compiled for.
template <typename K, bool V, int LOGE>
constexpr int max_threads_for() {
  return ((1 << LOGE) * (int(sizeof(K) / 4) + (V ? 1 : 0)) <= 16) ? 1024 : 512;
}

}  // namespace darm
