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
//   - MELDED is that region after DARM's region-region meld (Section IV-D,
//     IV-G): the loads and stores of both sides are aligned into one copy;
//     the two compares (key[l] < key[i] on one side, key[l] > key[i] on the
//     other) are aligned as one compare whose differing operands are chosen
//     by the direction (Algorithm 2, SetOperands) - the descending side's
//     keys enter complemented, x -> ~x, which reverses unsigned order - so
//     the warp reconverges before the swap.
//   The planner marks the rounds in which bit k can differ between lanes of
//   a warp; elsewhere the branch is warp-uniform, i.e. not a divergent
//   region (Definition 5), and both forms keep the plain branch.
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
enum Loc : uint8_t { LOC_GLOBAL = 0, LOC_SMEM = 1, LOC_NONE = 2 /* unused slot: no access */ };

struct Round {
  uint8_t kind;  // RoundKind
  uint8_t p;     // stage k = 2^p (window rounds)
  uint8_t a;     // lowest local bit of the register window
  uint8_t cnt;   // layers run: window bits a+LOGE-1 down to a+LOGE-cnt
  uint8_t src;   // Loc the round loads from
  uint8_t dst;   // Loc the round stores to
  uint8_t lanediv;  // 1: the direction can differ between lanes of a warp
  uint8_t pad;
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
  uint32_t flags;  // kSlotDesc | kSlotEmpty
};
constexpr uint32_t kSlotDesc = 1u;   // this segment sorts descending
constexpr uint32_t kSlotEmpty = 2u;  // unused slot of a packed block: no memory access
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
  uint8_t fill;        // first pass: apply the segment's key map and write
                       // sentinels beyond len
};

// The table sizes the C ABI documents for the no-allocation segmented sort.
static_assert(sizeof(SegSlot) == 16, "SegSlot is 16 bytes");
static_assert(sizeof(SegBlock) == 12, "SegBlock is 12 bytes");

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
  unsigned int* work_counter;  // persistent launches: next block to take
  uint32_t nblocks;            // persistent launches: blocks in the table
  uint32_t dir_base;           // single arrays: index of element 0 in the array
                               // whose network sets the directions (a chunk
                               // sorted on its own through its first stages:
                               // its offset); 0 otherwise
  Round rounds[kMaxRounds];
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

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

__device__ __forceinline__ uint32_t kmin(uint32_t a, uint32_t b) { return umin(a, b); }
__device__ __forceinline__ uint32_t kmax(uint32_t a, uint32_t b) { return umax(a, b); }
__device__ __forceinline__ uint64_t kmin(uint64_t a, uint64_t b) { return ullmin(a, b); }
__device__ __forceinline__ uint64_t kmax(uint64_t a, uint64_t b) { return ullmax(a, b); }

// 1 and 2^32 - 1 in constant memory: multiplied in, they keep an addition on
// the FMA pipe (an integer multiply-add) where the compiler would otherwise
// issue an add on the ALU pipe, which the min/max compare-exchanges keep busy.
// (static: every translation unit that includes this header keeps its own.)
static __constant__ uint32_t kFmaOne = 1u;
static __constant__ uint32_t kFmaMinusOne = 0xFFFFFFFFu;

// max(a, b) given lo = min(a, b): a + b - lo (mod 2^32), as two multiply-adds.
__device__ __forceinline__ uint32_t max_by_fma(uint32_t a, uint32_t b, uint32_t lo) {
  uint32_t t, hi;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(t) : "r"(a), "r"(kFmaOne), "r"(b));
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(hi) : "r"(lo), "r"(kFmaMinusOne), "r"(t));
  return hi;
}

// Keys-only compare-exchanges may alternate between two instruction mixes
// so that the ALU and FMA pipes share the work (MIX): one in three pairs
// computes (min, max) with two ALU operations, two in three compute the max
// on the FMA pipe (one ALU and two FMA operations).  `sel` is a compile-time
// pair index after unrolling.  Measured on 2^26 float keys: the merge pass
// 122.4 -> 117.5 us with the mix, but the tile pass 0.640 -> 0.684 ms (its
// longer dependency chains), so only the merge pass mixes.
__host__ __device__ constexpr bool fma_pair(int sel) { return (sel % 3) != 0; }

// The two sides of Fig. 1's direction branch.  Without a payload the strict
// swap leaves (min, max) ascending and (max, min) descending - equal keys
// are indistinguishable - so the side is one unsigned min and one max (or
// the max as a + b - min).  With a payload the swap predicate
// key[l] < key[i] (or >) moves the payload with its key.
template <typename K, bool V, bool ASC, bool MIX = false>
__device__ __forceinline__ void ce_side(K& a, K& b, uint32_t& va, uint32_t& vb, int sel = 0) {
  if constexpr (!V) {
    const K lo = kmin(a, b);
    K hi;
    if constexpr (MIX && sizeof(K) == 4) {
      hi = fma_pair(sel) ? K(max_by_fma(a, b, lo)) : kmax(a, b);
    } else {
      hi = kmax(a, b);
    }
    a = ASC ? lo : hi;
    b = ASC ? hi : lo;
  } else {
    cswap<K, V>(ASC ? (b < a) : (b > a), a, b, va, vb);
  }
}

// ---------------------------------------------------------------------------
// shared-memory layout
// ---------------------------------------------------------------------------

// Element l of a block lives at word phys(l) = l + 4 * (l / 32): four pad
// words after every 32 elements.  With this layout
//   - a warp whose lanes take 32 consecutive elements (window above bit 4)
//     hits 32 different banks;
//   - a warp whose lanes each take E consecutive elements (the bottom
//     window) reads them as 16-byte vectors without bank conflicts;
//   - the offset of register r in a window at bit a >= 5 is r * (2^a +
//     2^(a-3)), a multiply-add instead of bit twiddling.
__device__ __forceinline__ uint32_t phys(uint32_t l) { return l + ((l >> 5) << 2); }

// Key-value passes with 32-bit keys keep (key, payload) pairs together in
// 8-byte slots: pair l at slot phys8(l) = l + 2 * (l / 16).  The slot count
// of a tile equals the word count of phys(), so both layouts share
// smem_words().
__device__ __forceinline__ uint32_t phys8(uint32_t l) { return l + ((l >> 4) << 1); }

__host__ __device__ constexpr uint32_t smem_words(uint32_t elems) {
  return elems + ((elems >> 5) << 2) + 4;
}

// ---------------------------------------------------------------------------
// per-round element access
// ---------------------------------------------------------------------------

struct RoundAddr {
  uint32_t g_t;     // index within the segment of the thread's register 0
  uint32_t gsh;     // register r sits at g_t + (r << gsh) (non-vector rounds)
  uint32_t s_base;  // phys() of the thread's register 0
  uint32_t a;       // window position (local bit)
  uint32_t stride;  // phys offset per register when a >= 5
};

__device__ __forceinline__ uint32_t gmap(uint32_t l, uint32_t c, uint32_t w0) {
  return (l & ((1u << c) - 1u)) | ((l >> c) << w0);
}

// XOR of a key with the direction mask (melded rounds) after the key map.
template <typename K>
__device__ __forceinline__ K kx(K x, K m) { return x ^ m; }

// Load the thread's E elements of a round.  `m` is XORed into every key
// (all-ones turns a descending compare-exchange into an ascending one).  REV
// loads in the opposite register order: the descending side of the
// divergent form uses it so that the compiler cannot hoist the two sides'
// identical leading loads out of the branch (that would be a partial meld of
// exactly the code being compared).
template <typename K, bool V, int LOGE, bool REV>
__device__ __forceinline__ void load_elems(K (&kr)[1 << LOGE], uint32_t (&vr)[1 << LOGE],
                                           uint8_t src, bool vec, const RoundAddr& A,
                                           const K* __restrict__ gk,
                                           const uint32_t* __restrict__ gv,
                                           const K* sk, const uint32_t* sv, uint32_t mapf, K m) {
  constexpr int E = 1 << LOGE;
  constexpr int KPV = 16 / sizeof(K);  // keys per 16-byte vector
  if (src == LOC_NONE) {
#pragma unroll
    for (int r = 0; r < E; ++r) {
      kr[r] = K(0);
      vr[r] = 0u;
    }
    return;
  }
  if (src == LOC_GLOBAL) {
    if (vec && E >= KPV) {
#pragma unroll
      for (int q0 = 0; q0 < E / KPV; ++q0) {
        const int q = REV ? (E / KPV - 1 - q0) : q0;
        const uint4 w = *reinterpret_cast<const uint4*>(gk + A.g_t + q * KPV);
        const K* wk = reinterpret_cast<const K*>(&w);
#pragma unroll
        for (int u = 0; u < KPV; ++u) kr[q * KPV + u] = kx(key_in<K>(wk[u], mapf), m);
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        kr[r] = kx(key_in<K>(gk[A.g_t + (uint32_t(r) << A.gsh)], mapf), m);
      }
    }
    if (V) {
      if (vec && E >= 4) {
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
          vr[r] = gv[A.g_t + (uint32_t(r) << A.gsh)];
        }
      }
    }
  } else if (V && sizeof(K) == 4) {
    // interleaved (key, payload) slots
    const uint2* s2 = reinterpret_cast<const uint2*>(sk);
    if (A.a == 0 && E >= 2) {
#pragma unroll
      for (int q0 = 0; q0 < E / 2; ++q0) {
        const int q = REV ? (E / 2 - 1 - q0) : q0;
        const uint4 w = *reinterpret_cast<const uint4*>(s2 + A.s_base + phys8(uint32_t(2 * q)));
        kr[2 * q] = kx(K(w.x), m);
        vr[2 * q] = w.y;
        kr[2 * q + 1] = kx(K(w.z), m);
        vr[2 * q + 1] = w.w;
      }
    } else if (A.a >= 5) {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint2 w = s2[A.s_base + uint32_t(r) * A.stride];
        kr[r] = kx(K(w.x), m);
        vr[r] = w.y;
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint2 w = s2[A.s_base + phys8(uint32_t(r) << A.a)];
        kr[r] = kx(K(w.x), m);
        vr[r] = w.y;
      }
    }
  } else {
    if (A.a == 0 && E >= KPV) {
      // bottom window: the thread's E elements are consecutive in phys space
#pragma unroll
      for (int q0 = 0; q0 < E / KPV; ++q0) {
        const int q = REV ? (E / KPV - 1 - q0) : q0;
        const uint4 w = *reinterpret_cast<const uint4*>(sk + A.s_base + q * KPV);
        const K* wk = reinterpret_cast<const K*>(&w);
#pragma unroll
        for (int u = 0; u < KPV; ++u) kr[q * KPV + u] = kx(wk[u], m);
      }
      if (V) {
        if constexpr (E >= 4) {
#pragma unroll
          for (int q0 = 0; q0 < E / 4; ++q0) {
            const int q = REV ? (E / 4 - 1 - q0) : q0;
            const uint4 w = *reinterpret_cast<const uint4*>(sv + A.s_base + q * 4);
            vr[q * 4 + 0] = w.x;
            vr[q * 4 + 1] = w.y;
            vr[q * 4 + 2] = w.z;
            vr[q * 4 + 3] = w.w;
          }
        } else {
#pragma unroll
          for (int r0 = 0; r0 < E; ++r0) {
            const int r = REV ? (E - 1 - r0) : r0;
            vr[r] = sv[A.s_base + uint32_t(r)];
          }
        }
      }
    } else if (A.a >= 5) {
      // lanes take consecutive elements; register r is r * stride words away
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint32_t si = A.s_base + uint32_t(r) * A.stride;
        kr[r] = kx(sk[si], m);
        if (V) vr[r] = sv[si];
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint32_t si = A.s_base + phys(uint32_t(r) << A.a);
        kr[r] = kx(sk[si], m);
        if (V) vr[r] = sv[si];
      }
    }
  }
}

template <typename K, bool V, int LOGE, bool REV>
__device__ __forceinline__ void store_elems(const K (&kr)[1 << LOGE], const uint32_t (&vr)[1 << LOGE],
                                            uint8_t dst, bool vec, const RoundAddr& A,
                                            K* __restrict__ gk, uint32_t* __restrict__ gv,
                                            K* sk, uint32_t* sv, uint32_t mapf, K m) {
  constexpr int E = 1 << LOGE;
  constexpr int KPV = 16 / sizeof(K);
  if (dst == LOC_NONE) return;
  if (dst == LOC_GLOBAL) {
    if (vec && E >= KPV) {
#pragma unroll
      for (int q0 = 0; q0 < E / KPV; ++q0) {
        const int q = REV ? (E / KPV - 1 - q0) : q0;
        uint4 w;
        K* wk = reinterpret_cast<K*>(&w);
#pragma unroll
        for (int u = 0; u < KPV; ++u) wk[u] = key_out<K>(kx(kr[q * KPV + u], m), mapf);
        *reinterpret_cast<uint4*>(gk + A.g_t + q * KPV) = w;
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        gk[A.g_t + (uint32_t(r) << A.gsh)] = key_out<K>(kx(kr[r], m), mapf);
      }
    }
    if (V) {
      if (vec && E >= 4) {
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
          gv[A.g_t + (uint32_t(r) << A.gsh)] = vr[r];
        }
      }
    }
  } else if (V && sizeof(K) == 4) {
    uint2* s2 = reinterpret_cast<uint2*>(sk);
    if (A.a == 0 && E >= 2) {
#pragma unroll
      for (int q0 = 0; q0 < E / 2; ++q0) {
        const int q = REV ? (E / 2 - 1 - q0) : q0;
        uint4 w;
        w.x = uint32_t(kx(kr[2 * q], m));
        w.y = vr[2 * q];
        w.z = uint32_t(kx(kr[2 * q + 1], m));
        w.w = vr[2 * q + 1];
        *reinterpret_cast<uint4*>(s2 + A.s_base + phys8(uint32_t(2 * q))) = w;
      }
    } else if (A.a >= 5) {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        s2[A.s_base + uint32_t(r) * A.stride] = make_uint2(uint32_t(kx(kr[r], m)), vr[r]);
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        s2[A.s_base + phys8(uint32_t(r) << A.a)] = make_uint2(uint32_t(kx(kr[r], m)), vr[r]);
      }
    }
  } else {
    if (A.a == 0 && E >= KPV) {
#pragma unroll
      for (int q0 = 0; q0 < E / KPV; ++q0) {
        const int q = REV ? (E / KPV - 1 - q0) : q0;
        uint4 w;
        K* wk = reinterpret_cast<K*>(&w);
#pragma unroll
        for (int u = 0; u < KPV; ++u) wk[u] = kx(kr[q * KPV + u], m);
        *reinterpret_cast<uint4*>(sk + A.s_base + q * KPV) = w;
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
            *reinterpret_cast<uint4*>(sv + A.s_base + q * 4) = w;
          }
        } else {
#pragma unroll
          for (int r0 = 0; r0 < E; ++r0) {
            const int r = REV ? (E - 1 - r0) : r0;
            sv[A.s_base + uint32_t(r)] = vr[r];
          }
        }
      }
    } else if (A.a >= 5) {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint32_t si = A.s_base + uint32_t(r) * A.stride;
        sk[si] = kx(kr[r], m);
        if (V) sv[si] = vr[r];
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < E; ++r0) {
        const int r = REV ? (E - 1 - r0) : r0;
        const uint32_t si = A.s_base + phys(uint32_t(r) << A.a);
        sk[si] = kx(kr[r], m);
        if (V) sv[si] = vr[r];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// register layers
// ---------------------------------------------------------------------------

// Layers of one stage on the window: register bit q pairs r with r | 2^q.
// Window bit LOGE-1 is the highest; `cnt` layers run from the top down.
template <typename K, bool V, int LOGE, bool ASC, bool MIX = false>
__device__ __forceinline__ void window_side(K (&kr)[1 << LOGE], uint32_t (&vr)[1 << LOGE], int cnt) {
  constexpr int E = 1 << LOGE;
#pragma unroll
  for (int i = 0; i < LOGE; ++i) {
    if (i < cnt) {
      const int q = LOGE - 1 - i;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        if ((r >> q) & 1) continue;
        ce_side<K, V, ASC, MIX>(kr[r], kr[r | (1 << q)], vr[r], vr[r | (1 << q)], r);
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
          if (((r >> p) & 1) == 0 || final_stage)
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
__global__ void __launch_bounds__(MAXT, 1) darm_pass_kernel(const __grid_constant__ PassParams P) {
  constexpr int E = 1 << LOGE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  K* sk = reinterpret_cast<K*>(smem_raw);
  uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + size_t(sizeof(K)) * smem_words(1u << P.b));

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
    const uint32_t a = R.a;
    const uint32_t tl = (tid & ((1u << a) - 1u)) | ((tid >> a) << (a + LOGE));
    const uint32_t g_full = gmap(tl, P.c, P.w0) | gblk;  // index within the segment(s)
    RoundAddr A;
    A.a = a;
    A.gsh = (a >= P.c) ? (a - P.c + P.w0) : a;
    A.s_base = (V && sizeof(K) == 4) ? phys8(tl) : phys(tl);
    A.stride = (a >= 5) ? ((1u << a) + (1u << (a - 3))) : 0u;
    const bool vec = (a == 0) && (P.c >= uint32_t(LOGE));
    uint32_t min_ = 0, mout = 0;
    K* bk = gk;
    uint32_t* bv = gv;
    uint32_t seg_len = 0xFFFFFFFFu;
    bool skip_mem = false;
    if (slots != nullptr && (src == LOC_GLOBAL || dst == LOC_GLOBAL)) {
      // all E elements of this thread lie in one segment (E <= cap)
      const SegSlot S = slots[g_full >> log2cap];
      bk = gk + S.base;
      if (V) bv = gv + S.base;
      seg_len = S.len;
      skip_mem = (S.flags & kSlotEmpty) != 0;
      const uint32_t f = P.map_in | ((S.flags & kSlotDesc) ? kMapComplement : 0u);
      if (rd == 0 && src == LOC_GLOBAL && fill) min_ = f;
      if (last && final_pass) mout = f;
      A.g_t = g_full & capmask;
    } else {
      A.g_t = g_full;
      if (rd == 0 && src == LOC_GLOBAL) min_ = P.map_in;
      if (last) mout = P.map_out;
    }
    const uint8_t src_e = (skip_mem && src == LOC_GLOBAL) ? uint8_t(LOC_NONE) : src;
    const uint8_t dst_e = (skip_mem && dst == LOC_GLOBAL) ? uint8_t(LOC_NONE) : dst;
    // direction bits are read from the index within the segment (or, for a
    // chunk of a larger array, within that array)
    const uint32_t g_dir = (g_full | P.dir_base) & capmask;
    // the planner marks rounds whose direction can differ between the
    // lanes of a warp; only those are melded
    const bool lane_divergent = R.lanediv != 0;

    if (R.kind == RK_PHASE_A) {
      load_elems<K, V, LOGE, false>(kr, vr, src_e, vec, A, bk, bv, sk, sv, min_, K(0));
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
        if (VAR == kDivergent || !lane_divergent) {
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
      store_elems<K, V, LOGE, false>(kr, vr, dst_e, vec, A, bk, bv, sk, sv, mout, K(0));
    } else {
      const bool asc = ((g_dir & (1u << R.p) & capmask) == 0u);
      const int cnt = R.cnt;
      if (VAR == kDivergent || !lane_divergent) {
        // Fig. 1: one full copy of the body per direction
        if (asc) {
          load_elems<K, V, LOGE, false>(kr, vr, src_e, vec, A, bk, bv, sk, sv, min_, K(0));
          window_side<K, V, LOGE, true>(kr, vr, cnt);
          store_elems<K, V, LOGE, false>(kr, vr, dst_e, vec, A, bk, bv, sk, sv, mout, K(0));
        } else {
          load_elems<K, V, LOGE, true>(kr, vr, src_e, vec, A, bk, bv, sk, sv, min_, K(0));
          window_side<K, V, LOGE, false>(kr, vr, cnt);
          store_elems<K, V, LOGE, true>(kr, vr, dst_e, vec, A, bk, bv, sk, sv, mout, K(0));
        }
      } else {
        // melded: one copy of the loads, compares and stores.  The two sides'
        // compares (key[l] < key[i] and key[l] > key[i]) are aligned by
        // selecting their operands: the descending side's keys enter
        // complemented (x -> ~x reverses unsigned order), so both sides run
        // the same ascending compare-exchange, and the stores undo it.
        const K m = asc ? K(0) : ~K(0);
        load_elems<K, V, LOGE, false>(kr, vr, src_e, vec, A, bk, bv, sk, sv, min_, m);
        window_side<K, V, LOGE, true>(kr, vr, cnt);
        store_elems<K, V, LOGE, false>(kr, vr, dst_e, vec, A, bk, bv, sk, sv, mout, m);
      }
    }
    if (dst == LOC_SMEM) __syncthreads();
  }
}

// Largest block size a (K, V, E) instantiation is compiled for: 1024
// threads (64 registers each) while a thread's elements fit in 32 words,
// else 512 threads with up to 128 registers.
template <typename K, bool V, int LOGE>
constexpr int max_threads_for() {
  return ((1 << LOGE) * (int(sizeof(K) / 4) + (V ? 1 : 0)) <= 32) ? 1024 : 512;
}

}  // namespace darm
