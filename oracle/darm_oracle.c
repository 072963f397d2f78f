/*
 * CPU oracle for the bitonic compare-exchange network of DARM's running
 * example (Saumya, Sundararajah, Kulkarni, "DARM: Control-Flow Melding for
 * SIMT Thread Divergence Reduction", Fig. 1 and Section III).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or helper with the CUDA
 * library; the two are written independently so that one can check the other.
 *
 * Everything here is deliberately plain, single-threaded and slow:
 *
 *   - oracle_bitonic_{u32,u64}: the iterative network of Fig. 1, written
 *     with the same loop nest (k doubles from 2 to n, j halves from k/2 to 1,
 *     partner l = i ^ j, the lower index of a pair decides), generalised
 *     from "one element per thread" to a sequential loop over i.
 *   - oracle_bitonic_rec_{u32,u64}: an independent recursive formulation of
 *     the same comparator network (Batcher's sort/merge recursion), used to
 *     pin payload order under duplicate keys.
 *   - oracle_bitonic_f32: float keys through the IEEE-754 totalOrder bit map
 *     (not in the paper, whose keys are int; documented reading).
 *   - oracle_segmented_{u32,u64}: independent segments of power-of-two
 *     capacity, padded beyond their real length with the direction's
 *     extreme key before the network runs.
 *   - oracle_oddeven_u32 / oracle_oddeven_rec_u32: Batcher's odd-even merge
 *     sort network (PCM's base, Section VI-A), iterative and recursive.
 *   - oracle_pcm_u32 / oracle_pcm_rec_u32: PCM (Section VI-A), Batcher's
 *     network over buckets of sorted keys with merge-split comparators,
 *     iterative and recursive.
 *   - oracle_sb: the synthetic divergent kernels SB1-SB4 and their -R
 *     variants.
 *
 * Readings of the paper taken here (the paper is silent on them):
 *   - descending order flips every comparator: the ascending test of Fig. 1
 *     becomes ((i & k) == 0) XOR desc;
 *   - a swap happens only on strict inequality (Fig. 1 compares with < on the
 *     ascending side and > on the descending side), so equal keys never move
 *     relative to each other inside one comparator;
 *   - a payload travels with its key; only keys are compared.
 *
 * Status codes: 0 ok, 1 out of host memory (PCM), 2 length not a power of
 * two.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_NOT_POW2 2

static int is_pow2_u64(uint64_t n) { return n != 0 && (n & (n - 1)) == 0; }

#ifndef DARM_ORACLE_MUTANT
#define DARM_ORACLE_MUTANT 0
#endif

/*
 * Iterative network of Fig. 1.  For every stage k and every layer j, each
 * index i whose partner l = i ^ j lies above it compares (key[i], key[l]).
 * The block of size k that i belongs to runs ascending when bit k of i is
 * clear (Fig. 1's "(tid & k) == 0" test), flipped for a descending sort.
 * Ascending side: swap when key[l] < key[i]; descending side: swap when
 * key[l] > key[i].  `val` may be NULL (keys only).
 *
 * DARM_ORACLE_MUTANT (0 in every real build) plants one plausible mistake at
 * compile time so that the tests can show that the pins catch it:
 *   1 direction taken from bit j instead of bit k
 *   2 non-strict comparison (<= / >=)
 *   3 payload not swapped with its key
 *   4 descending flag ignored
 *   5 layer loop stops one layer early (j > 1)
 */
#define DEFINE_ITERATIVE(NAME, KT)                                             \
  int NAME(KT* key, uint32_t* val, uint64_t n, int desc) {                     \
    if (n <= 1) return ORACLE_OK;                                              \
    if (!is_pow2_u64(n)) return ORACLE_ERR_NOT_POW2;                           \
    for (uint64_t k = 2; k <= n; k <<= 1) {                                    \
      for (uint64_t j = k >> 1; j > (DARM_ORACLE_MUTANT == 5 ? 1u : 0u);       \
           j >>= 1) {                                                          \
        for (uint64_t i = 0; i < n; ++i) {                                     \
          uint64_t l = i ^ j;                                                  \
          if (l <= i) continue;                                                \
          uint64_t dirbit = (DARM_ORACLE_MUTANT == 1) ? (i & j) : (i & k);     \
          int up = (dirbit == 0);                                              \
          if (DARM_ORACLE_MUTANT != 4 && desc) up = !up;                       \
          int do_swap;                                                         \
          if (DARM_ORACLE_MUTANT == 2)                                         \
            do_swap = up ? (key[l] <= key[i]) : (key[l] >= key[i]);            \
          else                                                                 \
            do_swap = up ? (key[l] < key[i]) : (key[l] > key[i]);              \
          if (do_swap) {                                                       \
            KT tk = key[i];                                                    \
            key[i] = key[l];                                                   \
            key[l] = tk;                                                       \
            if (val && DARM_ORACLE_MUTANT != 3) {                              \
              uint32_t tv = val[i];                                            \
              val[i] = val[l];                                                 \
              val[l] = tv;                                                     \
            }                                                                  \
          }                                                                    \
        }                                                                      \
      }                                                                        \
    }                                                                          \
    return ORACLE_OK;                                                          \
  }

DEFINE_ITERATIVE(oracle_bitonic_u32, uint32_t)
DEFINE_ITERATIVE(oracle_bitonic_u64, uint64_t)

/*
 * Recursive formulation (Batcher's bitonic sorter) of the same network.
 * rec_sort(lo, n, up) sorts key[lo .. lo+n) in direction `up`: it sorts the
 * lower half ascending and the upper half descending (in Fig. 1 the halves
 * of a size-k block always take these two directions, whatever the block's
 * own direction), then merges.  rec_merge(lo, n, up) compares (i, i + n/2)
 * for every i in the lower half, then merges both halves in the same
 * direction.  A descending sort flips every direction.  Comparators of one
 * layer touch disjoint pairs, so the depth-first order gives the same result
 * as the layer-by-layer order of Fig. 1 whenever both describe the same
 * comparator set.
 */
#define DEFINE_RECURSIVE(NAME, KT)                                             \
  static void NAME##_merge(KT* key, uint32_t* val, uint64_t lo, uint64_t n,    \
                           int up) {                                           \
    if (n < 2) return;                                                         \
    uint64_t h = n / 2;                                                        \
    for (uint64_t i = lo; i < lo + h; ++i) {                                   \
      uint64_t l = i + h;                                                      \
      int do_swap = up ? (key[l] < key[i]) : (key[l] > key[i]);                \
      if (do_swap) {                                                           \
        KT tk = key[i];                                                        \
        key[i] = key[l];                                                       \
        key[l] = tk;                                                           \
        if (val) {                                                             \
          uint32_t tv = val[i];                                                \
          val[i] = val[l];                                                     \
          val[l] = tv;                                                         \
        }                                                                      \
      }                                                                        \
    }                                                                          \
    NAME##_merge(key, val, lo, h, up);                                         \
    NAME##_merge(key, val, lo + h, h, up);                                     \
  }                                                                            \
  static void NAME##_sort(KT* key, uint32_t* val, uint64_t lo, uint64_t n,     \
                          int up, int desc) {                                  \
    if (n < 2) return;                                                         \
    uint64_t h = n / 2;                                                        \
    NAME##_sort(key, val, lo, h, !desc, desc);                                 \
    NAME##_sort(key, val, lo + h, h, desc, desc);                              \
    NAME##_merge(key, val, lo, n, up);                                         \
  }                                                                            \
  int NAME(KT* key, uint32_t* val, uint64_t n, int desc) {                     \
    if (n <= 1) return ORACLE_OK;                                              \
    if (!is_pow2_u64(n)) return ORACLE_ERR_NOT_POW2;                           \
    NAME##_sort(key, val, 0, n, !desc, desc);                                  \
    return ORACLE_OK;                                                          \
  }

DEFINE_RECURSIVE(oracle_bitonic_rec_u32, uint32_t)
DEFINE_RECURSIVE(oracle_bitonic_rec_u64, uint64_t)

/*
 * Float keys.  The paper sorts int keys; float keys are ordered here by the
 * IEEE-754 totalOrder of their bit patterns (for non-NaN values): a
 * non-negative float gets its sign bit set, a negative float has every bit
 * inverted, so that unsigned order of the mapped word is numeric order with
 * -0.0 placed just below +0.0.  The mapped words go through the u32 network
 * and are mapped back.
 */
static uint32_t total_order_bits(uint32_t u) {
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
static uint32_t total_order_bits_inverse(uint32_t m) {
  return (m & 0x80000000u) ? (m & 0x7FFFFFFFu) : ~m;
}

int oracle_bitonic_f32(float* key, uint32_t* val, uint64_t n, int desc) {
  if (n <= 1) return ORACLE_OK;
  if (!is_pow2_u64(n)) return ORACLE_ERR_NOT_POW2;
  uint32_t* w = (uint32_t*)key; /* same storage, reinterpreted */
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t u;
    memcpy(&u, &key[i], sizeof u);
    u = total_order_bits(u);
    w[i] = u;
  }
  int rc = oracle_bitonic_u32(w, val, n, desc);
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t u = total_order_bits_inverse(w[i]);
    memcpy(&key[i], &u, sizeof u);
  }
  return rc;
}

/*
 * Segmented sort: segment s occupies [off[s], off[s+1]) of key/val; its
 * capacity off[s+1] - off[s] must be a power of two (paper: NUM is a power
 * of two).  Elements from len[s] up to the capacity are overwritten with the
 * sentinel (the largest key for ascending, 0 for descending; payload
 * 0xFFFFFFFF) and the whole capacity is sorted by the network of Fig. 1 with
 * indices local to the segment.  desc_per_seg may be NULL (all use `desc`).
 */
#define DEFINE_SEGMENTED(NAME, KT, NET, KMAX)                                  \
  int NAME(KT* key, uint32_t* val, const uint64_t* off, const uint32_t* len,   \
           uint64_t nseg, int desc, const uint8_t* desc_per_seg) {             \
    for (uint64_t s = 0; s < nseg; ++s) {                                      \
      uint64_t cap = off[s + 1] - off[s];                                      \
      if (cap == 0) continue;                                                  \
      if (!is_pow2_u64(cap)) return ORACLE_ERR_NOT_POW2;                       \
      int d = desc_per_seg ? (desc_per_seg[s] != 0) : (desc != 0);             \
      KT sentinel = d ? (KT)0 : (KT)KMAX;                                      \
      for (uint64_t i = len[s]; i < cap; ++i) {                                \
        key[off[s] + i] = sentinel;                                            \
        if (val) val[off[s] + i] = 0xFFFFFFFFu;                                \
      }                                                                        \
      int rc = NET(key + off[s], val ? val + off[s] : NULL, cap, d);           \
      if (rc) return rc;                                                       \
    }                                                                          \
    return ORACLE_OK;                                                          \
  }

DEFINE_SEGMENTED(oracle_segmented_u32, uint32_t, oracle_bitonic_u32, 0xFFFFFFFFu)
DEFINE_SEGMENTED(oracle_segmented_u64, uint64_t, oracle_bitonic_u64,
                 0xFFFFFFFFFFFFFFFFull)

/* Number of compare-exchange evaluations of the network for n = 2^m:
 * (n/2) * m(m+1)/2.  Used only to scale timing figures. */
uint64_t oracle_compare_exchanges(uint64_t n) {
  uint64_t m = 0;
  while ((1ull << m) < n) ++m;
  return (n / 2) * (m * (m + 1) / 2);
}

int oracle_mutant_id(void) { return DARM_ORACLE_MUTANT; }

/*
 * Batcher's odd-even merge sort network (the network PCM, Section VI-A, is
 * built on), ascending, strict swaps, payload travelling with its key.
 *
 * Iterative form: for every merge size p = 1, 2, 4, ... < n and every
 * distance k = p, p/2, ..., 1, x runs over [j, j + k) for
 * j = (k mod p), (k mod p) + 2k, ..., and (x, x + k) is compared when both
 * lie in the same block of 2p elements.  This is the textbook iterative
 * statement of the network (Knuth, TAOCP vol. 3, 5.3.4).
 * `ncmp` (nullable) receives the number of comparators evaluated.
 */
/* DARM_ORACLE_MUTANT 6 drops the same-block test of the iterative form,
 * 7 swaps equal keys too (non-strict compare); 0 in every real build. */
static void oe_cmpx(uint32_t* key, uint32_t* val, uint64_t a, uint64_t b) {
  if (DARM_ORACLE_MUTANT == 7 ? (key[b] <= key[a]) : (key[b] < key[a])) {
    uint32_t tk = key[a];
    key[a] = key[b];
    key[b] = tk;
    if (val) {
      uint32_t tv = val[a];
      val[a] = val[b];
      val[b] = tv;
    }
  }
}

int oracle_oddeven_u32(uint32_t* key, uint32_t* val, uint64_t n, uint64_t* ncmp) {
  uint64_t count = 0;
  if (n > 1 && !is_pow2_u64(n)) return ORACLE_ERR_NOT_POW2;
  for (uint64_t p = 1; p < n; p <<= 1) {
    for (uint64_t k = p; k >= 1; k >>= 1) {
      for (uint64_t j = k % p; j + k < n; j += 2 * k) {
        for (uint64_t i = 0; i < k && i + j + k < n; ++i) {
          const uint64_t x = i + j;
          if (DARM_ORACLE_MUTANT == 6 || x / (2 * p) == (x + k) / (2 * p)) {
            oe_cmpx(key, val, x, x + k);
            ++count;
          }
        }
      }
    }
  }
  if (ncmp) *ncmp = count;
  return ORACLE_OK;
}

/*
 * Recursive form of the same network: sort both halves, then merge them
 * with Batcher's odd-even merge, which merges the even- and the
 * odd-indexed subsequences (stride 2r) recursively and then compares the
 * neighbours (i, i + r) left out of place.  Each element meets its
 * comparators in the same order as in the iterative form, so the results
 * are identical, payload order under ties included.
 */
static void oe_merge(uint32_t* key, uint32_t* val, uint64_t lo, uint64_t n, uint64_t r) {
  const uint64_t step = 2 * r;
  if (step < n) {
    oe_merge(key, val, lo, n, step);
    oe_merge(key, val, lo + r, n, step);
    for (uint64_t i = lo + r; i + r < lo + n; i += step) oe_cmpx(key, val, i, i + r);
  } else {
    oe_cmpx(key, val, lo, lo + r);
  }
}

static void oe_sort(uint32_t* key, uint32_t* val, uint64_t lo, uint64_t n) {
  if (n < 2) return;
  const uint64_t h = n / 2;
  oe_sort(key, val, lo, h);
  oe_sort(key, val, lo + h, h);
  oe_merge(key, val, lo, n, 1);
}

int oracle_oddeven_rec_u32(uint32_t* key, uint32_t* val, uint64_t n) {
  if (n <= 1) return ORACLE_OK;
  if (!is_pow2_u64(n)) return ORACLE_ERR_NOT_POW2;
  oe_sort(key, val, 0, n);
  return ORACLE_OK;
}

/*
 * PCM, Partition and Concurrent Merge (Section VI-A): a parallel sort built on
 * Batcher's odd-even merge sort that odd-even merges buckets of sorted
 * elements.  Reading taken here: the n = B * S keys form B buckets of S
 * consecutive keys (B and S powers of two); every bucket is sorted by the
 * odd-even merge sort network above; then the same network runs over the B
 * buckets, each comparator (bucket x, bucket y), x < y, being a merge-split:
 * the two sorted buckets are merged - on equal keys bucket x's element comes
 * first, and within a bucket the order is kept - and the lower S keys of the
 * merge become bucket x, the upper S bucket y.  With S = 1 a merge-split is a
 * strict compare-exchange, so PCM is then the plain odd-even network.
 * Status 2 when B or S is not a power of two (or S does not divide n).
 */
/* DARM_ORACLE_MUTANT 8 takes bucket y's element first on equal keys. */
static void pcm_merge_split(uint32_t* key, uint32_t* val, uint64_t x, uint64_t y, uint64_t S,
                            uint32_t* tk, uint32_t* tv) {
  const uint32_t* a = key + x * S;
  const uint32_t* b = key + y * S;
  uint64_t i = 0, j = 0;
  for (uint64_t o = 0; o < 2 * S; ++o) {
    int take_a;
    if (i == S)
      take_a = 0;
    else if (j == S)
      take_a = 1;
    else
      take_a = (DARM_ORACLE_MUTANT == 8) ? (a[i] < b[j]) : (a[i] <= b[j]);
    if (take_a) {
      tk[o] = a[i];
      if (val) tv[o] = val[x * S + i];
      ++i;
    } else {
      tk[o] = b[j];
      if (val) tv[o] = val[y * S + j];
      ++j;
    }
  }
  memcpy(key + x * S, tk, S * sizeof(uint32_t));
  memcpy(key + y * S, tk + S, S * sizeof(uint32_t));
  if (val) {
    memcpy(val + x * S, tv, S * sizeof(uint32_t));
    memcpy(val + y * S, tv + S, S * sizeof(uint32_t));
  }
}

static int pcm_buckets(uint32_t* key, uint32_t* val, uint64_t n, uint64_t S, uint64_t* B) {
  if (S == 0 || !is_pow2_u64(S) || n % S != 0) return ORACLE_ERR_NOT_POW2;
  *B = n / S;
  if (*B == 0) return ORACLE_OK;
  if (!is_pow2_u64(*B)) return ORACLE_ERR_NOT_POW2;
  for (uint64_t b = 0; b < *B; ++b)
    oracle_oddeven_u32(key + b * S, val ? val + b * S : NULL, S, NULL);
  return ORACLE_OK;
}

int oracle_pcm_u32(uint32_t* key, uint32_t* val, uint64_t n, uint64_t S) {
  uint64_t B = 0;
  const int rc = pcm_buckets(key, val, n, S, &B);
  if (rc != ORACLE_OK || B < 2) return rc;
  uint32_t* tk = (uint32_t*)malloc(2 * S * sizeof(uint32_t));
  uint32_t* tv = (uint32_t*)malloc(2 * S * sizeof(uint32_t));
  if (!tk || !tv) {
    free(tk);
    free(tv);
    return 1;
  }
  /* the iterative network of oracle_oddeven_u32, over bucket indices */
  for (uint64_t p = 1; p < B; p <<= 1)
    for (uint64_t k = p; k >= 1; k >>= 1)
      for (uint64_t j = k % p; j + k < B; j += 2 * k)
        for (uint64_t i = 0; i < k && i + j + k < B; ++i) {
          const uint64_t x = i + j;
          if (x / (2 * p) == (x + k) / (2 * p)) pcm_merge_split(key, val, x, x + k, S, tk, tv);
        }
  free(tk);
  free(tv);
  return ORACLE_OK;
}

/* The recursive form over buckets (the recursion of oracle_oddeven_rec_u32
 * with merge-splits for compare-exchanges). */
static void pcm_rec_merge(uint32_t* key, uint32_t* val, uint64_t S, uint64_t lo, uint64_t nb,
                          uint64_t r, uint32_t* tk, uint32_t* tv) {
  const uint64_t step = 2 * r;
  if (step < nb) {
    pcm_rec_merge(key, val, S, lo, nb, step, tk, tv);
    pcm_rec_merge(key, val, S, lo + r, nb, step, tk, tv);
    for (uint64_t i = lo + r; i + r < lo + nb; i += step) pcm_merge_split(key, val, i, i + r, S, tk, tv);
  } else {
    pcm_merge_split(key, val, lo, lo + r, S, tk, tv);
  }
}

static void pcm_rec_sort(uint32_t* key, uint32_t* val, uint64_t S, uint64_t lo, uint64_t nb,
                         uint32_t* tk, uint32_t* tv) {
  if (nb < 2) return;
  const uint64_t h = nb / 2;
  pcm_rec_sort(key, val, S, lo, h, tk, tv);
  pcm_rec_sort(key, val, S, lo + h, h, tk, tv);
  pcm_rec_merge(key, val, S, lo, nb, 1, tk, tv);
}

int oracle_pcm_rec_u32(uint32_t* key, uint32_t* val, uint64_t n, uint64_t S) {
  uint64_t B = 0;
  const int rc = pcm_buckets(key, val, n, S, &B);
  if (rc != ORACLE_OK || B < 2) return rc;
  uint32_t* tk = (uint32_t*)malloc(2 * S * sizeof(uint32_t));
  uint32_t* tv = (uint32_t*)malloc(2 * S * sizeof(uint32_t));
  if (!tk || !tv) {
    free(tk);
    free(tv);
    return 1;
  }
  pcm_rec_sort(key, val, S, 0, B, tk, tv);
  free(tk);
  free(tv);
  return ORACLE_OK;
}

/*
 * Synthetic divergent kernels SB1, SB4 and their -R variants (Section VI-A:
 * two nested loops whose inner loop holds a divergent region; every path
 * works on different data of the thread's shared-memory slice; SB1 is a
 * two-way diamond, SB4 a three-way if-else-if-else; in SB1/SB4 the paths
 * compute identically, in the -R variants they do not).  The paper's figure
 * with their exact code is lost; this is the form the library implements:
 *
 *   block of 256 threads, thread t owns words s[q] = data[blk*1024 + q*256 + t],
 *   q = 0..3; for it in [0, iters), for j in [0, 4):
 *     SB1:  c = (t ^ j ^ it) & 1;  c == 1: (a, b) = (j, j+1), else (j+2, j+3)
 *     SB4:  c = (t + j + it) % 3;  (a, b) = (j + c, j + c + 1)
 *     (indices mod 4); then R rounds of  s[a] = g(s[a], s[b]):
 *       identical paths:  g(v, w) = 3v + w
 *       -R paths:         c = 0: 3v + w,  c = 1: 5v ^ w,  c = 2: 7v - w
 *   (all arithmetic modulo 2^32).
 *   SB2:  the SB1 paths, each holding an if-then region guarded by the
 *         data: if (s[b] & 1) run the rounds (paired regions B2 / B3);
 *   SB3:  the SB1 paths, each holding two if-then regions: the SB2 one,
 *         then if (s[a] & 2) run rounds of s[b] = g2(s[b], s[a]) (paired
 *         regions C2 / C3 and C6 / C5), g2 = 3v + w, or in SB3-R
 *         path 0: 7v - w, path 1: 3v + w.
 * pattern: 1 SB1, 2 SB2, 3 SB3, 4 SB4, 101..104 their -R variants.  Status 1
 * on a bad pattern.
 */
int oracle_sb(int pattern, uint32_t* data, uint64_t nblocks, int iters, int rounds) {
  const int base = pattern % 100;
  if (base < 1 || base > 4 || (pattern != base && pattern != base + 100)) return 1;
  const int three_way = (base == 4);
  const int same = (pattern < 100);
  for (uint64_t blk = 0; blk < nblocks; ++blk) {
    uint32_t* d = data + blk * 1024;
    for (uint32_t t = 0; t < 256; ++t) {
      uint32_t s[4];
      for (int q = 0; q < 4; ++q) s[q] = d[q * 256 + t];
      for (int it = 0; it < iters; ++it) {
        for (uint32_t j = 0; j < 4; ++j) {
          uint32_t c, a, b;
          if (three_way) {
            c = (t + j + (uint32_t)it) % 3u;
            a = (j + c) & 3u;
          } else {
            c = (t ^ j ^ (uint32_t)it) & 1u;
            a = c ? j : ((j + 2) & 3u);
            c = c ? 0u : 1u; /* path index: 0 = first path, 1 = second */
          }
          b = (a + 1) & 3u;
          if (base >= 2 && base <= 3 && (s[b] & 1u) == 0u) {
            /* first region not taken */
          } else {
            for (int r = 0; r < rounds; ++r) {
              const uint32_t v = s[a], w = s[b];
              if (same || c == 0)
                s[a] = 3u * v + w;
              else if (c == 1)
                s[a] = (5u * v) ^ w;
              else
                s[a] = 7u * v - w;
            }
          }
          if (base == 3 && (s[a] & 2u) != 0u) {
            for (int r = 0; r < rounds; ++r) {
              const uint32_t v = s[b], w = s[a];
              s[b] = (same || c == 1) ? 3u * v + w : 7u * v - w;
            }
          }
        }
      }
      for (int q = 0; q < 4; ++q) d[q * 256 + t] = s[q];
    }
  }
  return 0;
}
