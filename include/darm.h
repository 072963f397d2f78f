/*
 * darm.h - C ABI of the GB300 bitonic compare-exchange library.
 *
 * The library sorts arrays that already live in device memory with the
 * bitonic network of DARM's running example (Saumya, Sundararajah and
 * Kulkarni, "DARM: Control-Flow Melding for SIMT Thread Divergence
 * Reduction", Fig. 1 and Section III).  Every stage exists in two forms:
 *
 *   DARM_DIVERGENT  the direction test of Fig. 1 guards two full copies of
 *                   the compare-exchange body (loads, compare, stores), one
 *                   per direction, so threads whose blocks run in opposite
 *                   directions diverge;
 *   DARM_MELDED     the two copies melded as in Sections IV-D and IV-G
 *                   (a region-region meld): the loads and stores of both
 *                   sides are aligned into one copy, and the two
 *                   direction-specific compares (key[l] < key[i] ascending,
 *                   key[l] > key[i] descending) are aligned into one compare
 *                   whose differing operands are selected by the direction
 *                   (Algorithm 2's SetOperands rule): the descending side's
 *                   keys are XORed with an all-ones direction mask when the
 *                   round loads them (~x reverses unsigned order), one
 *                   ascending compare-exchange runs for both directions,
 *                   and the store XORs the mask back.  The paper's own
 *                   melded BIT keeps the two compares unaligned and selects
 *                   the swap condition; both forms compute the same
 *                   comparator network bit for bit.
 *
 * Both forms compute the same comparator network and give bit-identical
 * results.  Conventions shared by every sorting entry point:
 *
 *   - Sorting is in place.  The caller owns `keys` and `vals`; both are
 *     device pointers (e.g. from torch.empty(..., device="cuda")) aligned to
 *     16 bytes.  `vals` may be NULL (keys only); otherwise it is a uint32
 *     payload that travels with its key.
 *   - n must be a power of two (Fig. 1's NUM); n = 0 and n = 1 are no-ops.
 *     n is limited to 2^31.
 *   - dir: DARM_ASC or DARM_DESC.  Descending flips every comparator of
 *     Fig. 1 (the paper shows only the ascending network).
 *   - A swap happens only on strict inequality, so the payload order among
 *     equal keys is the one fixed by the network (not a stable order).
 *   - Float keys are ordered by the IEEE-754 totalOrder of their bits
 *     (-0.0 sorts just below +0.0); NaNs sort by bit pattern.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL is the legacy default stream).  Argument errors are returned
 *     synchronously before anything is enqueued; launch failures return
 *     DARM_ERR_CUDA.  Errors detected on the device (sentinel collisions,
 *     bounded waits that ran out) are latched in a device status word that
 *     darm_device_status() reads.
 *   - darm_sort_init must be called first (per process; idempotent).  All
 *     calls are safe from several host threads; kernels of different
 *     streams may overlap.
 */
#ifndef DARM_H_
#define DARM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DARM_OK = 0,
  DARM_ERR_INVALID_ARG = 1,
  DARM_ERR_NOT_POW2 = 2,
  DARM_ERR_NOT_INIT = 3,
  DARM_ERR_OOM = 4,
  DARM_ERR_CUDA = 5,
  DARM_ERR_BUDGET = 6,
  DARM_ERR_TIMEOUT = 7,
  DARM_ERR_SENTINEL_COLLISION = 8,
  DARM_ERR_BUSY = 9,
  DARM_ERR_NOT_FOUND = 10
} darm_status;

typedef enum { DARM_ASC = 0, DARM_DESC = 1 } darm_dir;

typedef enum {
  DARM_DIVERGENT = 0,
  DARM_MELDED = 1,
  DARM_AUTO = 2 /* the tuned choice (melded unless the tuner found better) */
} darm_variant;

typedef enum { DARM_U32 = 0, DARM_F32 = 1, DARM_U64 = 2 } darm_dtype;

/* ---- context --------------------------------------------------------- */

/* Select `device`, query its SM count, configure shared memory for every
 * kernel and allocate the device status word plus `workspace_bytes` of
 * scratch for host-buffer sorts (0 = grow on demand).  Idempotent: a second
 * call with the same device returns DARM_OK. */
int darm_sort_init(int device, size_t workspace_bytes);

/* Release everything darm_sort_init and later calls allocated (plans,
 * graphs, workspace, serving state).  The caller's buffers are untouched. */
int darm_sort_finalize(void);

/* Diagnostic of the bounded waits: enqueue on `stream` a one-warp kernel
 * that waits on an mbarrier nothing ever completes, with the same bounded
 * wait (about one second of %globaltimer) as the passes that stream tiles
 * with bulk copies.  The wait gives up and latches DARM_ERR_TIMEOUT in the
 * device status word (darm_device_status reads and clears it); the kernel
 * then returns, so the context stays usable.  Returns DARM_ERR_NOT_INIT,
 * DARM_ERR_CUDA (launch failed) or DARM_OK. */
int darm_check_bounded_wait(void* stream);

/* Human-readable name of a darm_status value (static storage). */
const char* darm_status_str(int status);

/* Read and clear the device status word (synchronises the device).
 * *status receives DARM_OK or the first device-detected error. */
int darm_device_status(int* status);

/* ---- whole-array sort (Fig. 1, one array of n = 2^m elements) ---------- */

/* Every comparator of stages 2 .. n/2 stays inside one half of the array.
 * Arrays of 2^22 elements or more are therefore sorted in a split schedule:
 * the second half's tile pass and stages run on a stream owned by the
 * library, concurrently with the first half's on `stream`, and the final
 * stage runs on `stream` once both are done.  Work enqueued on `stream`
 * before the call happens before both halves, and work enqueued on it after
 * the call happens after the whole sort, as for any stream-ordered call.
 * Calls are serialised while they enqueue (the library stream's fork and
 * join events are shared).  The result is the one network of Fig. 1 over
 * the whole array. */

/* uint32 keys, optional uint32 payload. */
int darm_bitonic_sort(uint32_t* keys, uint32_t* vals, size_t n, int dir,
                      int variant, void* stream);

/* float32 keys (totalOrder), optional uint32 payload. */
int darm_bitonic_sort_f32(float* keys, uint32_t* vals, size_t n, int dir,
                          int variant, void* stream);

/* uint64 keys, optional uint32 payload. */
int darm_bitonic_sort_u64(uint64_t* keys, uint32_t* vals, size_t n, int dir,
                          int variant, void* stream);

/* Same sort on HOST buffers: copies keys (and vals) into library-owned
 * device memory, sorts, copies back and synchronises.  `dtype` is a
 * darm_dtype.  Host buffers may be pageable; pinned memory is faster.
 * Returns after the result is in the host buffers. */
int darm_bitonic_sort_host(void* keys, uint32_t* vals, size_t n, int dtype,
                           int dir, int variant);

/* ---- one array split into shards (one per process or device) -------------- */

/* The network of one array of nshards * n elements whose shard `shard`
 * (elements shard*n .. shard*n + n - 1) lives in keys/vals (DEVICE, n a power
 * of two, nshards a power of two, n * nshards <= 2^31).  Composed as:
 *   darm_bitonic_sort_shard;
 *   for every stage k = 2n, 4n, .. nshards*n (log2k = log2 of k):
 *     for every layer j = k/2 .. n (log2j): exchange the shard with shard
 *       shard ^ (j / n) (the caller moves the peer's copy into peer_keys /
 *       peer_vals on this device) and call darm_bitonic_exchange;
 *     darm_bitonic_merge_shard(log2k).
 * Every comparator is the whole array's (Fig. 1), so the shards end holding
 * exactly the whole-array sort.  Between the first call and the final
 * stage's merge the keys are in the network's internal form (float keys as
 * totalOrder words, descending sorts complemented); the final merge restores
 * them.  With nshards = 1, darm_bitonic_sort_shard alone sorts the array.
 * Errors: DARM_ERR_NOT_POW2, DARM_ERR_INVALID_ARG (shard >= nshards,
 * misaligned or NULL buffers, a layer outside the schedule, a shard within
 * one tile for darm_bitonic_merge_shard), DARM_ERR_CUDA. */
int darm_bitonic_sort_shard(void* keys, uint32_t* vals, size_t n, int dtype, size_t shard,
                            size_t nshards, int dir, int variant, void* stream);

/* Layer j = 2^log2j (n <= j < k) of stage k = 2^log2k: element i of this
 * shard and element i of shard shard ^ (j / n) (peer_keys / peer_vals, the
 * peer's values before this layer) form one comparator; this shard keeps its
 * side of the pair.  One direction for the whole shard, so there is no
 * divergent and melded form. */
int darm_bitonic_exchange(void* keys, uint32_t* vals, const void* peer_keys,
                          const uint32_t* peer_vals, size_t n, int dtype, size_t shard,
                          size_t nshards, int log2k, int log2j, int dir, void* stream);

/* Layers j = n/2 .. 1 of stage k = 2^log2k (k > n) on this shard (n must
 * exceed one tile of the plan). */
int darm_bitonic_merge_shard(void* keys, uint32_t* vals, size_t n, int dtype, size_t shard,
                             size_t nshards, int log2k, int dir, int variant, void* stream);

/* ---- batched segmented sort ------------------------------------------ */

/* Sort num_segs independent segments in one batched launch sequence: the
 * paper's BIT benchmark sorts its input bucket by bucket, one thread block
 * per bucket (Section VI-A); here the buckets are arrays of uneven size.
 * Segment s occupies elements [seg_offsets[s], seg_offsets[s+1]) of keys
 * and vals; its capacity (the difference) must be a power of two and its
 * offset a multiple of min(capacity, 4) elements.  Only the first seg_len[s] elements are
 * real: the library writes the sentinel (UINT32_MAX for ascending, 0 for
 * descending; payload 0xFFFFFFFF) beyond them and sorts the whole capacity,
 * so the real keys end up first.  seg_offsets (uint64, num_segs + 1
 * entries) and seg_len (uint32) are HOST arrays, not device arrays: the
 * launch sequence (how many passes, how many blocks each, which segments
 * share a block) depends on the layout, so the host must read it anyway; the
 * library builds a longest-first work list from it, uploads it once and
 * replays the launch sequence as a CUDA graph on later calls with the same
 * layout.
 * seg_desc (HOST, uint8 per segment, nullable) overrides `dir` per segment.
 * With a payload, a real key equal to the sentinel makes the result
 * ambiguous; the kernel latches DARM_ERR_SENTINEL_COLLISION in the device
 * status word (see darm_device_status) and still sorts. */
int darm_segmented_sort(uint32_t* keys, uint32_t* vals, const uint64_t* seg_offsets,
                        const uint32_t* seg_len, uint32_t num_segs, int dir,
                        int variant, const uint8_t* seg_desc, void* stream);

/* Same sort as darm_segmented_sort for callers that cannot allocate device
 * memory - e.g. an application whose own allocator owns the whole GPU, or a
 * latency-critical loop that cannot take the device synchronisation
 * cudaMalloc/cudaFree bring.  (The paper has no counterpart; this is a
 * service of this library.)  The block tables and work counter that
 * darm_segmented_sort keeps in buffers it allocates are instead copied, on
 * `stream`, into one 1 MiB array compiled into the library, right before each
 * launch; nothing is allocated on the device and no graph is built.
 *   - Limit: the tables of any single launch must fit in 1 MiB:
 *     256 bytes of counter + 16 bytes per segment slot of the launch's phase
 *     (rounded up to a multiple of 256) + 12 bytes per block of the launch
 *     <= 1,048,576 bytes (so at most 65,520 slots, or 87,360 blocks, in one
 *     launch); larger layouts are rejected with DARM_ERR_INVALID_ARG and a
 *     message on stderr, before anything is enqueued.
 *   - The array is shared by every call and keeps the last call's contents:
 *     calls whose work overlaps on the GPU (other streams, other host
 *     threads) race on it.  Calls on one stream are ordered and safe.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it.
 *   - Each launch's tables are copied from host memory that the call reuses
 *     and frees before it returns, so the call must not be recorded into a
 *     CUDA graph: on a stream that is capturing it returns
 *     DARM_ERR_INVALID_ARG before enqueueing anything.
 * Arguments, layout rules and results are those of darm_segmented_sort. */
int darm_segmented_sort_noalloc(uint32_t* keys, uint32_t* vals, const uint64_t* seg_offsets,
                                const uint32_t* seg_len, uint32_t num_segs, int dir,
                                int variant, const uint8_t* seg_desc, void* stream);

/* ---- Batcher's odd-even merge sort network (one thread block) ------------ */

/* Sort n <= 4096 uint32 keys (power of two) ascending with Batcher's
 * odd-even merge sort network, the network the paper's PCM benchmark builds
 * on (Section VI-A), on one thread block in shared memory.  keys/vals are
 * DEVICE pointers (vals nullable: keys only; a payload travels with its
 * key; equal keys never move, so the payload order under ties is the
 * network's).  variant: DARM_DIVERGENT (one branch per comparator end) or
 * DARM_MELDED / DARM_AUTO (the two ends' loads and compares melded).
 * Asynchronous on `stream`.  Errors: DARM_ERR_NOT_POW2, DARM_ERR_INVALID_ARG
 * (n > 4096, NULL keys, bad variant), DARM_ERR_CUDA (launch). */
int darm_oddeven_sort_block(uint32_t* keys, uint32_t* vals, size_t n, int variant,
                            void* stream);

/* The same network on every aligned bucket of `bucket` keys (a power of two,
 * <= 4096) of an array of n keys (a multiple of `bucket`), one thread block
 * per bucket: the way the paper's benchmarks sort their input bucket by
 * bucket (Section VI-A).  Each bucket is sorted ascending on its own.
 * Errors: DARM_ERR_NOT_POW2 (bucket), DARM_ERR_INVALID_ARG (bucket > 4096,
 * n not a multiple of bucket, NULL keys, bad variant), DARM_ERR_CUDA. */
int darm_oddeven_sort_buckets(uint32_t* keys, uint32_t* vals, size_t n, size_t bucket,
                              int variant, void* stream);

/* PCM, Partition and Concurrent Merge (Section VI-A): a sort of the whole
 * array built on Batcher's odd-even merge sort.  The n keys form n / bucket
 * buckets (bucket a power of two <= 4096, the bucket count a power of two);
 * each bucket is sorted by the odd-even merge sort network
 * (darm_oddeven_sort_buckets), then the same network runs over the buckets
 * with every comparator (bucket x, bucket y > x) a merge-split: the two
 * sorted buckets are merged - on equal keys bucket x's key first, each
 * bucket's keys in order - and the lower half becomes bucket x, the upper
 * half bucket y.  The result is the whole array sorted ascending, the
 * payload order under equal keys being the one this network fixes.
 * keys/vals: DEVICE arrays sorted in place (vals nullable); scratch_keys
 * (and scratch_vals when vals is given): DEVICE arrays of n elements the
 * call may overwrite (not needed when there is one bucket); all 16-byte
 * aligned.  variant: DARM_DIVERGENT (the merge loop's data-dependent branch
 * with one copy of its body per side) or DARM_MELDED / DARM_AUTO (the two
 * sides melded by selects).  Asynchronous on `stream`.  Errors:
 * DARM_ERR_NOT_POW2 (bucket or bucket count), DARM_ERR_INVALID_ARG (bucket
 * > 4096, n not a multiple of bucket, n > 2^32, NULL or misaligned
 * buffers, bad variant), DARM_ERR_CUDA. */
int darm_pcm_sort(uint32_t* keys, uint32_t* vals, size_t n, size_t bucket,
                  uint32_t* scratch_keys, uint32_t* scratch_vals, int variant, void* stream);

/* ---- synthetic divergent kernels (Section VI-A) ------------------------- */

/* The paper's synthetic kernels, as built here: two nested loops whose inner
 * loop holds a divergent region; each path works on different words of the
 * thread's shared-memory slice.  pattern: 1 = SB1 (two-way diamond, paths
 * compute identically), 2 = SB2 (each path an if-then region guarded by the
 * data), 3 = SB3 (two such regions per path), 4 = SB4 (three-way
 * if-else-if-else); 101..104 = their -R variants (paths compute
 * differently).  data: DEVICE array
 * of nblocks * 1024 uint32 words, updated in place (block b owns words
 * [b*1024, (b+1)*1024), thread t of it the words q*256 + t, q = 0..3); the
 * outer loop runs `iters` times, each path `rounds` compute rounds.
 * variant: DARM_DIVERGENT or DARM_MELDED / DARM_AUTO.  Asynchronous on
 * `stream`.  Errors: DARM_ERR_INVALID_ARG (pattern, negative counts, NULL
 * data), DARM_ERR_CUDA. */
int darm_sb_run(int pattern, uint32_t* data, size_t nblocks, int iters, int rounds, int variant,
                void* stream);

/* ---- melding analysis (host only) -------------------------------------- */

/* One instruction of a divergent path: `opcode` is what the frequency
 * profile counts (an IR opcode), `type` refines it for alignment (operand
 * types, compare predicate), `latency` its static cost.  Instructions with
 * equal opcode must carry equal latency. */
typedef struct {
  int32_t opcode;
  int32_t type;
  int32_t latency;
} darm_inst;

/* Melding profitability of two basic blocks (Section IV-C, MP_B): the sum
 * over opcodes of min(frequency in b1, frequency in b2) x latency, over
 * lat(b1) + lat(b2).  Identical profiles give 0.5.  Host arrays; NaN on bad
 * arguments or inconsistent latencies. */
double darm_meld_mp_block(const darm_inst* b1, int n1, const darm_inst* b2, int n2);

/* Melding profitability of two isomorphic subgraphs (MP_S): nb corresponding
 * block pairs, block k of path 1 being i1[off1[k] .. off1[k+1]) (likewise
 * path 2); the latency-weighted mean of the pairs' MP_B.  NaN on bad
 * arguments. */
double darm_meld_mp_subgraph(const darm_inst* i1, const int32_t* off1, const darm_inst* i2,
                             const int32_t* off2, int nb);

/* Instruction alignment of two blocks (Smith-Waterman, Section IV-C):
 * compatible instructions (same opcode and type) align with score equal to
 * their latency, each unaligned instruction inside the aligned stretch costs
 * `gap` (>= 0).  Writes both sequences in program order as (i, j) pairs into
 * `pairs` (capacity 2 * (na + nb) int32): (i, j) aligned, (i, -1) or
 * (-1, j) unaligned.  Returns the number of pairs (-1 on bad arguments) and
 * the alignment score in *score (nullable). */
int darm_meld_align(const darm_inst* a, int na, const darm_inst* b, int nb, double gap,
                    int32_t* pairs, double* score);

/* A single-entry single-exit subgraph (Def. 3) of one path of a divergent
 * region: `nblocks` basic blocks linearised in pre-order, block k being
 * block `first_block + k` of a block table (block b = instructions
 * insts[block_off[b] .. block_off[b+1])).  Two subgraphs of more than one
 * block are isomorphic exactly when they have the same `shape` id (and
 * block count); `simple_region` is 1 for a simple region (Def. 1). */
typedef struct {
  int32_t first_block;
  int32_t nblocks;
  int32_t shape;
  int32_t simple_region;
} darm_subgraph;

/* The paper's default melding profitability threshold (Section V). */
#define DARM_MELD_THRESHOLD 0.2

/* Melding profitability of two SESE subgraphs (Def. 6, Section IV-C):
 * case 1, two isomorphic subgraphs of more than one block: MP_S over the
 * corresponding blocks; case 3, two single blocks: MP_B; case 2, a single
 * block A against a simple region M (region replication): A is placed
 * beside the block E of M with the highest MP_B(A, E) (first in pre-order
 * on ties) in a copy of M whose other blocks are empty, giving
 * MP_B(A, E) * (lat(A) + lat(E)) / (lat(A) + lat(M)).  Returns -1 when the
 * pair is not meldable (different shapes, or a block against a region that
 * is not simple); NaN on bad arguments or inconsistent latencies.  Host
 * arrays; block_off has nblocks_total + 1 entries. */
double darm_meld_mp_sese(const darm_inst* insts, const int32_t* block_off, int nblocks_total,
                         const darm_subgraph* s1, const darm_subgraph* s2);

/* Subgraph alignment (Def. 7) and the meld decision of Algorithm 1: the
 * ordered subgraphs st[0..m) of the true path and sf[0..n) of the false
 * path are aligned by Smith-Waterman, an aligned pair scoring its
 * profitability (darm_meld_mp_sese; non-meldable pairs cannot align) and
 * each unaligned subgraph inside the aligned stretch costing `gap` (>= 0).
 * Writes the k aligned pairs in order: (pairs[2i], pairs[2i+1]) = indices
 * into st and sf, profit[i] their profitability and meld[i] = 1 when
 * profit[i] >= threshold (Algorithm 1 melds those; pass
 * DARM_MELD_THRESHOLD for the paper's default).  Capacity: min(m, n)
 * pairs.  Returns k (-1 on bad arguments) and the alignment score in
 * *score (nullable). */
int darm_meld_subgraph_align(const darm_inst* insts, const int32_t* block_off, int nblocks_total,
                             const darm_subgraph* st, int m, const darm_subgraph* sf, int n,
                             double gap, double threshold, int32_t* pairs, double* profit,
                             int32_t* meld, double* score);

/* ---- tuning ----------------------------------------------------------- */

/* Time candidate tile sizes, elements per thread and per-stage variants for
 * arrays of n elements of `dtype` (with payload if has_vals), keep the
 * fastest as the plan DARM_AUTO uses, and append it to the text file
 * db_path (NULL: keep in memory only).  Allocates and frees its own scratch;
 * synchronises the device. */
int darm_autotune(int dtype, size_t n, int has_vals, const char* db_path);

/* Autotuner for batched segmented sorts (darm_segmented_sort with DARM_AUTO,
 * and darm_segmented_sort_noalloc).  The paper treats the block size as a
 * tunable evaluated per size (Section VI-A, "Block Size"); here every
 * candidate tuning - tile size, register windows per window pass, elements
 * per thread in window passes - is timed on whole batched sorts of the
 * caller's own layout (keys/vals: DEVICE buffers laid out as for
 * darm_segmented_sort; seg_offsets/seg_len: HOST arrays), then the
 * divergent or melded form per pass kind (tile, window, merge).  The
 * fastest becomes the batch tuning and is appended to db_path as a line
 * with log2 n = 0 (NULL: memory only).  The segments are sorted in place
 * several times (ascending); on return they hold the ascending sort.
 * Allocates and frees its tables; synchronises the device.
 * Errors: DARM_ERR_INVALID_ARG (no segments, misaligned buffers, or no
 * candidate could run), DARM_ERR_NOT_POW2 (a capacity is not a power of
 * two), DARM_ERR_CUDA. */
int darm_autotune_segmented(uint32_t* keys, uint32_t* vals, const uint64_t* seg_offsets,
                            const uint32_t* seg_len, uint32_t num_segs, const char* db_path);

/* Load plans previously written by darm_autotune and
 * darm_autotune_segmented (lines with log2 n = 0 are batch tunings).  A
 * line holds 13 to 16 whitespace-separated fields: key kind (0 32-bit, 1
 * 64-bit), payload flag, log2 n, log2 tile, log2 elements per thread in
 * tile/merge passes and in window passes, log2 threads of a one-window
 * pass, register windows per window pass, bulk-copy staging buffers of the
 * merge, the form (0 divergent, 1 melded) of tile, window and merge passes,
 * the tuner's time in ms, and optionally the shuffle field (bit 0: tile
 * pass with shuffle stages, bit 1: merge lane layers by shuffles), log2
 * elements per thread of merge passes and log2 tile of merge passes (each 0
 * when absent: the defaults). */
int darm_load_tune_db(const char* db_path);

/* Forget every tuning loaded or measured so far: later calls plan with the
 * library's defaults again. */
int darm_reset_tunings(void);

/* ---- introspection ----------------------------------------------------- */

/* Describe the launch sequence for a whole-array sort of n elements:
 * passes = number of full read+write sweeps over the array in HBM,
 * launches = kernel launches, tile = elements a tile pass keeps on chip. */
int darm_plan_info(int dtype, size_t n, int has_vals, int variant,
                   int* passes, int* launches, int* tile);

/* Text description of the launch sequence darm_plan_info counts, one line
 * per launch: pass kind ("tile", "window", "merge"; "*" marks a
 * compile-time schedule, "~" a tile pass with shuffle stages, "^" a pass
 * that streams its blocks through shared memory with TMA tensor copies and
 * works on them in place), elements per
 * thread, form, grid, threads, shared memory and the block bit map.  Writes
 * at most cap bytes into buf, NUL-terminated. */
int darm_plan_describe(int dtype, size_t n, int has_vals, int variant, char* buf, size_t cap);

/* The launch sequence of a whole-array sort as numbers, for checking the
 * planner on the host (no device needed, darm_sort_init not required).
 * tuning (nullable: the tuning a sort of this size would use): 8 int32 -
 * log2 tile, log2 elements per thread in tile/merge passes and in window
 * passes, log2 threads of a one-window pass, windows per window pass,
 * bulk-copy staging buffers, shuffle stages (bit 0 tile pass, bit 1 merge
 * passes), log2 tile of the merge passes (0: the tile pass's; smaller: the
 * window passes of each stage above the tile also cover the bits between).  smem_limit: shared
 * memory per block the plan may use (0: the device's, or 227 KiB before
 * init).  Writes, per launch, 21 int32 - pass kind (0 tile, 1 window,
 * 2 merge), compile-time tile/merge schedule, bulk-copy buffers (3: the
 * merge in place in swizzled buffers; 4: the same with two buffers per
 * CTA), one-window and two-window
 * compile-time shapes (two-window 2: streamed by TMA), shuffle stages,
 * log2 elements per
 * thread, form, grid, threads, shared memory bytes, then the block bit map
 * b, c, w0, s, log2 of the array length, rounds, persistent block count,
 * key map in and out, two-round shuffle merge - followed by 7 int32 per
 * round: kind (0 registers
 * only, 1 window), stage bit p, window bit a, layers, source and
 * destination (0 HBM, 1 shared memory), lane-divergent flag.  *count
 * receives the number of int32 needed; DARM_ERR_INVALID_ARG when cap is
 * smaller (nothing written). */
int darm_plan_dump(int dtype, size_t n, int has_vals, int variant, const int32_t* tuning,
                   size_t smem_limit, int32_t* out, int cap, int* count);

/* Profiling run of a whole-array sort: the launches of the array's plan in
 * plan order, all on `stream` (arrays of 2^22 elements or more: the whole
 * array's passes, not the split schedule of the plain call), with a CUDA
 * event pair recorded on `stream` around each one.  Synchronises
 * the stream, then writes for launch i < cap: ms[i] = its device time and
 * kind[i] = 0 tile pass, 1 window pass, 2 merge pass; *count = launches.
 * The keys are sorted exactly as by the plain call. */
int darm_sort_profile(void* keys, uint32_t* vals, size_t n, int dtype, int dir, int variant,
                      void* stream, float* ms, int* kind, int cap, int* count);

/* Number of kernels this library has launched since darm_sort_init
 * (graph replays count each kernel node). */
uint64_t darm_launch_count(void);

/* ---- serving: continuous batching of sort requests --------------------- */

typedef struct {
  size_t budget_bytes;  /* device memory all admitted jobs may hold */
  int max_inflight;     /* admitted jobs at once */
  int variant;          /* darm_variant for every job */
  int num_streams;      /* streams the scheduler spreads batched launches over */
} darm_serve_cfg;

/* Start the scheduler thread.  It owns a device arena of budget_bytes. */
int darm_sort_serve_start(const darm_serve_cfg* cfg);

/* Queue a sort of n keys (device pointer `keys` of `dtype`, optional device
 * payload `vals`) in direction `dir`.  n need not be a power of two: the
 * job is padded to the next power of two with sentinels inside the arena
 * and only the n real elements are written back.  The buffers must stay
 * valid until the request is reported done.  Returns DARM_ERR_BUDGET if the
 * job alone exceeds the budget. */
int darm_sort_serve_submit(void* keys, uint32_t* vals, size_t n, int dtype,
                           int dir, uint64_t* req_id);

/* Non-blocking: *done = 1 once the result is in the caller's buffers. */
int darm_sort_serve_poll(uint64_t req_id, int* done);

/* Block until done or timeout_ms passes (DARM_ERR_TIMEOUT). */
int darm_sort_serve_wait(uint64_t req_id, int timeout_ms);

/* Latency percentiles (submit to completion) and throughput of all
 * requests completed so far. */
int darm_sort_serve_stats(double* p50_ms, double* p99_ms, double* keys_per_s,
                          uint64_t* completed);

/* Fault injection for tests: the next tick's launches fail with `status`
 * (on the host, before anything is launched); every job that tick carried
 * completes with that status and its arena space is released.  No device
 * fault is involved. */
int darm_sort_serve_inject_fault(int status);

/* Drain outstanding jobs, stop the scheduler and free the arena. */
int darm_sort_serve_stop(void);

#ifdef __cplusplus
}
#endif

#endif /* DARM_H_ */
