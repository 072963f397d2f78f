// plan.h - host-side planner: turns a sort request into a list of pass
// launches of the round kernel (pass_kernel.cuh).
//
// Schedule for one array of n = 2^m elements and a tile of T = 2^t
// elements (t <= m):
//   tile pass     stages k = 2 .. T inside each tile (Phase A in registers
//                 for k <= E, then register windows through shared memory);
//   for every stage k = 2T .. n (p = log2 k):
//     window passes   layers j >= T, LOGE2 of them per pass, straight from
//                     HBM to registers and back (the direction is uniform per
//                     block because bit k lies above the window);
//     merge pass      layers j < T inside each tile.
// Every pass reads and writes the array once, so the HBM traffic of a sort
// is 2 * n * (bytes per element) * passes.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "pass_kernel.cuh"

namespace darm {

enum KeyKind { KEY_U32 = 0, KEY_U64 = 1 };
enum PassKind { PASS_TILE = 0, PASS_WINDOW = 1, PASS_MERGE = 2 };

struct Tuning {
  int t;      // log2 tile elements (tile and merge passes)
  int e1;     // log2 elements per thread in tile and merge passes
  int e2;     // log2 elements per thread in window passes
  int c2;     // log2 threads per block in one-round window passes
  int w2;     // register windows per window pass (1: registers only; 2: one
              // shared-memory exchange, 2*e2 layers per HBM sweep)
  int tma = 0; // merge passes of single arrays prefetch tiles with bulk copies
               // into this many staging buffers (0: plain merge kernel)
  int shfl = 0; // bit 0: tile passes of single arrays run stages 2E .. 32E
                // across lanes with shuffles (tile_shfl_kernel.cuh); bit 1:
                // bulk-copy merge passes run their lane layers by shuffles
                // (two rounds instead of three), where built
  int em = 0;   // log2 elements per thread in merge passes (0: e1)
  int tm = 0;   // log2 tile of merge passes (0: t); tm < t: the window passes
                // of every stage above the tile also cover bits tm .. t-1
  int var[3]; // variant per pass kind (used when DARM_AUTO is requested)
};

// SM count the planner sizes persistent launches for (set at init).
extern int g_sms_for_plans;

// The driver's tensor-map encoder (cuTensorMapEncodeTiled), looked up at
// init.  g_tensor_maps: 1 found, 0 missing (no merge pass then uses the
// swizzled in-place kernel, tma == 3), -1 before init (plans made for
// inspection assume a driver that has it, as every CUDA 12+ driver does).
extern void* g_encode_tiled;
extern int g_tensor_maps;

struct Launch {
  PassKind kind;
  bool fixed;  // compile-time-schedule tile/merge kernel (tile_kernel.cuh)
  int tma;     // persistent merge with bulk-copy prefetch into this many
               // staging buffers (tma_merge.cuh); 3: in place in three
               // swizzled tile buffers with bulk tensor stores
               // (tma_merge_swz.cuh); 4: the same with two buffers per CTA
               // (key-value tiles of 2^12 pairs: three CTAs per SM); 0:
               // plain merge kernel
  bool win2;   // two-window pass with a compile-time shape (window2_kernel.cuh)
  bool win1;   // one-window pass with a compile-time shape (window1_kernel.cuh)
  bool win2t;  // two-window pass streamed through shared memory by TMA
               // (window2_tma.cuh): persistent over P.nblocks blocks
  bool shfl;   // tile pass with shuffle stages (tile_shfl_kernel.cuh)
  bool mshfl;  // bulk-copy merge in two rounds with shuffle layers
  int loge;
  int variant;
  uint32_t grid;
  uint32_t threads;
  size_t smem;
  PassParams P;
};

// Bytes one element occupies (key + optional payload).
inline int elem_bytes(KeyKind kk, bool has_vals) {
  return (kk == KEY_U32 ? 4 : 8) + (has_vals ? 4 : 0);
}

Tuning default_tuning(KeyKind kk, bool has_vals);

// Clamp a tuning to what the compiled kernels and the device allow for an
// array of 2^m elements.  Returns false if no valid plan exists.
bool fit_tuning(Tuning& tn, KeyKind kk, bool has_vals, int m, size_t smem_limit);

// Rounds of a tile pass (stages 2 .. 2^t) and of a merge pass (layers
// t-1 .. 0 of one stage p > t).
std::vector<Round> tile_rounds(int t, int e);
std::vector<Round> merge_rounds(int t, int e, int p);
// Rounds of a tile pass whose first round also runs stages E+1 .. E+S
// (S = min(5, t - e)) across lanes with shuffles.
std::vector<Round> tile_rounds_shfl(int t, int e);

// Whole-array plan.  variant: 0/1 force divergent/melded everywhere, 2 uses
// tn.var per pass kind.  map_in/map_out: key transforms of the first load and
// last store.  Fills `out` (keys/vals pointers left null).
bool plan_array(std::vector<Launch>& out, KeyKind kk, bool has_vals, int m, const Tuning& tn,
                int variant, uint32_t map_in, uint32_t map_out, size_t smem_limit);

std::string describe(const std::vector<Launch>& plan);

}  // namespace darm
