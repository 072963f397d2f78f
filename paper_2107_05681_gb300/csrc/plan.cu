// plan.cu - host planner for the bitonic network's passes (see plan.h).
#include <algorithm>
#include <cstdio>
#include <sstream>

#include "kernel_table.h"
#include "plan.h"
#include "tile_kernel.cuh"

namespace darm {

int fixed_schedule_rounds(int logt, int loge, bool merge, SRound* out, int cap);
int shfl_schedule_rounds(int logt, int loge, SRound* out, int cap);

// A compile-time-schedule kernel is used only if one was built for this
// (key, payload, E, T) and its schedule equals the planner's round list.
static bool has_fixed(KeyKind kk, bool has_vals, int loge, int logt) {
  KernelEntry e = (kk == KEY_U32) ? tile_kernel_u32(has_vals, loge, logt, 1, false)
                                  : tile_kernel_u64(has_vals, loge, logt, 1, false);
  if (e.fn == nullptr) return false;
  for (int merge = 0; merge < 2; ++merge) {
    SRound sr[kMaxRounds];
    const int n = fixed_schedule_rounds(logt, loge, merge != 0, sr, kMaxRounds);
    const std::vector<Round> rs = merge ? merge_rounds(logt, loge, logt + 1) : tile_rounds(logt, loge);
    if (n != int(rs.size())) return false;
    for (int i = 0; i < n; ++i) {
      const Round& r = rs[i];
      if (sr[i].kind != r.kind || sr[i].a != r.a || sr[i].cnt != r.cnt || sr[i].src != r.src ||
          sr[i].dst != r.dst || (!merge && sr[i].p != r.p))
        return false;
    }
  }
  return true;
}

// A shuffle-stage tile kernel is used only if one was built for this shape
// and its compile-time schedule equals the planner's round list.
static bool has_shfl(KeyKind kk, bool has_vals, int loge, int logt) {
  if (kk != KEY_U32 || tile_shfl_kernel_u32(has_vals, loge, logt, 1).fn == nullptr) return false;
  SRound sr[kMaxRounds];
  const int n = shfl_schedule_rounds(logt, loge, sr, kMaxRounds);
  const std::vector<Round> rs = tile_rounds_shfl(logt, loge);
  if (n != int(rs.size())) return false;
  for (int i = 0; i < n; ++i) {
    const Round& r = rs[i];
    if (sr[i].kind != r.kind || sr[i].p != r.p || sr[i].a != r.a || sr[i].cnt != r.cnt ||
        sr[i].src != r.src || sr[i].dst != r.dst)
      return false;
  }
  return true;
}

int g_sms_for_plans = 152;
void* g_encode_tiled = nullptr;
int g_tensor_maps = -1;

static int max_threads(KeyKind kk, bool has_vals, int loge) {
  KernelEntry e = (kk == KEY_U32) ? kernel_u32(has_vals, loge, 1) : kernel_u64(has_vals, loge, 1);
  return e.fn ? e.max_threads : 0;
}

Tuning default_tuning(KeyKind kk, bool has_vals) {
  const int words = (kk == KEY_U32 ? 1 : 2) + (has_vals ? 1 : 0);
  Tuning tn;
  if (words == 1) {
    tn.t = 14;  // 16 Ki uint32 keys = 64 KiB of shared memory per tile
    tn.e1 = 5;  // 32 keys per thread: five layers per shared-memory round
    tn.e2 = 5;  // window passes: 10 layers per HBM sweep
    tn.c2 = 8;
    tn.w2 = 2;
    tn.tma = 3;  // in place, three swizzled tiles, bulk tensor stores: 2^26
                 // float keys, merge pass 117 -> 96 us (else 2: two dense
                 // staging buffers)
    tn.shfl = 1;  // 2^26 float keys: tile pass 0.686 -> 0.639 ms
  } else if (words == 2) {
    // tile pass on 8 Ki pairs, merges on 4 Ki-pair tiles (the window passes
    // take bit 12): 27 HBM sweeps instead of 29; 2^24 pairs 1.592 ->
    // 1.539 ms (tile pass 273 -> 307 us, one window and one merge pass
    // fewer).  For keys alone the 2^15-key tile pass costs about what the
    // two sweeps save (2.946 -> 2.926 ms), so they keep one tile size.
    tn.t = 13;
    tn.tm = 12;
    tn.e1 = 4;
    tn.e2 = 4;
    tn.c2 = 8;
    tn.w2 = 2;
    tn.tma = 4;   // in place, keys and payloads in swizzled buffers, two
                  // per CTA and three CTAs per SM: 2^24 pairs, merge pass
                  // 55.0 -> 51.0 us with three buffers (two CTAs per SM),
                  // 50.3 -> 49.3 us with two (sort 1.505 -> 1.486 ms)
    tn.shfl = 1;  // 2^24 key-value pairs: tile pass 0.335 -> 0.267 ms
  } else {
    tn.t = 12;  // 4 Ki elements of 12 bytes = 48 KiB
    tn.e1 = 3;
    tn.e2 = 3;
    tn.c2 = 8;
    tn.w2 = 2;
    tn.tma = 0;
  }
  tn.var[0] = tn.var[1] = tn.var[2] = kMelded;
  return tn;
}

static int count_tile_rounds(int t, int e) {
  int r = 1;
  for (int p = e + 1; p <= t; ++p) r += (p + e - 1) / e;
  return r;
}

bool fit_tuning(Tuning& tn, KeyKind kk, bool has_vals, int m, size_t smem_limit) {
  if (m < 1) return false;
  tn.e1 = std::max(1, std::min(tn.e1, 5));
  tn.e2 = std::max(1, std::min(tn.e2, 5));
  tn.t = std::min(tn.t, m);
  // shared memory: one tile of keys + payload
  while (tn.t > 1 && size_t(elem_bytes(kk, has_vals)) * smem_words(1u << tn.t) > smem_limit) --tn.t;
  tn.e1 = std::min(tn.e1, tn.t);
  if (tn.t >= 2) tn.e1 = std::max(tn.e1, 2);
  // block size of tile passes must fit the instantiation
  while ((1 << (tn.t - tn.e1)) > max_threads(kk, has_vals, tn.e1)) {
    if (tn.e1 < 5) {
      ++tn.e1;
    } else {
      --tn.t;
    }
  }
  while (count_tile_rounds(tn.t, tn.e1) > kMaxRounds) ++tn.e1;
  if (tn.e1 > 5 || tn.e1 > tn.t) return false;
  // window passes: threads cover low bits, window of e2 bits
  tn.c2 = std::max(0, std::min(tn.c2, 10));
  while ((1 << tn.c2) > max_threads(kk, has_vals, tn.e2)) --tn.c2;
  tn.w2 = std::max(1, std::min(tn.w2, 2));
  return true;
}

std::vector<Round> tile_rounds(int t, int e) {
  std::vector<Round> rs;
  Round a{};
  a.kind = RK_PHASE_A;
  a.p = uint8_t(e);
  a.a = 0;
  a.cnt = uint8_t(e);
  a.src = LOC_GLOBAL;
  a.dst = (t == e) ? LOC_GLOBAL : LOC_SMEM;
  rs.push_back(a);
  for (int p = e + 1; p <= t; ++p) {
    const int nw = (p + e - 1) / e;
    for (int i = nw - 1; i >= 0; --i) {
      const int lo = i * e;
      const int hi = std::min((i + 1) * e, p) - 1;
      Round r{};
      r.kind = RK_WINDOW;
      r.p = uint8_t(p);
      r.a = uint8_t(hi - e + 1);
      r.cnt = uint8_t(hi - lo + 1);
      r.src = LOC_SMEM;
      r.dst = LOC_SMEM;
      rs.push_back(r);
    }
  }
  rs.back().dst = LOC_GLOBAL;
  return rs;
}

std::vector<Round> tile_rounds_shfl(int t, int e) {
  const int last_shfl = e + std::min(5, t - e);
  std::vector<Round> rs;
  Round a{};
  a.kind = RK_PHASE_A;
  a.p = uint8_t(last_shfl);  // Phase A runs stages up to 2^last_shfl
  a.a = 0;
  a.cnt = uint8_t(e);
  a.src = LOC_GLOBAL;
  a.dst = (t == last_shfl) ? LOC_GLOBAL : LOC_SMEM;
  rs.push_back(a);
  for (int p = last_shfl + 1; p <= t; ++p) {
    const int nw = (p + e - 1) / e;
    for (int i = nw - 1; i >= 0; --i) {
      const int lo = i * e;
      const int hi = std::min((i + 1) * e, p) - 1;
      Round r{};
      r.kind = RK_WINDOW;
      r.p = uint8_t(p);
      r.a = uint8_t(hi - e + 1);
      r.cnt = uint8_t(hi - lo + 1);
      r.src = LOC_SMEM;
      r.dst = LOC_SMEM;
      rs.push_back(r);
    }
  }
  rs.back().dst = LOC_GLOBAL;
  return rs;
}

std::vector<Round> merge_rounds(int t, int e, int p) {
  std::vector<Round> rs;
  const int nw = (t + e - 1) / e;
  for (int i = nw - 1; i >= 0; --i) {
    const int lo = i * e;
    const int hi = std::min((i + 1) * e, t) - 1;
    Round r{};
    r.kind = RK_WINDOW;
    r.p = uint8_t(p);
    r.a = uint8_t(hi - e + 1);
    r.cnt = uint8_t(hi - lo + 1);
    r.src = LOC_SMEM;
    r.dst = LOC_SMEM;
    rs.push_back(r);
  }
  rs.front().src = LOC_GLOBAL;
  rs.back().dst = LOC_GLOBAL;
  return rs;
}

// Lane bit j (thread-index bit j < 5) of a round with window a..a+e-1 maps
// to local bit j (below the window) or j + e (above it).  The direction of
// stage 2^p can differ within a warp when local bit p is one of them.
static bool lane_divergent(int p, int a, int e, int b, int threads_log2) {
  if (p >= b) return false;  // block-index bit: uniform per block
  const int lanes = std::min(5, threads_log2);
  for (int j = 0; j < lanes; ++j) {
    const int pos = (j < a) ? j : j + e;
    if (pos == p) return true;
  }
  return false;
}

static void mark_lanes(std::vector<Round>& rs, int e, int b, int threads_log2) {
  for (Round& r : rs) r.lanediv = lane_divergent(r.p, r.a, e, b, threads_log2) ? 1 : 0;
}

static void set_rounds(PassParams& P, const std::vector<Round>& rs) {
  P.nrounds = uint32_t(rs.size());
  for (size_t i = 0; i < rs.size(); ++i) P.rounds[i] = rs[i];
}

static bool uses_smem(const std::vector<Round>& rs) {
  for (const Round& r : rs)
    if (r.src == LOC_SMEM || r.dst == LOC_SMEM) return true;
  return false;
}

static int pick_var(int variant, const Tuning& tn, PassKind k) {
  return (variant == 0 || variant == 1) ? variant : tn.var[k];
}

bool plan_array(std::vector<Launch>& out, KeyKind kk, bool has_vals, int m, const Tuning& tn0,
                int variant, uint32_t map_in, uint32_t map_out, size_t smem_limit) {
  out.clear();
  Tuning tn = tn0;
  if (!fit_tuning(tn, kk, has_vals, m, smem_limit)) return false;
  const int t = tn.t, e1 = tn.e1, e2 = tn.e2;
  const size_t tile_smem = size_t(elem_bytes(kk, has_vals)) * smem_words(1u << t);

  // tile pass
  {
    Launch L{};
    L.kind = PASS_TILE;
    L.fixed = has_fixed(kk, has_vals, e1, t);
    L.shfl = (tn.shfl & 1) != 0 && has_shfl(kk, has_vals, e1, t);
    L.loge = e1;
    L.variant = pick_var(variant, tn, PASS_TILE);
    L.grid = uint32_t(1u << (m - t));
    L.threads = 1u << (t - e1);
    std::vector<Round> rs = L.shfl ? tile_rounds_shfl(t, e1) : tile_rounds(t, e1);
    mark_lanes(rs, e1, t, t - e1);
    L.smem = uses_smem(rs) ? tile_smem : 0;
    L.P.b = uint32_t(t);
    L.P.c = uint32_t(t);
    L.P.w0 = uint32_t(t);
    L.P.s = 0;
    L.P.log2cap = uint32_t(m);
    L.P.map_in = map_in;
    L.P.map_out = (m == t) ? map_out : 0u;
    set_rounds(L.P, rs);
    out.push_back(L);
  }
  // Merge passes may take smaller tiles than the tile pass (tn.tm < t): the
  // window passes of every stage p > t then cover layer bits tg .. p-1 and
  // the merge the bits below tg.  Fewer, longer stages in the tile pass
  // trade its compute for whole HBM sweeps.
  const int tg = (tn.tm > 0 && tn.tm < t && tn.tm >= e1) ? tn.tm : t;
  const size_t merge_smem = size_t(elem_bytes(kk, has_vals)) * smem_words(1u << tg);
  for (int p = t + 1; p <= m; ++p) {
    // window passes over layer bits tg .. p-1, highest bits first.  A pass
    // covers up to w2 * e2 bits: one register window straight from HBM and
    // back, or (w2 = 2) two windows with one exchange through shared memory,
    // whose block holds 32 consecutive elements per window position so that
    // every warp access stays coalesced.
    // two-window passes hold 2^(c + 2*e2) elements in shared memory (no more
    // than a tile); the c low bits of a block are consecutive elements, at
    // least 8 of them so that every warp access fills whole 32-byte sectors
    const int c_sm = std::max(3, std::min(5, tg - 2 * e2));
    const bool two = tn.w2 >= 2 && (c_sm + 2 * e2 <= tg);
    const int w_max = two ? 2 * e2 : e2;
    int hi = p - 1;
    while (hi >= tg) {
      const int nbits = std::min(hi - tg + 1, w_max);
      const int lo = hi - nbits + 1;
      const int nr = (nbits + e2 - 1) / e2;
      Launch L{};
      L.kind = PASS_WINDOW;
      L.fixed = false;
      L.loge = e2;
      L.variant = pick_var(variant, tn, PASS_WINDOW);
      L.P.log2cap = uint32_t(m);
      if (nr == 1) {
        const int w0 = hi - e2 + 1;
        const int c = std::min(tn.c2, w0);
        L.threads = 1u << c;
        L.grid = uint32_t(1u << (m - c - e2));
        L.smem = 0;
        L.P.b = uint32_t(c + e2);
        L.P.c = uint32_t(c);
        L.P.w0 = uint32_t(w0);
        L.P.s = uint32_t(e2);
        Round r{};
        r.kind = RK_WINDOW;
        r.p = uint8_t(p);
        r.a = uint8_t(c);
        r.cnt = uint8_t(nbits);
        r.src = LOC_GLOBAL;
        r.dst = LOC_GLOBAL;
        r.lanediv = 0;  // bit p lies above the window: one direction per block
        set_rounds(L.P, std::vector<Round>{r});
        const KernelEntry w1e = window1_kernel(kk == KEY_U64, has_vals, e2, c);
        L.win1 = w1e.fn != nullptr && int(L.threads) == w1e.max_threads;
      } else {
        const int sbits = nr * e2;
        const int w0 = hi - sbits + 1;
        const int c = c_sm;
        const int b = c + sbits;
        L.threads = 1u << (b - e2);
        L.grid = uint32_t(1u << (m - b));
        L.smem = size_t(elem_bytes(kk, has_vals)) * smem_words(1u << b);
        L.P.b = uint32_t(b);
        L.P.c = uint32_t(c);
        L.P.w0 = uint32_t(w0);
        L.P.s = uint32_t(sbits);
        std::vector<Round> rs;
        int top = b - 1;                 // local bit of layer hi
        const int bottom = b - nbits;    // local bit of layer lo
        for (int i = 0; i < nr; ++i) {
          const int rhi = top - i * e2;
          const int rlo = std::max(rhi - e2 + 1, bottom);
          Round r{};
          r.kind = RK_WINDOW;
          r.p = uint8_t(p);
          r.a = uint8_t(rhi - e2 + 1);
          r.cnt = uint8_t(rhi - rlo + 1);
          r.src = (i == 0) ? LOC_GLOBAL : LOC_SMEM;
          r.dst = (i == nr - 1) ? LOC_GLOBAL : LOC_SMEM;
          r.lanediv = 0;
          rs.push_back(r);
        }
        set_rounds(L.P, rs);
        KernelEntry w2e = (kk == KEY_U32) ? window2_kernel_u32(has_vals, e2, c, L.variant)
                                          : window2_kernel_u64(has_vals, e2, c, L.variant);
        L.win2 = (nr == 2 && w2e.fn != nullptr && int(L.threads) == w2e.max_threads);
        // 32-bit keys, 16 consecutive elements per block, 32 keys (or 16
        // pairs) per thread: the TMA-streamed form where tensor maps are
        // available (tma mode 3)
        size_t w2t_smem = 0;
        const KernelEntry w2t = window2_tma_kernel_u32(has_vals, &w2t_smem);
        if (L.win2 && tn.tma >= 3 && g_tensor_maps != 0 && kk == KEY_U32 &&
            e2 == (has_vals ? 4 : 5) && c == 4 && rs[0].cnt == e2 && w2t.fn != nullptr &&
            int(L.threads) == w2t.max_threads && w2t_smem <= smem_limit) {
          int per_sm = 1;
          if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, w2t.fn, int(L.threads), w2t_smem) !=
                  cudaSuccess ||
              per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
          }
          L.win2 = false;
          L.win2t = true;
          L.smem = w2t_smem;
          L.P.nblocks = L.grid;
          L.grid = std::min<uint32_t>(L.grid, uint32_t(std::max(1, g_sms_for_plans) * per_sm));
        }
      }
      out.push_back(L);
      hi = lo - 1;
    }
    // merge pass: layers tg-1 .. 0 inside each tile
    Launch L{};
    L.kind = PASS_MERGE;
    // merge passes may run their own elements per thread (more, smaller
    // threads when the tile needs more resident warps)
    int em = e1;
    if (tn.em > 0 && tn.em <= 5 && tn.em <= tg && (1 << (tg - tn.em)) <= 1024 &&
        merge_round_count(tg, tn.em) <= kMaxRounds && has_fixed(kk, has_vals, tn.em, tg))
      em = tn.em;
    L.fixed = has_fixed(kk, has_vals, em, tg);
    L.loge = em;
    L.variant = pick_var(variant, tn, PASS_MERGE);
    L.grid = uint32_t(1u << (m - tg));
    L.threads = 1u << (tg - em);
    std::vector<Round> rs = merge_rounds(tg, em, p);
    mark_lanes(rs, em, tg, tg - em);
    L.smem = uses_smem(rs) ? merge_smem : 0;
    L.P.b = uint32_t(tg);
    L.P.c = uint32_t(tg);
    L.P.w0 = uint32_t(tg);
    L.P.s = 0;
    L.P.log2cap = uint32_t(m);
    L.P.map_in = 0;
    L.P.map_out = (p == m) ? map_out : 0u;
    set_rounds(L.P, rs);
    // single arrays: the persistent merge that streams the next tile in with
    // bulk copies while the current one is processed (one CTA per SM)
    size_t tma_smem = 0;
    int tma = tn.tma;
    if (tma == 4 && (g_tensor_maps == 0 ||
                     tma_merge_kernel_u32(has_vals, em, tg, 4, L.variant, &tma_smem).fn == nullptr ||
                     tma_smem > smem_limit))
      tma = 3;  // no two-buffer in-place kernel for this shape
    if (tma == 3 && (g_tensor_maps == 0 ||
                     tma_merge_kernel_u32(has_vals, em, tg, 3, L.variant, &tma_smem).fn == nullptr ||
                     tma_smem > smem_limit))
      tma = 2;  // no swizzled kernel for this shape (or no tensor maps)
    if (kk == KEY_U32 && tma &&
        tma_merge_kernel_u32(has_vals, em, tg, tma, L.variant, &tma_smem).fn != nullptr &&
        tma_smem <= smem_limit) {
      L.tma = tma;
      L.smem = tma_smem;
      if ((tn.shfl & 2) != 0 && !has_vals &&
          tma_merge_shfl_kernel_u32(em, tg, tma, L.variant, nullptr).fn != nullptr) {
        // two rounds: the top window from the staging buffer, then the lane
        // layers by shuffles and the register layers
        L.mshfl = true;
        std::vector<Round> two;
        Round r0{};
        r0.kind = RK_WINDOW;
        r0.p = uint8_t(p);
        r0.a = uint8_t(tg - em);
        r0.cnt = uint8_t(em);
        r0.src = LOC_GLOBAL;
        r0.dst = LOC_SMEM;
        Round r1{};
        r1.kind = RK_WINDOW;
        r1.p = uint8_t(p);
        r1.a = 0;
        r1.cnt = uint8_t(tg - em);  // lane layers tg-em-1 .. em, then em register layers
        r1.src = LOC_SMEM;
        r1.dst = LOC_GLOBAL;
        two.push_back(r0);
        two.push_back(r1);
        set_rounds(L.P, two);
      }
      L.P.nblocks = L.grid;
      int per_sm = 1;
      const void* tfn = tma_merge_kernel_u32(has_vals, em, tg, tma, L.variant, nullptr).fn;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tfn, int(L.threads), L.smem) !=
              cudaSuccess ||
          per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      L.grid = std::min<uint32_t>(L.grid, uint32_t(std::max(1, g_sms_for_plans) * per_sm));
    }
    out.push_back(L);
  }
  return true;
}

std::string describe(const std::vector<Launch>& plan) {
  std::ostringstream os;
  static const char* names[] = {"tile", "window", "merge"};
  for (const Launch& L : plan) {
    os << names[L.kind] << (L.fixed ? "*" : "") << (L.shfl ? "~" : "") << (L.win2t || L.tma >= 3 ? "^" : "") << " E=" << (1 << L.loge) << " var=" << L.variant << " grid=" << L.grid
       << " threads=" << L.threads << " smem=" << L.smem << " b=" << L.P.b << " c=" << L.P.c
       << " w0=" << L.P.w0 << " rounds=" << L.P.nrounds << "\n";
  }
  return os.str();
}

}  // namespace darm
