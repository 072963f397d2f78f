// meld_analysis.cu - melding profitability and instruction alignment of two
// divergent paths (host code; Section IV-C of the paper).
//
// An instruction is modelled as (opcode, type, latency): `opcode` is the
// instruction type the frequency profile counts (an IR opcode), `type`
// refines it for alignment (operand types, compare predicate): two
// instructions can be melded only when opcode and type both match.
//
//   MP_B(b1, b2) = sum over opcodes i of min(freq(i, b1), freq(i, b2)) * w_i
//                  / (lat(b1) + lat(b2))
// with w_i the latency of opcode i and lat(b) the sum of b's latencies: the
// share of instruction cycles melding could save.  Identical profiles give
// 0.5.
//   MP_S(S1, S2) = sum over corresponding blocks of MP_B * (lat(b1)+lat(b2))
//                  / sum of (lat(b1)+lat(b2)).
// Instruction alignment: Smith-Waterman local alignment; aligning two
// compatible instructions scores their latency, incompatible pairs cannot
// align, every unaligned instruction inside the aligned stretch costs `gap`.
//
// Subgraph alignment (Def. 7): the ordered SESE subgraphs of the true and
// false paths of a divergent region are aligned the same way, a pair scoring
// its melding profitability and allowed only when the two subgraphs are
// meldable (Def. 6); every unaligned subgraph inside the aligned stretch
// costs the gap penalty.  Algorithm 1 then melds an aligned pair when its
// profitability is at least the threshold (0.2 by default, Section V).
//   Def. 6 case 1 (both more than one block, isomorphic): MP_S over the
//   corresponding blocks (pre-order).  Case 3 (two single blocks): MP_B.
//   Case 2 (a simple region M and a single block A): region replication
//   copies M's structure around A, placing A beside the block E of M with
//   the highest MP_B(A, E) (the first in pre-order on ties); the copy's
//   other blocks are empty and share nothing, so its MP_S with M is
//   MP_B(A, E) * (lat(A) + lat(E)) / (lat(A) + lat(M)).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <vector>

#include "darm.h"

namespace {

// opcode -> latency, from every instruction of both blocks; false when one
// opcode is given two latencies
bool opcode_latencies(const darm_inst* a, int na, const darm_inst* b, int nb,
                      std::map<int32_t, int32_t>& w) {
  for (int s = 0; s < 2; ++s) {
    const darm_inst* p = s ? b : a;
    const int n = s ? nb : na;
    for (int i = 0; i < n; ++i) {
      auto it = w.find(p[i].opcode);
      if (it == w.end())
        w[p[i].opcode] = p[i].latency;
      else if (it->second != p[i].latency)
        return false;
    }
  }
  return true;
}

double mp_block(const darm_inst* b1, int n1, const darm_inst* b2, int n2, double* lat_sum) {
  std::map<int32_t, int32_t> w;
  if (!opcode_latencies(b1, n1, b2, n2, w)) return NAN;
  std::map<int32_t, int64_t> f1, f2;
  int64_t lat = 0;
  for (int i = 0; i < n1; ++i) {
    ++f1[b1[i].opcode];
    lat += b1[i].latency;
  }
  for (int i = 0; i < n2; ++i) {
    ++f2[b2[i].opcode];
    lat += b2[i].latency;
  }
  if (lat_sum) *lat_sum = double(lat);
  if (lat <= 0) return 0.0;
  int64_t common = 0;
  for (const auto& kv : f1) {
    auto it = f2.find(kv.first);
    if (it != f2.end()) common += std::min(kv.second, it->second) * int64_t(w[kv.first]);
  }
  return double(common) / double(lat);
}

// Melding profitability of two SESE subgraphs under Def. 6, or -1 when they
// are not meldable; NaN on inconsistent latencies.
double mp_sese(const darm_inst* insts, const int32_t* off, const darm_subgraph& s1,
               const darm_subgraph& s2) {
  auto blk = [&](const darm_subgraph& s, int k, const darm_inst** p, int* n) {
    const int b = s.first_block + k;
    *p = insts + off[b];
    *n = off[b + 1] - off[b];
  };
  if (s1.nblocks > 1 && s2.nblocks > 1) {
    if (s1.nblocks != s2.nblocks || s1.shape != s2.shape) return -1.0;  // not isomorphic
    double num = 0.0, den = 0.0;
    for (int k = 0; k < s1.nblocks; ++k) {
      const darm_inst *a, *b;
      int na, nb;
      blk(s1, k, &a, &na);
      blk(s2, k, &b, &nb);
      double lat = 0.0;
      const double mp = mp_block(a, na, b, nb, &lat);
      if (std::isnan(mp)) return NAN;
      num += mp * lat;
      den += lat;
    }
    return den > 0.0 ? num / den : 0.0;
  }
  if (s1.nblocks == 1 && s2.nblocks == 1) {
    const darm_inst *a, *b;
    int na, nb;
    blk(s1, 0, &a, &na);
    blk(s2, 0, &b, &nb);
    return mp_block(a, na, b, nb, nullptr);
  }
  // one single block against a region: only a simple region can be replicated
  const darm_subgraph& one = (s1.nblocks == 1) ? s1 : s2;
  const darm_subgraph& reg = (s1.nblocks == 1) ? s2 : s1;
  if (!reg.simple_region) return -1.0;
  const darm_inst* a;
  int na;
  blk(one, 0, &a, &na);
  double lat_a = 0.0;
  for (int i = 0; i < na; ++i) lat_a += a[i].latency;
  double lat_m = 0.0, best = -1.0, best_pair_lat = 0.0;
  for (int k = 0; k < reg.nblocks; ++k) {
    const darm_inst* b;
    int nb;
    blk(reg, k, &b, &nb);
    double lat = 0.0;
    const double mp = mp_block(a, na, b, nb, &lat);
    if (std::isnan(mp)) return NAN;
    lat_m += lat - lat_a;
    if (mp > best) {
      best = mp;
      best_pair_lat = lat;
    }
  }
  const double den = lat_a + lat_m;
  return den > 0.0 ? best * best_pair_lat / den : 0.0;
}

bool valid_subgraphs(const darm_subgraph* s, int n, int nblocks_total) {
  for (int i = 0; i < n; ++i)
    if (s[i].nblocks < 1 || s[i].first_block < 0 || s[i].first_block + s[i].nblocks > nblocks_total)
      return false;
  return true;
}

}  // namespace

extern "C" {

double darm_meld_mp_sese(const darm_inst* insts, const int32_t* block_off, int nblocks_total,
                         const darm_subgraph* s1, const darm_subgraph* s2) {
  if (!block_off || nblocks_total < 1 || !s1 || !s2) return NAN;
  for (int b = 0; b < nblocks_total; ++b)
    if (block_off[b + 1] < block_off[b] || block_off[b] < 0) return NAN;
  if (block_off[nblocks_total] > 0 && !insts) return NAN;
  if (!valid_subgraphs(s1, 1, nblocks_total) || !valid_subgraphs(s2, 1, nblocks_total)) return NAN;
  return mp_sese(insts, block_off, *s1, *s2);
}

int darm_meld_subgraph_align(const darm_inst* insts, const int32_t* block_off, int nblocks_total,
                             const darm_subgraph* st, int m, const darm_subgraph* sf, int n,
                             double gap, double threshold, int32_t* pairs, double* profit,
                             int32_t* meld, double* score) {
  if (m < 0 || n < 0 || gap < 0.0 || !(threshold >= 0.0) || !block_off || nblocks_total < 0)
    return -1;
  if ((m && !st) || (n && !sf) || (std::min(m, n) > 0 && (!pairs || !profit || !meld))) return -1;
  for (int b = 0; b < nblocks_total; ++b)
    if (block_off[b + 1] < block_off[b] || block_off[b] < 0) return -1;
  if (block_off[nblocks_total] > 0 && !insts) return -1;
  if (!valid_subgraphs(st, m, nblocks_total) || !valid_subgraphs(sf, n, nblocks_total)) return -1;
  // profitability of every pair (-1: not meldable)
  std::vector<double> F(size_t(m) * size_t(n), -1.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) {
      const double f = mp_sese(insts, block_off, st[i], sf[j]);
      if (std::isnan(f)) return -1;
      F[size_t(i) * n + j] = f;
    }
  const int W = n + 1;
  std::vector<double> H(size_t(m + 1) * W, 0.0);
  std::vector<uint8_t> from(size_t(m + 1) * W, 0);  // 0 stop, 1 diag, 2 up, 3 left
  double best = 0.0;
  int bi = 0, bj = 0;
  for (int i = 1; i <= m; ++i)
    for (int j = 1; j <= n; ++j) {
      double h = 0.0;
      uint8_t f = 0;
      const double fij = F[size_t(i - 1) * n + (j - 1)];
      if (fij >= 0.0) {
        const double d = H[size_t(i - 1) * W + (j - 1)] + fij;
        if (d > h) { h = d; f = 1; }
      }
      const double u = H[size_t(i - 1) * W + j] - gap;
      if (u > h) { h = u; f = 2; }
      const double l = H[size_t(i) * W + (j - 1)] - gap;
      if (l > h) { h = l; f = 3; }
      H[size_t(i) * W + j] = h;
      from[size_t(i) * W + j] = f;
      if (h > best) { best = h; bi = i; bj = j; }
    }
  std::vector<std::pair<int, int>> al;
  int i = bi, j = bj;
  while (i > 0 && j > 0 && from[size_t(i) * W + j] != 0) {
    const uint8_t f = from[size_t(i) * W + j];
    if (f == 1) {
      al.emplace_back(i - 1, j - 1);
      --i;
      --j;
    } else if (f == 2) {
      --i;
    } else {
      --j;
    }
  }
  std::reverse(al.begin(), al.end());
  for (size_t k = 0; k < al.size(); ++k) {
    pairs[2 * k] = al[k].first;
    pairs[2 * k + 1] = al[k].second;
    profit[k] = F[size_t(al[k].first) * n + al[k].second];
    meld[k] = profit[k] >= threshold ? 1 : 0;  // Algorithm 1: profit >= threshold
  }
  if (score) *score = best;
  return int(al.size());
}

double darm_meld_mp_block(const darm_inst* b1, int n1, const darm_inst* b2, int n2) {
  if (n1 < 0 || n2 < 0 || (n1 && !b1) || (n2 && !b2)) return NAN;
  return mp_block(b1, n1, b2, n2, nullptr);
}

double darm_meld_mp_subgraph(const darm_inst* i1, const int32_t* off1, const darm_inst* i2,
                             const int32_t* off2, int nb) {
  if (nb <= 0 || !off1 || !off2) return NAN;
  double num = 0.0, den = 0.0;
  for (int k = 0; k < nb; ++k) {
    const int a0 = off1[k], a1 = off1[k + 1], b0 = off2[k], b1 = off2[k + 1];
    if (a1 < a0 || b1 < b0) return NAN;
    double lat = 0.0;
    const double mp = mp_block(i1 + a0, a1 - a0, i2 + b0, b1 - b0, &lat);
    if (std::isnan(mp)) return NAN;
    num += mp * lat;
    den += lat;
  }
  return den > 0.0 ? num / den : 0.0;
}

int darm_meld_align(const darm_inst* a, int na, const darm_inst* b, int nb, double gap,
                    int32_t* pairs, double* score) {
  if (na < 0 || nb < 0 || gap < 0.0 || !pairs) return -1;
  const int W = nb + 1;
  std::vector<double> H(size_t(na + 1) * W, 0.0);
  std::vector<uint8_t> from(size_t(na + 1) * W, 0);  // 0 stop, 1 diag, 2 up, 3 left
  double best = 0.0;
  int bi = 0, bj = 0;
  for (int i = 1; i <= na; ++i)
    for (int j = 1; j <= nb; ++j) {
      double h = 0.0;
      uint8_t f = 0;
      const bool compat = a[i - 1].opcode == b[j - 1].opcode && a[i - 1].type == b[j - 1].type;
      if (compat) {
        const double d = H[size_t(i - 1) * W + (j - 1)] + double(a[i - 1].latency);
        if (d > h) { h = d; f = 1; }
      }
      const double u = H[size_t(i - 1) * W + j] - gap;
      if (u > h) { h = u; f = 2; }
      const double l = H[size_t(i) * W + (j - 1)] - gap;
      if (l > h) { h = l; f = 3; }
      H[size_t(i) * W + j] = h;
      from[size_t(i) * W + j] = f;
      if (h > best) { best = h; bi = i; bj = j; }
    }
  // aligned pairs of the best local alignment, collected backwards
  std::vector<std::pair<int, int>> al;
  int i = bi, j = bj;
  while (i > 0 && j > 0 && from[size_t(i) * W + j] != 0) {
    const uint8_t f = from[size_t(i) * W + j];
    if (f == 1) {
      al.emplace_back(i - 1, j - 1);
      --i;
      --j;
    } else if (f == 2) {
      --i;
    } else {
      --j;
    }
  }
  std::reverse(al.begin(), al.end());
  // both sequences in program order: aligned pairs, unaligned ones between
  int n = 0, x = 0, y = 0;
  for (const auto& p : al) {
    for (; x < p.first; ++x, ++n) { pairs[2 * n] = x; pairs[2 * n + 1] = -1; }
    for (; y < p.second; ++y, ++n) { pairs[2 * n] = -1; pairs[2 * n + 1] = y; }
    pairs[2 * n] = p.first;
    pairs[2 * n + 1] = p.second;
    ++n;
    ++x;
    ++y;
  }
  for (; x < na; ++x, ++n) { pairs[2 * n] = x; pairs[2 * n + 1] = -1; }
  for (; y < nb; ++y, ++n) { pairs[2 * n] = -1; pairs[2 * n + 1] = y; }
  if (score) *score = best;
  return n;
}

}  // extern "C"
