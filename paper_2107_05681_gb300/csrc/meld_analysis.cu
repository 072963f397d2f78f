// meld_analysis.cu - melding profitability and instruction alignment of two
// divergent paths (host code; Section IV-E of the paper).
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

}  // namespace

extern "C" {

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
