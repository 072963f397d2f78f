// tune.cu - autotuner: picks the tile size, elements per thread, window
// depth and the divergent or melded form of every pass kind by timing them.
//
// The paper treats the thread-block size as a tunable that the programmer
// picks per input (Section VI-A, "Block Size"), and notes that the block
// size best for the unmelded kernel was also best after melding.  Here the
// choice is measured: candidate (T, E) plans run on a scratch array of the
// requested size; then, for the fastest plan, each pass kind keeps whichever
// form (divergent or melded) has the lower total device time.
#include <cuda_runtime.h>

#include <cstdio>
#include <vector>

#include "darm.h"
#include "darm_internal.h"
#include "kernel_table.h"

namespace darm {
namespace {

__global__ void fill_hash_kernel(uint32_t* p, size_t words, uint32_t seed) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < words;
       i += size_t(gridDim.x) * blockDim.x) {
    uint32_t x = uint32_t(i) * 0x9E3779B1u ^ seed;
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    p[i] = x;
  }
}

// Device time of one sort with `plan`, per pass kind (ms); best of `reps`.
bool time_plan(const std::vector<Launch>& plan, KeyKind kk, void* keys, uint32_t* vals,
               size_t key_words, cudaStream_t s, int reps, float per_kind[3], float* total) {
  std::vector<cudaEvent_t> ev(plan.size() + 1);
  for (auto& e : ev) cudaEventCreate(&e);
  float best = 1e30f;
  float best_kind[3] = {0, 0, 0};
  bool ok = true;
  for (int r = 0; r < reps && ok; ++r) {
    fill_hash_kernel<<<1024, 256, 0, s>>>(static_cast<uint32_t*>(keys), key_words, 1234u + r);
    cudaEventRecord(ev[0], s);
    for (size_t i = 0; i < plan.size(); ++i) {
      std::vector<Launch> one(1, plan[i]);
      if (launch_plan(one, kk, keys, vals, s, false) != DARM_OK) ok = false;
      cudaEventRecord(ev[i + 1], s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) ok = false;
    float tot = 0, kind[3] = {0, 0, 0};
    for (size_t i = 0; i < plan.size() && ok; ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      kind[plan[i].kind] += ms;
      tot += ms;
    }
    if (tot < best) {
      best = tot;
      for (int k = 0; k < 3; ++k) best_kind[k] = kind[k];
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  *total = best;
  for (int k = 0; k < 3; ++k) per_kind[k] = best_kind[k];
  return ok;
}

}  // namespace
}  // namespace darm

using namespace darm;

extern "C" {

int darm_autotune(int dtype, size_t n, int has_vals, const char* db_path) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (dtype < DARM_U32 || dtype > DARM_U64) return DARM_ERR_INVALID_ARG;
  if (n < 2 || (n & (n - 1)) != 0 || n > (size_t(1) << 30)) return DARM_ERR_NOT_POW2;
  const KeyKind kk = dtype == DARM_U64 ? KEY_U64 : KEY_U32;
  const bool hv = has_vals != 0;
  int m = 0;
  while ((size_t(1) << m) < n) ++m;
  const size_t kbytes = n * (kk == KEY_U64 ? 8 : 4);
  void* keys = nullptr;
  uint32_t* vals = nullptr;
  if (cudaMalloc(&keys, kbytes) != cudaSuccess) return DARM_ERR_OOM;
  if (hv && cudaMalloc(&vals, n * 4) != cudaSuccess) {
    cudaFree(keys);
    return DARM_ERR_OOM;
  }
  cudaStream_t s;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  const Tuning base = default_tuning(kk, hv);
  Tuning best = base;
  float best_ms = 1e30f;
  const int t_cand[] = {base.t - 1, base.t, base.t + 1};
  const int e2_cand[] = {3, 4, 5};
  for (int t : t_cand)
    for (int e1 = base.e1 - 1; e1 <= base.e1; ++e1)
      for (int e2 : e2_cand)
        for (int w2 = 1; w2 <= 2; ++w2)
          for (int tma = 0; tma <= 4; ++tma) {
            Tuning tn = base;
            tn.tma = tma;
            tn.tm = 0;  // one tile size here; a smaller merge tile is tried below
            tn.t = t;
            tn.e1 = e1;
            tn.e2 = e2;
            tn.w2 = w2;
            tn.var[0] = tn.var[1] = tn.var[2] = kMelded;
            std::vector<Launch> plan;
            if (!plan_array(plan, kk, hv, m, tn, DARM_AUTO, 0, 0, g_ctx.smem_limit)) continue;
            float kind[3], tot;
            if (!time_plan(plan, kk, keys, vals, kbytes / 4, s, 3, kind, &tot)) continue;
            if (tot < best_ms) {
              best_ms = tot;
              best = tn;
            }
          }
  // shuffle stages: without them in the tile pass (0), and with the merge
  // passes in two rounds as well (3), where built for the chosen shape
  for (int shfl : {0, 3}) {
    if (shfl == best.shfl) continue;
    Tuning tn = best;
    tn.shfl = shfl;
    std::vector<Launch> plan;
    float kind[3], tot;
    if (plan_array(plan, kk, hv, m, tn, DARM_AUTO, 0, 0, g_ctx.smem_limit) &&
        time_plan(plan, kk, keys, vals, kbytes / 4, s, 3, kind, &tot) && tot < best_ms) {
      best_ms = tot;
      best = tn;
    }
  }
  // merge passes on tiles half the tile pass's (the window passes take the
  // bit between): two sweeps fewer for a longer tile pass
  if (best.t - 1 >= best.e1) {
    Tuning tn = best;
    tn.tm = best.t - 1;
    std::vector<Launch> plan;
    float kind[3], tot;
    if (plan_array(plan, kk, hv, m, tn, DARM_AUTO, 0, 0, g_ctx.smem_limit) &&
        time_plan(plan, kk, keys, vals, kbytes / 4, s, 3, kind, &tot) && tot < best_ms) {
      best_ms = tot;
      best = tn;
    }
  }
  // per pass kind: divergent or melded
  float kind_of[2][3];
  for (int v = 0; v < 2; ++v) {
    Tuning tn = best;
    tn.var[0] = tn.var[1] = tn.var[2] = v;
    std::vector<Launch> plan;
    float tot;
    plan_array(plan, kk, hv, m, tn, DARM_AUTO, 0, 0, g_ctx.smem_limit);
    time_plan(plan, kk, keys, vals, kbytes / 4, s, 3, kind_of[v], &tot);
  }
  for (int k = 0; k < 3; ++k) best.var[k] = (kind_of[kDivergent][k] < kind_of[kMelded][k]) ? kDivergent : kMelded;
  {
    std::lock_guard<std::mutex> lk(g_ctx.mu);
    g_ctx.tuned[std::make_tuple(int(kk), int(hv), m)] = best;
    g_ctx.plans.clear();
  }
  cudaStreamDestroy(s);
  cudaFree(keys);
  if (vals) cudaFree(vals);
  if (cudaGetLastError() != cudaSuccess) return DARM_ERR_CUDA;
  if (db_path) {
    FILE* f = fopen(db_path, "a");
    if (!f) return DARM_ERR_INVALID_ARG;
    fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %.6f %d %d %d\n", int(kk), int(hv), m, best.t,
            best.e1, best.e2, best.c2, best.w2, best.tma, best.var[0], best.var[1], best.var[2],
            double(best_ms), best.shfl, best.em, best.tm);
    fclose(f);
  }
  return DARM_OK;
}

int darm_reset_tunings(void) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  std::lock_guard<std::mutex> lk(g_ctx.mu);
  g_ctx.tuned.clear();
  g_ctx.plans.clear();
  return DARM_OK;
}

int darm_load_tune_db(const char* db_path) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (!db_path) return DARM_ERR_INVALID_ARG;
  FILE* f = fopen(db_path, "r");
  if (!f) return DARM_ERR_NOT_FOUND;
  int kk, hv, m;
  double ms;
  int loaded = 0;
  char line[512];
  std::lock_guard<std::mutex> lk(g_ctx.mu);
  // one tuning per line: 13 fields, then optionally shuffle stages, merge
  // elements per thread and merge tile
  while (fgets(line, sizeof line, f)) {
    Tuning tn;
    const int got = sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d %d %lf %d %d %d", &kk, &hv, &m,
                           &tn.t, &tn.e1, &tn.e2, &tn.c2, &tn.w2, &tn.tma, &tn.var[0], &tn.var[1],
                           &tn.var[2], &ms, &tn.shfl, &tn.em, &tn.tm);
    if (got < 13) continue;
    if (got < 14) tn.shfl = 0;
    if (got < 15) tn.em = 0;
    if (got < 16) tn.tm = 0;
    if (kk < 0 || kk > 1 || m < 0 || m > 31) continue;
    g_ctx.tuned[std::make_tuple(kk, hv, m)] = tn;  // m == 0: a batch tuning
    ++loaded;
  }
  fclose(f);
  g_ctx.plans.clear();  // batch graphs are keyed by their tuning
  return loaded ? DARM_OK : DARM_ERR_NOT_FOUND;
}

}  // extern "C"
