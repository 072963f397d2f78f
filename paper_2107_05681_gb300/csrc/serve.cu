// serve.cu - continuous-batching sort service.
//
// A scheduler thread owns a device arena of the configured budget and runs
// "ticks".  Each tick advances every admitted job by one phase of its network
// (tile pass, or one stage 2^p > T: window passes + merge pass) with batched
// launches: all jobs in the same phase share one block table and one launch
// per pass kind, whatever their sizes (batch.h).  Requests that arrive while
// others are on the GPU are admitted at the next tick as soon as a slot and
// arena space are free, so their work overlaps with the jobs already running.
//
// Memory.  A job of n keys occupies cap = next power of two of n elements in
// the arena: 8 bytes of key space (uint64; uint32/float keys are widened on
// the way in and narrowed on the way out) and 4 bytes of payload space, so a
// job's budget cost is 12 * cap bytes.  Element ranges come from a buddy
// allocator; the keys and payload arenas use the same element index.
//
// Pacing.  A stream has at most two ticks in flight; the scheduler polls
// completion events and never blocks the device.  Latency is the host time
// from submit to the moment the scheduler sees the job's completion event.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "batch.h"
#include "darm.h"
#include "darm_internal.h"

namespace darm {
namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

// uint32 / float keys -> uint64 arena keys (float through the totalOrder
// map).  The +1 keeps every widened key strictly between the two sentinels
// (0 and UINT64_MAX), so padding never ties with a real key.
__global__ void widen_keys_kernel(uint64_t* dst, const uint32_t* src, size_t n, int is_f32) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t u = src[i];
  if (is_f32) u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  dst[i] = uint64_t(u) + 1u;
}

__global__ void narrow_keys_kernel(uint32_t* dst, const uint64_t* src, size_t n, int is_f32) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t u = uint32_t(src[i] - 1u);
  if (is_f32) u = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
  dst[i] = u;
}

// Buddy allocator over [0, total) elements in power-of-two blocks.
class Buddy {
 public:
  void init(uint64_t total) {
    free_.assign(64, {});
    uint64_t off = 0;
    for (int o = 63; o >= 0; --o) {
      const uint64_t sz = uint64_t(1) << o;
      if (total & sz) {
        free_[o].insert(off);
        off += sz;
      }
    }
    used_ = 0;
  }
  bool alloc(int order, uint64_t* off) {
    int o = order;
    while (o < 64 && free_[o].empty()) ++o;
    if (o >= 64) return false;
    uint64_t b = *free_[o].begin();
    free_[o].erase(free_[o].begin());
    while (o > order) {  // split, keep the lower half
      --o;
      free_[o].insert(b + (uint64_t(1) << o));
    }
    *off = b;
    used_ += uint64_t(1) << order;
    return true;
  }
  void release(uint64_t off, int order) {
    used_ -= uint64_t(1) << order;
    int o = order;
    uint64_t b = off;
    while (o < 63) {
      const uint64_t buddy = b ^ (uint64_t(1) << o);
      auto it = free_[o].find(buddy);
      if (it == free_[o].end()) break;
      free_[o].erase(it);
      b = std::min(b, buddy);
      ++o;
    }
    free_[o].insert(b);
  }

 private:
  std::vector<std::set<uint64_t>> free_;
  uint64_t used_ = 0;
};

struct Job {
  uint64_t id = 0;
  void* ukeys = nullptr;
  uint32_t* uvals = nullptr;
  size_t n = 0;
  int dtype = DARM_U64;
  bool desc = false;
  int c = 0;             // log2 capacity
  uint64_t off = 0;      // arena element offset
  int phase = -1;        // next phase to issue: 0 tile pass, p > t stage 2^p
  bool last_issued = false;
  bool finished = false;
  int status = DARM_OK;
  int stream = 0;
  cudaEvent_t ev = nullptr;
  double t_submit = 0, t_done = 0;
};

struct StreamState {
  cudaStream_t s = nullptr;
  // tick ring: tables uploaded for a tick stay alive until its event fires
  struct Slot {
    cudaEvent_t ev = nullptr;
    bool busy = false;
    SegSlot* d_slots = nullptr;
    SegBlock* d_blocks = nullptr;
    unsigned int* d_counters = nullptr;
    size_t cap_slots = 0, cap_blocks = 0, cap_counters = 0;
  };
  Slot ring[3];
  int next = 0;
};

struct Server {
  darm_serve_cfg cfg{};
  uint64_t* d_keys = nullptr;
  uint32_t* d_vals = nullptr;
  uint64_t elems = 0;
  Buddy buddy;
  std::vector<StreamState> streams;
  std::thread thread;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> queue;
  std::vector<std::shared_ptr<Job>> active;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  uint64_t next_id = 1;
  bool stopping = false;
  int inject = DARM_OK;  // fault injected into the next tick's launches
  std::vector<double> lat_ms;
  double keys_done = 0, t_first = 0, t_last = 0;
  int rr = 0;
};

std::mutex g_srv_mu;  // guards g_srv itself (start/stop)
std::unique_ptr<Server> g_srv;

int log2_ceil(uint64_t v) {
  int m = 0;
  while ((uint64_t(1) << m) < v) ++m;
  return m;
}

void finish_job(Server& S, Job& j, int status) {
  j.finished = true;
  j.status = status;
  j.t_done = now_s();
  if (j.c >= 0 && j.phase != -2) S.buddy.release(j.off, j.c);
  j.phase = -2;
  if (status == DARM_OK) {
    S.lat_ms.push_back((j.t_done - j.t_submit) * 1e3);
    S.keys_done += double(j.n);
    if (S.t_first == 0 || j.t_submit < S.t_first) S.t_first = j.t_submit;
    S.t_last = std::max(S.t_last, j.t_done);
  }
  if (j.ev) {
    cudaEventDestroy(j.ev);
    j.ev = nullptr;
  }
}

// Upload a tick's tables into a ring slot (growing it if needed) and launch.
int run_tick(Server& S, StreamState& st, BatchTables& bt) {
  if (bt.launches.empty()) return DARM_OK;
  StreamState::Slot& slot = st.ring[st.next];
  st.next = (st.next + 1) % 3;
  if (slot.busy) {
    cudaEventSynchronize(slot.ev);  // only reached when three ticks are queued
    slot.busy = false;
  }
  auto grow = [](auto*& p, size_t& cap, size_t need) {
    if (need <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t n = std::max<size_t>(need, 1024);
    const cudaError_t e = cudaMalloc(&p, n * sizeof(*p));
    if (e == cudaSuccess) cap = n;
    return e;
  };
  if (grow(slot.d_slots, slot.cap_slots, bt.slots.size()) != cudaSuccess ||
      grow(slot.d_blocks, slot.cap_blocks, bt.blocks.size()) != cudaSuccess ||
      grow(slot.d_counters, slot.cap_counters, std::max<size_t>(1, bt.persistent.size())) !=
          cudaSuccess)
    return DARM_ERR_OOM;
  cudaMemcpyAsync(slot.d_slots, bt.slots.data(), bt.slots.size() * sizeof(SegSlot),
                  cudaMemcpyHostToDevice, st.s);
  cudaMemcpyAsync(slot.d_blocks, bt.blocks.data(), bt.blocks.size() * sizeof(SegBlock),
                  cudaMemcpyHostToDevice, st.s);
  cudaMemsetAsync(slot.d_counters, 0, std::max<size_t>(1, bt.persistent.size()) * sizeof(unsigned),
                  st.s);
  batch_bind(bt, slot.d_blocks, slot.d_slots, slot.d_counters);
  int rc = S.inject;
  if (rc == DARM_OK) rc = launch_plan(bt.launches, KEY_U64, S.d_keys, S.d_vals, st.s);
  S.inject = DARM_OK;
  cudaEventRecord(slot.ev, st.s);
  slot.busy = true;
  return rc;
}

void copy_in(Server& S, Job& j, cudaStream_t s) {
  uint64_t* dk = S.d_keys + j.off;
  if (j.dtype == DARM_U64) {
    cudaMemcpyAsync(dk, j.ukeys, j.n * 8, cudaMemcpyDeviceToDevice, s);
  } else {
    widen_keys_kernel<<<unsigned((j.n + 255) / 256), 256, 0, s>>>(
        dk, static_cast<const uint32_t*>(j.ukeys), j.n, j.dtype == DARM_F32);
  }
  if (j.uvals) cudaMemcpyAsync(S.d_vals + j.off, j.uvals, j.n * 4, cudaMemcpyDeviceToDevice, s);
}

void copy_out(Server& S, Job& j, cudaStream_t s) {
  const uint64_t* dk = S.d_keys + j.off;
  if (j.dtype == DARM_U64) {
    cudaMemcpyAsync(j.ukeys, dk, j.n * 8, cudaMemcpyDeviceToDevice, s);
  } else {
    narrow_keys_kernel<<<unsigned((j.n + 255) / 256), 256, 0, s>>>(
        static_cast<uint32_t*>(j.ukeys), dk, j.n, j.dtype == DARM_F32);
  }
  if (j.uvals) cudaMemcpyAsync(j.uvals, S.d_vals + j.off, j.n * 4, cudaMemcpyDeviceToDevice, s);
}

void scheduler(Server* Sp) {
  Server& S = *Sp;
  if (cudaSetDevice(g_ctx.device) != cudaSuccess) return;
  const Tuning tn = batch_tuning(KEY_U64, true, 31);
  const int t = tn.t;
  std::unique_lock<std::mutex> lk(S.mu);
  for (;;) {
    // 1. retire jobs whose copy-out has completed
    bool any_done = false;
    for (auto& jp : S.active) {
      Job& j = *jp;
      if (j.last_issued && !j.finished && cudaEventQuery(j.ev) == cudaSuccess) {
        finish_job(S, j, DARM_OK);
        any_done = true;
      }
    }
    if (any_done) {
      S.active.erase(std::remove_if(S.active.begin(), S.active.end(),
                                    [](const std::shared_ptr<Job>& j) { return j->finished; }),
                     S.active.end());
      S.cv_done.notify_all();
    }
    // 2. admit queued jobs in arrival order while slots and arena space last
    for (auto it = S.queue.begin(); it != S.queue.end() &&
                                    int(S.active.size()) < S.cfg.max_inflight;) {
      Job& j = **it;
      uint64_t off = 0;
      if (S.buddy.alloc(j.c, &off)) {
        j.off = off;
        j.phase = 0;
        j.stream = S.rr;
        S.rr = (S.rr + 1) % int(S.streams.size());
        S.active.push_back(*it);
        it = S.queue.erase(it);
      } else {
        break;  // keep arrival order: the head waits for space
      }
    }
    if (S.stopping && S.queue.empty() && S.active.empty()) break;
    // 3. one tick per stream: every job not yet finishing advances one phase
    bool issued = false;
    for (size_t si = 0; si < S.streams.size(); ++si) {
      StreamState& st = S.streams[si];
      // pacing: at most two ticks of this stream in flight
      int inflight = 0;
      for (auto& sl : st.ring)
        if (sl.busy) {
          if (cudaEventQuery(sl.ev) == cudaSuccess)
            sl.busy = false;
          else
            ++inflight;
        }
      if (inflight >= 2) continue;
      std::vector<Job*> mine;
      for (auto& jp : S.active)
        if (jp->stream == int(si) && !jp->last_issued) mine.push_back(jp.get());
      if (mine.empty()) continue;
      BatchTables bt;
      std::vector<BatchSeg> tile_segs;
      std::map<int, std::vector<BatchSeg>> stage_segs;
      std::vector<Job*> finishing;
      for (Job* j : mine) {
        BatchSeg bs{j->off, uint32_t(j->n), j->c, j->desc};
        if (j->phase == 0) {
          copy_in(S, *j, st.s);
          if (j->c >= 1) tile_segs.push_back(bs);
          if (j->c <= t) finishing.push_back(j);
          j->phase = (j->c <= t) ? -1 : t + 1;
        } else if (j->phase > t) {
          stage_segs[j->phase].push_back(bs);
          if (j->phase == j->c) {
            finishing.push_back(j);
            j->phase = -1;
          } else {
            ++j->phase;
          }
        }
      }
      int rc = DARM_OK;
      if (!tile_segs.empty())
        rc = batch_append(bt, KEY_U64, true, tn, S.cfg.variant, tile_segs, 0, 0);
      for (auto& kv : stage_segs)
        if (rc == DARM_OK) rc = batch_append(bt, KEY_U64, true, tn, S.cfg.variant, kv.second, kv.first, 0);
      if (rc == DARM_OK) rc = run_tick(S, st, bt);
      for (Job* j : finishing) {
        if (rc != DARM_OK) {
          continue;
        }
        copy_out(S, *j, st.s);
        cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming);
        cudaEventRecord(j->ev, st.s);
        j->last_issued = true;
      }
      if (rc != DARM_OK) {
        // a failed tick fails every job it carried; their memory is released
        // once the stream has drained what was enqueued before the failure
        cudaStreamSynchronize(st.s);
        for (Job* j : mine) finish_job(S, *j, rc);
        S.active.erase(std::remove_if(S.active.begin(), S.active.end(),
                                      [](const std::shared_ptr<Job>& j) { return j->finished; }),
                       S.active.end());
        S.cv_done.notify_all();
      }
      issued = true;
    }
    if (!issued) {
      // nothing to launch: wait for an arrival or poll in-flight work
      if (S.active.empty() && S.queue.empty())
        S.cv_work.wait_for(lk, std::chrono::milliseconds(5));
      else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      }
    }
  }
}

}  // namespace
}  // namespace darm

using namespace darm;

extern "C" {

int darm_sort_serve_start(const darm_serve_cfg* cfg) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (!cfg || cfg->budget_bytes < 12 || cfg->max_inflight < 1 || cfg->num_streams < 1 ||
      cfg->variant < DARM_DIVERGENT || cfg->variant > DARM_AUTO)
    return DARM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_srv_mu);
  if (g_srv) return DARM_ERR_BUSY;
  auto S = std::make_unique<Server>();
  S->cfg = *cfg;
  S->elems = cfg->budget_bytes / 12;
  if (cudaMalloc(&S->d_keys, S->elems * 8) != cudaSuccess) return DARM_ERR_OOM;
  if (cudaMalloc(&S->d_vals, S->elems * 4) != cudaSuccess) {
    cudaFree(S->d_keys);
    return DARM_ERR_OOM;
  }
  S->buddy.init(S->elems);
  S->streams.resize(size_t(cfg->num_streams));
  for (auto& st : S->streams) {
    cudaStreamCreateWithFlags(&st.s, cudaStreamNonBlocking);
    for (auto& sl : st.ring) cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
  }
  if (cudaGetLastError() != cudaSuccess) return DARM_ERR_CUDA;
  S->thread = std::thread(scheduler, S.get());
  g_srv = std::move(S);
  return DARM_OK;
}

int darm_sort_serve_submit(void* keys, uint32_t* vals, size_t n, int dtype, int dir,
                           uint64_t* req_id) {
  if (dtype < DARM_U32 || dtype > DARM_U64 || (dir != DARM_ASC && dir != DARM_DESC) || !req_id)
    return DARM_ERR_INVALID_ARG;
  if (n > 0 && !keys) return DARM_ERR_INVALID_ARG;
  if (n > (size_t(1) << 31)) return DARM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_srv_mu);
  if (!g_srv) return DARM_ERR_NOT_INIT;
  Server& S = *g_srv;
  auto j = std::make_shared<Job>();
  j->ukeys = keys;
  j->uvals = vals;
  j->n = n;
  j->dtype = dtype;
  j->desc = dir == DARM_DESC;
  j->c = n <= 1 ? 0 : log2_ceil(n);
  j->t_submit = now_s();
  if ((uint64_t(1) << j->c) > S.elems) return DARM_ERR_BUDGET;
  std::lock_guard<std::mutex> lk(S.mu);
  if (S.stopping) return DARM_ERR_BUSY;
  j->id = S.next_id++;
  *req_id = j->id;
  S.jobs[j->id] = j;
  if (n <= 1) {
    // nothing to sort: done at once
    j->c = 0;
    j->phase = -2;
    j->finished = true;
    j->t_done = j->t_submit;
    S.lat_ms.push_back(0.0);
    S.keys_done += double(n);
    S.cv_done.notify_all();
    return DARM_OK;
  }
  S.queue.push_back(j);
  S.cv_work.notify_one();
  return DARM_OK;
}

int darm_sort_serve_poll(uint64_t req_id, int* done) {
  if (!done) return DARM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_srv_mu);
  if (!g_srv) return DARM_ERR_NOT_INIT;
  std::lock_guard<std::mutex> lk(g_srv->mu);
  auto it = g_srv->jobs.find(req_id);
  if (it == g_srv->jobs.end()) return DARM_ERR_NOT_FOUND;
  *done = it->second->finished ? 1 : 0;
  return it->second->finished ? it->second->status : DARM_OK;
}

int darm_sort_serve_wait(uint64_t req_id, int timeout_ms) {
  Server* S;
  {
    std::lock_guard<std::mutex> g(g_srv_mu);
    if (!g_srv) return DARM_ERR_NOT_INIT;
    S = g_srv.get();
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(req_id);
  if (it == S->jobs.end()) return DARM_ERR_NOT_FOUND;
  std::shared_ptr<Job> j = it->second;
  const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  while (!j->finished) {
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !j->finished)
      return DARM_ERR_TIMEOUT;
  }
  return j->status;
}

int darm_sort_serve_stats(double* p50_ms, double* p99_ms, double* keys_per_s, uint64_t* completed) {
  std::lock_guard<std::mutex> g(g_srv_mu);
  if (!g_srv) return DARM_ERR_NOT_INIT;
  std::lock_guard<std::mutex> lk(g_srv->mu);
  std::vector<double> v = g_srv->lat_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) {
    if (v.empty()) return 0.0;
    const size_t i = size_t(q * double(v.size() - 1) + 0.5);
    return v[std::min(i, v.size() - 1)];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  const double span = g_srv->t_last - g_srv->t_first;
  if (keys_per_s) *keys_per_s = span > 0 ? g_srv->keys_done / span : 0.0;
  if (completed) *completed = uint64_t(v.size());
  return DARM_OK;
}

int darm_sort_serve_inject_fault(int status) {
  std::lock_guard<std::mutex> g(g_srv_mu);
  if (!g_srv) return DARM_ERR_NOT_INIT;
  std::lock_guard<std::mutex> lk(g_srv->mu);
  g_srv->inject = status;
  return DARM_OK;
}

int darm_sort_serve_stop(void) {
  std::unique_ptr<Server> S;
  {
    std::lock_guard<std::mutex> g(g_srv_mu);
    if (!g_srv) return DARM_OK;
    {
      std::lock_guard<std::mutex> lk(g_srv->mu);
      g_srv->stopping = true;
      g_srv->cv_work.notify_all();
    }
    S = std::move(g_srv);
  }
  if (S->thread.joinable()) S->thread.join();
  cudaDeviceSynchronize();
  for (auto& st : S->streams) {
    for (auto& sl : st.ring) {
      if (sl.ev) cudaEventDestroy(sl.ev);
      if (sl.d_slots) cudaFree(sl.d_slots);
      if (sl.d_blocks) cudaFree(sl.d_blocks);
      if (sl.d_counters) cudaFree(sl.d_counters);
    }
    if (st.s) cudaStreamDestroy(st.s);
  }
  for (auto& kv : S->jobs)
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
  cudaFree(S->d_keys);
  cudaFree(S->d_vals);
  return DARM_OK;
}

}  // extern "C"
