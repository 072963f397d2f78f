// darm_api.cu - the C ABI (include/darm.h): context, whole-array sorts,
// host-buffer sorts, plan introspection and the launch path shared by the
// segmented sort and the serving loop.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "darm.h"
#include "darm_internal.h"
#include "kernel_table.h"
#include "plan.h"

namespace darm {

Context g_ctx;

const void* kernel_fn(KeyKind kk, bool has_vals, int loge, int variant) {
  KernelEntry e = (kk == KEY_U32) ? kernel_u32(has_vals, loge, variant)
                                  : kernel_u64(has_vals, loge, variant);
  return e.fn;
}

const void* fixed_kernel_fn(KeyKind kk, bool has_vals, int loge, int logt, int variant, bool merge) {
  KernelEntry e = (kk == KEY_U32) ? tile_kernel_u32(has_vals, loge, logt, variant, merge)
                                  : tile_kernel_u64(has_vals, loge, logt, variant, merge);
  return e.fn;
}

// The tile-pass blocks of batched segments that lie wholly beyond their
// segment's real length (a tile launch with no rounds; batch.cu).  Every
// key of such a block is the sentinel, so the tile's network moves nothing
// there and its result is the sentinel key (all ones in the sort's internal
// key order: the segment is longer than the tile, its later passes read
// keys unmapped) and payload 0xFFFFFFFF at each of the block's 2^b
// positions.  One CTA per table entry writes it in 16-byte stores (segment
// offsets are multiples of 4 elements).
template <typename K>
__global__ void darm_padding_tile_kernel(const __grid_constant__ PassParams P) {
  const SegBlock B = P.blocks[blockIdx.x];
  const uint64_t at = P.slots[B.first_slot].base + (uint64_t(B.blk_in_seg) << P.b);
  const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
  uint4* k4 = reinterpret_cast<uint4*>(static_cast<K*>(P.keys) + at);
  const uint32_t kvec = uint32_t((uint64_t(sizeof(K)) << P.b) / 16u);
  for (uint32_t i = threadIdx.x; i < kvec; i += blockDim.x) k4[i] = ones;
  if (P.vals != nullptr) {
    uint4* v4 = reinterpret_cast<uint4*>(P.vals + at);
    const uint32_t vvec = (1u << P.b) / 4u;
    for (uint32_t i = threadIdx.x; i < vvec; i += blockDim.x) v4[i] = ones;
  }
}

// Tensor map of `rows` rows of 32 uint32 keys (128 bytes) from `keys`,
// read and written in boxes of `box_rows` rows with the 128-byte swizzle
// (the swizzled in-place merge pass).
static bool encode_key_rows(CUtensorMap* tm, void* keys, uint64_t rows, uint32_t box_rows) {
  if (g_encode_tiled == nullptr) return false;
  auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(g_encode_tiled);
  const cuuint64_t dims[2] = {32, rows};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t box[2] = {32, box_rows};
  const cuuint32_t elem_strides[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, keys, dims, strides, box, elem_strides,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of a two-window pass over `nblocks` blocks of 16 x 2^(2e)
// uint32 elements from `base` (keys or payloads), window bits w0 ..
// w0+2e-1: dimensions (16 consecutive elements, the 2^(w0-4) positions
// between them and the windows, bottom window, top window, the blocks
// above), one box = one block.
static bool encode_window2_blocks(CUtensorMap* tm, void* base, uint32_t nblocks, uint32_t w0,
                                  int loge) {
  if (g_encode_tiled == nullptr || w0 < 4 || w0 + 2 * uint32_t(loge) + 2 > 40) return false;
  const uint32_t nmid = w0 - 4;
  if ((uint64_t(nblocks) & ((uint64_t(1) << nmid) - 1)) != 0) return false;
  auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(g_encode_tiled);
  const cuuint64_t win = cuuint64_t(1) << loge;
  const cuuint64_t dims[5] = {16, cuuint64_t(1) << nmid, win, win, cuuint64_t(nblocks) >> nmid};
  const cuuint64_t strides[4] = {64, cuuint64_t(4) << w0, cuuint64_t(4) << (w0 + loge),
                                 cuuint64_t(4) << (w0 + 2 * loge)};
  const cuuint32_t box[5] = {16, 1, cuuint32_t(win), cuuint32_t(win), 1};
  const cuuint32_t elem_strides[5] = {1, 1, 1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, base, dims, strides, box, elem_strides,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int launch_plan(const std::vector<Launch>& plan, KeyKind kk, void* keys, uint32_t* vals,
                cudaStream_t stream, bool count) {
  return launch_range(plan.data(), plan.data() + plan.size(), kk, keys, vals, stream, count);
}

int launch_range(const Launch* first, const Launch* last, KeyKind kk, void* keys, uint32_t* vals,
                 cudaStream_t stream, bool count) {
  const bool has_vals = vals != nullptr;
  for (const Launch* it = first; it != last; ++it) {
    const Launch& L = *it;
    PassParams P = L.P;
    P.keys = keys;
    P.vals = vals;
    P.status = g_ctx.d_status;
    const bool padding = (L.kind == PASS_TILE && L.P.nrounds == 0);
    const void* fn =
        padding ? ((kk == KEY_U32) ? reinterpret_cast<const void*>(&darm_padding_tile_kernel<uint32_t>)
                                   : reinterpret_cast<const void*>(&darm_padding_tile_kernel<uint64_t>))
        : L.win2t ? window2_tma_kernel_u32(has_vals, nullptr).fn
        : L.win1 ? window1_kernel(kk == KEY_U64, has_vals, L.loge, int(L.P.c)).fn
        : L.win2 ? ((kk == KEY_U32) ? window2_kernel_u32(has_vals, L.loge, int(L.P.c), L.variant)
                                  : window2_kernel_u64(has_vals, L.loge, int(L.P.c), L.variant)).fn
        : L.mshfl ? tma_merge_shfl_kernel_u32(L.loge, int(L.P.b), L.tma, L.variant, nullptr).fn
        : L.tma ? tma_merge_kernel_u32(has_vals, L.loge, int(L.P.b), L.tma, L.variant, nullptr).fn
        : L.shfl ? (L.P.blocks ? tile_shfl_seg_kernel_u32(has_vals, L.loge, int(L.P.b), L.variant)
                               : tile_shfl_kernel_u32(has_vals, L.loge, int(L.P.b), L.variant)).fn
        : L.fixed ? fixed_kernel_fn(kk, has_vals, L.loge, int(L.P.b), L.variant, L.kind == PASS_MERGE)
                  : kernel_fn(kk, has_vals, L.loge, L.variant);
    if (!fn) return DARM_ERR_INVALID_ARG;
    CUtensorMap tmap, tmap2;
    void* args[] = {&P, &tmap, &tmap2};
    if (L.win2t && (!encode_window2_blocks(&tmap, keys, L.P.nblocks, L.P.w0, L.loge) ||
                    (has_vals && !encode_window2_blocks(&tmap2, vals, L.P.nblocks, L.P.w0, L.loge)))) {
      fprintf(stderr, "darm: encoding the window pass's tensor map failed\n");
      return DARM_ERR_CUDA;
    }
    if (L.tma >= 3) {
      // the tiles this launch covers, as rows of 32 keys (and payloads)
      const int rows_log2 = int(L.P.b) - 5;
      const uint64_t rows = uint64_t(L.P.nblocks) << rows_log2;
      const uint32_t box = rows_log2 >= 8 ? 256u : (1u << rows_log2);
      if (!encode_key_rows(&tmap, keys, rows, box) ||
          (has_vals && !encode_key_rows(&tmap2, vals, rows, box))) {
        fprintf(stderr, "darm: encoding the merge pass's tensor map failed\n");
        return DARM_ERR_CUDA;
      }
    }
    cudaError_t err = cudaLaunchKernel(fn, dim3(L.grid), dim3(L.threads), args, L.smem, stream);
    if (err != cudaSuccess) {
      fprintf(stderr, "darm: launch failed: %s\n", cudaGetErrorString(err));
      return DARM_ERR_CUDA;
    }
    if (count) g_ctx.launches.fetch_add(1, std::memory_order_relaxed);
  }
  return DARM_OK;
}

static int log2_exact(size_t n) {
  int m = 0;
  while ((size_t(1) << m) < n) ++m;
  return m;
}

Tuning tuning_for(KeyKind kk, bool has_vals, int m) {
  std::lock_guard<std::mutex> lk(g_ctx.mu);
  auto it = g_ctx.tuned.find(std::make_tuple(int(kk), int(has_vals), m));
  if (it != g_ctx.tuned.end()) return it->second;
  Tuning tn = default_tuning(kk, has_vals);
  // a keys-only array of one small tile is sorted by one CTA whose time is
  // latency: 16 keys per thread (256 threads for 4096 keys) beat 32 (4096
  // uint32 keys: 31.1 -> 27.8 us melded, 36.7 -> 30.6 us divergent)
  if (kk == KEY_U32 && !has_vals && m <= 12) tn.e1 = 4;
  return tn;
}

const std::vector<Launch>* cached_plan(KeyKind kk, bool has_vals, int m, int variant,
                                       uint32_t map_in, uint32_t map_out) {
  const Tuning tn = tuning_for(kk, has_vals, m);
  PlanKey key{int(kk), int(has_vals), m, variant, map_in, map_out, tn.t, tn.e1, tn.e2, tn.c2,
              tn.w2 * 16 + tn.tma + tn.shfl * 256 + tn.em * 1024 + tn.tm * 8192,
              tn.var[0] * 4 + tn.var[1] * 2 + tn.var[2]};
  std::lock_guard<std::mutex> lk(g_ctx.mu);
  auto it = g_ctx.plans.find(key);
  if (it != g_ctx.plans.end()) return &it->second;
  std::vector<Launch> plan;
  if (!plan_array(plan, kk, has_vals, m, tn, variant, map_in, map_out, g_ctx.smem_limit))
    return nullptr;
  auto res = g_ctx.plans.emplace(key, std::move(plan));
  return &res.first->second;
}

int check_common(const void* keys, const void* vals, size_t n, int dir, int variant) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (dir != DARM_ASC && dir != DARM_DESC) return DARM_ERR_INVALID_ARG;
  if (variant < DARM_DIVERGENT || variant > DARM_AUTO) return DARM_ERR_INVALID_ARG;
  if (n <= 1) return DARM_OK;
  if ((n & (n - 1)) != 0) return DARM_ERR_NOT_POW2;
  if (n > (size_t(1) << 31)) return DARM_ERR_INVALID_ARG;
  if (keys == nullptr) return DARM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(keys) & 15u) != 0) return DARM_ERR_INVALID_ARG;
  if (vals != nullptr && (reinterpret_cast<uintptr_t>(vals) & 15u) != 0) return DARM_ERR_INVALID_ARG;
  return -1;  // proceed
}

// Whole arrays of 2^kSplitMinLog2 elements or more run split: every
// comparator of stages 2 .. 2^(m-1) stays inside one half of the array, so
// the two halves go through the tile pass and those stages at the same time,
// the first on the caller's stream and the second on the library's split
// stream (one half's launches fill the other's launch ramps and tails, and
// its HBM-bound passes can run beside the other's ALU-bound tile pass), and
// the final stage runs over the whole array once both are done.  Every comparator, with its direction, is the whole
// array's: the halves' passes take their directions from their index in the
// whole array (dir_base, log2cap = m).
constexpr int kSplitMinLog2 = 22;
constexpr int kSplitVariantTag = 0x100;  // plan-cache key of a split plan

// The split plan, cached beside the whole-array plans: for each half h its
// tile pass and stages 2^(t+1) .. 2^(m-1) (entries [h * per, (h + 1) * per)),
// then the final stage's launches.  Returns nullptr where the array does
// not split (a plan the split does not fit).
const std::vector<Launch>* cached_split_plan(KeyKind kk, bool hv, int m, int variant, uint32_t map,
                                             size_t* per) {
  const Tuning tn = tuning_for(kk, hv, m);
  const std::vector<Launch>* full = cached_plan(kk, hv, m, variant, map, map);
  if (!full || full->empty() || full->front().kind != PASS_TILE) return nullptr;
  PlanKey key{int(kk), int(hv), m, variant | kSplitVariantTag, map, map, tn.t, tn.e1, tn.e2, tn.c2,
              tn.w2 * 16 + tn.tma + tn.shfl * 256 + tn.em * 1024 + tn.tm * 8192,
              tn.var[0] * 4 + tn.var[1] * 2 + tn.var[2]};
  std::lock_guard<std::mutex> lk(g_ctx.mu);
  auto it = g_ctx.plans.find(key);
  if (it == g_ctx.plans.end()) {
    std::vector<Launch> out;
    std::vector<Launch> hplan;
    const Launch& tile = full->front();
    const int t = int(tile.P.b);
    // the half-size plan with the whole array's tuning starts where the
    // whole array's tile pass ends
    const bool ok = tile.P.work_counter == nullptr && m - 1 > t &&
                    plan_array(hplan, kk, hv, m - 1, tn, variant, map, 0u, g_ctx.smem_limit) &&
                    !hplan.empty() && hplan.front().kind == PASS_TILE && hplan.front().P.b == tile.P.b;
    if (ok) {
      for (int h = 0; h < 2; ++h) {
        const uint32_t off = uint32_t(h) << (m - 1);
        Launch T = tile;
        T.grid = 1u << (m - 1 - t);
        T.P.dir_base = off;
        out.push_back(T);
        for (size_t i = 1; i < hplan.size(); ++i) {
          Launch L = hplan[i];
          L.P.log2cap = uint32_t(m);
          L.P.dir_base = off;
          out.push_back(L);
        }
      }
      for (size_t i = 1; i < full->size(); ++i)
        if (int((*full)[i].P.rounds[0].p) == m) out.push_back((*full)[i]);
    }
    it = g_ctx.plans.emplace(key, std::move(out)).first;
  }
  if (it->second.empty()) return nullptr;
  *per = 0;
  for (size_t i = 1; i < it->second.size() && it->second[i].kind != PASS_TILE; ++i) *per = i;
  *per += 1;
  return &it->second;
}

int sort_device(KeyKind kk, bool f32, void* keys, uint32_t* vals, size_t n, int dir, int variant,
                cudaStream_t stream) {
  const int rc = check_common(keys, vals, n, dir, variant);
  if (rc >= 0) return rc;
  const int m = log2_exact(n);
  const uint32_t map = (f32 ? kMapF32 : 0u) | (dir == DARM_DESC ? kMapComplement : 0u);
  if (m >= kSplitMinLog2) {
    size_t per = 0;
    const std::vector<Launch>* sp = cached_split_plan(kk, vals != nullptr, m, variant, map, &per);
    if (sp) {
      const Launch* L0 = sp->data();
      const size_t hn = size_t(1) << (m - 1);
      const size_t ksz = (kk == KEY_U64) ? 8 : 4;
      cudaStream_t s2 = g_ctx.split_stream;
      // one split sort enqueues at a time: the fork and join events are shared
      static std::mutex split_mu;
      std::lock_guard<std::mutex> lk(split_mu);
      if (cudaEventRecord(g_ctx.split_fork_ev, stream) != cudaSuccess ||
          cudaStreamWaitEvent(s2, g_ctx.split_fork_ev, 0) != cudaSuccess)
        return DARM_ERR_CUDA;
      int r = launch_range(L0, L0 + per, kk, keys, vals, stream);
      if (r != DARM_OK) return r;
      r = launch_range(L0 + per, L0 + 2 * per, kk, static_cast<char*>(keys) + hn * ksz,
                       vals ? vals + hn : nullptr, s2);
      if (r != DARM_OK) return r;
      if (cudaEventRecord(g_ctx.split_join_ev, s2) != cudaSuccess ||
          cudaStreamWaitEvent(stream, g_ctx.split_join_ev, 0) != cudaSuccess)
        return DARM_ERR_CUDA;
      return launch_range(L0 + 2 * per, L0 + sp->size(), kk, keys, vals, stream);
    }
  }
  const std::vector<Launch>* plan = cached_plan(kk, vals != nullptr, m, variant, map, map);
  if (!plan) return DARM_ERR_INVALID_ARG;
  return launch_plan(*plan, kk, keys, vals, stream);
}

// Allow each kernel the device's opt-in shared memory minus what it
// declares statically.
static void set_smem_attr(const void* fn, void* ctx) {
  int* st = static_cast<int*>(ctx);  // {opt-in bytes, first error}
  cudaFuncAttributes fa;
  cudaError_t err = cudaFuncGetAttributes(&fa, fn);
  if (err == cudaSuccess) {
    const int bytes = st[0] - int(fa.sharedSizeBytes);
    err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  }
  if (err != cudaSuccess && st[1] == 0) st[1] = int(err);
}

}  // namespace darm

using namespace darm;

extern "C" {

int darm_sort_init(int device, size_t workspace_bytes) {
  std::lock_guard<std::mutex> lk(g_ctx.mu);
  if (g_ctx.inited) return device == g_ctx.device ? DARM_OK : DARM_ERR_BUSY;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return DARM_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return DARM_ERR_CUDA;
  int sms = 0, optin = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  g_ctx.device = device;
  g_ctx.sms = sms;
  g_sms_for_plans = sms;
  {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    cudaGetLastError();
    g_encode_tiled = fn;
    g_tensor_maps = fn != nullptr ? 1 : 0;
  }
  g_ctx.smem_limit = size_t(optin);
  int st[2] = {optin, 0};
  for_each_kernel_u32(set_smem_attr, st);
  for_each_kernel_u64(set_smem_attr, st);
  for_each_tile_kernel_u32(set_smem_attr, st);
  for_each_tile_kernel_u64(set_smem_attr, st);
  for_each_tma_kernel_u32(set_smem_attr, st);
  for_each_tile_shfl_kernel_u32(set_smem_attr, st);
  for_each_pcm_kernel(set_smem_attr, st);
  for_each_oddeven_kernel(set_smem_attr, st);
  for_each_window2_kernel(set_smem_attr, st);
  if (st[1] != 0) {
    fprintf(stderr, "darm: configuring shared memory failed: %s\n",
            cudaGetErrorString(cudaError_t(st[1])));
    cudaGetLastError();
    return DARM_ERR_CUDA;
  }
  g_ctx.smem_limit = size_t(optin) - 64;  // room for the kernels' static shared memory
  if (cudaMalloc(&g_ctx.d_status, sizeof(int)) != cudaSuccess) return DARM_ERR_OOM;
  if (cudaMemset(g_ctx.d_status, 0, sizeof(int)) != cudaSuccess) return DARM_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&g_ctx.host_stream, cudaStreamNonBlocking) != cudaSuccess)
    return DARM_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&g_ctx.host_copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return DARM_ERR_CUDA;
  for (cudaEvent_t& e : g_ctx.host_chunk_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return DARM_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&g_ctx.host_stream2, cudaStreamNonBlocking) != cudaSuccess)
    return DARM_ERR_CUDA;
  if (cudaEventCreateWithFlags(&g_ctx.host_join_ev, cudaEventDisableTiming) != cudaSuccess)
    return DARM_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&g_ctx.split_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g_ctx.split_fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g_ctx.split_join_ev, cudaEventDisableTiming) != cudaSuccess)
    return DARM_ERR_CUDA;
  if (workspace_bytes) {
    if (cudaMalloc(&g_ctx.ws, workspace_bytes) != cudaSuccess) return DARM_ERR_OOM;
    g_ctx.ws_bytes = workspace_bytes;
  }
  if (cudaGetLastError() != cudaSuccess) return DARM_ERR_CUDA;
  g_ctx.launches.store(0);
  g_ctx.inited = true;
  return DARM_OK;
}

int darm_sort_finalize(void) {
  darm_sort_serve_stop();
  segmented_release_all();
  std::lock_guard<std::mutex> lk(g_ctx.mu);
  if (!g_ctx.inited) return DARM_OK;
  cudaDeviceSynchronize();
  if (g_ctx.ws) cudaFree(g_ctx.ws);
  if (g_ctx.d_status) cudaFree(g_ctx.d_status);
  if (g_ctx.host_stream) cudaStreamDestroy(g_ctx.host_stream);
  if (g_ctx.host_copy_stream) cudaStreamDestroy(g_ctx.host_copy_stream);
  if (g_ctx.host_stream2) cudaStreamDestroy(g_ctx.host_stream2);
  if (g_ctx.host_join_ev) cudaEventDestroy(g_ctx.host_join_ev);
  g_ctx.host_stream2 = nullptr;
  g_ctx.host_join_ev = nullptr;
  if (g_ctx.split_stream) cudaStreamDestroy(g_ctx.split_stream);
  if (g_ctx.split_fork_ev) cudaEventDestroy(g_ctx.split_fork_ev);
  if (g_ctx.split_join_ev) cudaEventDestroy(g_ctx.split_join_ev);
  g_ctx.split_stream = nullptr;
  g_ctx.split_fork_ev = nullptr;
  g_ctx.split_join_ev = nullptr;
  for (cudaEvent_t& e : g_ctx.host_chunk_ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  g_ctx.host_copy_stream = nullptr;
  g_ctx.ws = nullptr;
  g_ctx.ws_bytes = 0;
  g_ctx.d_status = nullptr;
  g_ctx.host_stream = nullptr;
  g_ctx.plans.clear();
  g_ctx.inited = false;
  return DARM_OK;
}

const char* darm_status_str(int status) {
  switch (status) {
    case DARM_OK: return "DARM_OK";
    case DARM_ERR_INVALID_ARG: return "DARM_ERR_INVALID_ARG";
    case DARM_ERR_NOT_POW2: return "DARM_ERR_NOT_POW2";
    case DARM_ERR_NOT_INIT: return "DARM_ERR_NOT_INIT";
    case DARM_ERR_OOM: return "DARM_ERR_OOM";
    case DARM_ERR_CUDA: return "DARM_ERR_CUDA";
    case DARM_ERR_BUDGET: return "DARM_ERR_BUDGET";
    case DARM_ERR_TIMEOUT: return "DARM_ERR_TIMEOUT";
    case DARM_ERR_SENTINEL_COLLISION: return "DARM_ERR_SENTINEL_COLLISION";
    case DARM_ERR_BUSY: return "DARM_ERR_BUSY";
    case DARM_ERR_NOT_FOUND: return "DARM_ERR_NOT_FOUND";
    default: return "DARM_ERR_UNKNOWN";
  }
}

int darm_device_status(int* status) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (!status) return DARM_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return DARM_ERR_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, g_ctx.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DARM_ERR_CUDA;
  if (cudaMemset(g_ctx.d_status, 0, sizeof(int)) != cudaSuccess) return DARM_ERR_CUDA;
  *status = h;
  return DARM_OK;
}

int darm_check_bounded_wait(void* stream) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (launch_bounded_wait_check(g_ctx.d_status, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return DARM_ERR_CUDA;
  g_ctx.launches.fetch_add(1, std::memory_order_relaxed);
  return DARM_OK;
}

int darm_bitonic_sort(uint32_t* keys, uint32_t* vals, size_t n, int dir, int variant,
                      void* stream) {
  return sort_device(KEY_U32, false, keys, vals, n, dir, variant,
                     static_cast<cudaStream_t>(stream));
}

int darm_bitonic_sort_f32(float* keys, uint32_t* vals, size_t n, int dir, int variant,
                          void* stream) {
  return sort_device(KEY_U32, true, keys, vals, n, dir, variant,
                     static_cast<cudaStream_t>(stream));
}

int darm_bitonic_sort_u64(uint64_t* keys, uint32_t* vals, size_t n, int dir, int variant,
                          void* stream) {
  return sort_device(KEY_U64, false, keys, vals, n, dir, variant,
                     static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace darm {
namespace {

// Host-buffer sorts of 2^m >= 2^kHostChunkMinLog2 elements overlap the
// host<->device copies with the sort.  A stage 2^p compares elements of one
// aligned 2^p-element block only, so:
//   - the input is copied in 8 chunks on a copy stream, and the tile pass of
//     each chunk runs as soon as it has arrived;
//   - once the first half (4 chunks) has arrived and been tiled, stages
//     2^(t+1) .. 2^(m-1) run on that half while the second half is still
//     being copied; the second half's tile passes run on a second stream as
//     its chunks arrive, beside those stages; then the second half's stages;
//   - the final stage runs over the whole array; its trailing passes whose
//     blocks lie inside one chunk (the merge, and window passes below bit
//     m-3) run chunk by chunk, and each chunk is copied back while the next
//     one is processed.
// A chunk or half reads its comparator directions from its index in the
// whole array (dir_base), so every comparator is the whole-array network's
// and the result is identical.  (Running all stages below 2^(m-3) per chunk
// was slower: those launches are too small to fill the GPU.)
constexpr int kHostChunkMinLog2 = 20;
constexpr int kHostChunks = 8;

int sort_host_chunked(KeyKind kk, bool f32, void* keys_out, uint32_t* vals_out, void* dk,
                      uint32_t* dv, int m, int dir, int variant, cudaStream_t s) {
  const void* keys = keys_out;
  const uint32_t* vals = vals_out;
  const int mc = m - 3, mh = m - 1;
  const size_t cn = size_t(1) << mc, hn = size_t(1) << mh;
  const size_t ksz = (kk == KEY_U64) ? 8 : 4;
  const bool hv = vals != nullptr;
  const uint32_t map = (f32 ? kMapF32 : 0u) | (dir == DARM_DESC ? kMapComplement : 0u);
  const std::vector<Launch>* full = cached_plan(kk, hv, m, variant, map, map);
  if (!full || full->empty() || full->front().kind != PASS_TILE) return DARM_ERR_INVALID_ARG;
  // the half-size plan takes the whole array's tuning, so that its passes
  // start where the whole array's tile pass ends
  std::vector<Launch> hplan_v;
  if (!plan_array(hplan_v, kk, hv, mh, tuning_for(kk, hv, m), variant, map, 0u, g_ctx.smem_limit))
    return DARM_ERR_INVALID_ARG;
  const std::vector<Launch>* hplan = &hplan_v;
  if (hplan->empty() || hplan->front().kind != PASS_TILE ||
      hplan->front().P.b != full->front().P.b)
    return DARM_ERR_INVALID_ARG;
  std::vector<Launch> tile(1, full->front());
  const int t = int(tile[0].P.b);
  if (mc < t || tile[0].P.work_counter != nullptr) return DARM_ERR_INVALID_ARG;
  tile[0].grid = uint32_t(1u << (mc - t));
  // stages t+1 .. m-1 on one half: the half-size plan without its tile pass
  std::vector<Launch> half(hplan->begin() + 1, hplan->end());
  for (Launch& L : half) L.P.log2cap = uint32_t(m);  // directions of the whole array
  // the final stage of the whole-array plan, split into a whole-array body
  // and a chunk-local tail
  size_t first = full->size();
  while (first > 1 && (*full)[first - 1].kind != PASS_TILE &&
         int((*full)[first - 1].P.rounds[0].p) == m)
    --first;
  size_t tail_begin = full->size();
  while (tail_begin > first) {
    const Launch& L = (*full)[tail_begin - 1];
    if (L.P.work_counter != nullptr) break;
    const bool local = (L.kind == PASS_MERGE) ||
                       (L.kind == PASS_WINDOW && int(L.P.w0 + L.P.s) <= mc && int(L.P.b) <= mc);
    if (!local) break;
    --tail_begin;
  }
  const std::vector<Launch> body(full->begin() + first, full->begin() + tail_begin);
  std::vector<Launch> tail(full->begin() + tail_begin, full->end());
  for (Launch& L : tail) {
    if (L.tma) {
      L.P.nblocks = uint32_t(1u << (mc - int(L.P.b)));
      L.grid = std::min(L.grid, L.P.nblocks);
    } else if (L.win2t) {
      L.P.nblocks >>= 3;  // 2^(m - b) blocks -> 2^(mc - b) per chunk
      L.grid = std::min(L.grid, L.P.nblocks);
    } else {
      L.grid >>= 3;  // 2^(m - b) blocks -> 2^(mc - b) per chunk
    }
  }
  cudaStream_t cps = g_ctx.host_copy_stream;
  for (int c = 0; c < kHostChunks; ++c) {
    const size_t off = size_t(c) * cn;
    if (cudaMemcpyAsync(static_cast<char*>(dk) + off * ksz,
                        static_cast<const char*>(keys) + off * ksz, cn * ksz,
                        cudaMemcpyHostToDevice, cps) != cudaSuccess)
      return DARM_ERR_CUDA;
    if (hv && cudaMemcpyAsync(dv + off, vals + off, cn * 4, cudaMemcpyHostToDevice, cps) !=
                  cudaSuccess)
      return DARM_ERR_CUDA;
    if (cudaEventRecord(g_ctx.host_chunk_ev[c], cps) != cudaSuccess) return DARM_ERR_CUDA;
  }
  int rc;
  // Tile passes as the chunks arrive: the first half's on `s`, the second
  // half's on a second stream, so that they run while `s` works through the
  // first half's stages (the tile passes are bound by the ALU, those stages
  // by HBM); `s` joins them before the second half's stages.
  cudaStream_t s2 = g_ctx.host_stream2;
  for (int c = 0; c < kHostChunks; ++c) {
    cudaStream_t ts = (c < kHostChunks / 2) ? s : s2;
    const size_t off = size_t(c) * cn;
    if (cudaStreamWaitEvent(ts, g_ctx.host_chunk_ev[c], 0) != cudaSuccess) return DARM_ERR_CUDA;
    tile[0].P.dir_base = uint32_t(off);
    rc = launch_plan(tile, kk, static_cast<char*>(dk) + off * ksz, hv ? dv + off : nullptr, ts);
    if (rc != DARM_OK) return rc;
  }
  if (cudaEventRecord(g_ctx.host_join_ev, s2) != cudaSuccess) return DARM_ERR_CUDA;
  for (int h = 0; h < 2; ++h) {
    if (h == 1 && cudaStreamWaitEvent(s, g_ctx.host_join_ev, 0) != cudaSuccess) return DARM_ERR_CUDA;
    const size_t off = size_t(h) * hn;
    for (Launch& L : half) L.P.dir_base = uint32_t(off);
    rc = launch_plan(half, kk, static_cast<char*>(dk) + off * ksz, hv ? dv + off : nullptr, s);
    if (rc != DARM_OK) return rc;
  }
  rc = launch_plan(body, kk, dk, dv, s);
  if (rc != DARM_OK) return rc;
  for (int c = 0; c < kHostChunks; ++c) {
    const size_t off = size_t(c) * cn;
    char* kd = static_cast<char*>(dk) + off * ksz;
    if (!tail.empty()) {
      rc = launch_plan(tail, kk, kd, hv ? dv + off : nullptr, s);
      if (rc != DARM_OK) return rc;
    }
    if (cudaEventRecord(g_ctx.host_chunk_ev[c], s) != cudaSuccess) return DARM_ERR_CUDA;
    if (cudaStreamWaitEvent(cps, g_ctx.host_chunk_ev[c], 0) != cudaSuccess) return DARM_ERR_CUDA;
    if (cudaMemcpyAsync(static_cast<char*>(keys_out) + off * ksz, kd, cn * ksz,
                        cudaMemcpyDeviceToHost, cps) != cudaSuccess)
      return DARM_ERR_CUDA;
    if (hv && cudaMemcpyAsync(vals_out + off, dv + off, cn * 4, cudaMemcpyDeviceToHost, cps) !=
                  cudaSuccess)
      return DARM_ERR_CUDA;
  }
  // the caller synchronises `s`: make it wait for the last copies
  if (cudaEventRecord(g_ctx.host_chunk_ev[0], cps) != cudaSuccess) return DARM_ERR_CUDA;
  if (cudaStreamWaitEvent(s, g_ctx.host_chunk_ev[0], 0) != cudaSuccess) return DARM_ERR_CUDA;
  return DARM_OK;
}

}  // namespace
}  // namespace darm

extern "C" {

int darm_bitonic_sort_host(void* keys, uint32_t* vals, size_t n, int dtype, int dir,
                           int variant) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (dtype < DARM_U32 || dtype > DARM_U64) return DARM_ERR_INVALID_ARG;
  if (n <= 1) return DARM_OK;
  if ((n & (n - 1)) != 0) return DARM_ERR_NOT_POW2;
  if (!keys) return DARM_ERR_INVALID_ARG;
  const size_t kbytes = n * (dtype == DARM_U64 ? 8 : 4);
  const size_t vbytes = vals ? n * 4 : 0;
  const size_t need = kbytes + ((vbytes + 255) & ~size_t(255)) + 256;
  std::lock_guard<std::mutex> lk(g_ctx.host_mu);
  if (g_ctx.ws_bytes < need) {
    if (g_ctx.ws) cudaFree(g_ctx.ws);
    g_ctx.ws = nullptr;
    g_ctx.ws_bytes = 0;
    if (cudaMalloc(&g_ctx.ws, need) != cudaSuccess) return DARM_ERR_OOM;
    g_ctx.ws_bytes = need;
  }
  char* base = static_cast<char*>(g_ctx.ws);
  void* dk = base;
  uint32_t* dv = vals ? reinterpret_cast<uint32_t*>(base + ((kbytes + 255) & ~size_t(255))) : nullptr;
  cudaStream_t s = g_ctx.host_stream;
  const KeyKind kk = dtype == DARM_U64 ? KEY_U64 : KEY_U32;
  const int m = log2_exact(n);
  if (m >= kHostChunkMinLog2) {
    // copies in both directions happen inside, overlapped with passes
    const int rc = sort_host_chunked(kk, dtype == DARM_F32, keys, vals, dk, dv, m, dir, variant, s);
    if (rc != DARM_OK) {
      // copies already enqueued must not outlive the call: the workspace and
      // the caller's buffers are reused once it returns
      cudaStreamSynchronize(g_ctx.host_copy_stream);
      cudaStreamSynchronize(g_ctx.host_stream2);
      cudaStreamSynchronize(s);
      return rc;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return DARM_ERR_CUDA;
    return DARM_OK;
  }
  if (cudaMemcpyAsync(dk, keys, kbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return DARM_ERR_CUDA;
  if (vals && cudaMemcpyAsync(dv, vals, vbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return DARM_ERR_CUDA;
  const int rc = sort_device(kk, dtype == DARM_F32, dk, dv, n, dir, variant, s);
  if (rc != DARM_OK) {
    cudaStreamSynchronize(s);  // let the enqueued copies finish before returning
    return rc;
  }
  if (cudaMemcpyAsync(keys, dk, kbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return DARM_ERR_CUDA;
  if (vals && cudaMemcpyAsync(vals, dv, vbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return DARM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DARM_ERR_CUDA;
  return DARM_OK;
}

int darm_plan_info(int dtype, size_t n, int has_vals, int variant, int* passes, int* launches,
                   int* tile) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (dtype < DARM_U32 || dtype > DARM_U64) return DARM_ERR_INVALID_ARG;
  if (n < 2 || (n & (n - 1)) != 0) return DARM_ERR_NOT_POW2;
  const KeyKind kk = dtype == DARM_U64 ? KEY_U64 : KEY_U32;
  const int m = log2_exact(n);
  const std::vector<Launch>* plan = cached_plan(kk, has_vals != 0, m, variant, 0, 0);
  if (!plan) return DARM_ERR_INVALID_ARG;
  if (passes) *passes = int(plan->size());
  if (launches) *launches = int(plan->size());
  if (tile) *tile = plan->empty() ? 0 : int(1u << plan->front().P.b);
  return DARM_OK;
}

int darm_plan_describe(int dtype, size_t n, int has_vals, int variant, char* buf, size_t cap) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (dtype < DARM_U32 || dtype > DARM_U64 || !buf || cap == 0) return DARM_ERR_INVALID_ARG;
  if (n < 2 || (n & (n - 1)) != 0) return DARM_ERR_NOT_POW2;
  const KeyKind kk = dtype == DARM_U64 ? KEY_U64 : KEY_U32;
  const std::vector<Launch>* plan = cached_plan(kk, has_vals != 0, log2_exact(n), variant, 0, 0);
  if (!plan) return DARM_ERR_INVALID_ARG;
  const std::string d = describe(*plan);
  const size_t k = std::min(d.size(), cap - 1);
  std::memcpy(buf, d.data(), k);
  buf[k] = '\0';
  return DARM_OK;
}

int darm_plan_dump(int dtype, size_t n, int has_vals, int variant, const int32_t* tuning,
                   size_t smem_limit, int32_t* out, int cap, int* count) {
  if (dtype < DARM_U32 || dtype > DARM_U64) return DARM_ERR_INVALID_ARG;
  if (variant < DARM_DIVERGENT || variant > DARM_AUTO || !count) return DARM_ERR_INVALID_ARG;
  if (n < 2 || (n & (n - 1)) != 0 || n > (size_t(1) << 31)) return DARM_ERR_NOT_POW2;
  const KeyKind kk = dtype == DARM_U64 ? KEY_U64 : KEY_U32;
  const bool hv = has_vals != 0;
  const int m = log2_exact(n);
  Tuning tn = tuning_for(kk, hv, m);
  if (tuning) {
    tn.t = tuning[0];
    tn.e1 = tuning[1];
    tn.e2 = tuning[2];
    tn.c2 = tuning[3];
    tn.w2 = tuning[4];
    tn.tma = tuning[5];
    tn.shfl = tuning[6];
    tn.tm = tuning[7];
  }
  if (smem_limit == 0) smem_limit = g_ctx.inited ? g_ctx.smem_limit : size_t(232448 - 64);
  const uint32_t map = dtype == DARM_F32 ? kMapF32 : 0u;
  std::vector<Launch> plan;
  if (!plan_array(plan, kk, hv, m, tn, variant, map, map, smem_limit)) return DARM_ERR_INVALID_ARG;
  std::vector<int32_t> v;
  for (const Launch& L : plan) {
    const int32_t head[] = {int32_t(L.kind), L.fixed, L.tma, L.win1, L.win2t ? 2 : int(L.win2), L.shfl, L.loge,
                            L.variant, int32_t(L.grid), int32_t(L.threads), int32_t(L.smem),
                            int32_t(L.P.b), int32_t(L.P.c), int32_t(L.P.w0), int32_t(L.P.s),
                            int32_t(L.P.log2cap), int32_t(L.P.nrounds), int32_t(L.P.nblocks),
                            int32_t(L.P.map_in), int32_t(L.P.map_out), L.mshfl};
    v.insert(v.end(), head, head + 21);
    for (uint32_t r = 0; r < L.P.nrounds; ++r) {
      const Round& R = L.P.rounds[r];
      const int32_t row[] = {R.kind, R.p, R.a, R.cnt, R.src, R.dst, R.lanediv};
      v.insert(v.end(), row, row + 7);
    }
  }
  *count = int(v.size());
  if (!out || cap < int(v.size())) return DARM_ERR_INVALID_ARG;
  std::copy(v.begin(), v.end(), out);
  return DARM_OK;
}

uint64_t darm_launch_count(void) { return g_ctx.launches.load(); }

int darm_sort_profile(void* keys, uint32_t* vals, size_t n, int dtype, int dir, int variant,
                      void* stream, float* ms, int* kind, int cap, int* count) {
  if (dtype < DARM_U32 || dtype > DARM_U64) return DARM_ERR_INVALID_ARG;
  const int rc0 = check_common(keys, vals, n, dir, variant);
  if (rc0 >= 0) return rc0;
  const KeyKind kk = dtype == DARM_U64 ? KEY_U64 : KEY_U32;
  const int m = log2_exact(n);
  const uint32_t map = (dtype == DARM_F32 ? kMapF32 : 0u) | (dir == DARM_DESC ? kMapComplement : 0u);
  const std::vector<Launch>* plan = cached_plan(kk, vals != nullptr, m, variant, map, map);
  if (!plan) return DARM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t L = plan->size();
  std::vector<cudaEvent_t> ev(L + 1);
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return DARM_ERR_CUDA;
  int rc = DARM_OK;
  cudaEventRecord(ev[0], s);
  for (size_t i = 0; i < L && rc == DARM_OK; ++i) {
    std::vector<Launch> one(1, (*plan)[i]);
    rc = launch_plan(one, kk, keys, vals, s);
    cudaEventRecord(ev[i + 1], s);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = DARM_ERR_CUDA;
  for (size_t i = 0; i < L && rc == DARM_OK; ++i) {
    if (int(i) < cap) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
      if (ms) ms[i] = t;
      if (kind) kind[i] = int((*plan)[i].kind);
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (count) *count = int(L);
  return rc;
}

}  // extern "C"
