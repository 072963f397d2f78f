// pcm.cu - PCM, Partition and Concurrent Merge (Section VI-A): a sort built on
// Batcher's odd-even merge sort that odd-even merges buckets of sorted keys.
//
// The n = B * S keys form B buckets of S consecutive keys (B, S powers of
// two, S <= 4096).  Every bucket is first sorted by the odd-even merge sort
// network on one thread block (oddeven.cu).  Then the same network runs over
// the B buckets: stage s = 0 .. log2 B - 1 (p = 2^s), layer t = s .. 0
// (k = 2^t) compares bucket x with bucket x + k
//   - for every x with bit s clear when k == p;
//   - for every x with (x mod 2p) in [k, 2p - k) and bit t set when k < p;
// and every comparator is a merge-split: the two sorted buckets are merged -
// on equal keys bucket x's key first, each bucket's keys in order - and the
// lower S keys of the merge become bucket x, the upper S bucket x + k.  With
// S = 1 a merge-split is a strict compare-exchange and PCM is the plain
// odd-even network.
//
// One launch per layer, one CTA per comparator.  The CTA stages both buckets
// in shared memory, each thread finds where its 2S/T outputs start on the
// merge path (a binary search for the split (i, j), i + j = its first
// output, with A[i-1] <= B[j] and B[j-1] < A[i]) and merges them one by one:
// the loop whose data-dependent branch - take from A or from B - the paper's
// PCM kernel diverges on.
//   divergent: if (A wins) { emit A[i]; i++; reload A[i] } else { the same
//              with B } - two copies of the body, one per side, each with its
//              own shared-memory load;
//   melded:    the two sides aligned into one copy (Algorithm 2): the
//              emitted value, the advanced index and the reloaded array are
//              chosen by select on the branch condition, so the warp issues
//              one shared-memory load per output.
// Merges go out of place: buffers 0 (the caller's keys) and 1 (the caller's
// scratch) alternate per bucket.  Which buffer holds bucket x before a layer
// is the parity of the comparators x has taken part in so far, a closed
// form (pcm_parts), so no location table is kept; a last launch copies the
// buckets that end in the scratch back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "darm.h"
#include "darm_internal.h"

namespace darm {
namespace {

constexpr uint32_t kPcmMaxBucket = 4096;
constexpr uint32_t kPcmThreads = 512;
constexpr uint32_t kPcmPerThread = 16;  // outputs per thread at full size

struct PcmLayer {
  uint32_t* k[2];  // buffer 0: the caller's keys, 1: the caller's scratch
  uint32_t* v[2];  // payloads (nullptr: keys only)
  uint32_t S;      // keys per bucket
  uint32_t s, t;   // stage p = 2^s, layer k = 2^t
};

// Layers t' in [t_lo, s] of stage s in which bucket x takes part: the first
// layer (t' = s) always; a later one (t' < s) when x mod 2^(s+1) lies in
// [2^t', 2^(s+1) - 2^t'), i.e. when 2^t' <= w = min(z, 2^(s+1) - 1 - z).
__device__ __forceinline__ uint32_t pcm_stage_parts(uint32_t x, uint32_t s, uint32_t t_lo) {
  const uint32_t z = x & ((2u << s) - 1u);
  const uint32_t w = min(z, (2u << s) - 1u - z);
  const uint32_t bits = 32u - __clz(w);  // floor(log2 w) + 1, 0 when w == 0
  const uint32_t below = min(s, bits);
  return (below > t_lo ? below - t_lo : 0u) + (s >= t_lo ? 1u : 0u);
}

// Comparators bucket x took part in before layer (s, t): the buffer holding
// it now is this count's parity.
__device__ __forceinline__ uint32_t pcm_parts(uint32_t x, uint32_t s, uint32_t t) {
  uint32_t n = 0;
  for (uint32_t q = 0; q < s; ++q) n += pcm_stage_parts(x, q, 0);
  return n + pcm_stage_parts(x, s, t + 1);
}

// Buffer `sel` of the keys or payloads, chosen by select (indexing the
// parameter arrays with a run-time value would copy them to local memory).
__device__ __forceinline__ uint32_t* kbuf(const PcmLayer& L, uint32_t sel) {
  return sel ? L.k[1] : L.k[0];
}
__device__ __forceinline__ uint32_t* vbuf(const PcmLayer& L, uint32_t sel) {
  return sel ? L.v[1] : L.v[0];
}

// Shared-memory slot of element e of a 2S-element region: one pad word per
// 32 elements, so that the lanes of a warp, whose merge positions are about
// 2S/T apart, fall on distinct banks.
__device__ __forceinline__ uint32_t pad(uint32_t e) { return e + (e >> 5); }
__host__ __device__ constexpr uint32_t padded_words(uint32_t n) { return n + (n >> 5) + 1; }

__device__ __forceinline__ void put4(uint32_t* dst, uint32_t e, uint4 w) {
  dst[pad(e)] = w.x;
  dst[pad(e + 1)] = w.y;
  dst[pad(e + 2)] = w.z;
  dst[pad(e + 3)] = w.w;
}

__device__ __forceinline__ uint4 get4(const uint32_t* src, uint32_t e) {
  return make_uint4(src[pad(e)], src[pad(e + 1)], src[pad(e + 2)], src[pad(e + 3)]);
}

template <bool V, int VAR>
__global__ void __launch_bounds__(kPcmThreads) darm_pcm_layer_kernel(const PcmLayer L) {
  extern __shared__ __align__(16) uint32_t pcm_smem[];
  const uint32_t S = L.S;
  const uint32_t R = padded_words(2 * S);  // words of one region
  uint32_t* sAB = pcm_smem;            // [A | B], 2S keys
  uint32_t* sOut = pcm_smem + R;       // 2S merged keys
  uint32_t* sVAB = pcm_smem + 2 * R;   // payloads of A and B
  uint32_t* sVOut = pcm_smem + 3 * R;  // merged payloads

  // comparator of this CTA
  const uint32_t c = blockIdx.x;
  const uint32_t p = 1u << L.s, k = 1u << L.t;
  uint32_t x;
  if (L.t == L.s) {
    x = ((c >> L.s) << (L.s + 1)) | (c & (p - 1u));
  } else {
    const uint32_t per = p - k;
    const uint32_t q = c / per, r = c - q * per;
    x = (q << (L.s + 1)) + k + ((r >> L.t) << (L.t + 1)) + (r & (k - 1u));
  }
  const uint32_t y = x + k;
  const uint32_t la = pcm_parts(x, L.s, L.t) & 1u;
  const uint32_t lb = pcm_parts(y, L.s, L.t) & 1u;
  const uint32_t* gA = kbuf(L, la) + size_t(x) * S;
  const uint32_t* gB = kbuf(L, lb) + size_t(y) * S;
  const uint32_t tid = threadIdx.x, nt = blockDim.x;

  // stage both buckets (128-bit global loads where the bucket allows)
  if (S >= 4) {
    for (uint32_t e = tid * 4; e < S; e += nt * 4) {
      put4(sAB, e, *reinterpret_cast<const uint4*>(gA + e));
      put4(sAB, S + e, *reinterpret_cast<const uint4*>(gB + e));
      if (V) {
        put4(sVAB, e, *reinterpret_cast<const uint4*>(vbuf(L, la) + size_t(x) * S + e));
        put4(sVAB, S + e, *reinterpret_cast<const uint4*>(vbuf(L, lb) + size_t(y) * S + e));
      }
    }
  } else {
    for (uint32_t e = tid; e < S; e += nt) {
      sAB[pad(e)] = gA[e];
      sAB[pad(S + e)] = gB[e];
      if (V) {
        sVAB[pad(e)] = vbuf(L, la)[size_t(x) * S + e];
        sVAB[pad(S + e)] = vbuf(L, lb)[size_t(y) * S + e];
      }
    }
  }
  __syncthreads();

  // merge path: outputs [d, d + Q) of this thread start at split (i, j)
  const uint32_t Q = (2 * S) / nt;
  const uint32_t d = tid * Q;
  uint32_t lo = d > S ? d - S : 0u, hi = d < S ? d : S;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (sAB[pad(mid)] <= sAB[pad(S + (d - mid - 1))])
      lo = mid + 1;
    else
      hi = mid;
  }
  uint32_t i = lo, j = d - lo;
  uint32_t a = (i < S) ? sAB[pad(i)] : 0u;
  uint32_t b = (j < S) ? sAB[pad(S + j)] : 0u;
#pragma unroll 4
  for (uint32_t o = 0; o < Q; ++o) {
    uint32_t key, val = 0;
    if (VAR == kDivergent) {
      if (j >= S || (i < S && a <= b)) {
        key = a;
        if (V) val = sVAB[pad(i)];
        ++i;
        if (i < S) a = sAB[pad(i)];
      } else {
        key = b;
        if (V) val = sVAB[pad(S + j)];
        ++j;
        if (j < S) b = sAB[pad(S + j)];
      }
    } else {
      const bool ta = (j >= S) || (i < S && a <= b);
      key = ta ? a : b;
      const uint32_t src = ta ? i : S + j;  // the emitted element's slot
      if (V) val = sVAB[pad(src)];
      i += ta ? 1u : 0u;
      j += ta ? 0u : 1u;
      const uint32_t nxt = ta ? i : j;      // the side's next element
      const uint32_t nslot = ta ? i : S + j;
      const uint32_t fresh = (nxt < S) ? sAB[pad(nslot)] : 0u;
      a = ta ? fresh : a;
      b = ta ? b : fresh;
    }
    sOut[pad(d + o)] = key;
    if (V) sVOut[pad(d + o)] = val;
  }
  __syncthreads();

  // lower half -> bucket x, upper half -> bucket y, each in the buffer it
  // does not occupy now
  uint32_t* oA = kbuf(L, la ^ 1u) + size_t(x) * S;
  uint32_t* oB = kbuf(L, lb ^ 1u) + size_t(y) * S;
  if (S >= 4) {
    for (uint32_t e = tid * 4; e < S; e += nt * 4) {
      *reinterpret_cast<uint4*>(oA + e) = get4(sOut, e);
      *reinterpret_cast<uint4*>(oB + e) = get4(sOut, S + e);
      if (V) {
        *reinterpret_cast<uint4*>(vbuf(L, la ^ 1u) + size_t(x) * S + e) = get4(sVOut, e);
        *reinterpret_cast<uint4*>(vbuf(L, lb ^ 1u) + size_t(y) * S + e) = get4(sVOut, S + e);
      }
    }
  } else {
    for (uint32_t e = tid; e < S; e += nt) {
      oA[e] = sOut[pad(e)];
      oB[e] = sOut[pad(S + e)];
      if (V) {
        vbuf(L, la ^ 1u)[size_t(x) * S + e] = sVOut[pad(e)];
        vbuf(L, lb ^ 1u)[size_t(y) * S + e] = sVOut[pad(S + e)];
      }
    }
  }
}

// Buckets of 256 keys or more: 2S/16 threads (at least 32), 16 outputs each.
// Same algorithm as darm_pcm_layer_kernel with less bookkeeping: the
// buckets' locations are summed by the lanes of each warp (one stage per
// lane) instead of a serial loop in every thread; a side's next key is
// read without a bound check (the slot after A is B's first, the slot after
// B is the region's spare word, and neither is used once that side is
// exhausted); and a thread's 16 outputs are contiguous slots, so their
// addresses are immediates.
constexpr uint32_t kPcmQ = 16;

__device__ __forceinline__ uint32_t pcm_parity_warp(uint32_t x, uint32_t s, uint32_t t) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t n = 0;
  if (lane < s)
    n = pcm_stage_parts(x, lane, 0);
  else if (lane == s)
    n = pcm_stage_parts(x, s, t + 1);
  return __reduce_add_sync(0xFFFFFFFFu, n) & 1u;
}

template <bool V, int VAR>
__global__ void __launch_bounds__(kPcmThreads) darm_pcm_layer16_kernel(const PcmLayer L) {
  extern __shared__ __align__(16) uint32_t pcm_smem[];
  const uint32_t S = L.S;
  const uint32_t R = padded_words(2 * S);
  uint32_t* sAB = pcm_smem;
  uint32_t* sOut = pcm_smem + R;
  uint32_t* sVAB = pcm_smem + 2 * R;
  uint32_t* sVOut = pcm_smem + 3 * R;

  const uint32_t c = blockIdx.x;
  const uint32_t p = 1u << L.s, k = 1u << L.t;
  uint32_t x;
  if (L.t == L.s) {
    x = ((c >> L.s) << (L.s + 1)) | (c & (p - 1u));
  } else {
    const uint32_t per = p - k;
    const uint32_t q = c / per, r = c - q * per;
    x = (q << (L.s + 1)) + k + ((r >> L.t) << (L.t + 1)) + (r & (k - 1u));
  }
  const uint32_t y = x + k;
  const uint32_t la = pcm_parity_warp(x, L.s, L.t);
  const uint32_t lb = pcm_parity_warp(y, L.s, L.t);
  const uint32_t tid = threadIdx.x, nt = blockDim.x;
  {
    const uint4* gA = reinterpret_cast<const uint4*>(kbuf(L, la) + size_t(x) * S);
    const uint4* gB = reinterpret_cast<const uint4*>(kbuf(L, lb) + size_t(y) * S);
    const uint4* vA = V ? reinterpret_cast<const uint4*>(vbuf(L, la) + size_t(x) * S) : nullptr;
    const uint4* vB = V ? reinterpret_cast<const uint4*>(vbuf(L, lb) + size_t(y) * S) : nullptr;
    for (uint32_t e = tid; e < S / 4; e += nt) {
      const uint4 ka = __ldg(gA + e), kb = __ldg(gB + e);
      put4(sAB, 4 * e, ka);
      put4(sAB, S + 4 * e, kb);
      if (V) {
        put4(sVAB, 4 * e, __ldg(vA + e));
        put4(sVAB, S + 4 * e, __ldg(vB + e));
      }
    }
  }
  __syncthreads();

  const uint32_t d = tid * kPcmQ;
  uint32_t lo = d > S ? d - S : 0u, hi = d < S ? d : S;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (sAB[pad(mid)] <= sAB[pad(S + (d - mid - 1))])
      lo = mid + 1;
    else
      hi = mid;
  }
  uint32_t i = lo, j = d - lo;  // next unread of A, of B
  uint32_t a = sAB[pad(i)];      // read unconditionally: see above
  uint32_t b = sAB[pad(S + j)];
  const uint32_t po = pad(d);    // the 16 outputs are slots po .. po + 15
#pragma unroll
  for (uint32_t o = 0; o < kPcmQ; ++o) {
    const bool ta = (j >= S) || (i < S && a <= b);
    uint32_t key, val = 0;
    if (VAR == kDivergent) {
      if (ta) {
        key = a;
        if (V) val = sVAB[pad(i)];
        ++i;
        a = sAB[pad(i)];
      } else {
        key = b;
        if (V) val = sVAB[pad(S + j)];
        ++j;
        b = sAB[pad(S + j)];
      }
    } else {
      key = ta ? a : b;
      const uint32_t slot = ta ? i : S + j;
      if (V) val = sVAB[pad(slot)];
      i += ta ? 1u : 0u;
      j += ta ? 0u : 1u;
      const uint32_t fresh = sAB[pad(slot + 1)];
      a = ta ? fresh : a;
      b = ta ? b : fresh;
    }
    sOut[po + o] = key;
    if (V) sVOut[po + o] = val;
  }
  __syncthreads();

  uint4* oA = reinterpret_cast<uint4*>(kbuf(L, la ^ 1u) + size_t(x) * S);
  uint4* oB = reinterpret_cast<uint4*>(kbuf(L, lb ^ 1u) + size_t(y) * S);
  uint4* wA = V ? reinterpret_cast<uint4*>(vbuf(L, la ^ 1u) + size_t(x) * S) : nullptr;
  uint4* wB = V ? reinterpret_cast<uint4*>(vbuf(L, lb ^ 1u) + size_t(y) * S) : nullptr;
  for (uint32_t e = tid; e < S / 4; e += nt) {
    oA[e] = get4(sOut, 4 * e);
    oB[e] = get4(sOut, S + 4 * e);
    if (V) {
      wA[e] = get4(sVOut, 4 * e);
      wB[e] = get4(sVOut, S + 4 * e);
    }
  }
}

// Buckets whose last merge-split left them in the scratch: copy them back.
template <bool V>
__global__ void __launch_bounds__(256) darm_pcm_gather_kernel(const PcmLayer L, uint32_t nstages) {
  const uint32_t x = blockIdx.x;
  uint32_t n = 0;
  for (uint32_t q = 0; q < nstages; ++q) n += pcm_stage_parts(x, q, 0);
  if ((n & 1u) == 0u) return;
  const size_t base = size_t(x) * L.S;
  for (uint32_t e = threadIdx.x; e < L.S; e += blockDim.x) {
    L.k[0][base + e] = L.k[1][base + e];
    if (V) L.v[0][base + e] = L.v[1][base + e];
  }
}

size_t pcm_smem_bytes(bool has_vals, uint32_t S) {
  return size_t(has_vals ? 4 : 2) * padded_words(2 * S) * sizeof(uint32_t);
}

}  // namespace

void for_each_pcm_kernel(void (*fn)(const void*, void*), void* ctx) {
  fn(reinterpret_cast<const void*>(&darm_pcm_layer16_kernel<false, 0>), ctx);
  fn(reinterpret_cast<const void*>(&darm_pcm_layer16_kernel<false, 1>), ctx);
  fn(reinterpret_cast<const void*>(&darm_pcm_layer16_kernel<true, 0>), ctx);
  fn(reinterpret_cast<const void*>(&darm_pcm_layer16_kernel<true, 1>), ctx);
  fn(reinterpret_cast<const void*>(&darm_pcm_layer_kernel<false, 0>), ctx);
  fn(reinterpret_cast<const void*>(&darm_pcm_layer_kernel<false, 1>), ctx);
  fn(reinterpret_cast<const void*>(&darm_pcm_layer_kernel<true, 0>), ctx);
  fn(reinterpret_cast<const void*>(&darm_pcm_layer_kernel<true, 1>), ctx);
}

}  // namespace darm

using namespace darm;

extern "C" int darm_pcm_sort(uint32_t* keys, uint32_t* vals, size_t n, size_t bucket,
                             uint32_t* scratch_keys, uint32_t* scratch_vals, int variant,
                             void* stream) {
  if (!g_ctx.inited) return DARM_ERR_NOT_INIT;
  if (variant < DARM_DIVERGENT || variant > DARM_AUTO) return DARM_ERR_INVALID_ARG;
  if (n == 0) return DARM_OK;
  if (bucket == 0 || (bucket & (bucket - 1)) != 0) return DARM_ERR_NOT_POW2;
  if (bucket > kPcmMaxBucket || n % bucket != 0 || !keys) return DARM_ERR_INVALID_ARG;
  const size_t nb = n / bucket;
  if ((nb & (nb - 1)) != 0) return DARM_ERR_NOT_POW2;
  if (nb > (size_t(1) << 31) || n > (size_t(1) << 32)) return DARM_ERR_INVALID_ARG;
  auto misaligned = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) != 0; };
  if (misaligned(keys) || (vals && misaligned(vals))) return DARM_ERR_INVALID_ARG;
  if (nb > 1 && (!scratch_keys || misaligned(scratch_keys) ||
                 (vals && (!scratch_vals || misaligned(scratch_vals)))))
    return DARM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = darm_oddeven_sort_buckets(keys, vals, n, bucket, variant, stream);
  if (rc != DARM_OK || nb == 1) return rc;

  const uint32_t S = uint32_t(bucket);
  const bool melded = variant != DARM_DIVERGENT;
  const bool hv = vals != nullptr;
  PcmLayer L{};
  L.k[0] = keys;
  L.k[1] = scratch_keys;
  L.v[0] = vals;
  L.v[1] = hv ? scratch_vals : nullptr;
  L.S = S;
  const uint32_t threads = uint32_t(std::max<size_t>(1, std::min<size_t>(kPcmThreads, 2 * S / kPcmPerThread)));
  const size_t smem = pcm_smem_bytes(hv, S);
  const bool q16 = S >= 256;  // 2S/16 >= 32 threads: the warp-summing kernel
  const void* fn =
      q16 ? (hv ? (melded ? reinterpret_cast<const void*>(&darm_pcm_layer16_kernel<true, 1>)
                          : reinterpret_cast<const void*>(&darm_pcm_layer16_kernel<true, 0>))
                : (melded ? reinterpret_cast<const void*>(&darm_pcm_layer16_kernel<false, 1>)
                          : reinterpret_cast<const void*>(&darm_pcm_layer16_kernel<false, 0>)))
          : (hv ? (melded ? reinterpret_cast<const void*>(&darm_pcm_layer_kernel<true, 1>)
                          : reinterpret_cast<const void*>(&darm_pcm_layer_kernel<true, 0>))
                : (melded ? reinterpret_cast<const void*>(&darm_pcm_layer_kernel<false, 1>)
                          : reinterpret_cast<const void*>(&darm_pcm_layer_kernel<false, 0>)));
  uint32_t nstages = 0;
  while ((size_t(1) << nstages) < nb) ++nstages;
  const uint32_t B = uint32_t(nb);
  for (uint32_t st = 0; st < nstages; ++st) {
    for (int t = int(st); t >= 0; --t) {
      L.s = st;
      L.t = uint32_t(t);
      const uint32_t ncmp = (uint32_t(t) == st) ? B / 2 : (B >> (st + 1)) * ((1u << st) - (1u << t));
      void* args[] = {&L};
      if (cudaLaunchKernel(fn, dim3(ncmp), dim3(threads), args, smem, s) != cudaSuccess)
        return DARM_ERR_CUDA;
      g_ctx.launches.fetch_add(1, std::memory_order_relaxed);
    }
  }
  void* gargs[] = {&L, &nstages};
  const void* gfn = hv ? reinterpret_cast<const void*>(&darm_pcm_gather_kernel<true>)
                       : reinterpret_cast<const void*>(&darm_pcm_gather_kernel<false>);
  if (cudaLaunchKernel(gfn, dim3(B), dim3(std::min<uint32_t>(256, S)), gargs, 0, s) != cudaSuccess)
    return DARM_ERR_CUDA;
  g_ctx.launches.fetch_add(1, std::memory_order_relaxed);
  return DARM_OK;
}
