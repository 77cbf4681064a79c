// Stable LSD radix sort of the (tile, depth) pairs: 9-bit digits (512 values; 45-bit keys of
// a 1080p frame take 5 passes), one "onesweep" pass per digit with decoupled look-back (Merrill & Garland's single-pass prefix scan, as used by
// onesweep sorting), all sizes read on the device.
//
//   k_hist   one read of all keys: the histograms of every digit at once; clears the first
//            look-back table.
//   k_plan   per digit: exclusive digit offsets; a digit on which all keys agree is marked
//            inactive and costs nothing; ping-pong buffer and look-back table per pass.
//   k_pass   persistent CTAs take 4096-key partitions in ticket order. Per partition:
//            warp-level ranking with one match.any per key (stable: lane, round, warp order =
//            input order), publish the per-digit counts (aggregate), look back over
//            predecessors until an inclusive prefix is found, publish the inclusive prefix,
//            reorder the partition in shared memory and write each digit's run contiguously.
//
// Every wait on a predecessor is bounded; when the bound is hit the kernel sets
// FLOD_DEV_TIMEOUT in the status word and continues (the output is then invalid, the
// caller sees the status).
#include "common.cuh"
#include "kernels.h"

namespace flod {

// look-back words: 2 flag bits over a 62-bit count
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1ull;
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr int kWindow = 8;         // predecessors read per look-back step

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void __launch_bounds__(256) k_hist(Ws ws, int n_passes) {
  __shared__ uint32_t h[kPlanPasses * kRadixBins];
  for (int i = threadIdx.x; i < kPlanPasses * kRadixBins; i += 256) h[i] = 0;
  __syncthreads();
  const unsigned long long P0 = *ws.pair_count;
  const uint32_t P = (uint32_t)(P0 < ws.pair_capacity ? P0 : ws.pair_capacity);
  const unsigned long long* keys = ws.keys[0];
  const uint32_t stride = gridDim.x * 256u;
  for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < P; i += stride) {
    const unsigned long long k = keys[i];
    for (int p = 0; p < n_passes; ++p)
      atomicAdd(&h[p * kRadixBins + (uint32_t)((k >> (kRadixBits * p)) & (kRadixBins - 1))], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_passes * kRadixBins; i += 256)
    if (h[i]) atomicAdd(&ws.hist[i], h[i]);
  const uint32_t nparts = ws.plan[kPlanNParts];
  for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < nparts * (uint32_t)kRadixBins; i += stride)
    ws.lookback[i] = 0;
}

__global__ void __launch_bounds__(kRadixBins) k_plan(Ws ws, int n_passes) {
  __shared__ uint32_t wsum[kRadixBins / 32];
  const unsigned long long P0 = *ws.pair_count;
  const uint32_t P = (uint32_t)(P0 < ws.pair_capacity ? P0 : ws.pair_capacity);
  const int d = threadIdx.x, lane = d & 31, wid = d >> 5;
  int src = 0, nact = 0;
  for (int p = 0; p < n_passes; ++p) {
    const uint32_t c = ws.hist[p * kRadixBins + d];
    const int one_bin = __syncthreads_or(c == P);
    const bool active = P > 0 && !one_bin;
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < wid; ++w) pre += wsum[w];
    ws.hist[p * kRadixBins + d] = pre + x - c;
    __syncthreads();
    if (d == 0) {
      ws.plan[kPlanActive + p] = active ? 1u : 0u;
      ws.plan[kPlanSrc + p] = (uint32_t)src;
      ws.plan[kPlanLb + p] = (uint32_t)(nact & 1);
    }
    if (active) {
      src ^= 1;
      ++nact;
    }
  }
  for (int p = n_passes + d; p < kPlanPasses; p += kRadixBins) {
    if (p >= n_passes) ws.plan[kPlanActive + p] = 0;
  }
  if (d == 0) ws.plan[kPlanFinal] = (uint32_t)src;
}

constexpr int kSortWarps = kSortThreads / 32;
static_assert(kSortThreads == kRadixBins, "one thread per digit value in the partition steps");

struct SortSmem {
  unsigned long long keys[kSortPart];
  uint32_t vals[kSortPart];
  uint32_t whist[kSortWarps][kRadixBins];   // per-warp digit counts, then per-warp prefixes
  uint32_t local_start[kRadixBins];
  uint32_t gbase[kRadixBins];
  uint32_t wsum[kSortWarps];
  uint32_t part;
};

// One digit pass. kSortThreads threads, kSortKeysPerThread keys each: warp w ranks the
// 32 * kSortKeysPerThread consecutive keys starting at w * 32 * kSortKeysPerThread, round by
// round, so (warp, round, lane) order is input order and the ranking is stable. Thread d
// then owns digit value d for the partition-level steps.
__global__ void __launch_bounds__(kSortThreads, 2) k_pass(Ws ws, int pass) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
  if (!ws.plan[kPlanActive + pass]) return;
  const int src = (int)ws.plan[kPlanSrc + pass];
  const int lbt = (int)ws.plan[kPlanLb + pass];
  const unsigned long long* __restrict__ kin = ws.keys[src];
  const uint32_t* __restrict__ vin = ws.vals[src];
  unsigned long long* __restrict__ kout = ws.keys[src ^ 1];
  uint32_t* __restrict__ vout = ws.vals[src ^ 1];
  const unsigned long long P0 = *ws.pair_count;
  const uint32_t P = (uint32_t)(P0 < ws.pair_capacity ? P0 : ws.pair_capacity);
  const uint32_t nparts = ws.plan[kPlanNParts];
  unsigned long long* lb = ws.lookback + (size_t)lbt * ws.max_parts * kRadixBins;
  unsigned long long* lb_next = ws.lookback + (size_t)(lbt ^ 1) * ws.max_parts * kRadixBins;
  const uint32_t* goff = ws.hist + pass * kRadixBins;
  const int shift = kRadixBits * pass;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int d = tid;   // digit value owned in the partition steps

  for (;;) {
    if (tid == 0) sm.part = atomicAdd(&ws.plan[kPlanCounter + pass], 1u);
    for (int i = tid; i < kSortWarps * kRadixBins; i += kSortThreads) (&sm.whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t part = sm.part;
    if (part >= nparts) break;
    const uint32_t base = part * (uint32_t)kSortPart;
    const uint32_t wbase = base + wid * (32 * kSortKeysPerThread) + lane;

    unsigned long long k[kSortKeysPerThread];
    uint32_t v[kSortKeysPerThread];
    uint32_t rank[kSortKeysPerThread];
#pragma unroll
    for (int r = 0; r < kSortKeysPerThread; ++r) {
      const uint32_t idx = wbase + r * 32;
      k[r] = idx < P ? kin[idx] : ~0ull;
      v[r] = idx < P ? vin[idx] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kSortKeysPerThread; ++r) {
      const bool valid = wbase + r * 32 < P;
      const uint32_t dg = (uint32_t)(k[r] >> shift) & (kRadixBins - 1);
      // lanes holding the same digit (a lane past the end matches only itself)
      const uint32_t peers = __match_any_sync(0xffffffffu, valid ? dg : 0x10000u | (uint32_t)lane);
      uint32_t before = 0;
      if (valid) before = sm.whist[wid][dg];
      __syncwarp();
      if (valid && (peers & lt_mask) == 0) sm.whist[wid][dg] = before + __popc(peers);
      __syncwarp();
      rank[r] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    // digit d: exclusive prefix over warps and the partition's digit total
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = sm.whist[w][d];
      sm.whist[w][d] = total;
      total += c;
    }
    // publish the aggregate (or the inclusive prefix for the first partition)
    if (part == 0) st_relaxed(lb + d, kFlagInc | total);
    else st_relaxed(lb + (size_t)part * kRadixBins + d, kFlagAgg | total);
    lb_next[(size_t)part * kRadixBins + d] = 0;
    uint32_t x = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sm.wsum[wid] = x;
    __syncthreads();
    {
      uint32_t pre = 0;
      for (int w = 0; w < wid; ++w) pre += sm.wsum[w];
      sm.local_start[d] = pre + x - total;
    }
    __syncthreads();
    // reorder the partition in shared memory (needs no global offset)
#pragma unroll
    for (int r = 0; r < kSortKeysPerThread; ++r) {
      if (wbase + r * 32 < P) {
        const uint32_t dd = (uint32_t)(k[r] >> shift) & (kRadixBins - 1);
        const uint32_t pos = sm.local_start[dd] + sm.whist[wid][dd] + rank[r];
        sm.keys[pos] = k[r];
        sm.vals[pos] = v[r];
      }
    }
    // windowed look-back: read up to kWindow predecessors at once, nearest first; sum their
    // aggregates up to the nearest inclusive prefix; re-poll from the first one not ready
    unsigned long long excl = 0;
    if (part > 0) {
      int q = (int)part - 1;
      uint32_t spins = 0;
      bool done = false;
      while (!done && q >= 0) {
        unsigned long long wv[kWindow];
#pragma unroll
        for (int i = 0; i < kWindow; ++i)
          wv[i] = (q - i >= 0) ? ld_relaxed(lb + (size_t)(q - i) * kRadixBins + d) : kFlagInc;
        int consumed = 0;
        bool stalled = false;
#pragma unroll
        for (int i = 0; i < kWindow; ++i) {
          if (done || stalled) continue;
          const unsigned long long flag = wv[i] & ~kValMask;
          if (flag == 0) {
            stalled = true;
            continue;
          }
          if (q - i >= 0) excl += wv[i] & kValMask;
          ++consumed;
          if (flag == kFlagInc) done = true;
        }
        q -= consumed;
        if (stalled && !done) {
          if (++spins > kSpinLimit) {
            set_status(ws.status, FLOD_DEV_TIMEOUT);
            break;
          }
          if (spins > 8) __nanosleep(64);
        }
      }
      st_relaxed(lb + (size_t)part * kRadixBins + d, kFlagInc | ((excl + total) & kValMask));
    }
    sm.gbase[d] = goff[d] + (uint32_t)excl;
    __syncthreads();
    const uint32_t nvalid = min((uint32_t)kSortPart, P - base);
    for (uint32_t i = tid; i < nvalid; i += kSortThreads) {
      const unsigned long long key = sm.keys[i];
      const uint32_t dd = (uint32_t)(key >> shift) & (kRadixBins - 1);
      const uint32_t dst = sm.gbase[dd] + (i - sm.local_start[dd]);
      kout[dst] = key;
      vout[dst] = sm.vals[i];
    }
    __syncthreads();
  }
}

int sort_kernel_smem_bytes() { return (int)sizeof(SortSmem); }

cudaError_t sort_kernel_prepare() {
  return cudaFuncSetAttribute(k_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(SortSmem));
}

const void* sort_kernel_ptr() { return reinterpret_cast<const void*>(&k_pass); }

cudaError_t launch_radix_sort(const Ws& ws, int n_passes, int resident_hist, int resident_sort,
                              cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ws.hist, 0, sizeof(uint32_t) * kPlanPasses * kRadixBins, st);
  if (e != cudaSuccess) return e;
  k_hist<<<resident_hist, 256, 0, st>>>(ws, n_passes);
  k_plan<<<1, kRadixBins, 0, st>>>(ws, n_passes);
  for (int p = 0; p < n_passes; ++p)
    k_pass<<<resident_sort, kSortThreads, sizeof(SortSmem), st>>>(ws, p);
  return cudaGetLastError();
}

}  // namespace flod
