// Stable LSD radix sort of the (tile, depth) pairs, 9-bit digits, one "onesweep" pass per
// digit with decoupled look-back (Merrill & Garland's single-pass prefix scan, as used by
// onesweep sorting), all sizes read on the device.
//
// Every pair of a unit carries the same 32 depth bits, so the depth digits (the low half of
// the key) are sorted over units before any pair exists (stage "units": key = depth bits,
// value = unit); the pairs are then emitted in that order and only the tile digits (the
// high half) are sorted over the pairs (stage "pairs": key = tile id, value = unit). Both
// stages are stable and the units start in index order, so the result is the stable sort of
// (tile << 32 | depth bits) over pairs emitted in unit order: within a tile by depth, ties
// by unit index.
//
//   k_unit_keys  unit keys (depth bits, or all ones for a unit with no tile) and the digit
//                histograms of stage "units"; clears the first look-back table.
//   k_hist       the digit histograms of the pair keys; clears the first look-back table.
//   k_plan       per digit: exclusive digit offsets; a digit on which all keys agree is
//                marked inactive and costs nothing; ping-pong buffer and table per pass.
//   k_pass       persistent CTAs take 4096-key partitions in ticket order. Per partition:
//                warp-level ranking with one match.any per key (stable: lane, round, warp
//                order = input order), publish the per-digit counts (aggregate), reorder the
//                partition in shared memory, look back over predecessors until an inclusive
//                prefix is found, publish the inclusive prefix, write each digit's run.
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

// One sort stage: ping-pong key/value buffers, its element count and its plan slots.
struct Stage {
  uint32_t* keys[2];
  uint32_t* vals[2];
  const unsigned long long* count;   // device element count (pair stage), or NULL
  uint32_t fixed_count;              // element count when `count` is NULL (unit stage)
  uint64_t cap;                      // elements beyond cap are ignored
  int slot0;                         // first plan slot (digit d uses slot slot0 + d)
  int nparts_word;                   // plan word holding the partition count
  int final_word;                    // plan word receiving the result's buffer index
  uint32_t shifts;                   // digit d: bits [shift_d, shift_d + width_d) of the key,
  uint32_t widths;                   //   shift_d, width_d = byte d of shifts, widths
};

__device__ __forceinline__ uint32_t digit_of(uint32_t key, const Stage& s, int d) {
  const uint32_t sh = (s.shifts >> (8 * d)) & 0xffu, wd = (s.widths >> (8 * d)) & 0xffu;
  return (key >> sh) & ((1u << wd) - 1u);
}

__device__ __forceinline__ uint32_t stage_count(const Stage& s) {
  if (!s.count) return s.fixed_count;
  const unsigned long long c = *s.count;
  return (uint32_t)(c < s.cap ? c : s.cap);
}

__device__ __forceinline__ void block_hist_flush(const uint32_t* h, uint32_t* hist, int n_digits) {
  for (int i = threadIdx.x; i < n_digits * kRadixBins; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Stage "units": key = float bits of the view-space depth of a unit with tiles (positive, so
// the bits order like the values), all ones otherwise; value = unit index.
__global__ void __launch_bounds__(256) k_unit_keys(Ws ws, Stage st, int n_digits) {
  __shared__ uint32_t h[4 * kRadixBins];
  for (int i = threadIdx.x; i < 4 * kRadixBins; i += 256) h[i] = 0;
  __syncthreads();
  const uint32_t U = st.fixed_count;
  const uint32_t stride = gridDim.x * 256u;
  for (uint32_t u = blockIdx.x * 256u + threadIdx.x; u < U; u += stride) {
    const uint32_t key = ws.tiles_touched[u] ? __float_as_uint(ws.depth[u]) : 0xffffffffu;
    st.keys[0][u] = key;
    st.vals[0][u] = u;
    for (int d = 0; d < n_digits; ++d) atomicAdd(&h[d * kRadixBins + digit_of(key, st, d)], 1u);
  }
  __syncthreads();
  block_hist_flush(h, ws.hist + st.slot0 * kRadixBins, n_digits);
  const uint32_t nparts = (U + kSortPart - 1) / kSortPart;
  for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < nparts * (uint32_t)kRadixBins; i += stride)
    ws.lookback[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x < 4) ws.plan[kPlanCounter + st.slot0 + threadIdx.x] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) ws.plan[st.nparts_word] = nparts;
}

// Stage "pairs": histograms of the tile keys the emission wrote.
__global__ void __launch_bounds__(256) k_hist(Ws ws, Stage st, int n_digits) {
  __shared__ uint32_t h[4 * kRadixBins];
  for (int i = threadIdx.x; i < 4 * kRadixBins; i += 256) h[i] = 0;
  __syncthreads();
  const uint32_t P = stage_count(st);
  const uint32_t* keys = st.keys[0];
  const uint32_t stride = gridDim.x * 256u;
  for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < P; i += stride) {
    const uint32_t k = keys[i];
    for (int d = 0; d < n_digits; ++d) atomicAdd(&h[d * kRadixBins + digit_of(k, st, d)], 1u);
  }
  __syncthreads();
  block_hist_flush(h, ws.hist + st.slot0 * kRadixBins, n_digits);
  const uint32_t nparts = ws.plan[st.nparts_word];
  for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < nparts * (uint32_t)kRadixBins; i += stride)
    ws.lookback[i] = 0;
}

__global__ void __launch_bounds__(kRadixBins) k_plan(Ws ws, Stage st, int n_digits) {
  __shared__ uint32_t wsum[kRadixBins / 32];
  const uint32_t P = stage_count(st);
  const int d = threadIdx.x, lane = d & 31, wid = d >> 5;
  int src = 0, nact = 0;
  for (int p = 0; p < 4; ++p) {
    const int slot = st.slot0 + p;
    const uint32_t c = p < n_digits ? ws.hist[slot * kRadixBins + d] : 0u;
    const int one_bin = __syncthreads_or(c == P);
    const bool active = p < n_digits && P > 0 && !one_bin;
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
    ws.hist[slot * kRadixBins + d] = pre + x - c;
    __syncthreads();
    if (d == 0) {
      ws.plan[kPlanActive + slot] = active ? 1u : 0u;
      ws.plan[kPlanSrc + slot] = (uint32_t)src;
      ws.plan[kPlanLb + slot] = (uint32_t)(nact & 1);
    }
    if (active) {
      src ^= 1;
      ++nact;
    }
  }
  if (d == 0) ws.plan[st.final_word] = (uint32_t)src;
}

constexpr int kSortWarps = kSortThreads / 32;
static_assert(kSortThreads == kRadixBins, "one thread per digit value in the partition steps");

struct SortSmem {
  uint32_t keys[kSortPart];
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
__global__ void __launch_bounds__(kSortThreads, 2) k_pass(Ws ws, Stage st, int digit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
  const int slot = st.slot0 + digit;
  if (!ws.plan[kPlanActive + slot]) return;
  const int src = (int)ws.plan[kPlanSrc + slot];
  const int lbt = (int)ws.plan[kPlanLb + slot];
  const uint32_t* __restrict__ kin = src ? st.keys[1] : st.keys[0];
  const uint32_t* __restrict__ vin = src ? st.vals[1] : st.vals[0];
  uint32_t* __restrict__ kout = src ? st.keys[0] : st.keys[1];
  uint32_t* __restrict__ vout = src ? st.vals[0] : st.vals[1];
  const uint32_t P = stage_count(st);
  const uint32_t nparts = ws.plan[st.nparts_word];
  unsigned long long* lb = ws.lookback + (size_t)lbt * ws.max_parts * kRadixBins;
  unsigned long long* lb_next = ws.lookback + (size_t)(lbt ^ 1) * ws.max_parts * kRadixBins;
  const uint32_t* goff = ws.hist + slot * kRadixBins;
  const int shift = (int)((st.shifts >> (8 * digit)) & 0xffu);
  const uint32_t dmask = (1u << ((st.widths >> (8 * digit)) & 0xffu)) - 1u;
  const bool live_d = (uint32_t)threadIdx.x <= dmask;   // digit values this pass can take
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int d = tid;   // digit value owned in the partition steps

  for (;;) {
    if (tid == 0) sm.part = atomicAdd(&ws.plan[kPlanCounter + slot], 1u);
    for (int i = tid; i < kSortWarps * kRadixBins; i += kSortThreads) (&sm.whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t part = sm.part;
    if (part >= nparts) break;
    const uint32_t base = part * (uint32_t)kSortPart;
    const uint32_t wbase = base + wid * (32 * kSortKeysPerThread) + lane;

    uint32_t k[kSortKeysPerThread];
    uint32_t v[kSortKeysPerThread];
    uint32_t rank[kSortKeysPerThread];
#pragma unroll
    for (int r = 0; r < kSortKeysPerThread; ++r) {
      const uint32_t idx = wbase + r * 32;
      k[r] = idx < P ? kin[idx] : ~0u;
      v[r] = idx < P ? vin[idx] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kSortKeysPerThread; ++r) {
      const bool valid = wbase + r * 32 < P;
      const uint32_t dg = (k[r] >> shift) & dmask;
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
    // publish the aggregate (or the inclusive prefix for the first partition); values the
    // digit cannot take have no run and no look-back
    if (live_d) {
      if (part == 0) st_relaxed(lb + d, kFlagInc | total);
      else st_relaxed(lb + (size_t)part * kRadixBins + d, kFlagAgg | total);
    }
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
        const uint32_t dd = (k[r] >> shift) & dmask;
        const uint32_t pos = sm.local_start[dd] + sm.whist[wid][dd] + rank[r];
        sm.keys[pos] = k[r];
        sm.vals[pos] = v[r];
      }
    }
    // windowed look-back: read up to kWindow predecessors at once, nearest first; sum their
    // aggregates up to the nearest inclusive prefix; re-poll from the first one not ready
    unsigned long long excl = 0;
    if (part > 0 && live_d) {
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
      const uint32_t key = sm.keys[i];
      const uint32_t dd = (key >> shift) & dmask;
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

static Stage unit_stage(const Ws& ws) {
  Stage s;
  s.keys[0] = ws.ukeys[0];
  s.keys[1] = ws.ukeys[1];
  s.vals[0] = ws.uvals[0];
  s.vals[1] = ws.uvals[1];
  s.count = nullptr;
  s.fixed_count = ws.units;
  s.cap = ws.units;
  s.slot0 = 0;
  s.nparts_word = kPlanNPartsUnits;
  s.final_word = kPlanFinalUnits;
  s.shifts = 0x18100800u;   // four 8-bit digits of the 32 depth bits
  s.widths = 0x08080808u;
  return s;
}

// The tile bits split into n_digits digits of near-equal width (each at most 9 bits).
static Stage pair_stage(const Ws& ws, int n_digits, int tile_bits) {
  Stage s;
  s.keys[0] = ws.keys[0];
  s.keys[1] = ws.keys[1];
  s.vals[0] = ws.vals[0];
  s.vals[1] = ws.vals[1];
  s.count = ws.pair_count;
  s.fixed_count = 0;
  s.cap = ws.pair_capacity;
  s.slot0 = 4;
  s.nparts_word = kPlanNParts;
  s.final_word = kPlanFinal;
  s.shifts = s.widths = 0;
  int shift = 0;
  for (int d = 0; d < n_digits; ++d) {
    const int w = tile_bits / n_digits + (d < tile_bits % n_digits ? 1 : 0);
    s.shifts |= (uint32_t)shift << (8 * d);
    s.widths |= (uint32_t)w << (8 * d);
    shift += w;
  }
  return s;
}

// Stage "units": depth digits (32 bits -> 4 passes of 8 bits).
cudaError_t launch_unit_sort(const Ws& ws, int resident_small, int resident_sort, cudaStream_t st) {
  const Stage s = unit_stage(ws);
  const int n_digits = 4;
  cudaError_t e = cudaMemsetAsync(ws.hist, 0, sizeof(uint32_t) * 4 * kRadixBins, st);
  if (e != cudaSuccess) return e;
  k_unit_keys<<<resident_small, 256, 0, st>>>(ws, s, n_digits);
  k_plan<<<1, kRadixBins, 0, st>>>(ws, s, n_digits);
  for (int p = 0; p < n_digits; ++p)
    k_pass<<<resident_sort, kSortThreads, sizeof(SortSmem), st>>>(ws, s, p);
  return cudaGetLastError();
}

// Stage "pairs": tile digits (n_digits passes over the emitted pairs).
cudaError_t launch_pair_sort(const Ws& ws, int n_digits, int tile_bits, int resident_small,
                             int resident_sort, cudaStream_t st) {
  const Stage s = pair_stage(ws, n_digits, tile_bits);
  cudaError_t e = cudaMemsetAsync(ws.hist + 4 * kRadixBins, 0, sizeof(uint32_t) * 4 * kRadixBins, st);
  if (e != cudaSuccess) return e;
  k_hist<<<resident_small, 256, 0, st>>>(ws, s, n_digits);
  k_plan<<<1, kRadixBins, 0, st>>>(ws, s, n_digits);
  for (int p = 0; p < n_digits; ++p)
    k_pass<<<resident_sort, kSortThreads, sizeof(SortSmem), st>>>(ws, s, p);
  return cudaGetLastError();
}

}  // namespace flod
