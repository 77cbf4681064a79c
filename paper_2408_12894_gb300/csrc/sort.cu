// Stable LSD radix sort of the (tile, depth) pairs, all sizes read on the device.
//
// Every pair of a unit carries the same 32 depth bits, so the depth digits (the low half of
// the key) are sorted over units before any pair exists (stage "units": key = depth bits,
// value = unit); the pairs are then emitted in that order and only the tile digits (the
// high half) are sorted over the pairs (stage "pairs": key = tile id, value = unit). Both
// stages are stable and the units start in index order, so the result is the stable sort of
// (tile << 32 | depth bits) over pairs emitted in unit order: within a tile by depth, ties
// by unit index.
//
// Each digit is one reduce-then-scan pass over 4,096-key partitions (the classic
// three-phase radix pass, with the scan spread over one CTA per digit value):
//   k_count  per partition, its digit histogram -> counts[digit value][partition]
//   k_scan   one CTA per digit value: exclusive scan of its counts over the partitions and
//            their total; the CTA that finishes last (a ticket, nothing waits) turns the
//            totals into digit bases and writes the pass plan: whether the pass moves keys
//            (a digit on which all keys agree costs no scatter), its source buffer, the next
//            pass's source
//   k_pass   per partition: warp-level ranking, the lanes of equal digit found with one
//            ballot per digit bit (stable: lane, round, warp order = input order), digit
//            offsets within the partition, reorder in shared memory, and a coalesced
//            scatter of each digit's run to base[digit] + counts[digit][partition] + offset.
// No CTA ever waits for another, so no pass can hang on a CTA that is not scheduled.
#include "common.cuh"
#include "kernels.h"

namespace flod {

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
  int keybits_word;                  // plan word with the keys' significant bits, or -1
};

// Whether digit d has any significant key bits (digits above them are skipped outright).
__device__ __forceinline__ bool digit_live(const Ws& ws, const Stage& s, int d) {
  return s.keybits_word < 0 || ((s.shifts >> (8 * d)) & 0xffu) < ws.plan[s.keybits_word];
}

__device__ __forceinline__ uint32_t stage_count(const Stage& s) {
  if (!s.count) return s.fixed_count;
  const unsigned long long c = *s.count;
  return (uint32_t)(c < s.cap ? c : s.cap);
}

__device__ __forceinline__ const uint32_t* src_keys(const Stage& s, int src) {
  return src ? s.keys[1] : s.keys[0];
}

// Stage "units": only units with tiles take part. Per 1024 units their count and the
// smallest and largest depth bits (k_vis_count), an exclusive scan of those counts with the
// total (k_vis_scan, one CTA; the total is the stage's element count), then the keys in unit
// order (k_unit_keys): key = float bits of the view-space depth minus the smallest (depths
// are positive, so the bits order like the values, and the difference keeps that order with
// fewer significant bits: digits above them are skipped), value = unit index.
__global__ void __launch_bounds__(256) k_vis_count(Ws ws, uint32_t n_tiles) {
  pdl_entry();
  // the tile ranges of this frame start empty (k_ranges sets those of tiles with pairs)
  for (uint32_t t = blockIdx.x * 256u + threadIdx.x; t < n_tiles; t += gridDim.x * 256u)
    ws.ranges[t] = make_uint2(0u, 0u);
  __shared__ uint32_t red[3][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t i4 = blockIdx.x * 256u + threadIdx.x;
  const uint4 t = reinterpret_cast<const uint4*>(ws.tiles_touched)[i4];
  const uint4 d = reinterpret_cast<const uint4*>(ws.depth)[i4];   // the float bits
  const uint32_t vis[4] = {t.x != 0, t.y != 0, t.z != 0, t.w != 0};
  const uint32_t bits[4] = {d.x, d.y, d.z, d.w};
  uint32_t s = 0, lo = 0xffffffffu, hi = 0u;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (!vis[j]) continue;
    ++s;
    lo = min(lo, bits[j]);
    hi = max(hi, bits[j]);
  }
  s = __reduce_add_sync(0xffffffffu, s);
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if (lane == 0) {
    red[0][wid] = s;
    red[1][wid] = lo;
    red[2][wid] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t c = 0, l = 0xffffffffu, h = 0u;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      c += red[0][w];
      l = min(l, red[1][w]);
      h = max(h, red[2][w]);
    }
    ws.slices[blockIdx.x] = c;
    ws.block_sums[blockIdx.x] = (unsigned long long)h << 32 | l;   // scratch until the scan
  }
}

__global__ void __launch_bounds__(1024) k_vis_scan(Ws ws, Stage st, uint32_t nblocks) {
  pdl_entry();
  __shared__ uint32_t warp_tot[32], warp_lo[32], warp_hi[32];
  __shared__ uint32_t s_carry, s_lo, s_hi;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    s_carry = 0;
    s_lo = 0xffffffffu;
    s_hi = 0u;
  }
  __syncthreads();
  for (uint32_t b0 = 0; b0 < nblocks; b0 += 1024) {
    const uint32_t i = b0 + tid;
    const uint32_t v = i < nblocks ? ws.slices[i] : 0u;
    const unsigned long long mm = i < nblocks ? ws.block_sums[i] : 0xffffffffull;
    const uint32_t lo = __reduce_min_sync(0xffffffffu, (uint32_t)mm);
    const uint32_t hi = __reduce_max_sync(0xffffffffu, (uint32_t)(mm >> 32));
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    if (lane == 0) {
      warp_lo[wid] = lo;
      warp_hi[wid] = hi;
    }
    __syncthreads();
    uint32_t pre = s_carry, all = 0;
    for (int q = 0; q < 32; ++q) {
      if (q < wid) pre += warp_tot[q];
      all += warp_tot[q];
    }
    if (i < nblocks) ws.slices[i] = pre + x - v;
    __syncthreads();
    if (tid == 0) {
      s_carry += all;
      for (int q = 0; q < 32; ++q) {
        s_lo = min(s_lo, warp_lo[q]);
        s_hi = max(s_hi, warp_hi[q]);
      }
    }
    __syncthreads();
  }
  if (tid < 4) ws.plan[kPlanCounter + st.slot0 + tid] = 0;
  if (tid == 0) {
    // keys become depth bits minus the smallest: same order, fewer significant bits
    const uint32_t span = (s_carry && s_hi >= s_lo) ? s_hi - s_lo : 0u;
    ws.plan[kPlanDepthMin] = s_lo;
    ws.plan[kPlanKeyBits] = span ? 32u - (uint32_t)__clz(span) : 0u;
    *reinterpret_cast<unsigned long long*>(ws.plan + kPlanNVis) = s_carry;
    ws.plan[st.nparts_word] = (s_carry + kSortPart - 1) / kSortPart;
    ws.plan[kPlanSrc + st.slot0] = 0;
  }
}

__global__ void __launch_bounds__(256) k_unit_keys(Ws ws, Stage st) {
  pdl_entry();
  __shared__ uint32_t red[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t u0 = blockIdx.x * 1024u + 4u * tid;
  const uint4 t = reinterpret_cast<const uint4*>(ws.tiles_touched)[blockIdx.x * 256u + tid];
  const uint32_t vis[4] = {t.x != 0, t.y != 0, t.z != 0, t.w != 0};
  const uint32_t s = vis[0] + vis[1] + vis[2] + vis[3];
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) red[wid] = x;
  __syncthreads();
  uint32_t pos = ws.slices[blockIdx.x] + x - s;
  for (int q = 0; q < wid; ++q) pos += red[q];
  const uint32_t lo = ws.plan[kPlanDepthMin];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (!vis[j]) continue;
    st.keys[0][pos] = __float_as_uint(ws.depth[u0 + j]) - lo;
    st.vals[0][pos] = u0 + j;
    ++pos;
  }
}

// Phase 1: digit histogram of every partition, stored digit-major.
__global__ void __launch_bounds__(256) k_count(Ws ws, Stage st, int digit) {
  pdl_entry();
  __shared__ uint32_t h[8][kRadixBins];   // one histogram per warp (fewer colliding atomics)
  if (!digit_live(ws, st, digit)) return;
  const int slot = st.slot0 + digit;
  const uint32_t* __restrict__ kin = src_keys(st, (int)ws.plan[kPlanSrc + slot]);
  const uint32_t P = stage_count(st);
  const uint32_t nparts = ws.plan[st.nparts_word];
  const int shift = (int)((st.shifts >> (8 * digit)) & 0xffu);
  const uint32_t width = (st.widths >> (8 * digit)) & 0xffu;
  const uint32_t dmask = (1u << width) - 1u, nbins = 1u << width;
  const int tid = threadIdx.x;
  uint32_t* hw = h[tid >> 5];
  for (uint32_t part = blockIdx.x; part < nparts; part += gridDim.x) {
    for (uint32_t d = tid; d < 8 * nbins; d += 256) h[d / nbins][d % nbins] = 0;
    __syncthreads();
    const uint32_t base = part * (uint32_t)kSortPart;
#pragma unroll
    for (int r = 0; r < kSortPart / 1024; ++r) {    // 16 keys per thread, 16-byte loads
      const uint32_t i = base + 4u * (r * 256u + tid);
      if (i + 3 < P) {
        const uint4 v = reinterpret_cast<const uint4*>(kin)[i >> 2];
        atomicAdd(&hw[(v.x >> shift) & dmask], 1u);
        atomicAdd(&hw[(v.y >> shift) & dmask], 1u);
        atomicAdd(&hw[(v.z >> shift) & dmask], 1u);
        atomicAdd(&hw[(v.w >> shift) & dmask], 1u);
      } else {
        for (uint32_t j = 0; j < 4; ++j)
          if (i + j < P) atomicAdd(&hw[(kin[i + j] >> shift) & dmask], 1u);
      }
    }
    __syncthreads();
    for (uint32_t d = tid; d < nbins; d += 256) {
      uint32_t c = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) c += h[w][d];
      ws.counts[(size_t)d * ws.max_parts + part] = c;
    }
    __syncthreads();
  }
}

// Phase 2: one CTA per digit value (grid = 2^width): exclusive scan of its partition counts
// in place and its total; the last CTA to finish writes the digit bases and the pass plan.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_scan(Ws ws, Stage st, int digit, int last) {
  pdl_entry();
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  __shared__ uint32_t s_carry;
  __shared__ int s_last;
  const int slot = st.slot0 + digit;
  const uint32_t nparts = ws.plan[st.nparts_word];
  const uint32_t nbins = 1u << ((st.widths >> (8 * digit)) & 0xffu);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint32_t* col = ws.counts + (size_t)blockIdx.x * ws.max_parts;
  uint32_t* tot = ws.hist + slot * kRadixBins;
  if (!digit_live(ws, st, digit)) {   // all keys agree on this digit: the pass moves nothing
    if (blockIdx.x == 0 && tid == 0) {
      const uint32_t src = ws.plan[kPlanSrc + slot];
      ws.plan[kPlanActive + slot] = 0;
      if (last) ws.plan[st.final_word] = src;
      else ws.plan[kPlanSrc + slot + 1] = src;
    }
    return;
  }
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < nparts; b0 += 4u * kScanThreads) {
    uint32_t v[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t i = b0 + 4u * tid + j;
      v[j] = i < nparts ? col[i] : 0u;
      s += v[j];
    }
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    uint32_t run = s_carry, all = 0;
    for (int q = 0; q < kScanThreads / 32; ++q) {
      if (q < wid) run += warp_tot[q];
      all += warp_tot[q];
    }
    run += x - s;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t i = b0 + 4u * tid + j;
      if (i < nparts) col[i] = run;
      run += v[j];
    }
    __syncthreads();
    if (tid == 0) s_carry += all;
    __syncthreads();
  }
  if (tid == 0) {
    tot[blockIdx.x] = s_carry;
    __threadfence();
    s_last = atomicAdd(&ws.plan[kPlanCounter + slot], 1u) == nbins - 1;
  }
  __syncthreads();
  if (!s_last) return;
  // the last CTA: totals -> exclusive digit bases; the plan of this pass
  __threadfence();
  const uint32_t P = stage_count(st);
  const uint32_t t = (uint32_t)tid < nbins ? reinterpret_cast<volatile uint32_t*>(tot)[tid] : 0u;
  const int one_bin = __syncthreads_or(t == P);
  uint32_t x = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  uint32_t pre = 0;
  for (int q = 0; q < wid; ++q) pre += warp_tot[q];
  if ((uint32_t)tid < nbins) tot[tid] = pre + x - t;
  if (tid == 0) {
    const uint32_t active = (P > 0 && !one_bin) ? 1u : 0u;
    const uint32_t src = ws.plan[kPlanSrc + slot];
    ws.plan[kPlanActive + slot] = active;
    if (last) ws.plan[st.final_word] = src ^ active;
    else ws.plan[kPlanSrc + slot + 1] = src ^ active;
  }
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
};

// Phase 3. kSortThreads threads, kSortKeysPerThread keys each: warp w ranks the
// 32 * kSortKeysPerThread consecutive keys starting at w * 32 * kSortKeysPerThread, round by
// round, so (warp, round, lane) order is input order and the ranking is stable. Thread d
// then owns digit value d for the partition-level steps.
// W: the digit's width in bits, a compile-time constant so that the ranking's ballot loop
// unrolls (one instantiation per width 1..9).
template <int W>
__global__ void __launch_bounds__(kSortThreads, 2) k_pass(Ws ws, Stage st, int digit) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
  const int slot = st.slot0 + digit;
  if (!ws.plan[kPlanActive + slot]) return;
  const int src = (int)ws.plan[kPlanSrc + slot];
  const uint32_t* __restrict__ kin = src ? st.keys[1] : st.keys[0];
  const uint32_t* __restrict__ vin = src ? st.vals[1] : st.vals[0];
  uint32_t* __restrict__ kout = src ? st.keys[0] : st.keys[1];
  uint32_t* __restrict__ vout = src ? st.vals[0] : st.vals[1];
  const uint32_t P = stage_count(st);
  const uint32_t nparts = ws.plan[st.nparts_word];
  const uint32_t* goff = ws.hist + slot * kRadixBins;
  const int shift = (int)((st.shifts >> (8 * digit)) & 0xffu);
  constexpr int width = W;
  constexpr uint32_t dmask = (1u << W) - 1u;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int d = tid;   // digit value owned in the partition steps

  for (uint32_t part = blockIdx.x; part < nparts; part += gridDim.x) {
    for (int i = tid; i < (kSortWarps << width); i += kSortThreads)   // the bins this digit has
      sm.whist[i >> width][i & dmask] = 0;
    // this partition's global offset of every digit value (the scan of phase 2)
    if ((uint32_t)d <= dmask) sm.gbase[d] = goff[d] + ws.counts[(size_t)d * ws.max_parts + part];
    __syncthreads();
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
      // lanes holding the same digit, one ballot per digit bit (valid lanes only)
      uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
      for (int b = 0; b < width; ++b) {
        const bool bit = (dg >> b) & 1u;
        const uint32_t m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
      }
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
    if ((uint32_t)d <= dmask) {
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = sm.whist[w][d];
        sm.whist[w][d] = total;
        total += c;
      }
    }
    uint32_t x = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
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
    // reorder the partition in shared memory
#pragma unroll
    for (int r = 0; r < kSortKeysPerThread; ++r) {
      if (wbase + r * 32 < P) {
        const uint32_t dd = (k[r] >> shift) & dmask;
        const uint32_t pos = sm.local_start[dd] + sm.whist[wid][dd] + rank[r];
        sm.keys[pos] = k[r];
        sm.vals[pos] = v[r];
      }
    }
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

// The scatter kernel of each digit width (1..9 bits).
using PassFn = void (*)(Ws, Stage, int);
static const PassFn kPassFns[10] = {nullptr,   k_pass<1>, k_pass<2>, k_pass<3>, k_pass<4>,
                                    k_pass<5>, k_pass<6>, k_pass<7>, k_pass<8>, k_pass<9>};

cudaError_t sort_kernel_prepare() {
  for (int w = 1; w <= 9; ++w) {
    const cudaError_t e = cudaFuncSetAttribute(kPassFns[w], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)sizeof(SortSmem));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Occupancy is taken from the 8-bit instantiation (every width has the same launch shape
// and shared memory, and at most the registers that two CTAs per SM allow).
const void* sort_kernel_ptr() { return reinterpret_cast<const void*>(kPassFns[8]); }

static Stage unit_stage(const Ws& ws) {
  Stage s;
  s.keys[0] = ws.ukeys[0];
  s.keys[1] = ws.ukeys[1];
  s.vals[0] = ws.uvals[0];
  s.vals[1] = ws.uvals[1];
  s.count = reinterpret_cast<const unsigned long long*>(ws.plan + kPlanNVis);
  s.fixed_count = 0;
  s.cap = ws.units;
  s.slot0 = 0;
  s.nparts_word = kPlanNPartsUnits;
  s.final_word = kPlanFinalUnits;
  s.shifts = 0x18100800u;   // four 8-bit digits of the 32 depth bits
  s.widths = 0x08080808u;
  s.keybits_word = kPlanKeyBits;
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
  s.keybits_word = -1;
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

static cudaError_t run_passes(const Ws& ws, const Stage& s, int n_digits, int resident_small,
                              int resident_sort, cudaStream_t st) {
  for (int p = 0; p < n_digits; ++p) {
    const int width = (int)((s.widths >> (8 * p)) & 0xffu);
    if (width < 1 || width > 9) return cudaErrorInvalidValue;
    const uint32_t nbins = 1u << width;
    launch_k(k_count, dim3(resident_small), dim3(256), 0, st, ws, s, p);
    launch_k(k_scan, dim3(nbins), dim3(kScanThreads), 0, st, ws, s, p, p + 1 == n_digits ? 1 : 0);
    launch_k(kPassFns[width], dim3(resident_sort), dim3(kSortThreads), sizeof(SortSmem), st, ws, s, p);
  }
  return cudaGetLastError();
}

// Stage "units": depth digits (32 bits -> 4 passes of 8 bits) of the units with tiles.
cudaError_t launch_unit_sort(const Ws& ws, uint32_t n_tiles, int resident_small, int resident_sort,
                             cudaStream_t st) {
  const Stage s = unit_stage(ws);
  const uint32_t nblocks = ws.units / kScanBlock;
  launch_k(k_vis_count, dim3(nblocks), dim3(256), 0, st, ws, n_tiles);
  launch_k(k_vis_scan, dim3(1), dim3(1024), 0, st, ws, s, nblocks);
  launch_k(k_unit_keys, dim3(nblocks), dim3(256), 0, st, ws, s);
  return run_passes(ws, s, 4, resident_small, resident_sort, st);
}

// Stage "pairs": tile digits (n_digits passes over the emitted pairs). The emission's scan
// kernel has reset the stage's plan words.
cudaError_t launch_pair_sort(const Ws& ws, int n_digits, int tile_bits, int resident_small,
                             int resident_sort, cudaStream_t st) {
  return run_passes(ws, pair_stage(ws, n_digits, tile_bits), n_digits, resident_small,
                    resident_sort, st);
}

}  // namespace flod
