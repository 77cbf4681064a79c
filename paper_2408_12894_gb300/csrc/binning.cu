// Tile binning. The sort key of a pair is (global tile id << 32) | float bits of its unit's
// view-space depth t_z (t_z > z_near > 0, so the bits order like the values). The depth half
// is sorted over units first (sort.cu, stage "units"); this file then walks the units in that
// order ("slots"): per-1024-slot pair counts, their exclusive scan, emission of each unit's
// tiles in row-major order with the 32-bit tile id as key, the stable sort of the tile half
// (stage "pairs"), and the per-tile [start, end) ranges of the result. Within a tile the
// pairs end up by depth with ties by unit index. Pair counts never leave the device: the
// scan writes the total and the partition count that the sort kernels read.
#include "common.cuh"
#include "kernels.h"

namespace flod {

// Pair count of every 1024 slots of the depth-sorted unit order.
__global__ void __launch_bounds__(256) k_block_sums(Ws ws) {
  __shared__ uint32_t red[8];
  const uint32_t* order = ws.uvals[ws.plan[kPlanFinalUnits]];
  const uint4 o = reinterpret_cast<const uint4*>(order)[blockIdx.x * 256u + threadIdx.x];
  uint32_t s = ws.tiles_touched[o.x] + ws.tiles_touched[o.y] + ws.tiles_touched[o.z] +
               ws.tiles_touched[o.w];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w];
    ws.block_sums[blockIdx.x] = t;
  }
}

// One CTA: exclusive scan of the block sums, pair total, partition count, counters reset.
__global__ void __launch_bounds__(1024) k_scan_blocks(Ws ws, uint32_t nblocks,
                                                      unsigned long long* user_count) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ uint32_t warp_sl[32];
  __shared__ unsigned long long carry_s;
  __shared__ uint32_t carry_sl;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    carry_s = 0;
    carry_sl = 0;
  }
  __syncthreads();
  for (uint32_t base = 0; base < nblocks; base += 1024) {
    const uint32_t i = base + tid;
    unsigned long long v = i < nblocks ? ws.block_sums[i] : 0ull;
    const uint32_t sl = (uint32_t)((v + kEmitSlice - 1) / kEmitSlice);   // emission slices
    unsigned long long x = v;
    uint32_t xs = sl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      uint32_t ys = __shfl_up_sync(0xffffffffu, xs, o);
      if (lane >= o) {
        x += y;
        xs += ys;
      }
    }
    if (lane == 31) {
      warp_tot[wid] = x;
      warp_sl[wid] = xs;
    }
    __syncthreads();
    if (wid == 0) {
      unsigned long long w = warp_tot[lane];
      uint32_t ws_ = warp_sl[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
        uint32_t ys = __shfl_up_sync(0xffffffffu, ws_, o);
        if (lane >= o) {
          w += y;
          ws_ += ys;
        }
      }
      warp_tot[lane] = w;   // inclusive over warps
      warp_sl[lane] = ws_;
    }
    __syncthreads();
    const unsigned long long carry = carry_s;
    const unsigned long long excl = carry + (wid ? warp_tot[wid - 1] : 0ull) + x - v;
    const uint32_t excl_sl = carry_sl + (wid ? warp_sl[wid - 1] : 0u) + xs - sl;
    if (i < nblocks) {
      ws.block_sums[i] = excl;
      ws.slices[i] = excl_sl;
    }
    __syncthreads();
    if (tid == 1023) {
      carry_s = excl + v;
      carry_sl = excl_sl + sl;
    }
    __syncthreads();
  }
  if (tid == 0) {
    const unsigned long long P = carry_s;
    *ws.pair_count = P;
    if (user_count) *user_count = P;
    unsigned long long pe = P;
    if (P > ws.pair_capacity) {
      set_status(ws.status, FLOD_DEV_CAPACITY);
      pe = ws.pair_capacity;
    }
    uint32_t nparts = (uint32_t)((pe + kSortPart - 1) / kSortPart);
    ws.plan[kPlanNParts] = nparts;
#pragma unroll
    for (int p = 4; p < kPlanPasses; ++p) ws.plan[kPlanCounter + p] = 0;   // pair-stage tickets
    ws.plan[kPlanQueue] = 0;
    ws.plan[kPlanQueue + 1] = 0;
    ws.plan[kPlanSlices] = carry_sl;
  }
}

// Key emission in depth-sorted unit order, load-balanced over output positions. Each
// 1024-slot block's contiguous range of pairs is cut into slices of kEmitSlice positions;
// persistent CTAs take slices in turn. For its slice a CTA rescans the block's 1024 pair
// counts in shared memory, fetches the tile rectangle of the units that overlap the slice,
// and its threads walk the slice's positions: position p belongs to the slot whose prefix
// range holds it (binary search in shared memory) and its tile is the (p - start)-th tile of
// that unit's rectangle in row-major order. Writes are coalesced, and a block of huge
// splats is spread over many CTAs.
template <int MAXV>
__global__ void __launch_bounds__(256) k_emit(const __grid_constant__ Batch<MAXV> b, Ws ws,
                                              uint32_t nblocks) {
  __shared__ uint32_t s_pre[kScanBlock + 1];
  __shared__ uint32_t s_rect[kScanBlock];     // tx0 | (rect width << 16)
  __shared__ uint32_t s_tile0[kScanBlock];    // global id of the rectangle's first row, column 0
  __shared__ uint32_t s_tx[kScanBlock];       // tiles per row of the unit's view
  __shared__ uint32_t warp_tot[8];
  __shared__ uint32_t s_blk;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t n_slices = ws.plan[kPlanSlices];
  const unsigned long long cap = ws.pair_capacity;
  const uint32_t* order = ws.uvals[ws.plan[kPlanFinalUnits]];
  uint32_t* keys = ws.keys[0];
  uint32_t* vals = ws.vals[0];
  for (uint32_t w = blockIdx.x; w < n_slices; w += gridDim.x) {
    if (tid == 0) {                       // the block holding slice w
      uint32_t lo = 0, hi = nblocks - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (ws.slices[mid] <= w) lo = mid; else hi = mid - 1;
      }
      s_blk = lo;
    }
    __syncthreads();
    const uint32_t blk = s_blk;
    const uint32_t r0 = (w - ws.slices[blk]) * (uint32_t)kEmitSlice;
    const uint4 un = reinterpret_cast<const uint4*>(order)[blk * 256u + tid];
    const uint32_t unit[4] = {un.x, un.y, un.z, un.w};
    uint32_t cnt[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) cnt[j] = ws.tiles_touched[unit[j]];
    const uint32_t s = cnt[0] + cnt[1] + cnt[2] + cnt[3];
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    uint32_t run = 0;
    for (int q = 0; q < wid; ++q) run += warp_tot[q];
    run += x - s;
    const uint32_t r1_full = r0 + (uint32_t)kEmitSlice;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int sl = 4 * tid + j;
      s_pre[sl] = run;
      if (cnt[j] && run < r1_full && run + cnt[j] > r0) {
        const uint32_t u = unit[j];
        const ViewP& V = b.views[view_of_unit(b, u)];
        const float2 xy = ws.xy[u];
        int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
        tile_rect(xy.x, xy.y, ws.radius[u], V.width, V.height, b.cfg.tile_w, b.cfg.tile_h, tx0,
                  tx1, ty0, ty1);
        s_rect[sl] = (uint32_t)tx0 | ((uint32_t)(tx1 - tx0 + 1) << 16);
        s_tile0[sl] = V.tile_off + (uint32_t)ty0 * V.tiles_x;
        s_tx[sl] = V.tiles_x;
      }
      run += cnt[j];
    }
    if (tid == 255) s_pre[kScanBlock] = run;
    __syncthreads();
    const uint32_t total = s_pre[kScanBlock];
    const uint32_t r1 = min(r1_full, total);
    const unsigned long long base = ws.block_sums[blk];
    for (uint32_t p = r0 + tid; p < r1; p += 256) {
      if (base + p >= cap) break;
      int lo = 0, hi = kScanBlock - 1;        // last slot with s_pre[slot] <= p
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pre[mid] <= p) lo = mid; else hi = mid - 1;
      }
      const uint32_t k = p - s_pre[lo];
      const uint32_t r = s_rect[lo];
      const uint32_t wdt = r >> 16;
      keys[base + p] = s_tile0[lo] + (k / wdt) * s_tx[lo] + (r & 0xffffu) + k % wdt;
      vals[base + p] = order[blk * (uint32_t)kScanBlock + lo];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_ranges(Ws ws) {
  const unsigned long long P0 = *ws.pair_count;
  const uint32_t P = (uint32_t)(P0 < ws.pair_capacity ? P0 : ws.pair_capacity);
  const uint32_t* keys = ws.keys[ws.plan[kPlanFinal]];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ws.ranges[t].x = i;
    if (i == P - 1 || keys[i + 1] != t) ws.ranges[t].y = i + 1;
  }
}

// Largest-first render order: every tile goes to bucket floor(log2(pairs)) + 1 (0 for an
// empty tile), buckets are laid out from the largest down, and tiles land in their bucket
// in arrival order. Persistent render CTAs then take the most expensive tiles first.
__global__ void __launch_bounds__(256) k_queue_count(Ws ws, uint32_t n_tiles) {
  __shared__ uint32_t h[33];
  if (threadIdx.x < 33) h[threadIdx.x] = 0;
  __syncthreads();
  for (uint32_t t = blockIdx.x * 256u + threadIdx.x; t < n_tiles; t += gridDim.x * 256u) {
    const uint2 r = ws.ranges[t];
    const uint32_t n = r.y - r.x;
    atomicAdd(&h[n ? 32 - __clz(n) : 0], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(&ws.queue[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_queue_offsets(Ws ws) {
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int bkt = 32; bkt >= 0; --bkt) {
      ws.queue[33 + bkt] = run;
      run += ws.queue[bkt];
    }
  }
}

__global__ void __launch_bounds__(256) k_queue_fill(Ws ws, uint32_t n_tiles) {
  for (uint32_t t = blockIdx.x * 256u + threadIdx.x; t < n_tiles; t += gridDim.x * 256u) {
    const uint2 r = ws.ranges[t];
    const uint32_t n = r.y - r.x;
    const uint32_t slot = atomicAdd(&ws.queue[33 + (n ? 32 - __clz(n) : 0)], 1u);
    ws.queue[kQueueHeader + slot] = t;
  }
}

template <int MAXV>
cudaError_t launch_binning(const Batch<MAXV>& b, const Ws& ws, int n_passes, int resident_sort,
                           int resident_small, unsigned long long* d_pair_count, bool build_queue,
                           cudaStream_t st) {
  const uint32_t nblocks = b.units / kScanBlock;
  cudaError_t e;
  if (b.tiles) {
    e = cudaMemsetAsync(ws.ranges, 0, sizeof(uint2) * b.tiles, st);
    if (e != cudaSuccess) return e;
  }
  if (nblocks) {
    if ((e = launch_unit_sort(ws, resident_small, resident_sort, st)) != cudaSuccess) return e;
    k_block_sums<<<nblocks, 256, 0, st>>>(ws);
  }
  k_scan_blocks<<<1, 1024, 0, st>>>(ws, nblocks, d_pair_count);
  if (nblocks) k_emit<MAXV><<<resident_small, 256, 0, st>>>(b, ws, nblocks);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_pair_sort(ws, n_passes, resident_small, resident_sort, st)) != cudaSuccess) return e;
  k_ranges<<<resident_small, 256, 0, st>>>(ws);
  if (build_queue && b.tiles) {
    if ((e = cudaMemsetAsync(ws.queue, 0, sizeof(uint32_t) * kQueueHeader, st)) != cudaSuccess)
      return e;
    const uint32_t g = min((uint32_t)resident_small, (b.tiles + 255) / 256);
    k_queue_count<<<g, 256, 0, st>>>(ws, b.tiles);
    k_queue_offsets<<<1, 32, 0, st>>>(ws);
    k_queue_fill<<<g, 256, 0, st>>>(ws, b.tiles);
  }
  return cudaGetLastError();
}

template cudaError_t launch_binning<kMaxViewsSmall>(const BatchS&, const Ws&, int, int, int,
                                                    unsigned long long*, bool, cudaStream_t);
template cudaError_t launch_binning<FLOD_MAX_VIEWS>(const BatchL&, const Ws&, int, int, int,
                                                    unsigned long long*, bool, cudaStream_t);

}  // namespace flod
