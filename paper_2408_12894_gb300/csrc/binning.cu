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

constexpr uint32_t kLightPairs = 16 * kEmitSlice;   // blocks up to this many pairs: k_emit_light
constexpr uint32_t kBigPerGroup = 1;   // k_emit_big: units per half-warp and step
constexpr uint32_t kSmallTiles = 32;   // light emission, one pair per lane: units of at most
                                       //   this many tiles, rows from their tile record

// The list of units k_emit_big writes: entry e is (first position, unit), held in the pair
// sort's second key and value buffers (free until the first tile pass writes them). Only
// units with a first position below the pair capacity are listed, so the list (at most one
// entry per position) always fits.
struct BigUnits {
  uint32_t* pos;
  uint32_t* unit;
};
__device__ __forceinline__ BigUnits big_units(const Ws& ws) { return {ws.keys[1], ws.vals[1]}; }

// Pair count of every 1024 slots of the depth-sorted unit order. The tile count of every slot
// is also stored in slot order (in the unit sort's key buffer 0, free once the sort is done;
// 0 past the visible units), so that the emission reads it without a gather.
__global__ void __launch_bounds__(256) k_block_sums(Ws ws) {
  pdl_entry();
  __shared__ uint32_t red[8];
  const uint32_t* order = ws.uvals[ws.plan[kPlanFinalUnits]];
  const uint32_t nvis = visible_units(ws);
  const uint32_t s0 = blockIdx.x * 1024u + 4u * threadIdx.x;
  uint4 c = make_uint4(0u, 0u, 0u, 0u);
  if (s0 < nvis) {   // slots past the visible units hold no unit
    const uint4 o = reinterpret_cast<const uint4*>(order)[blockIdx.x * 256u + threadIdx.x];
    c.x = ws.tiles_touched[o.x];
    c.y = s0 + 1 < nvis ? ws.tiles_touched[o.y] : 0u;
    c.z = s0 + 2 < nvis ? ws.tiles_touched[o.z] : 0u;
    c.w = s0 + 3 < nvis ? ws.tiles_touched[o.w] : 0u;
  }
  reinterpret_cast<uint4*>(slot_counts(ws))[blockIdx.x * 256u + threadIdx.x] = c;
  uint32_t s = c.x + c.y + c.z + c.w;
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
  pdl_entry();
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
    // emission slices, for the blocks the light emission leaves out
    const uint32_t sl = v > kLightPairs ? (uint32_t)((v + kEmitSlice - 1) / kEmitSlice) : 0u;
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
    for (int p = 4; p < kPlanPasses; ++p) ws.plan[kPlanCounter + p] = 0;   // pair-stage scan tickets
    ws.plan[kPlanSrc + 4] = 0;                                             // pair stage reads buffer 0
    ws.plan[kPlanQueue] = 0;
    ws.plan[kPlanQueue + 1] = 0;
    ws.plan[kPlanSlices] = carry_sl;
    ws.plan[kPlanBigUnits] = 0;
  }
}

// Key emission in depth-sorted unit order, load-balanced over output positions. Each
// 1024-slot block's contiguous range of pairs is cut into slices of kEmitSlice positions;
// persistent CTAs take slices in turn. For its slice [r0, r1) a CTA
//   1. rescans the block's 1024 pair counts (slot start positions);
//   2. counts the tile rows of the slots that overlap the slice and scans them: each
//      (slot, tile row) is one work item;
//   3. evaluates the items, split evenly over the threads (consecutive items per thread, at
//      most kEmitPerThread per round): the row's tile columns (UnitTiles/unit_row, the rule
//      preprocess counted with), a block scan of their counts for the row's first
//      position, and, for a row that overlaps the slice, a
//      "segment": its first tile id (minus its first slice position) and its unit, with the
//      segment's id marked at that position;
//   4. fills every position with the id of the last mark at or before it (a block scan);
//   5. writes keys (tile ids) and values (units), one position per thread and step.
// Threads stay converged whatever the mix of splat sizes, writes are coalesced, and a block
// of huge splats is spread over many CTAs. A slot whose rows hold another tile count than
// preprocess stored sets FLOD_DEV_TILESET.
constexpr uint32_t kEmitPerThread = 8;
constexpr uint16_t kNoSeg = 0xffffu;

template <int MAXV>
__device__ __forceinline__ bool slot_tiles(const Batch<MAXV>& b, const Ws& ws, uint32_t u,
                                           UnitTiles& t, uint32_t& row_base, uint32_t& tiles_x) {
  const ViewP& V = b.views[view_of_unit(b, u)];
  const float2 xy = ws.xy[u];
  row_base = V.tile_off;
  tiles_x = V.tiles_x;
  const bool rows = b.cfg.extent_rule == 2;
  const float r = rows ? 0.f : ws.radius[u];
  return unit_tiles(xy.x, xy.y, rows ? ws.ext[u] : make_float4(0.f, 0.f, r, r), V.width,
                    V.height, b.cfg.tile_w, b.cfg.tile_h, rows, t);
}

// Block-wide exclusive sum over 256 threads (8 warps); also returns the total.
__device__ __forceinline__ uint32_t block_excl_sum(uint32_t x, uint32_t* warp_tot, uint32_t& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  uint32_t pre = 0;
  total = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint32_t t = warp_tot[q];
    if (q < wid) pre += t;
    total += t;
  }
  return pre + inc - x;
}

template <int MAXV>
__global__ void __launch_bounds__(256) k_emit(const __grid_constant__ Batch<MAXV> b, Ws ws,
                                              uint32_t nblocks) {
  pdl_entry();
  __shared__ uint32_t s_pre[kScanBlock + 1];     // slot start positions (block-relative)
  __shared__ uint32_t s_row[kScanBlock + 1];     // first item of each slot
  __shared__ uint32_t s_unit[kScanBlock];
  __shared__ uint16_t s_owner[kEmitSlice];       // segment id per slice position
  __shared__ uint32_t s_seg_tile[kEmitSlice];    // tile id at slice position 0 (mod 2^32)
  __shared__ uint16_t s_seg_slot[kEmitSlice];
  __shared__ uint32_t warp_tot[8];
  __shared__ uint32_t s_blkmap[256];             // block of each of my next 256 slices
  __shared__ uint32_t s_nseg;
  const int tid = threadIdx.x;
  const uint32_t n_slices = ws.plan[kPlanSlices];
  const unsigned long long cap = ws.pair_capacity;
  const uint32_t* order = ws.uvals[ws.plan[kPlanFinalUnits]];
  const uint32_t nvis = visible_units(ws);
  uint32_t* keys = ws.keys[0];
  uint32_t* vals = ws.vals[0];
  for (uint32_t it = 0;; ++it) {
    const uint32_t w = blockIdx.x + it * gridDim.x;
    if (w >= n_slices) break;
    if ((it & 255u) == 0) {               // the blocks of my next 256 slices, searched at once
      __syncthreads();
      const uint32_t wt = blockIdx.x + (it + (uint32_t)tid) * gridDim.x;
      if (wt < n_slices) {
        uint32_t lo = 0, hi = nblocks - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (ws.slices[mid] <= wt) lo = mid; else hi = mid - 1;
        }
        s_blkmap[tid] = lo;
      }
    }
    if (tid == 0) s_nseg = 0;
    for (int i = tid; i < kEmitSlice; i += 256) s_owner[i] = kNoSeg;
    __syncthreads();
    const uint32_t blk = s_blkmap[it & 255u];
    const uint32_t r0 = (w - ws.slices[blk]) * (uint32_t)kEmitSlice;
    // 1. slot start positions (slots past the visible units hold no unit)
    const uint32_t s0 = blk * 1024u + 4u * tid;
    uint4 un = make_uint4(0u, 0u, 0u, 0u);
    if (s0 < nvis) un = reinterpret_cast<const uint4*>(order)[blk * 256u + tid];
    const uint32_t unit[4] = {un.x, un.y, un.z, un.w};
    uint32_t cnt[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      cnt[j] = s0 + j < nvis ? ws.tiles_touched[unit[j]] : 0u;
      s_unit[4 * tid + j] = unit[j];
    }
    uint32_t total;
    uint32_t run = block_excl_sum(cnt[0] + cnt[1] + cnt[2] + cnt[3], warp_tot, total);
    uint32_t pre[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      pre[j] = run;
      s_pre[4 * tid + j] = run;
      run += cnt[j];
    }
    if (tid == 255) s_pre[kScanBlock] = run;
    const uint32_t r1 = min(r0 + (uint32_t)kEmitSlice, total);
    // 2. tile rows of the slots that overlap the slice (from their tile records)
    uint32_t nrow[4];
    uint4 rec[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      nrow[j] = 0;
      if (cnt[j] && pre[j] < r1 && pre[j] + cnt[j] > r0) {
        rec[j] = ws.trec[unit[j]];
        nrow[j] = rec[j].y & 0xffffu;
        if (!nrow[j]) set_status(ws.status, FLOD_DEV_TILESET);
      }
    }
    uint32_t n_items;
    run = block_excl_sum(nrow[0] + nrow[1] + nrow[2] + nrow[3], warp_tot, n_items);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      s_row[4 * tid + j] = run;
      run += nrow[j];
    }
    if (tid == 255) s_row[kScanBlock] = run;
    __syncthreads();
    // the first overlapping slot: its start is the position of item 0
    uint32_t p_first = 0;
    {
      int lo = 0, hi = kScanBlock - 1;         // first slot whose end exceeds r0
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_pre[mid + 1] > r0) hi = mid; else lo = mid + 1;
      }
      p_first = s_pre[lo];
    }
    // 3. items, `per` consecutive items per thread and round
    uint32_t carry = p_first;
    const uint32_t per = min(kEmitPerThread, (n_items + 255u) / 256u);
    for (uint32_t ib = 0; ib < n_items; ib += 256u * per) {
      const uint32_t i0 = ib + per * tid;
      int slot = -1;
      UnitTiles t;
      uint4 rc = make_uint4(0u, 0u, 0u, 0u);
      uint32_t row_base = 0, tiles_x = 0;
      uint32_t nn[kEmitPerThread], tile0[kEmitPerThread];
      int sl[kEmitPerThread];
      uint32_t mine = 0;
#pragma unroll
      for (int k = 0; k < (int)kEmitPerThread; ++k) {
        nn[k] = 0;
        sl[k] = -1;
        const uint32_t i = i0 + k;
        if (k >= (int)per || i >= n_items) continue;
        bool fresh = false;
        if (slot < 0) {                        // last slot whose first item is <= i
          int lo = 0, hi = kScanBlock - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_row[mid] <= i) lo = mid; else hi = mid - 1;
          }
          slot = lo;
          fresh = true;
        }
        while (s_row[slot + 1] <= i) {         // next slot with rows
          ++slot;
          fresh = true;
        }
        if (fresh) {
          const uint32_t uu = s_unit[slot];
          rc = ws.trec[uu];
          const ViewP& V = b.views[view_of_unit(b, uu)];
          row_base = V.tile_off;
          tiles_x = V.tiles_x;
          if ((rc.y >> 16) == kRecCompute) slot_tiles(b, ws, uu, t, row_base, tiles_x);
        }
        const int r = (int)(i - s_row[slot]);
        const uint32_t mode = rc.y >> 16;
        const uint32_t tx0 = rc.x & 0xffffu, ty = (rc.x >> 16) + (uint32_t)r;
        if (mode == kRecCompute) {
          int cx0, cx1;
          if (unit_row(t, t.ty0 + r, cx0, cx1)) {
            nn[k] = (uint32_t)(cx1 - cx0 + 1);
            tile0[k] = row_base + ty * tiles_x + (uint32_t)cx0;
          }
        } else {
          uint32_t off = 0, cnt = rc.z;
          if (mode == kRecTable) rec_row(rc, r, off, cnt);
          nn[k] = cnt;
          tile0[k] = row_base + ty * tiles_x + tx0 + off;
        }
        sl[k] = slot;
        mine += nn[k];
      }
      uint32_t round_total;
      const uint32_t pos0 = carry + block_excl_sum(mine, warp_tot, round_total);
      // segment ids: one shared-memory atomic per warp
      uint32_t nmine = 0, pos = pos0;
#pragma unroll
      for (int k = 0; k < (int)kEmitPerThread; ++k) {
        if (nn[k] && pos < r1 && pos + nn[k] > r0) ++nmine;
        pos += nn[k];
      }
      const int lane = tid & 31;
      uint32_t incl = nmine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      uint32_t wbase = 0;
      if (lane == 31 && incl) wbase = atomicAdd(&s_nseg, incl);
      wbase = __shfl_sync(0xffffffffu, wbase, 31);
      uint32_t id = wbase + incl - nmine;
      pos = pos0;
#pragma unroll
      for (int k = 0; k < (int)kEmitPerThread; ++k) {
        if (nn[k] && pos < r1 && pos + nn[k] > r0) {
          const uint32_t first = max(pos, r0);
          if (id < (uint32_t)kEmitSlice) {
            s_owner[first - r0] = (uint16_t)id;
            s_seg_tile[id] = tile0[k] + (first - pos) - (first - r0);
            s_seg_slot[id] = (uint16_t)sl[k];
          }
          ++id;
        }
        pos += nn[k];
      }
      carry += round_total;
    }
    // the rows of the overlapping slots must add up to their stored counts
    if (tid == 0) {
      int lo = 0, hi = kScanBlock - 1;         // last slot starting before r1
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pre[mid] < r1) lo = mid; else hi = mid - 1;
      }
      if (carry != s_pre[lo + 1] || s_nseg > (uint32_t)kEmitSlice)
        set_status(ws.status, FLOD_DEV_TILESET);
    }
    __syncthreads();
    // 4. fill: each position takes the last segment marked at or before it
    constexpr int kPer = kEmitSlice / 256;
    uint16_t last = kNoSeg;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const uint16_t o = s_owner[tid * kPer + k];
      if (o != kNoSeg) last = o;
    }
    {
      // carry-in: the last mark of the nearest preceding thread that has one
      const int lane = tid & 31, wid = tid >> 5;
      uint32_t v = last;                       // kNoSeg = none
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o && v == kNoSeg) v = y;
      }
      // v: inclusive "last mark" up to this lane; the exclusive one comes from lane - 1
      uint32_t ex = __shfl_up_sync(0xffffffffu, v, 1);
      if (lane == 0) ex = kNoSeg;
      __syncthreads();
      if (lane == 31) warp_tot[wid] = v;
      __syncthreads();
      if (ex == kNoSeg) {
        for (int q = wid - 1; q >= 0; --q) {
          if (warp_tot[q] != kNoSeg) {
            ex = warp_tot[q];
            break;
          }
        }
      }
      uint16_t cur = (uint16_t)ex;
      for (int k = 0; k < kPer; ++k) {
        const uint16_t o = s_owner[tid * kPer + k];
        if (o != kNoSeg) cur = o;
        else s_owner[tid * kPer + k] = cur;
      }
    }
    __syncthreads();
    // 5. write
    const unsigned long long base = ws.block_sums[blk];
    for (uint32_t p = r0 + tid; p < r1; p += 256) {
      if (base + p >= cap) break;
      const uint32_t rel = p - r0;
      const uint16_t sgi = s_owner[rel];
      if (sgi == kNoSeg) continue;             // only with an inconsistent tile set
      keys[base + p] = s_seg_tile[sgi] + rel;
      vals[base + p] = s_unit[s_seg_slot[sgi]];
    }
    __syncthreads();
  }
}

// Key emission of a light block (at most kLightPairs pairs), one CTA per 1024-slot block.
// Each warp owns 128 consecutive slots, taken as 4 rounds of 32 (one slot per lane); the
// block's pair counts are scanned per warp and across the 8 warps. In a round:
//   - "small" units (at most kSmallTiles tiles, rows given by the tile record's table or
//     uniform form) are written one pair per lane: each unit's lane builds its row table, the
//     round's small pairs are numbered 0..n-1, lane i finds the unit holding pair i by a
//     binary search over the units' first numbers (shuffles) and its row from the row
//     starts, and writes keys and values of 32 consecutive positions of a unit run at once;
//   - the other units (more tiles, rows recomputed from the ellipse, or a record that does
//     not add up) are listed for k_emit_big, where half a warp writes each: rows 16 at a time
//     (one per lane, their columns from the record or recomputed), then the pairs one per
//     lane. A CTA's run time then no longer depends on how many of them its slots hold.
// Heavier blocks are left to the sliced k_emit.
template <int MAXV>
__device__ __forceinline__ bool rec_row_tiles(const Batch<MAXV>& b, const Ws& ws, uint32_t u,
                                              const uint4& rc, const UnitTiles& t, uint32_t r,
                                              uint32_t row_base, uint32_t tiles_x, uint32_t& n,
                                              uint32_t& tile0) {
  const uint32_t mode = rc.y >> 16;
  const uint32_t ty = (rc.x >> 16) + r;
  if (mode == kRecCompute) {
    int cx0, cx1;
    if (!unit_row(t, t.ty0 + (int)r, cx0, cx1)) return false;
    n = (uint32_t)(cx1 - cx0 + 1);
    tile0 = row_base + ty * tiles_x + (uint32_t)cx0;
    return true;
  }
  uint32_t off = 0, c = rc.z;
  if (mode == kRecTable) rec_row(rc, (int)r, off, c);
  n = c;
  tile0 = row_base + ty * tiles_x + (rc.x & 0xffffu) + off;
  return c > 0;
}

// A group of GW lanes (the whole warp, or one half of it) writes the n_all pairs of unit u
// (tile record rc; centre xy and extent ext, (m, h, rx, ry) or (0, 0, r, r), for rows
// recomputed) from position p0 on: rows GW at a time, one per lane (first tile and count,
// from the record or recomputed), then their pairs one per lane. The group's lanes take the
// same path; the shuffles involve only them.
template <int MAXV, int GW>
__device__ __forceinline__ void emit_unit_group(const Batch<MAXV>& b, const Ws& ws, uint32_t u,
                                                const uint4& rc, float2 xy, float4 ext,
                                                unsigned long long p0, uint32_t n_all,
                                                uint32_t* keys, uint32_t* vals,
                                                unsigned long long cap) {
  static_assert(GW == 16 || GW == 32, "a warp or half a warp");
  const int lane = threadIdx.x & (GW - 1);
  const uint32_t mask = GW == 32 ? 0xffffffffu : 0xffffu << (threadIdx.x & 16);
  const ViewP& V = b.views[view_of_unit(b, u)];
  const uint32_t row_base = V.tile_off, tiles_x = V.tiles_x;
  UnitTiles t;
  if ((rc.y >> 16) == kRecCompute)
    unit_tiles(xy.x, xy.y, ext, V.width, V.height, b.cfg.tile_w, b.cfg.tile_h,
               b.cfg.extent_rule == 2, t);
  const uint32_t nrows = rc.y & 0xffffu;
  uint32_t done = 0;
  for (uint32_t r0 = 0; r0 < nrows; r0 += GW) {
    // rows r0..r0+GW-1, one per lane: their first tile and tile count
    const uint32_t r = r0 + lane;
    uint32_t rn = 0, rt0 = 0;
    if (r < nrows && !rec_row_tiles(b, ws, u, rc, t, r, row_base, tiles_x, rn, rt0)) rn = 0;
    uint32_t incl = rn;
#pragma unroll
    for (int o = 1; o < GW; o <<= 1) {
      const uint32_t y = __shfl_up_sync(mask, incl, o, GW);
      if (lane >= o) incl += y;
    }
    const uint32_t excl = incl - rn;                      // the row's first pair (chunk-relative)
    const uint32_t chunk = __shfl_sync(mask, incl, GW - 1, GW);
    // the chunk's pairs, one per lane: the row holding pair q is the last row whose first
    // pair is <= q (a row without tiles shares its first pair with the next one)
    for (uint32_t q0 = 0; q0 < chunk; q0 += GW) {
      const uint32_t q = q0 + lane;
      int v = 0;
#pragma unroll
      for (int step = GW / 2; step > 0; step >>= 1) {
        const uint32_t ev = __shfl_sync(mask, excl, v + step, GW);
        if (ev <= q) v += step;
      }
      const uint32_t tile = __shfl_sync(mask, rt0, v, GW) + (q - __shfl_sync(mask, excl, v, GW));
      if (q < chunk && done + q < n_all) {
        const unsigned long long p = p0 + done + q;
        if (p < cap) {
          keys[p] = tile;
          vals[p] = u;
        }
      }
    }
    done += chunk;
  }
  if (lane == 0 && done != n_all) set_status(ws.status, FLOD_DEV_TILESET);
}

// Row table of a small unit (rows given by its record's table or uniform form, at most
// kRecRows rows): for row r, K_r = (tile id of the row's first tile) - (tiles in rows before
// r), so that its j-th tile is K_row + j, where row = the number of rows r >= 1 starting at or
// before j (cum = bytes 0..2: start of rows 1..3, 255 past the last row). False if the rows
// do not hold exactly c tiles or the form has more rows.
__device__ __forceinline__ bool small_unit_rows(const uint4& rc, uint32_t c, uint32_t tb,
                                                uint32_t tx, uint4& K, uint32_t& cum) {
  const uint32_t mode = rc.y >> 16, nrows = rc.y & 0xffffu;
  if (mode == kRecCompute || nrows > (uint32_t)kRecRows) return false;
  uint32_t k[kRecRows], start = 0;
  cum = 0;
#pragma unroll
  for (int r = 0; r < kRecRows; ++r) {
    uint32_t off = 0, n = 0;
    if ((uint32_t)r < nrows) {
      if (mode == kRecUniform) n = rc.z;
      else rec_row(rc, r, off, n);
    }
    if (r > 0) cum |= ((uint32_t)r < nrows ? start : 255u) << (8 * (r - 1));
    k[r] = tb + (uint32_t)r * tx + off - start;
    start += n;
  }
  K = make_uint4(k[0], k[1], k[2], k[3]);
  return start == c;
}

template <int MAXV>
__global__ void __launch_bounds__(256, 4) k_emit_light(const __grid_constant__ Batch<MAXV> b, Ws ws) {
  pdl_entry();
  constexpr int kRounds = kScanBlock / 256;   // rounds of 32 slots per warp
  __shared__ uint32_t warp_tot[8];
  __shared__ uint4 s_K[8][32];                 // row tables of the round's small units
  __shared__ uint32_t s_cum[8][32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const size_t slot0 = (size_t)blockIdx.x * kScanBlock + (size_t)wid * (32 * kRounds) + lane;
  const uint32_t* order = ws.uvals[ws.plan[kPlanFinalUnits]];
  const uint32_t* counts = slot_counts(ws);   // 0 past the visible units
  uint32_t unit[kRounds], cnt[kRounds];
  uint32_t wsum = 0;
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    cnt[r] = counts[slot0 + 32 * r];
    unit[r] = order[slot0 + 32 * r];
    wsum += cnt[r];
  }
  uint4 rc[kRounds];   // tile records, requested before the block scan
#pragma unroll
  for (int r = 0; r < kRounds; ++r)
    rc[r] = cnt[r] ? ws.trec[unit[r]] : make_uint4(0u, 0u, 0u, 0u);
  // the units whose rows are recomputed (taken by the whole warp later): their centre and
  // extent brought into L2 now
#pragma unroll
  for (int r = 0; r < kRounds; ++r)
    if ((rc[r].y >> 16) == kRecCompute) {
      prefetch_l2(ws.xy + unit[r]);
      prefetch_l2(ws.ext + unit[r]);
    }
  wsum = __reduce_add_sync(0xffffffffu, wsum);
  if (lane == 0) warp_tot[wid] = wsum;
  __syncthreads();
  uint32_t total = 0, wpre = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint32_t t = warp_tot[q];
    if (q < wid) wpre += t;
    total += t;
  }
  if (total == 0 || total > kLightPairs) return;   // nothing, or the sliced emission's
  const unsigned long long cap = ws.pair_capacity;
  uint32_t* keys = ws.keys[0];
  uint32_t* vals = ws.vals[0];
  unsigned long long base = ws.block_sums[blockIdx.x] + wpre;
#pragma unroll 1
  for (int r = 0; r < kRounds; ++r) {
    // this round's slot (a select chain keeps the per-round arrays in registers)
    uint32_t c = cnt[0], u = unit[0];
    uint4 rr = rc[0];
#pragma unroll
    for (int q = 1; q < kRounds; ++q)
      if (q == r) {
        c = cnt[q];
        u = unit[q];
        rr = rc[q];
      }
    // small units: their row table, for the lanes that write their pairs
    bool small = false;
    if (c && c <= kSmallTiles) {
      const ViewP& V = b.views[view_of_unit(b, u)];
      const uint32_t tx = V.tiles_x;
      const uint32_t tb = V.tile_off + (rr.x >> 16) * tx + (rr.x & 0xffffu);
      uint4 K;
      uint32_t cum;
      small = small_unit_rows(rr, c, tb, tx, K, cum);
      s_K[wid][lane] = K;
      s_cum[wid][lane] = cum;
    }
    // one scan for both: all pairs (low 17 bits: a light block has at most 2^16) and the
    // small units' pairs (high bits: at most 32 x kSmallTiles)
    const uint32_t x = c | (small ? c : 0u) << 17;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t excl = (incl - x) & 0x1ffffu;           // first position (round-relative)
    const uint32_t vstart = (incl - x) >> 17;               // first small-pair number
    const uint32_t rtot = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t vtot = rtot >> 17;
    __syncwarp();
    for (uint32_t i0 = 0; i0 < vtot; i0 += 32) {
      const uint32_t i = i0 + lane;
      int v = 0;   // the last lane whose first small-pair number is <= i
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t sv = __shfl_sync(0xffffffffu, vstart, v + step);
        if (sv <= i) v += step;
      }
      const uint32_t j = i - __shfl_sync(0xffffffffu, vstart, v);
      const uint32_t pr = __shfl_sync(0xffffffffu, excl, v);
      const uint32_t uv = __shfl_sync(0xffffffffu, u, v);
      if (i < vtot) {
        const uint4 K = s_K[wid][v];
        const uint32_t cum = s_cum[wid][v];
        const uint32_t row = (uint32_t)(j >= (cum & 0xffu)) + (uint32_t)(j >= ((cum >> 8) & 0xffu)) +
                             (uint32_t)(j >= (cum >> 16));
        const uint32_t key = (row == 0 ? K.x : row == 1 ? K.y : row == 2 ? K.z : K.w) + j;
        const unsigned long long p = base + pr + j;
        if (p < cap) {
          keys[p] = key;
          vals[p] = uv;
        }
      }
    }
    __syncwarp();
    // the other units: listed for k_emit_big (one warp per unit there)
    const unsigned long long pos = base + excl;
    const bool other = c && !small && pos < cap;
    const uint32_t om = __ballot_sync(0xffffffffu, other);
    if (om) {
      uint32_t first = 0;
      if (lane == 0) first = atomicAdd(&ws.plan[kPlanBigUnits], (uint32_t)__popc(om));
      first = __shfl_sync(0xffffffffu, first, 0);
      if (other) {
        const uint32_t idx = first + (uint32_t)__popc(om & ((1u << lane) - 1u));
        const BigUnits L = big_units(ws);
        L.pos[idx] = (uint32_t)pos;
        L.unit[idx] = u;
      }
    }
    base += rtot & 0x1ffffu;
  }
}

// The units the light emission listed (more than kSmallTiles tiles, rows recomputed, or a
// record that does not add up): each half-warp takes kBigPerGroup entries, its first lanes
// fetch their units' data at once, then it writes the units one after the other (the two
// halves of a warp side by side).
template <int MAXV>
__global__ void __launch_bounds__(256) k_emit_big(const __grid_constant__ Batch<MAXV> b, Ws ws) {
  pdl_entry();
  constexpr uint32_t G = kBigPerGroup;
  constexpr int GW = 16;   // lanes per group: two units of a warp are written side by side
  const uint32_t n = ws.plan[kPlanBigUnits];
  const BigUnits L = big_units(ws);
  const int gl = threadIdx.x & (GW - 1);
  const uint32_t mask = 0xffffu << (threadIdx.x & 16);
  const uint32_t ng = (gridDim.x * blockDim.x) / GW;
  const unsigned long long cap = ws.pair_capacity;
  const bool rows = b.cfg.extent_rule == 2;
  for (uint32_t e0 = ((blockIdx.x * blockDim.x + threadIdx.x) / GW) * G; e0 < n; e0 += ng * G) {
    // the group's lanes 0..G-1 fetch one unit's data each, all requests in flight together
    const uint32_t e = e0 + (uint32_t)gl;
    uint32_t u = 0, pos = 0, c = 0;
    uint4 rc = make_uint4(0u, 0u, 0u, 0u);
    float2 xy = make_float2(0.f, 0.f);
    float4 ext = make_float4(0.f, 0.f, 0.f, 0.f);
    if ((uint32_t)gl < G && e < n) {
      u = L.unit[e];
      pos = L.pos[e];
      c = ws.tiles_touched[u];
      rc = ws.trec[u];
      xy = ws.xy[u];
      if (rows) {
        ext = ws.ext[u];
      } else {
        const float r = ws.radius[u];
        ext = make_float4(0.f, 0.f, r, r);
      }
    }
    const int m = (int)min(G, n - e0);
    for (int k = 0; k < m; ++k) {
      const uint4 rk = make_uint4(__shfl_sync(mask, rc.x, k, GW), __shfl_sync(mask, rc.y, k, GW),
                                  __shfl_sync(mask, rc.z, k, GW), __shfl_sync(mask, rc.w, k, GW));
      const float2 xk = make_float2(__shfl_sync(mask, xy.x, k, GW), __shfl_sync(mask, xy.y, k, GW));
      const float4 ek = make_float4(__shfl_sync(mask, ext.x, k, GW), __shfl_sync(mask, ext.y, k, GW),
                                    __shfl_sync(mask, ext.z, k, GW), __shfl_sync(mask, ext.w, k, GW));
      emit_unit_group<MAXV, GW>(b, ws, __shfl_sync(mask, u, k, GW), rk, xk, ek,
                                __shfl_sync(mask, pos, k, GW), __shfl_sync(mask, c, k, GW),
                                ws.keys[0], ws.vals[0], cap);
    }
  }
}

// Tile ranges from the sorted tile keys: four consecutive keys per thread (one 16-byte load),
// a range starts or ends where a key differs from its neighbour.
__global__ void __launch_bounds__(256) k_ranges(Ws ws, uint32_t n_tiles) {
  pdl_entry();
  const unsigned long long P0 = *ws.pair_count;
  const uint32_t P = (uint32_t)(P0 < ws.pair_capacity ? P0 : ws.pair_capacity);
  const uint32_t* keys = ws.keys[ws.plan[kPlanFinal]];
  constexpr uint32_t kNone = 0xffffffffu;   // never a tile id
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; 4ull * q < P; q += gridDim.x * blockDim.x) {
    const uint32_t i0 = 4u * q;
    uint32_t k[4];
    if (i0 + 3 < P) {
      const uint4 v = reinterpret_cast<const uint4*>(keys)[q];
      k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) k[j] = i0 + j < P ? keys[i0 + j] : kNone;
    }
    const uint32_t prev = i0 ? keys[i0 - 1] : kNone;
    const uint32_t next = i0 + 4 < P ? keys[i0 + 4] : kNone;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t t = k[j];
      if (t >= n_tiles) continue;   // past the end, or an inconsistent tile set (FLOD_DEV_TILESET)
      const uint32_t before = j ? k[j - 1] : prev;
      const uint32_t after = j < 3 ? k[j + 1] : next;
      if (before != t) ws.ranges[t].x = i0 + j;
      if (after != t) ws.ranges[t].y = i0 + j + 1;
    }
  }
}

__global__ void __launch_bounds__(256) k_queue_count(Ws ws, uint32_t n_tiles) {
  pdl_entry();
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
  pdl_entry();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int bkt = 32; bkt >= 0; --bkt) {
      ws.queue[33 + bkt] = run;
      run += ws.queue[bkt];
    }
  }
}

__global__ void __launch_bounds__(256) k_queue_fill(Ws ws, uint32_t n_tiles) {
  pdl_entry();
  for (uint32_t t = blockIdx.x * 256u + threadIdx.x; t < n_tiles; t += gridDim.x * 256u) {
    const uint2 r = ws.ranges[t];
    const uint32_t n = r.y - r.x;
    const uint32_t slot = atomicAdd(&ws.queue[33 + (n ? 32 - __clz(n) : 0)], 1u);
    ws.queue[kQueueHeader + slot] = t;
  }
}

template <int MAXV>
cudaError_t launch_binning(const Batch<MAXV>& b, const Ws& ws, int n_passes, int tile_bits,
                           int resident_sort,
                           int resident_small, unsigned long long* d_pair_count, bool build_queue,
                           int phase, cudaStream_t st) {
  const uint32_t nblocks = b.units / kScanBlock;
  cudaError_t e;
  if (phase == 0 || phase == 1) {   // depth order of the units with tiles
    if (b.tiles && !nblocks) {   // with units, the unit sort's first kernel clears them
      e = cudaMemsetAsync(ws.ranges, 0, sizeof(uint2) * b.tiles, st);
      if (e != cudaSuccess) return e;
    }
    if (nblocks &&
        (e = launch_unit_sort(ws, b.tiles, resident_small, resident_sort, st)) != cudaSuccess)
      return e;
  }
  if (phase == 0 || phase == 2) {   // pair offsets and key emission
    if (nblocks) launch_k(k_block_sums, dim3(nblocks), dim3(256), 0, st, ws);
    launch_k(k_scan_blocks, dim3(1), dim3(1024), 0, st, ws, nblocks, d_pair_count);
    if (nblocks) {
      launch_k(k_emit_light<MAXV>, dim3(nblocks), dim3(256), 0, st, b, ws);
      launch_k(k_emit_big<MAXV>, dim3(resident_small), dim3(256), 0, st, b, ws);
      launch_k(k_emit<MAXV>, dim3(resident_small), dim3(256), 0, st, b, ws, nblocks);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (phase == 0 || phase == 3) {   // tile digits over the pairs
    if ((e = launch_pair_sort(ws, n_passes, tile_bits, resident_small, resident_sort, st)) !=
        cudaSuccess)
      return e;
  }
  if (phase != 0 && phase != 4) return cudaGetLastError();
  launch_k(k_ranges, dim3(resident_small), dim3(256), 0, st, ws, b.tiles);
  if (build_queue && b.tiles) {
    if ((e = cudaMemsetAsync(ws.queue, 0, sizeof(uint32_t) * kQueueHeader, st)) != cudaSuccess)
      return e;
    const uint32_t g = min((uint32_t)resident_small, (b.tiles + 255) / 256);
    launch_k(k_queue_count, dim3(g), dim3(256), 0, st, ws, b.tiles);
    launch_k(k_queue_offsets, dim3(1), dim3(32), 0, st, ws);
    launch_k(k_queue_fill, dim3(g), dim3(256), 0, st, ws, b.tiles);
  }
  return cudaGetLastError();
}

template cudaError_t launch_binning<kMaxViewsSmall>(const BatchS&, const Ws&, int, int, int, int,
                                                    unsigned long long*, bool, int, cudaStream_t);
template cudaError_t launch_binning<FLOD_MAX_VIEWS>(const BatchL&, const Ws&, int, int, int, int,
                                                    unsigned long long*, bool, int, cudaStream_t);

}  // namespace flod
