// Overlap pruning (Sec. 4.3): a Gaussian is removed when the average distance to its three
// nearest neighbours in its level, d_avg = (d1 + d2 + d3) / 3, is below d_OP (= s_min / 2 of
// the level being trained).
//
// Only neighbours within R = 3 d_OP can decide it: if fewer than three other means lie
// within R, then d3 > R and d_avg > d_OP, so the Gaussian is kept whatever they are. The
// means are therefore binned into a uniform grid of cell edge R (cells relative to the
// set's bounding box, hashed into an open-addressing table), and each Gaussian looks at the
// 27 cells around its own: every mean within R lies there, so when three are found within
// R they are exactly the three nearest and d_avg is exact; otherwise the Gaussian is kept
// and its d_avg reported as +inf. Kernels (one grid-stride pass each, none waits for
// another CTA): table clear and box init, bounding box, cell insert (atomic CAS on the
// 64-bit cell key, linear probing bounded by the table size), cell ranges (atomic
// allocation), cell fill, the 3-nearest search, then the kept indices compacted in order
// (per-block counts, a one-CTA scan, ordered writes).
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace flod {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kCellBits = 21;                       // per axis in the packed key
constexpr uint32_t kCellMax = (1u << kCellBits) - 1u;
constexpr int kPruneBlock = 1024;                   // Gaussians per compaction block

struct PruneScratch {
  uint32_t* hdr;                 // [0..5] box min/max as ordered ints, [6] allocated points,
                                 // [7] status bits
  unsigned long long* keys;      // [S] packed cell keys
  uint32_t* count;               // [S] points per cell
  uint32_t* start;               // [S] first position of the cell's points in `order`
  uint32_t* fill;                // [S] points placed so far
  uint32_t* pslot;               // [n] the table slot of each point's cell
  uint32_t* order;               // [n] point indices grouped by cell
  uint32_t* blocks;              // [n / kPruneBlock + 1] kept per block, then offsets
  uint32_t S;                    // table slots (a power of two >= 2n)
};

struct PruneP {
  const float* means;
  uint32_t n;
  float d_op, cell;              // d_OP and the cell edge R = 3 d_OP
  uint8_t* keep;
  float* d_avg;
  uint32_t* out_kept;
  uint32_t* d_kept;
  uint32_t* d_status;
  PruneScratch s;
};

// float <-> int order-preserving map (for atomicMin / atomicMax on floats)
__device__ __forceinline__ int f2o(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__device__ __forceinline__ uint32_t hash_key(unsigned long long k, uint32_t S) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return (uint32_t)k & (S - 1u);
}

__device__ __forceinline__ unsigned long long pack_cell(uint32_t x, uint32_t y, uint32_t z) {
  return (unsigned long long)x | ((unsigned long long)y << kCellBits) |
         ((unsigned long long)z << (2 * kCellBits));
}

// Cell of a mean (clamped to the key range; a clamp is reported and the pruning skipped).
__device__ __forceinline__ bool cell_of(const PruneP& p, const float* m, uint32_t& cx, uint32_t& cy,
                                        uint32_t& cz) {
  bool ok = true;
  uint32_t c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float lo = o2f((int)p.s.hdr[a]);
    float f = floorf((m[a] - lo) / p.cell);
    if (!(f >= 0.f)) f = 0.f;
    if (f > (float)kCellMax) {
      f = (float)kCellMax;
      ok = false;
    }
    c[a] = (uint32_t)f;
  }
  cx = c[0];
  cy = c[1];
  cz = c[2];
  return ok;
}

// Slot of a cell key: inserts it when `insert`, else returns S when the cell is absent.
__device__ __forceinline__ uint32_t find_slot(const PruneScratch& s, unsigned long long key, bool insert) {
  uint32_t h = hash_key(key, s.S);
  for (uint32_t probe = 0; probe < s.S; ++probe) {
    const unsigned long long k = s.keys[h];
    if (k == key) return h;
    if (k == kEmptyKey) {
      if (!insert) return s.S;
      const unsigned long long prev = atomicCAS(&s.keys[h], kEmptyKey, key);
      if (prev == kEmptyKey || prev == key) return h;
    }
    h = (h + 1u) & (s.S - 1u);
  }
  return s.S;   // the table is sized 2n: not reached
}

__global__ void __launch_bounds__(256) k_prune_clear(const __grid_constant__ PruneP p) {
  pdl_entry();
  const uint32_t stride = gridDim.x * 256u;
  for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < p.s.S; i += stride) {
    p.s.keys[i] = kEmptyKey;
    p.s.count[i] = 0u;
    p.s.fill[i] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x < 8) {
    const uint32_t v = threadIdx.x < 3 ? (uint32_t)f2o(FLT_MAX) : threadIdx.x < 6 ? (uint32_t)f2o(-FLT_MAX) : 0u;
    p.s.hdr[threadIdx.x] = v;
  }
}

__global__ void __launch_bounds__(256) k_prune_box(const __grid_constant__ PruneP p) {
  pdl_entry();
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  const uint32_t stride = gridDim.x * 256u;
  for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < p.n; i += stride) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float v = p.means[3ull * i + a];
      lo[a] = fminf(lo[a], v);
      hi[a] = fmaxf(hi[a], v);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      atomicMin(reinterpret_cast<int*>(&p.s.hdr[a]), f2o(lo[a]));
      atomicMax(reinterpret_cast<int*>(&p.s.hdr[3 + a]), f2o(hi[a]));
    }
  }
}

__global__ void __launch_bounds__(256) k_prune_insert(const __grid_constant__ PruneP p) {
  pdl_entry();
  const uint32_t stride = gridDim.x * 256u;
  for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < p.n; i += stride) {
    uint32_t cx, cy, cz;
    if (!cell_of(p, p.means + 3ull * i, cx, cy, cz)) atomicOr(&p.s.hdr[7], 1u);
    const uint32_t h = find_slot(p.s, pack_cell(cx, cy, cz), true);
    p.s.pslot[i] = h;
    if (h < p.s.S) atomicAdd(&p.s.count[h], 1u);
  }
}

__global__ void __launch_bounds__(256) k_prune_ranges(const __grid_constant__ PruneP p) {
  pdl_entry();
  const uint32_t stride = gridDim.x * 256u;
  for (uint32_t h = blockIdx.x * 256u + threadIdx.x; h < p.s.S; h += stride) {
    const uint32_t c = p.s.count[h];
    if (c) p.s.start[h] = atomicAdd(&p.s.hdr[6], c);
  }
}

__global__ void __launch_bounds__(256) k_prune_fill(const __grid_constant__ PruneP p) {
  pdl_entry();
  const uint32_t stride = gridDim.x * 256u;
  for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < p.n; i += stride) {
    const uint32_t h = p.s.pslot[i];
    if (h < p.s.S) p.s.order[p.s.start[h] + atomicAdd(&p.s.fill[h], 1u)] = i;
  }
}

// Keeps the three smallest (d^2, index) pairs, ties by index.
__device__ __forceinline__ void push3(float d2, uint32_t j, float (&bd)[3], uint32_t (&bj)[3]) {
  if (d2 > bd[2] || (d2 == bd[2] && j > bj[2])) return;
  if (d2 < bd[1] || (d2 == bd[1] && j < bj[1])) {
    bd[2] = bd[1];
    bj[2] = bj[1];
    if (d2 < bd[0] || (d2 == bd[0] && j < bj[0])) {
      bd[1] = bd[0];
      bj[1] = bj[0];
      bd[0] = d2;
      bj[0] = j;
    } else {
      bd[1] = d2;
      bj[1] = j;
    }
  } else {
    bd[2] = d2;
    bj[2] = j;
  }
}

__device__ __forceinline__ bool knn_keep(const PruneP& p, uint32_t i, float& davg) {
  const float* mi = p.means + 3ull * i;
  const float x = mi[0], y = mi[1], z = mi[2];
  uint32_t cx, cy, cz;
  const bool in_range = cell_of(p, mi, cx, cy, cz);
  float bd[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
  uint32_t bj[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu};
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const long long nx = (long long)cx + dx, ny = (long long)cy + dy, nz = (long long)cz + dz;
        if (nx < 0 || ny < 0 || nz < 0 || nx > kCellMax || ny > kCellMax || nz > kCellMax) continue;
        const uint32_t h = find_slot(p.s, pack_cell((uint32_t)nx, (uint32_t)ny, (uint32_t)nz), false);
        if (h >= p.s.S) continue;
        const uint32_t b = p.s.start[h], e = b + p.s.count[h];
        for (uint32_t k = b; k < e; ++k) {
          const uint32_t j = p.s.order[k];
          if (j == i) continue;
          const float* mj = p.means + 3ull * j;
          const float ex = __fsub_rn(mj[0], x), ey = __fsub_rn(mj[1], y), ez = __fsub_rn(mj[2], z);
          const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
          push3(d2, j, bd, bj);
        }
      }
  const float R2 = p.cell * p.cell;
  if (!in_range || bj[2] == 0xffffffffu || bd[2] > R2) {   // fewer than three within R
    davg = INFINITY;
    return true;
  }
  davg = (__fsqrt_rn(bd[0]) + __fsqrt_rn(bd[1]) + __fsqrt_rn(bd[2])) / 3.f;
  return !(davg < p.d_op);
}

// One thread per Gaussian of a block of kPruneBlock: the search, the keep mask, d_avg and
// the block's kept count.
__global__ void __launch_bounds__(256) k_prune_knn(const __grid_constant__ PruneP p) {
  pdl_entry();
  __shared__ uint32_t red[8];
  uint32_t c = 0;
  const bool grid_ok = !(p.s.hdr[7] & 1u);
  for (int r = 0; r < kPruneBlock / 256; ++r) {
    const uint32_t i = blockIdx.x * (uint32_t)kPruneBlock + r * 256u + threadIdx.x;
    if (i >= p.n) break;
    float davg = INFINITY;
    bool keep = true;
    if (grid_ok) keep = knn_keep(p, i, davg);
    p.keep[i] = keep ? 1u : 0u;
    if (p.d_avg) p.d_avg[i] = davg;
    c += keep ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    p.s.blocks[blockIdx.x] = t;
  }
}

// Exclusive scan of the block counts (one CTA) and the kept total.
__global__ void __launch_bounds__(1024) k_prune_scan(const __grid_constant__ PruneP p, uint32_t nblocks) {
  pdl_entry();
  __shared__ uint32_t wt[32];
  __shared__ uint32_t carry_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  for (uint32_t base = 0; base < nblocks; base += 1024) {
    const uint32_t i = base + tid;
    const uint32_t v = i < nblocks ? p.s.blocks[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wt[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint32_t w = wt[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wt[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = carry_s + (wid ? wt[wid - 1] : 0u) + x - v;
    if (i < nblocks) p.s.blocks[i] = excl;
    __syncthreads();
    if (tid == 1023) carry_s = excl + v;
    __syncthreads();
  }
  if (tid == 0) {
    *p.d_kept = carry_s;
    if (p.d_status) *p.d_status = p.s.hdr[7];
  }
}

// Kept indices in index order.
__global__ void __launch_bounds__(256) k_prune_write(const __grid_constant__ PruneP p) {
  pdl_entry();
  __shared__ uint32_t wcnt[8];
  __shared__ uint32_t base_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) base_s = p.s.blocks[blockIdx.x];
  for (int r = 0; r < kPruneBlock / 256; ++r) {
    const uint32_t i = blockIdx.x * (uint32_t)kPruneBlock + r * 256u + threadIdx.x;
    const bool keep = i < p.n && p.keep[i];
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wcnt[wid] = __popc(bal);
    __syncthreads();
    uint32_t pre = base_s;
    for (int w = 0; w < wid; ++w) pre += wcnt[w];
    pre += __popc(bal & ((1u << lane) - 1u));
    if (keep) p.out_kept[pre] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (int w = 0; w < 8; ++w) t += wcnt[w];
      base_s += t;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
static uint32_t table_slots(uint32_t n) {
  uint32_t S = 1024;
  while (S < 2u * n && S < (1u << 31)) S <<= 1;
  return S;
}

size_t prune_scratch_bytes(uint32_t n) {
  const size_t S = table_slots(n);
  const size_t nb = n / kPruneBlock + 1;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  return up(64) + up(8 * S) + 3 * up(4 * S) + 2 * up(4 * (size_t)n) + up(4 * nb);
}

cudaError_t launch_prune(const float* means, uint32_t n, float d_op, uint8_t* keep, float* d_avg,
                         uint32_t* out_kept, uint32_t* d_kept, uint32_t* d_status, void* scratch,
                         int grid, cudaStream_t st) {
  PruneP p;
  p.means = means;
  p.n = n;
  p.d_op = d_op;
  p.cell = 3.f * d_op;
  p.keep = keep;
  p.d_avg = d_avg;
  p.out_kept = out_kept;
  p.d_kept = d_kept;
  p.d_status = d_status;
  const uint32_t S = table_slots(n);
  const size_t nb = n / kPruneBlock + 1;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  unsigned char* b = static_cast<unsigned char*>(scratch);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* at = b + off;
    off += up(bytes);
    return at;
  };
  p.s.hdr = reinterpret_cast<uint32_t*>(take(64));
  p.s.keys = reinterpret_cast<unsigned long long*>(take(8ull * S));
  p.s.count = reinterpret_cast<uint32_t*>(take(4ull * S));
  p.s.start = reinterpret_cast<uint32_t*>(take(4ull * S));
  p.s.fill = reinterpret_cast<uint32_t*>(take(4ull * S));
  p.s.pslot = reinterpret_cast<uint32_t*>(take(4ull * n));
  p.s.order = reinterpret_cast<uint32_t*>(take(4ull * n));
  p.s.blocks = reinterpret_cast<uint32_t*>(take(4 * nb));
  p.s.S = S;
  const uint32_t nblocks = (n + kPruneBlock - 1) / kPruneBlock;
  const unsigned gs = (unsigned)grid;
  launch_k(k_prune_clear, dim3(gs), dim3(256), 0, st, p);
  if (n) {
    launch_k(k_prune_box, dim3(gs), dim3(256), 0, st, p);
    launch_k(k_prune_insert, dim3(gs), dim3(256), 0, st, p);
    launch_k(k_prune_ranges, dim3(gs), dim3(256), 0, st, p);
    launch_k(k_prune_fill, dim3(gs), dim3(256), 0, st, p);
    launch_k(k_prune_knn, dim3(nblocks), dim3(256), 0, st, p);
  }
  launch_k(k_prune_scan, dim3(1), dim3(1024), 0, st, p, nblocks);
  if (n && out_kept) launch_k(k_prune_write, dim3(nblocks), dim3(256), 0, st, p);
  return cudaGetLastError();
}

}  // namespace flod
