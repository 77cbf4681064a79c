// Level selection (Eq. 6 with the thresholds of Eq. 7, Sec. 5.2) and AdjustScale (Eq. 5,
// Sec. 4.2).
//
// Selection is a stream compaction over the concatenation of the levels: a Gaussian of
// level k is kept iff lo_k <= d < hi_k with d = ||mean - origin|| in float32 (each
// difference, square and sum rounded to nearest, then a correctly rounded square root), so
// that the decision is reproducible by any float32 implementation. Three launches: per-block
// counts, one-CTA scan of the counts, ordered write. The output is in (level, index) order.
// With room in the scratch, the count kernel also stores each block's keep bits (one ballot
// word per warp and round), and the write kernel places the kept entries from those bits
// and one 64-entry scan per block, without reading the means or deciding again; with only
// the counts (the fixed scratch of the allocation-free entry point) it decides again.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace flod {

constexpr int kSelThreads = 256;
constexpr int kSelPerThread = 8;
constexpr int kSelBlock = kSelThreads * kSelPerThread;   // 2048 Gaussians per block

struct SelP {
  SetP lv[FLOD_MAX_SETS];
  float lo[FLOD_MAX_SETS], hi[FLOD_MAX_SETS];
  uint32_t start[FLOD_MAX_SETS + 1];   // first global index of each level (block aligned)
  int n_levels;
  float ox, oy, oz;
  uint32_t total_blocks;
};

__device__ __forceinline__ bool sel_keep(const SelP& s, int lv, uint32_t i) {
  const float* m = s.lv[lv].means + 3ull * i;
  const float dx = __fsub_rn(__ldg(m), s.ox);
  const float dy = __fsub_rn(__ldg(m + 1), s.oy);
  const float dz = __fsub_rn(__ldg(m + 2), s.oz);
  const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  const float d = __fsqrt_rn(d2);
  return d >= s.lo[lv] && d < s.hi[lv];
}

__device__ __forceinline__ int level_of_block(const SelP& s, uint32_t blk) {
  const uint32_t g = blk * (uint32_t)kSelBlock;
  int lv = 0;
  while (lv + 1 < s.n_levels && g >= s.start[lv + 1]) ++lv;
  return lv;
}

constexpr int kSelWords = kSelPerThread * (kSelThreads / 32);   // keep-bit words per block

__global__ void __launch_bounds__(kSelThreads) k_sel_count(const __grid_constant__ SelP s,
                                                           uint32_t* counts, uint32_t* masks) {
  pdl_entry();
  __shared__ uint32_t red[kSelThreads / 32];
  const int lv = level_of_block(s, blockIdx.x);
  const uint32_t i0 = blockIdx.x * (uint32_t)kSelBlock - s.start[lv];
  const uint32_t n = (uint32_t)s.lv[lv].n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t c = 0;
#pragma unroll
  for (int j = 0; j < kSelPerThread; ++j) {
    const uint32_t i = i0 + j * kSelThreads + threadIdx.x;
    const bool keep = i < n && sel_keep(s, lv, i);
    c += keep;
    if (masks) {   // word (round j, warp wid): bit lane = Gaussian i0 + 256 j + 32 wid + lane
      const uint32_t bal = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) masks[(size_t)blockIdx.x * kSelWords + j * (kSelThreads / 32) + wid] = bal;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) t += red[w];
    counts[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_sel_scan(uint32_t* counts, uint32_t nblocks,
                                                   uint32_t* d_count) {
  pdl_entry();
  __shared__ uint32_t wt[32];
  __shared__ uint32_t carry_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  for (uint32_t base = 0; base < nblocks; base += 1024) {
    const uint32_t i = base + tid;
    const uint32_t v = i < nblocks ? counts[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wt[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint32_t w = wt[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      wt[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = carry_s + (wid ? wt[wid - 1] : 0u) + x - v;
    if (i < nblocks) counts[i] = excl;
    __syncthreads();
    if (tid == 1023) carry_s = excl + v;
    __syncthreads();
  }
  if (tid == 0) *d_count = carry_s;
}

__global__ void __launch_bounds__(kSelThreads) k_sel_write(const __grid_constant__ SelP s,
                                                           const uint32_t* offsets,
                                                           const uint32_t* masks, uint32_t* out,
                                                           uint32_t cap) {
  pdl_entry();
  __shared__ uint32_t wcnt[kSelThreads / 32];
  __shared__ uint32_t base_s;
  const int lv = level_of_block(s, blockIdx.x);
  const uint32_t i0 = blockIdx.x * (uint32_t)kSelBlock - s.start[lv];
  const uint32_t n = (uint32_t)s.lv[lv].n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (masks) {
    static_assert(kSelWords == 64, "two keep-bit words per lane of one warp");
    __shared__ uint32_t m[kSelWords], pre[kSelWords];
    if (threadIdx.x < kSelWords) m[threadIdx.x] = masks[(size_t)blockIdx.x * kSelWords + threadIdx.x];
    __syncthreads();
    if (wid == 0) {   // exclusive prefix of the words' counts, in (round, warp) order
      const uint32_t a = __popc(m[2 * lane]), b = __popc(m[2 * lane + 1]);
      uint32_t x = a + b;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      pre[2 * lane] = x - a - b;
      pre[2 * lane + 1] = x - b;
    }
    __syncthreads();
    const uint32_t base = offsets[blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kSelPerThread; ++j) {
      const int q = j * (kSelThreads / 32) + wid;
      const uint32_t bal = m[q];
      if ((bal >> lane) & 1u) {
        const uint32_t pos = base + pre[q] + __popc(bal & lt);
        if (pos < cap) out[pos] = ((uint32_t)lv << FLOD_SEL_SHIFT) | (i0 + j * kSelThreads + threadIdx.x);
      }
    }
    return;
  }
  if (threadIdx.x == 0) base_s = offsets[blockIdx.x];
  // rounds of 256 consecutive Gaussians; inside a round, order = thread order
  for (int j = 0; j < kSelPerThread; ++j) {
    const uint32_t i = i0 + j * kSelThreads + threadIdx.x;
    const bool keep = i < n && sel_keep(s, lv, i);
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wcnt[wid] = __popc(bal);
    __syncthreads();
    uint32_t pre = base_s;
    for (int w = 0; w < wid; ++w) pre += wcnt[w];
    pre += __popc(bal & ((1u << lane) - 1u));
    if (keep && pre < cap) out[pre] = ((uint32_t)lv << FLOD_SEL_SHIFT) | i;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (int w = 0; w < kSelThreads / 32; ++w) t += wcnt[w];
      base_s += t;
    }
    __syncthreads();
  }
}

cudaError_t launch_select(const SetP* levels, int n_levels, const float* lo, const float* hi,
                          const float origin[3], uint32_t* out, uint32_t cap, uint32_t* d_count,
                          uint32_t* scratch, uint32_t* masks, uint32_t n_blocks, cudaStream_t st) {
  SelP s{};
  s.n_levels = n_levels;
  uint32_t g = 0;
  for (int l = 0; l < n_levels; ++l) {
    s.lv[l] = levels[l];
    s.lo[l] = lo[l];
    s.hi[l] = hi[l];
    s.start[l] = g;
    g += (uint32_t)((levels[l].n + kSelBlock - 1) / kSelBlock) * kSelBlock;
  }
  s.start[n_levels] = g;
  s.ox = origin[0];
  s.oy = origin[1];
  s.oz = origin[2];
  s.total_blocks = n_blocks;
  if (n_blocks == 0) {
    return cudaMemsetAsync(d_count, 0, sizeof(uint32_t), st);
  }
  launch_k(k_sel_count, dim3(n_blocks), dim3(kSelThreads), 0, st, s, scratch, masks);
  launch_k(k_sel_scan, dim3(1), dim3(1024), 0, st, scratch, n_blocks, d_count);
  launch_k(k_sel_write, dim3(n_blocks), dim3(kSelThreads), 0, st, s, (const uint32_t*)scratch,
           (const uint32_t*)masks, out, cap);
  return cudaGetLastError();
}

uint32_t select_mask_words() { return (uint32_t)kSelWords; }

uint32_t select_blocks(const int* ns, int n_levels) {
  uint32_t b = 0;
  for (int l = 0; l < n_levels; ++l) b += (uint32_t)((ns[l] + kSelBlock - 1) / kSelBlock);
  return b;
}

// Eq. 5 in float32 with the library exp/log (full precision).
__global__ void k_adjust_scale(float* s_opt, int64_t n, float s_cur, float s_next) {
  pdl_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s_opt[i] = logf(expf(s_opt[i]) + (s_cur - s_next));
}

cudaError_t launch_adjust_scale(float* s_opt, int64_t n, float s_cur, float s_next,
                                cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  launch_k(k_adjust_scale, dim3((unsigned)blocks), dim3(256), 0, st, s_opt, n, s_cur, s_next);
  return cudaGetLastError();
}

}  // namespace flod

// ---------------------------------------------------------------------------------------
// allocation-free variant of the selection: the block-count scratch is a fixed array in
// the library's device image instead of caller memory
// ---------------------------------------------------------------------------------------
static __device__ __align__(256) uint32_t g_select_scratch[FLOD_SELECT_NOALLOC_MAX_BLOCKS + 1];

namespace {
std::mutex g_scratch_mu;
bool g_scratch_ready[64];
void* g_scratch_ptr[64];

// Device address of g_select_scratch for the current device (looked up once per device,
// with that device current). In host code the array's name is only a host-side stand-in.
cudaError_t static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ready[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_select_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
    g_scratch_ready[dev] = true;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" flod_status flod_select_levels_noalloc(const flod_gaussians* levels, int n_levels,
                                                  const float* d_thresh, float gamma,
                                                  float focal, const float origin[3],
                                                  uint32_t* out_sel, uint32_t sel_capacity,
                                                  uint32_t* d_count, flod_stream stream) {
  if (!levels || n_levels < 1 || n_levels > FLOD_MAX_SETS) return FLOD_ERR_INVALID_ARG;
  int ns[FLOD_MAX_SETS];
  for (int l = 0; l < n_levels; ++l) {
    if (levels[l].n < 0 || levels[l].n >= (1 << FLOD_SEL_SHIFT)) return FLOD_ERR_INVALID_ARG;
    ns[l] = levels[l].n;
  }
  // too many Gaussians for the fixed scratch: refuse before anything is enqueued
  if (flod::select_blocks(ns, n_levels) > (uint32_t)FLOD_SELECT_NOALLOC_MAX_BLOCKS)
    return FLOD_ERR_INVALID_ARG;
  void* scratch = nullptr;
  if (static_scratch(&scratch) != cudaSuccess) return FLOD_ERR_CUDA;
  return flod_select_levels(levels, n_levels, d_thresh, gamma, focal, origin, out_sel,
                            sel_capacity, d_count, scratch,
                            sizeof(uint32_t) * (FLOD_SELECT_NOALLOC_MAX_BLOCKS + 1), stream);
}
