// Internal definitions shared by the CUDA translation units of the FLoD splatting path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/flod.h"

namespace flod {

// ---------------------------------------------------------------------------------------
// constants of the blending rule (Sec. 3, after Eq. 2; 3DGS prior art)
// ---------------------------------------------------------------------------------------
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kClampFov = 1.3f;        // Jacobian off-screen guard, x tan(half fov)
constexpr float kExtentMargin = 1.0f + 1.0f / 1024.0f;   // rule 2: tau widened by 2^-10

constexpr int kScanBlock = 1024;         // units per block-sum entry; view capacities are
                                         // rounded up to a multiple of it
constexpr int kMaxViewsSmall = 8;        // views carried in the small parameter table

// ---------------------------------------------------------------------------------------
// per-view / per-set tables, passed by value as __grid_constant__ kernel parameters
// ---------------------------------------------------------------------------------------
struct ViewP {
  float vm[12];
  float fx, fy, cx, cy;
  int width, height;
  float cpx, cpy, cpz;
  int set;
  const uint32_t* sel;
  const uint32_t* sel_count;
  uint32_t cap;        // units reserved (not rounded)
  uint32_t unit_off;   // first unit of the view (multiple of kScanBlock)
  uint32_t tile_off;   // first global tile id
  uint32_t tiles_x, tiles_y;
  uint64_t pix_off;    // first pixel of the view in the concatenated outputs
};

struct SetP {
  const float* means;
  const float* quats;
  const float* s_opt;
  const float* logit;
  const float* sh;
  int n, deg;
  float s_min;
  int bulk_ok;   // every array 16-byte aligned: a CTA's chunk can be staged by cp.async
};

struct CfgP {
  int tile_w, tile_h, batch, extent_rule;
  float dilation, z_near;
  float bg[3];
};

template <int MAXV>
struct Batch {
  int n_views, n_sets;
  uint32_t units, tiles;
  CfgP cfg;
  SetP sets[FLOD_MAX_SETS];
  ViewP views[MAXV];
  uint32_t unit_end[MAXV];  // exclusive prefix ends, for unit -> view lookup
  uint32_t tile_end[MAXV];
};

using BatchS = Batch<kMaxViewsSmall>;
using BatchL = Batch<FLOD_MAX_VIEWS>;

// workspace pointers derived from the layout
struct Ws {
  uint32_t* status;
  unsigned long long* pair_count;
  uint32_t* plan;
  float2* xy;
  float* depth;
  float4* conic_o;
  float4* rgb;
  float* radius;
  float4* ext;             // (m, h, rx, ry): the unit's support ellipse (see UnitTiles)
  uint4* trec;             // the unit's tile record (see rec_row)
  uint32_t* tiles_touched;
  unsigned long long* block_sums;
  uint32_t* slices;
  uint32_t* ukeys[2];      // unit-stage sort: depth keys
  uint32_t* uvals[2];      // unit-stage sort: unit indices (the result is the emission order)
  uint32_t* keys[2];       // pair-stage sort: tile keys
  uint32_t* vals[2];       // pair-stage sort: unit indices (the result is what renders read)
  uint32_t* hist;
  uint32_t* counts;        // radix sort: per-partition digit counts, digit-major
  uint2* ranges;
  float* grad2d;           // per unit 9 floats: du, dv, dopacity, da, db, dc, dr, dg, db
  uint32_t* queue;
  uint64_t pair_capacity;
  uint32_t max_parts;
  uint32_t units;
};

// radix-sort plan words (uint32 plan[64])
constexpr int kPlanPasses = 8;       // slots 0-3: depth digits over units; 4-7: tile digits over pairs
constexpr int kPlanActive = 0;       // plan[kPlanActive + p] = 1 if pass p moves keys
constexpr int kPlanSrc = 8;          // plan[kPlanSrc + p] = source buffer of pass p
constexpr int kPlanNVis = 16;        // uint64 at plan[16]: units with tiles (the sorted unit slots)
constexpr int kPlanDepthMin = 18;    // smallest depth bits of those units
constexpr int kPlanKeyBits = 20;     // significant bits of (depth bits - smallest)
constexpr int kPlanCounter = 24;     // plan[kPlanCounter + p] = finished digit-scan CTAs of pass p
constexpr int kPlanNParts = 40;      // number of partitions
constexpr int kPlanQueue = 41;       // render work-queue ticket counter (x2: fwd, bwd)
constexpr int kPlanSlices = 43;      // number of key-emission slices
constexpr int kPlanNPartsUnits = 44; // partitions of the unit-stage sort
constexpr int kPlanFinalUnits = 45;  // buffer holding the depth-sorted unit order
constexpr int kPlanBigUnits = 46;    // units the light emission leaves to k_emit_big
constexpr int kEmitSlice = 4096;     // output positions per emission slice
constexpr int kQueueHeader = 66;     // queue[0..32] bucket counts, [33..65] offsets, then tiles
constexpr int kPlanEvalFwd = 48;     // uint64 running count of forward evaluations
constexpr int kPlanEvalBwd = 50;     // uint64 running count of backward evaluations
constexpr int kPlanBlended = 52;     // uint64 running count of blended (pixel, Gaussian) pairs
constexpr int kPlanFinal = 63;       // buffer holding the sorted result

constexpr int kRadixBits = 9;                        // digit width of one sort pass
constexpr int kRadixBins = 1 << kRadixBits;          // 512 digit values
constexpr int kSortThreads = 512;                    // one thread per digit value
constexpr int kSortKeysPerThread = 8;
constexpr int kSortPart = kSortThreads * kSortKeysPerThread;   // 4096 keys per partition

template <int MAXV>
__device__ __forceinline__ int view_of_unit(const Batch<MAXV>& b, uint32_t u) {
  int lo = 0, hi = b.n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (u < b.unit_end[mid]) hi = mid; else lo = mid + 1;
  }
  return lo;
}

template <int MAXV>
__device__ __forceinline__ int view_of_tile(const Batch<MAXV>& b, uint32_t t) {
  int lo = 0, hi = b.n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (t < b.tile_end[mid]) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// The pixel rectangle rule, every step rounded to nearest in float32 so that a float32
// reference takes the same decisions: columns ceil((u - r) - 0.5) .. floor((u + r) - 0.5),
// clamped to the image; then tiles. Returns false if empty.
__device__ __forceinline__ bool pixel_rect(float u, float v, float rx, float ry, int W, int H,
                                           int& px0, int& px1, int& py0, int& py1) {
  float x0 = ceilf(__fsub_rn(__fsub_rn(u, rx), 0.5f));
  float x1 = floorf(__fsub_rn(__fadd_rn(u, rx), 0.5f));
  float y0 = ceilf(__fsub_rn(__fsub_rn(v, ry), 0.5f));
  float y1 = floorf(__fsub_rn(__fadd_rn(v, ry), 0.5f));
  // NaN compares false: treat as empty
  if (!(x0 <= x1) || !(y0 <= y1)) return false;
  x0 = fmaxf(x0, 0.f);
  y0 = fmaxf(y0, 0.f);
  x1 = fminf(x1, (float)(W - 1));
  y1 = fminf(y1, (float)(H - 1));
  if (x0 > x1 || y0 > y1) return false;
  px0 = (int)x0;
  px1 = (int)x1;
  py0 = (int)y0;
  py1 = (int)y1;
  return true;
}

// Tile sizes are powers of two (8, 16, 32 pixels: the configurations accepted), so the tile
// of a (non-negative) pixel coordinate is a shift.
__device__ __forceinline__ int tile_shift(int t) { return __ffs(t) - 1; }

// ---------------------------------------------------------------------------------------
// Tile sets of a unit ("segments": one run of tile columns per tile row)
// ---------------------------------------------------------------------------------------
// ext = (m, h, rx, ry) of the unit's support ellipse {d : d^T Sigma'^-1 d <= tau} (extent
// rule 2; rules 0 and 1 store (0, 0, r, r) and list full rectangle rows). Row dy of the
// ellipse is x in u + m dy +- h sqrt(ry^2 - dy^2); its rightmost point lies at
// dy = m ry^2 / rx (the leftmost at minus that) and the right boundary is concave in dy, so
// over a band of rows the extremes are at those points clamped to the band. Every
// operation is rounded explicitly, so that preprocess (which counts the tiles) and emission
// (which lists them) take identical decisions and a float32 reference can repeat them.
struct UnitTiles {
  float u, v;
  float4 e;
  float dyx, ry2;
  int px0, px1, py0, py1;   // pixel rectangle (clamped to the image)
  int ty0, ty1;             // its tile rows
  int tw, th;
  int lw;                   // log2 of the tile width
  bool rows;                // rule 2: per-row column ranges
};

__device__ __forceinline__ bool unit_tiles(float u, float v, float4 e, int W, int H, int tw,
                                           int th, bool rows, UnitTiles& t) {
  if (!pixel_rect(u, v, e.z, e.w, W, H, t.px0, t.px1, t.py0, t.py1)) return false;
  t.u = u;
  t.v = v;
  t.e = e;
  t.ry2 = __fmul_rn(e.w, e.w);
  t.dyx = e.z > 0.f ? __fdiv_rn(__fmul_rn(e.x, t.ry2), e.z) : 0.f;
  const int lh = tile_shift(th);
  t.ty0 = t.py0 >> lh;
  t.ty1 = t.py1 >> lh;
  t.tw = tw;
  t.th = th;
  t.lw = tile_shift(tw);
  t.rows = rows;
  return true;
}

// A unit's tile set as preprocess found it, for the emission ("tile record", uint4):
//   x = tx0 | ty0 << 16       first tile column and row of the rectangle (within the view)
//   y = rows | mode << 16     tile rows of the rectangle, and how the rows are given:
//   mode kRecTable   z, w = up to 4 rows of (column offset from tx0, count) in 8 + 8 bits
//   mode kRecUniform z = tile count of every row (offset 0: rectangle rules)
//   mode kRecCompute the rows are recomputed from (u, v, ext) with unit_row
constexpr uint32_t kRecTable = 0, kRecUniform = 1, kRecCompute = 2;
constexpr int kRecRows = 4;

__device__ __forceinline__ void rec_row(const uint4 r, int row, uint32_t& off, uint32_t& cnt) {
  const uint32_t word = row < 2 ? r.z : r.w;
  const uint32_t h = (word >> (16 * (row & 1))) & 0xffffu;
  off = h & 0xffu;
  cnt = h >> 8;
}

// Tile columns [cx0, cx1] of tile row ty (ty0 <= ty <= ty1); false if the row has none.
__device__ __forceinline__ bool unit_row(const UnitTiles& t, int ty, int& cx0, int& cx1) {
  if (!t.rows) {
    cx0 = t.px0 >> t.lw;
    cx1 = t.px1 >> t.lw;
    return true;
  }
  const int jy0 = max(ty * t.th, t.py0);
  const int jy1 = min(ty * t.th + t.th - 1, t.py1);
  const float dy0 = __fsub_rn((float)jy0 + 0.5f, t.v);
  const float dy1 = __fsub_rn((float)jy1 + 0.5f, t.v);
  const float dr = fminf(fmaxf(t.dyx, dy0), dy1);
  const float dl = fminf(fmaxf(-t.dyx, dy0), dy1);
  const float wr = __fmul_rn(t.e.y, __fsqrt_rn(fmaxf(__fsub_rn(t.ry2, __fmul_rn(dr, dr)), 0.f)));
  const float wl = dl == dr ? wr  // same point: the same value, one square root fewer
                            : __fmul_rn(t.e.y, __fsqrt_rn(fmaxf(__fsub_rn(t.ry2, __fmul_rn(dl, dl)), 0.f)));
  const float xr = __fadd_rn(__fadd_rn(t.u, __fmul_rn(t.e.x, dr)), wr);
  const float xl = __fsub_rn(__fadd_rn(t.u, __fmul_rn(t.e.x, dl)), wl);
  const float c0 = fmaxf(ceilf(__fsub_rn(xl, 0.5f)), (float)t.px0);
  const float c1 = fminf(floorf(__fsub_rn(xr, 0.5f)), (float)t.px1);
  if (!(c0 <= c1)) return false;
  cx0 = (int)c0 >> t.lw;
  cx1 = (int)c1 >> t.lw;
  return true;
}

// Per-pixel opacity of a splat: alpha = min(0.99, o * exp(-q/2)) with
// q = a dx^2 + 2 b dx dy + c dy^2, dx = px - u. The conic arrives pre-scaled by -log2(e)/2
// (see scale_conic), so exp(-q/2) = 2^(q') with one hardware ex2 (splat_alpha). Written with explicit
// roundings so that the forward and the backward pass recompute bit-identical values.
constexpr float kNegHalfLog2e = -0.5f * 1.4426950408889634f;

// (a, b, c, o) -> (a k, 2 b k, c k, o) with k = -log2(e)/2
__device__ __forceinline__ float4 scale_conic(float4 co) {
  return make_float4(co.x * kNegHalfLog2e, 2.f * co.y * kNegHalfLog2e, co.z * kNegHalfLog2e, co.w);
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// With t0 = (a' dx) dx and t1 = (2b') dx computed once per Gaussian and column,
// q' = t0 + dy (t1 + c' dy) for each pixel row of that column.
__device__ __forceinline__ float splat_q(float t0, float t1, float dy, float4 cs) {
  return __fmaf_rn(dy, __fmaf_rn(cs.z, dy, t1), t0);
}

// The skip rule alpha < 1/255 taken on q' before any exponential: o 2^q' >= 1/255 <=>
// q' >= -log2(255 o) (the splat's threshold, computed once per batch load). The forward and
// the backward take the decision with the same numbers.
__device__ __forceinline__ float splat_qmin(float o) {
  float l;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(255.f * o));
  return -l;
}

// alpha = min(0.99, o 2^q'), with g = 2^q' (= exp(-q/2)) returned for the backward.
__device__ __forceinline__ float splat_alpha(float qs, float o, float& g) {
  g = ex2_approx(qs);
  return fminf(kAlphaMax, __fmul_rn(o, g));
}

// Pairs of float32 values in one instruction (sm_100 and later): where two results share an
// operand, one packed instruction does the work of two scalar ones.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// ---------------------------------------------------------------------------------------
// Programmatic dependent launch. Every kernel is launched so that it may be scheduled while
// the previous kernel of its stream drains (launch_k). Its first statement waits for that
// kernel to complete and its writes to be visible (before any global memory access, so the
// order of the stream is kept), then lets the next kernel be scheduled.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------------------------------
// Asynchronous copies global -> shared memory (cp.async, 16 bytes per request). The
// requests of a CTA are spread over its threads and complete with one wait_all per thread
// followed by a barrier: no copy can still be writing into a CTA's shared memory once its
// threads have passed that barrier, so no exit path leaves a copy in flight.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// dst, src 16-byte aligned, bytes a multiple of 16; every thread of the CTA takes part
// (blockDim.x a multiple of 32). Each warp copies one contiguous share of the range, 512
// bytes per instruction: at 3M Gaussians the preprocess staged this way ran 0.168 ms
// against 0.188 ms with the range strided over the whole CTA (DRAM locality).
__device__ __forceinline__ void async_copy(void* dst, const void* src, uint32_t bytes) {
  const char* s = static_cast<const char*>(src);
  const uint32_t d = smem_addr(dst);
  const uint32_t nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t per = (bytes + nw * 512u - 1u) / (nw * 512u) * 512u;   // bytes per warp
  const uint32_t end = min(bytes, (w + 1u) * per);
  for (uint32_t o = w * per + lane * 16u; o < end; o += 512u)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + o), "l"(s + o) : "memory");
}

// Waits for every cp.async this thread issued (the caller then synchronises the CTA).
__device__ __forceinline__ void async_copy_wait() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Named CTA barriers (ids 1..15; 0 is __syncthreads) for producer / consumer hand-offs
// between warp groups: `arrive` counts the calling warp in and goes on, `sync` waits until
// n threads (a multiple of 32) have arrived or synced; both order the shared-memory
// accesses before them against those after the barrier completes. The warps of both
// groups stay resident in the same CTA, so every wait ends once the other group reaches
// its matching arrive.
__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Tile count of every depth-sorted unit slot (written by the binning after the unit sort,
// into the unit sort's key buffer 0, whose keys are no longer needed then).
__device__ __forceinline__ uint32_t* slot_counts(const Ws& ws) { return ws.ukeys[0]; }

// Number of depth-sorted unit slots (units with at least one tile).
__device__ __forceinline__ uint32_t visible_units(const Ws& ws) {
  return (uint32_t)*reinterpret_cast<const unsigned long long*>(ws.plan + kPlanNVis);
}

__device__ __forceinline__ void set_status(uint32_t* status, uint32_t bits) {
  atomicOr(status, bits);
}

}  // namespace flod
