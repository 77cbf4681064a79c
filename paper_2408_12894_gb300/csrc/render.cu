// Per-tile alpha blending (Sec. 3, after Eq. 2: the image is the alpha blend of the
// projected Gaussians in depth order) and its backward.
//
// Forward: a CTA renders one tile; each thread owns PIX pixels of one column. The tile's
// sorted Gaussians are staged into shared memory in batches (mean, conic pre-scaled by
// -log2(e)/2 with the opacity, colour); every pixel walks them front to back:
//   alpha = min(0.99, o exp(-q/2)); skip alpha < 1/255 (decided on q before the exponential);
//   stop before the Gaussian that would take T below 1e-4; C += rgb alpha T; T *= 1 - alpha.
// The CTA leaves the tile as soon as every pixel has stopped (__syncthreads_count).
//
// Backward: the same tiles, every pixel walking back to front from its last blended
// Gaussian (n_contrib) and recovering T by multiplying with 1 / (1 - alpha), so no per-pair
// state is stored. d(alpha) = T (g . rgb) - P / (1 - alpha), with P = g . S the upstream
// gradient against the colour behind (S, background T_final bg included), kept as one
// scalar per pixel. The conic and mean gradients are linear in dL/dq times dx^2, dx dy,
// dy^2, dx, dy; dx is fixed per thread (one column), so a thread sums only the moments
// (1, dy, dy^2) of dL/dq over its PIX pixels and expands them once per Gaussian. A warp then
// reduces the nine per-Gaussian gradients with a transposing butterfly and the owning lanes
// add them with atomics; warps where no pixel touches the Gaussian skip the reduction.
//
// Launch modes: one CTA per tile in tile order, or persistent CTAs (about the number that
// fit on the GPU) taking tiles from the largest-first queue that flod_bin_sort builds.
#include "common.cuh"
#include "kernels.h"

namespace flod {

// one 64-bit atomic per CTA: a count of (pixel, Gaussian) pairs of the launch
__device__ __forceinline__ void add_evals(uint32_t* counter, uint32_t evals) {
  __shared__ unsigned long long s_ev;
  if (threadIdx.x == 0) s_ev = 0;
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
  if ((threadIdx.x & 31) == 0 && evals) atomicAdd(&s_ev, (unsigned long long)evals);
  __syncthreads();
  if (threadIdx.x == 0 && s_ev) atomicAdd(reinterpret_cast<unsigned long long*>(counter), s_ev);
}

// Next tile for this CTA: the block index (one-shot mode) or a queue ticket (persistent).
template <bool PERSIST>
__device__ __forceinline__ bool next_tile(const Ws& ws, uint32_t n_tiles, int counter,
                                          bool first, uint32_t& tile) {
  __shared__ uint32_t s_item;
  if (!PERSIST) {
    tile = blockIdx.x;
    return first;
  }
  __syncthreads();
  if (threadIdx.x == 0) s_item = atomicAdd(&ws.plan[kPlanQueue + counter], 1u);
  __syncthreads();
  const uint32_t item = s_item;
  if (item >= n_tiles) return false;
  tile = ws.queue[kQueueHeader + item];
  return true;
}

// ---------------------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------------------
template <int MAXV, int PIX, bool PERSIST>
__global__ void __launch_bounds__(256 / PIX) k_render_fwd(const __grid_constant__ Batch<MAXV> b,
                                                          Ws ws, float* __restrict__ out_rgb,
                                                          float* __restrict__ out_T,
                                                          uint32_t* __restrict__ out_nc) {
  __shared__ float4 s_xq[256];    // mean x, y and the skip threshold q'_min
  __shared__ float4 s_cs[256];
  __shared__ float4 s_rgb[256];
  const uint32_t* __restrict__ vals = ws.vals[ws.plan[kPlanFinal]];
  const int tw = b.cfg.tile_w;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int batch = b.cfg.batch;
  uint32_t evals = 0, blended = 0;
  uint32_t tile;
  for (bool first = true; next_tile<PERSIST>(ws, b.tiles, 0, first, tile); first = false) {
    const ViewP& V = b.views[view_of_tile(b, tile)];
    const uint32_t lt = tile - V.tile_off;
    const int px = (int)(lt % V.tiles_x) * tw + tid % tw;
    const int py0 = (int)(lt / V.tiles_x) * b.cfg.tile_h + (tid / tw) * PIX;
    const uint2 rg = ws.ranges[tile];
    const float fx = (float)px + 0.5f;
    float T[PIX], c0[PIX], c1[PIX], c2[PIX], fy[PIX];
    uint32_t last[PIX], stop[PIX];
    bool live[PIX];
    bool done = true;
#pragma unroll
    for (int j = 0; j < PIX; ++j) {
      T[j] = 1.f;
      c0[j] = c1[j] = c2[j] = 0.f;
      last[j] = 0;
      stop[j] = 0;
      fy[j] = (float)(py0 + j) + 0.5f;
      live[j] = px < V.width && py0 + j < V.height;
      done = done && !live[j];
    }
    uint32_t pos = 0;   // Gaussians of the tile list walked so far
    for (uint32_t start = rg.x; start < rg.y; start += batch) {
      if (__syncthreads_count(done) == nthr) break;
      const int cnt = (int)min((uint32_t)batch, rg.y - start);
      for (int k = tid; k < cnt; k += nthr) {
        const uint32_t id = vals[start + k];
        const float2 m = ws.xy[id];
        const float4 co = ws.conic_o[id];
        s_xq[k] = make_float4(m.x, m.y, splat_qmin(co.w), 0.f);
        s_cs[k] = scale_conic(co);
        s_rgb[k] = ws.rgb[id];
      }
      __syncthreads();
      if (!done) {
#pragma unroll 4
        for (int k = 0; k < cnt; ++k) {
          const float4 mq = s_xq[k];
          const float4 cs = s_cs[k];
          const float dx = fx - mq.x;
          const float t0 = __fmul_rn(__fmul_rn(cs.x, dx), dx);
          const float t1 = __fmul_rn(cs.y, dx);
          ++pos;
#pragma unroll
          for (int j = 0; j < PIX; ++j) {
            const float qs = splat_q(t0, t1, fy[j] - mq.y, cs);
            if (!live[j] || qs < mq.z) continue;     // stopped, or alpha < 1/255
            float g;
            const float a = splat_alpha(qs, cs.w, g);
            const float Tn = T[j] * (1.f - a);
            if (Tn < kTMin) {
              live[j] = false;
              stop[j] = pos;
              continue;
            }
            const float4 c = s_rgb[k];
            const float w = a * T[j];
            c0[j] += w * c.x;
            c1[j] += w * c.y;
            c2[j] += w * c.z;
            T[j] = Tn;
            last[j] = pos;
            ++blended;
          }
          if ((k & 7) == 7) {              // every eighth splat: leave once all pixels stopped
            bool any_live = false;
#pragma unroll
            for (int j = 0; j < PIX; ++j) any_live = any_live || live[j];
            if (!any_live) {
              done = true;
              break;
            }
          }
        }
        if (!done) {
          bool any_live = false;
#pragma unroll
          for (int j = 0; j < PIX; ++j) any_live = any_live || live[j];
          done = !any_live;
        }
      }
    }
    const uint64_t npix = (uint64_t)V.width * V.height;
#pragma unroll
    for (int j = 0; j < PIX; ++j) {
      const int py = py0 + j;
      if (px < V.width && py < V.height) {
        evals += live[j] ? pos : stop[j];
        const uint64_t p = (uint64_t)py * V.width + px;
        out_rgb[3 * V.pix_off + p] = c0[j] + T[j] * b.cfg.bg[0];
        out_rgb[3 * V.pix_off + npix + p] = c1[j] + T[j] * b.cfg.bg[1];
        out_rgb[3 * V.pix_off + 2 * npix + p] = c2[j] + T[j] * b.cfg.bg[2];
        out_T[V.pix_off + p] = T[j];
        out_nc[V.pix_off + p] = last[j];
      }
    }
  }
  add_evals(ws.plan + kPlanEvalFwd, evals);
  add_evals(ws.plan + kPlanBlended, blended);
}

// ---------------------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------------------

// Sums nine per-lane values over the warp and adds each total to its slot of a unit's
// 2D-gradient record (du, dv, dop | da, db, dc | dr, dg, db). A transposing butterfly: at
// each shuffle distance a lane keeps one half of its values, sends the other half to its
// partner and adds what it receives, so after distances 16, 8, 4, 2 every lane holds one
// partial sum; distance 1 completes it. 12 shuffles instead of 45.
__device__ __forceinline__ void warp_reduce_add9(float (&v)[9], float4* rec) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float w[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {                 // 10 slots (slot 9 is empty) -> 5
    const float lo = v[i], hi = i < 4 ? v[5 + i] : 0.f;
    const float send = b4 ? lo : hi;
    w[i] = (b4 ? hi : lo) + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float x[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {                 // 6 slots (slot 5 empty) -> 3
    const float lo = w[i], hi = i < 2 ? w[3 + i] : 0.f;
    const float send = b3 ? lo : hi;
    x[i] = (b3 ? hi : lo) + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float y[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {                 // 4 slots (slot 3 empty) -> 2
    const float lo = x[i], hi = i < 1 ? x[2 + i] : 0.f;
    const float send = b2 ? lo : hi;
    y[i] = (b2 ? hi : lo) + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  float z;
  {
    const float send = b1 ? y[0] : y[1];
    z = (b1 ? y[1] : y[0]) + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  // which of the nine values this lane now holds
  const int i3 = (b2 ? 2 : 0) + (b1 ? 1 : 0);   // index into x (valid < 3)
  const int i2 = (b3 ? 3 : 0) + i3;             // index into w (valid < 5)
  const int i1 = (b4 ? 5 : 0) + i2;             // original index (valid < 9)
  if ((lane & 1) == 0 && i3 < 3 && i2 < 5 && i1 < 9 && z != 0.f)
    atomicAdd(reinterpret_cast<float*>(rec) + i1 + i1 / 3, z);
}

template <int MAXV, int PIX, bool PERSIST>
__global__ void __launch_bounds__(256 / PIX) k_render_bwd(const __grid_constant__ Batch<MAXV> b,
                                                          Ws ws, const float* __restrict__ dL,
                                                          const float* __restrict__ fwd_T,
                                                          const uint32_t* __restrict__ fwd_nc) {
  __shared__ uint32_t s_id[256];
  __shared__ float2 s_xy[256];
  __shared__ float4 s_co[256];
  __shared__ float4 s_cs[256];
  __shared__ float4 s_rgb[256];
  __shared__ uint32_t s_max;
  const uint32_t* __restrict__ vals = ws.vals[ws.plan[kPlanFinal]];
  const int tw = b.cfg.tile_w;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int batch = b.cfg.batch;
  uint32_t evals = 0;
  uint32_t tile;
  for (bool first = true; next_tile<PERSIST>(ws, b.tiles, 1, first, tile); first = false) {
    const ViewP& V = b.views[view_of_tile(b, tile)];
    const uint32_t lt = tile - V.tile_off;
    const int px = (int)(lt % V.tiles_x) * tw + tid % tw;
    const int py0 = (int)(lt / V.tiles_x) * b.cfg.tile_h + (tid / tw) * PIX;
    const uint2 rg = ws.ranges[tile];
    const float fx = (float)px + 0.5f;
    const uint64_t npix = (uint64_t)V.width * V.height;
    // per pixel: T, the upstream gradient g, and P = g . (colour behind the current splat,
    // background included), the only use of that colour in the chain rule
    float T[PIX], g0[PIX], g1[PIX], g2[PIX], P[PIX], fy[PIX];
    uint32_t last[PIX];
    uint32_t my_max = 0;
#pragma unroll
    for (int j = 0; j < PIX; ++j) {
      const int py = py0 + j;
      fy[j] = (float)py + 0.5f;
      T[j] = g0[j] = g1[j] = g2[j] = 0.f;
      last[j] = 0;
      if (px < V.width && py < V.height) {
        const uint64_t p = (uint64_t)py * V.width + px;
        T[j] = fwd_T[V.pix_off + p];
        last[j] = fwd_nc[V.pix_off + p];
        g0[j] = dL[3 * V.pix_off + p];
        g1[j] = dL[3 * V.pix_off + npix + p];
        g2[j] = dL[3 * V.pix_off + 2 * npix + p];
      }
      P[j] = T[j] * (g0[j] * b.cfg.bg[0] + g1[j] * b.cfg.bg[1] + g2[j] * b.cfg.bg[2]);
      my_max = max(my_max, last[j]);
      evals += last[j];
    }
    if (tid == 0) s_max = 0;
    __syncthreads();
    if (my_max) atomicMax(&s_max, my_max);
    __syncthreads();
    const uint32_t end = rg.x + s_max;
    for (uint32_t bend = end; bend > rg.x;) {
      const uint32_t bstart = bend - rg.x > (uint32_t)batch ? bend - batch : rg.x;
      const int cnt = (int)(bend - bstart);
      __syncthreads();
      for (int k = tid; k < cnt; k += nthr) {
        const uint32_t id = vals[bstart + k];
        s_id[k] = id;
        s_xy[k] = ws.xy[id];
        const float4 co = ws.conic_o[id];
        s_co[k] = co;
        float4 cs = scale_conic(co);
        cs.w = splat_qmin(co.w);     // the opacity stays in s_co
        s_cs[k] = cs;
        s_rgb[k] = ws.rgb[id];
      }
      __syncthreads();
#pragma unroll 4
      for (int k = cnt - 1; k >= 0; --k) {
        const uint32_t pos = bstart - rg.x + (uint32_t)k + 1u;
        const float2 m = s_xy[k];
        const float4 co = s_co[k];
        const float4 cs = s_cs[k];   // (a', 2b', c', q'_min)
        const float4 c = s_rgb[k];
        const float dx = fx - m.x;
        const float t0 = __fmul_rn(__fmul_rn(cs.x, dx), dx);
        const float t1 = __fmul_rn(cs.y, dx);
        // this thread's sums over its pixels: colour gradient, and the moments
        // E0 = sum e, E1 = sum e dy, E2 = sum e dy^2 of e = G dL/dalpha (unclamped alpha)
        float r0 = 0.f, r1 = 0.f, r2 = 0.f, E0 = 0.f, E1 = 0.f, E2 = 0.f;
        bool any = false;
#pragma unroll
        for (int j = 0; j < PIX; ++j) {
          if (pos > last[j]) continue;
          const float dy = fy[j] - m.y;
          const float qs = splat_q(t0, t1, dy, cs);
          if (qs < cs.w) continue;                   // alpha < 1/255
          any = true;
          float gg;
          const float a = splat_alpha(qs, co.w, gg);
          const float ioma = rcp_approx(1.f - a);
          T[j] *= ioma;                              // T in front of this splat
          const float w = a * T[j];
          r0 += w * g0[j];
          r1 += w * g1[j];
          r2 += w * g2[j];
          const float gc = g0[j] * c.x + g1[j] * c.y + g2[j] * c.z;
          const float dalpha = T[j] * gc - ioma * P[j];
          P[j] += w * gc;
          if (co.w * gg < kAlphaMax) {
            const float e = gg * dalpha;
            const float ed = e * dy;
            E0 += e;
            E1 += ed;
            E2 += ed * dy;
          }
        }
        if (__any_sync(0xffffffffu, any)) {
          // dL/dq = -o/2 e; q = a dx^2 + 2 b dx dy + c dy^2, dq/du = -2 (a dx + b dy), ...
          const float hq = -0.5f * co.w;
          const float Q0 = hq * E0, Q1 = hq * E1;
          float acc[9];
          acc[0] = -2.f * (co.x * dx * Q0 + co.y * Q1);
          acc[1] = -2.f * (co.y * dx * Q0 + co.z * Q1);
          acc[2] = E0;
          acc[3] = dx * dx * Q0;
          acc[4] = 2.f * dx * Q1;
          acc[5] = hq * E2;
          acc[6] = r0;
          acc[7] = r1;
          acc[8] = r2;
          warp_reduce_add9(acc, ws.grad2d + 3ull * s_id[k]);
        }
      }
      bend = bstart;
    }
  }
  add_evals(ws.plan + kPlanEvalBwd, evals);
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
// Persistent grid size: CTAs of `kernel` that fit on the device at once.
static int resident_ctas(const void* kernel, int threads, int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * sms;
}

template <int MAXV, int PIX>
static cudaError_t fwd_launch(const Batch<MAXV>& b, const Ws& ws, float* out_rgb, float* out_T,
                              uint32_t* out_nc, int resident, bool persistent, cudaStream_t st) {
  const int thr = b.cfg.tile_w * b.cfg.tile_h / PIX;
  if (persistent) {
    cudaError_t e = cudaMemsetAsync(ws.plan + kPlanQueue, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    static int cached = 0;
    if (!cached) cached = resident_ctas((const void*)k_render_fwd<MAXV, PIX, true>, thr, resident);
    const uint32_t grid = min((uint32_t)cached, b.tiles);
    k_render_fwd<MAXV, PIX, true><<<grid, thr, 0, st>>>(b, ws, out_rgb, out_T, out_nc);
  } else {
    k_render_fwd<MAXV, PIX, false><<<b.tiles, thr, 0, st>>>(b, ws, out_rgb, out_T, out_nc);
  }
  return cudaGetLastError();
}

template <int MAXV, int PIX>
static cudaError_t bwd_launch(const Batch<MAXV>& b, const Ws& ws, const float* dL,
                              const float* fwd_T, const uint32_t* fwd_nc, int resident,
                              bool persistent, cudaStream_t st) {
  const int thr = b.cfg.tile_w * b.cfg.tile_h / PIX;
  if (persistent) {
    cudaError_t e = cudaMemsetAsync(ws.plan + kPlanQueue + 1, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    static int cached = 0;
    if (!cached) cached = resident_ctas((const void*)k_render_bwd<MAXV, PIX, true>, thr, resident);
    const uint32_t grid = min((uint32_t)cached, b.tiles);
    k_render_bwd<MAXV, PIX, true><<<grid, thr, 0, st>>>(b, ws, dL, fwd_T, fwd_nc);
  } else {
    k_render_bwd<MAXV, PIX, false><<<b.tiles, thr, 0, st>>>(b, ws, dL, fwd_T, fwd_nc);
  }
  return cudaGetLastError();
}

// resident: the device's SM count (the persistent grid is SMs x resident CTAs per SM); one
// thread per 2 (forward) or 4 (backward; 2 for 8x8 tiles) pixels
template <int MAXV>
cudaError_t launch_render_fwd(const Batch<MAXV>& b, const Ws& ws, float* out_rgb, float* out_T,
                              uint32_t* out_nc, int resident, bool persistent, cudaStream_t st) {
  if (b.tiles == 0) return cudaSuccess;
  return fwd_launch<MAXV, 2>(b, ws, out_rgb, out_T, out_nc, resident, persistent, st);
}

template <int MAXV>
cudaError_t launch_render_bwd(const Batch<MAXV>& b, const Ws& ws, const float* dL,
                              const float* fwd_T, const uint32_t* fwd_nc, int resident,
                              bool persistent, cudaStream_t st) {
  if (b.tiles == 0) return cudaSuccess;
  if (b.cfg.tile_w * b.cfg.tile_h >= 128)
    return bwd_launch<MAXV, 4>(b, ws, dL, fwd_T, fwd_nc, resident, persistent, st);
  return bwd_launch<MAXV, 2>(b, ws, dL, fwd_T, fwd_nc, resident, persistent, st);
}

template cudaError_t launch_render_fwd<kMaxViewsSmall>(const BatchS&, const Ws&, float*, float*,
                                                       uint32_t*, int, bool, cudaStream_t);
template cudaError_t launch_render_fwd<FLOD_MAX_VIEWS>(const BatchL&, const Ws&, float*, float*,
                                                       uint32_t*, int, bool, cudaStream_t);
template cudaError_t launch_render_bwd<kMaxViewsSmall>(const BatchS&, const Ws&, const float*,
                                                       const float*, const uint32_t*, int, bool,
                                                       cudaStream_t);
template cudaError_t launch_render_bwd<FLOD_MAX_VIEWS>(const BatchL&, const Ws&, const float*,
                                                       const float*, const uint32_t*, int, bool,
                                                       cudaStream_t);

}  // namespace flod
