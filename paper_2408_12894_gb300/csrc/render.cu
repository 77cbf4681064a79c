// Per-tile alpha blending (Sec. 3, after Eq. 2: the image is the alpha blend of the
// projected Gaussians in depth order) and its backward.
//
// Forward: one CTA per tile (one thread per pixel). The tile's sorted Gaussians are staged
// into shared memory in batches; every pixel walks them front to back:
//   alpha = min(0.99, o exp(-q/2)); skip alpha < 1/255; stop before the Gaussian that
//   would take T below 1e-4; C += rgb alpha T; T *= 1 - alpha.
// The CTA leaves as soon as every pixel has stopped (__syncthreads_count).
//
// Backward: the same tiles, every pixel walking back to front from its last blended
// Gaussian (n_contrib) and recovering T by division by (1 - alpha), so no per-pair state is
// stored. d(alpha) = sum_c g_c (rgb_c T - S_c / (1 - alpha)), S = colour behind + T_final bg.
// The nine per-Gaussian gradients of a warp are reduced with shuffles and one lane adds
// them with float4 atomics; warps where no pixel touches the Gaussian skip the reduction.
#include "common.cuh"
#include "kernels.h"

namespace flod {

__device__ __forceinline__ void add_evals(uint32_t* counter, uint32_t evals);

template <int MAXV>
__device__ __forceinline__ void tile_pixel(const Batch<MAXV>& b, uint32_t tile, int& vi,
                                           int& px, int& py) {
  vi = view_of_tile(b, tile);
  const ViewP& V = b.views[vi];
  const uint32_t lt = tile - V.tile_off;
  const int tx = (int)(lt % V.tiles_x), ty = (int)(lt / V.tiles_x);
  px = tx * b.cfg.tile_w + (int)(threadIdx.x % (unsigned)b.cfg.tile_w);
  py = ty * b.cfg.tile_h + (int)(threadIdx.x / (unsigned)b.cfg.tile_w);
}

template <int MAXV>
__global__ void __launch_bounds__(256) k_render_fwd(const __grid_constant__ Batch<MAXV> b, Ws ws,
                                                    float* __restrict__ out_rgb,
                                                    float* __restrict__ out_T,
                                                    uint32_t* __restrict__ out_nc) {
  __shared__ float2 s_xy[256];
  __shared__ float4 s_co[256];
  __shared__ float4 s_rgb[256];
  const uint32_t tile = blockIdx.x;
  int vi, px, py;
  tile_pixel(b, tile, vi, px, py);
  const ViewP& V = b.views[vi];
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  const bool inside = px < V.width && py < V.height;
  const uint32_t* __restrict__ vals = ws.vals[ws.plan[kPlanFinal]];
  const uint2 rg = ws.ranges[tile];
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const int batch = b.cfg.batch;
  float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
  uint32_t last = 0, evals = 0;
  bool done = !inside;
  for (uint32_t start = rg.x; start < rg.y; start += batch) {
    if (__syncthreads_count(done) == nthr) break;
    const int cnt = (int)min((uint32_t)batch, rg.y - start);
    for (int k = tid; k < cnt; k += nthr) {
      const uint32_t id = vals[start + k];
      s_xy[k] = ws.xy[id];
      s_co[k] = ws.conic_o[id];
      s_rgb[k] = ws.rgb[id];
    }
    __syncthreads();
    if (!done) {
      int k = 0;
      for (; k < cnt; ++k) {
        const float2 m = s_xy[k];
        float g;
        const float a = splat_alpha(fx - m.x, fy - m.y, s_co[k], g);
        if (a < kAlphaMin) continue;
        const float Tn = T * (1.f - a);
        if (Tn < kTMin) {
          done = true;
          ++k;
          break;
        }
        const float4 c = s_rgb[k];
        const float w = a * T;
        c0 += w * c.x;
        c1 += w * c.y;
        c2 += w * c.z;
        T = Tn;
        last = start - rg.x + (uint32_t)k + 1u;
      }
      evals += (uint32_t)k;
    }
  }
  add_evals(ws.plan + kPlanEvalFwd, evals);
  if (inside) {
    const uint64_t npix = (uint64_t)V.width * V.height;
    const uint64_t p = (uint64_t)py * V.width + px;
    out_rgb[3 * V.pix_off + p] = c0 + T * b.cfg.bg[0];
    out_rgb[3 * V.pix_off + npix + p] = c1 + T * b.cfg.bg[1];
    out_rgb[3 * V.pix_off + 2 * npix + p] = c2 + T * b.cfg.bg[2];
    out_T[V.pix_off + p] = T;
    out_nc[V.pix_off + p] = last;
  }
}

// one 64-bit atomic per CTA: the number of (pixel, Gaussian) evaluations of the launch
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

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int MAXV>
__global__ void __launch_bounds__(256) k_render_bwd(const __grid_constant__ Batch<MAXV> b, Ws ws,
                                                    const float* __restrict__ dL,
                                                    const float* __restrict__ fwd_T,
                                                    const uint32_t* __restrict__ fwd_nc) {
  __shared__ uint32_t s_id[256];
  __shared__ float2 s_xy[256];
  __shared__ float4 s_co[256];
  __shared__ float4 s_rgb[256];
  __shared__ uint32_t s_max;
  const uint32_t tile = blockIdx.x;
  int vi, px, py;
  tile_pixel(b, tile, vi, px, py);
  const ViewP& V = b.views[vi];
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  const bool inside = px < V.width && py < V.height;
  const uint32_t* __restrict__ vals = ws.vals[ws.plan[kPlanFinal]];
  const uint2 rg = ws.ranges[tile];
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const int batch = b.cfg.batch;
  const uint64_t npix = (uint64_t)V.width * V.height;
  const uint64_t p = inside ? (uint64_t)py * V.width + px : 0;
  float T = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
  uint32_t last = 0;
  if (inside) {
    T = fwd_T[V.pix_off + p];
    last = fwd_nc[V.pix_off + p];
    g0 = dL[3 * V.pix_off + p];
    g1 = dL[3 * V.pix_off + npix + p];
    g2 = dL[3 * V.pix_off + 2 * npix + p];
  }
  const float Tf = T;
  float S0 = Tf * b.cfg.bg[0], S1 = Tf * b.cfg.bg[1], S2 = Tf * b.cfg.bg[2];
  if (tid == 0) s_max = 0;
  __syncthreads();
  if (last) atomicMax(&s_max, last);
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
      s_co[k] = ws.conic_o[id];
      s_rgb[k] = ws.rgb[id];
    }
    __syncthreads();
    for (int k = cnt - 1; k >= 0; --k) {
      const uint32_t pos = bstart - rg.x + (uint32_t)k + 1u;
      const float2 m = s_xy[k];
      const float4 co = s_co[k];
      const float dx = fx - m.x, dy = fy - m.y;
      float gg = 0.f, a = 0.f;
      bool on = inside && pos <= last;
      if (on) {
        a = splat_alpha(dx, dy, co, gg);
        on = a >= kAlphaMin;
      }
      float du = 0.f, dv = 0.f, dop = 0.f, dca = 0.f, dcb = 0.f, dcc = 0.f;
      float dr = 0.f, dg = 0.f, dbl = 0.f;
      if (on) {
        const float4 c = s_rgb[k];
        const float om = 1.f - a;
        T = T / om;
        const float w = a * T;
        dr = w * g0;
        dg = w * g1;
        dbl = w * g2;
        const float ioma = 1.f / om;
        const float dalpha = g0 * (c.x * T - S0 * ioma) + g1 * (c.y * T - S1 * ioma) +
                             g2 * (c.z * T - S2 * ioma);
        S0 += c.x * w;
        S1 += c.y * w;
        S2 += c.z * w;
        if (co.w * gg < kAlphaMax) {
          dop = gg * dalpha;
          const float dq = -0.5f * co.w * gg * dalpha;   // dL/dq
          dca = dq * dx * dx;
          dcb = dq * 2.f * dx * dy;
          dcc = dq * dy * dy;
          du = -dq * 2.f * (co.x * dx + co.y * dy);
          dv = -dq * 2.f * (co.y * dx + co.z * dy);
        }
      }
      if (__any_sync(0xffffffffu, on)) {
        du = warp_sum(du);
        dv = warp_sum(dv);
        dop = warp_sum(dop);
        dca = warp_sum(dca);
        dcb = warp_sum(dcb);
        dcc = warp_sum(dcc);
        dr = warp_sum(dr);
        dg = warp_sum(dg);
        dbl = warp_sum(dbl);
        if ((tid & 31) == 0) {
          float4* gp = ws.grad2d + 3ull * s_id[k];
          atomicAdd(gp, make_float4(du, dv, dop, 0.f));
          atomicAdd(gp + 1, make_float4(dca, dcb, dcc, 0.f));
          atomicAdd(gp + 2, make_float4(dr, dg, dbl, 0.f));
        }
      }
    }
    bend = bstart;
  }
  add_evals(ws.plan + kPlanEvalBwd, last);
}

template <int MAXV>
cudaError_t launch_render_fwd(const Batch<MAXV>& b, const Ws& ws, float* out_rgb, float* out_T,
                              uint32_t* out_nc, int resident, bool persistent, cudaStream_t st) {
  (void)resident;
  (void)persistent;
  if (b.tiles == 0) return cudaSuccess;
  k_render_fwd<MAXV><<<b.tiles, b.cfg.tile_w * b.cfg.tile_h, 0, st>>>(b, ws, out_rgb, out_T, out_nc);
  return cudaGetLastError();
}

template <int MAXV>
cudaError_t launch_render_bwd(const Batch<MAXV>& b, const Ws& ws, const float* dL,
                              const float* fwd_T, const uint32_t* fwd_nc, int resident,
                              bool persistent, cudaStream_t st) {
  (void)resident;
  (void)persistent;
  if (b.tiles == 0) return cudaSuccess;
  k_render_bwd<MAXV><<<b.tiles, b.cfg.tile_w * b.cfg.tile_h, 0, st>>>(b, ws, dL, fwd_T, fwd_nc);
  return cudaGetLastError();
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
