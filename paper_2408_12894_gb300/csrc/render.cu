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
// add them with atomics. A warp none of whose pixels blends a Gaussian skips it after one
// vote; the others take every pixel pair without branching (G = 0 where a pixel does not blend).
//
// Both walks take a thread's pixels in pairs (rows 2p, 2p + 1 of its column): the pair's
// values sit in the two halves of a float2 and every operation on them is one packed
// float32 instruction (add/mul/fma .f32x2), with the per-Gaussian operands stored twice in
// shared memory so that one 16-byte load yields two ready pair operands. A pixel of a pair
// that does not blend the splat gets G = 0, which leaves its T, colour and P unchanged.
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
// Both walks stage at most 128 Gaussians per batch (a configured batch of 256 is taken as
// 128): the smaller shared arrays leave more of each SM's L1 to the batch loads' gathers
// (backward 0.58 -> 0.52 ms, forward 0.256 -> 0.249 ms at 3M / 1080p, against 256).
constexpr int kStageMax = 128;

template <int MAXV, int PIX, bool PERSIST>
__global__ void __launch_bounds__(256 / PIX) k_render_fwd(const __grid_constant__ Batch<MAXV> b,
                                                          Ws ws, float* __restrict__ out_rgb,
                                                          float* __restrict__ out_T,
                                                          uint32_t* __restrict__ out_nc) {
  pdl_entry();
  static_assert(PIX % 2 == 0, "pixels are walked in pairs");
  constexpr int NP = PIX / 2;
  __shared__ float4 s_x[kStageMax];     // (mean x, a', 2b', q'_min)
  __shared__ float4 s_y[kStageMax];     // (-mean y, -mean y, c', c')
  __shared__ float4 s_o[kStageMax];     // (-o, -o, r, r)
  __shared__ float4 s_c[kStageMax];     // (g, g, b, b)
  const uint32_t* __restrict__ vals = ws.vals[ws.plan[kPlanFinal]];
  const int tw = b.cfg.tile_w;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int batch = min(b.cfg.batch, kStageMax);
  const float2 one2 = dup2(1.f);
  uint32_t evals = 0, blended = 0;
  uint32_t tile;
  for (bool first = true; next_tile<PERSIST>(ws, b.tiles, 0, first, tile); first = false) {
    const ViewP& V = b.views[view_of_tile(b, tile)];
    const uint32_t lt = tile - V.tile_off;
    const int px = (int)(lt % V.tiles_x) * tw + tid % tw;
    const int py0 = (int)(lt / V.tiles_x) * b.cfg.tile_h + (tid / tw) * PIX;
    const uint2 rg = ws.ranges[tile];
    const float fx = (float)px + 0.5f;
    // per pixel pair: T and the colour sums (negated); per pixel: liveness, stop position
    float2 T[NP], NC0[NP], NC1[NP], NC2[NP], FY[NP];
    uint32_t last[PIX], stop[PIX];
    bool live[PIX];
    bool done = true;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      T[p] = one2;
      NC0[p] = NC1[p] = NC2[p] = dup2(0.f);
      FY[p] = make_float2((float)(py0 + 2 * p) + 0.5f, (float)(py0 + 2 * p + 1) + 0.5f);
    }
#pragma unroll
    for (int j = 0; j < PIX; ++j) {
      last[j] = 0;
      stop[j] = 0;
      live[j] = px < V.width && py0 + j < V.height;
      done = done && !live[j];
    }
    done = __all_sync(0xffffffffu, done);   // warps walk and stop together (votes below)
    uint32_t pos = 0;   // Gaussians of the tile list walked so far
    for (uint32_t start = rg.x; start < rg.y; start += batch) {
      if (__syncthreads_count(done) == nthr) break;
      const int cnt = (int)min((uint32_t)batch, rg.y - start);
      for (int k = tid; k < cnt; k += nthr) {
        const uint32_t id = vals[start + k];
        const float2 m = ws.xy[id];
        const float4 co = ws.conic_o[id];
        const float4 cs = scale_conic(co);
        const float4 c = ws.rgb[id];
        s_x[k] = make_float4(m.x, cs.x, cs.y, splat_qmin(co.w));
        s_y[k] = make_float4(-m.y, -m.y, cs.z, cs.z);
        s_o[k] = make_float4(-co.w, -co.w, c.x, c.x);
        s_c[k] = make_float4(c.y, c.y, c.z, c.z);
      }
      __syncthreads();
      if (!done) {
#pragma unroll 8
        for (int k = 0; k < cnt; ++k) {
          const float4 sx = s_x[k];
          const float4 sy = s_y[k];
          const float dx = fx - sx.x;
          const float2 t0 = dup2(__fmul_rn(__fmul_rn(sx.y, dx), dx));
          const float2 t1 = dup2(__fmul_rn(sx.z, dx));
          const float2 nmy = make_float2(sy.x, sy.y), cz = make_float2(sy.z, sy.w);
          ++pos;
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const float2 dy = add2(FY[p], nmy);
            const float2 q = fma2(dy, fma2(cz, dy, t1), t0);
            const bool pa = live[2 * p] && !(q.x < sx.w);       // live and alpha >= 1/255
            const bool pb = live[2 * p + 1] && !(q.y < sx.w);
            if (!__any_sync(0xffffffffu, pa || pb)) continue;   // no pixel of the warp blends
            const float4 so = s_o[k];
            float2 g;
            g.x = pa ? ex2_approx(q.x) : 0.f;
            g.y = pb ? ex2_approx(q.y) : 0.f;
            const float2 nog = mul2(make_float2(so.x, so.y), g);   // -o G
            float2 na = make_float2(fmaxf(-kAlphaMax, nog.x), fmaxf(-kAlphaMax, nog.y));
            float2 Tn = mul2(T[p], add2(one2, na));                // T (1 - alpha)
            const bool sa = Tn.x < kTMin, sb = Tn.y < kTMin;      // only a blended pixel can
            if (sa || sb) {                                       // fall below: it stops here
              if (sa) {
                live[2 * p] = false;
                stop[2 * p] = pos;
                na.x = 0.f;
                Tn.x = T[p].x;
              }
              if (sb) {
                live[2 * p + 1] = false;
                stop[2 * p + 1] = pos;
                na.y = 0.f;
                Tn.y = T[p].y;
              }
            }
            const float4 sc = s_c[k];
            const float2 nw = mul2(na, T[p]);                      // -alpha T
            NC0[p] = fma2(nw, make_float2(so.z, so.w), NC0[p]);
            NC1[p] = fma2(nw, make_float2(sc.x, sc.y), NC1[p]);
            NC2[p] = fma2(nw, make_float2(sc.z, sc.w), NC2[p]);
            T[p] = Tn;
            const bool ba = pa && !sa, bb = pb && !sb;
            last[2 * p] = ba ? pos : last[2 * p];
            last[2 * p + 1] = bb ? pos : last[2 * p + 1];
            blended += (uint32_t)ba + (uint32_t)bb;
          }
          if ((k & 7) == 7) {     // every eighth splat: the warp leaves once all its pixels stopped
            bool any_live = false;
#pragma unroll
            for (int j = 0; j < PIX; ++j) any_live = any_live || live[j];
            if (!__any_sync(0xffffffffu, any_live)) {
              done = true;
              break;
            }
          }
        }
        if (!done) {
          bool any_live = false;
#pragma unroll
          for (int j = 0; j < PIX; ++j) any_live = any_live || live[j];
          done = !__any_sync(0xffffffffu, any_live);
        }
      }
    }
    const uint64_t npix = (uint64_t)V.width * V.height;
#pragma unroll
    for (int j = 0; j < PIX; ++j) {
      const int py = py0 + j;
      if (px < V.width && py < V.height) {
        const int p = j / 2;
        const bool hi = j & 1;
        const float t = hi ? T[p].y : T[p].x;
        evals += live[j] ? pos : stop[j];
        const uint64_t i = (uint64_t)py * V.width + px;
        out_rgb[3 * V.pix_off + i] = t * b.cfg.bg[0] - (hi ? NC0[p].y : NC0[p].x);
        out_rgb[3 * V.pix_off + npix + i] = t * b.cfg.bg[1] - (hi ? NC1[p].y : NC1[p].x);
        out_rgb[3 * V.pix_off + 2 * npix + i] = t * b.cfg.bg[2] - (hi ? NC2[p].y : NC2[p].x);
        out_T[V.pix_off + i] = t;
        out_nc[V.pix_off + i] = last[j];
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
// 2D-gradient record (du, dv, dop, da, db, dc, dr, dg, db). A transposing butterfly: at
// each shuffle distance a lane keeps one half of its values, sends the other half to its
// partner and adds what it receives, so after distances 16, 8, 4, 2 every lane holds one
// partial sum; distance 1 completes it. 12 shuffles instead of 45.
__device__ __forceinline__ void warp_reduce_add9(float (&v)[9], float* rec) {
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
    atomicAdd(rec + i1, z);
}

template <int MAXV, int PIX, bool PERSIST>
__global__ void __launch_bounds__(256 / PIX) k_render_bwd(const __grid_constant__ Batch<MAXV> b,
                                                          Ws ws, const float* __restrict__ dL,
                                                          const float* __restrict__ fwd_T,
                                                          const uint32_t* __restrict__ fwd_nc) {
  pdl_entry();
  static_assert(PIX % 2 == 0, "pixels are walked in pairs");
  constexpr int NP = PIX / 2;
  // per staged Gaussian: the scalars of its column terms, and the operands the pixel pairs
  // share, each stored twice so that one 16-byte load yields two pair operands
  __shared__ uint32_t s_id[kStageMax];
  __shared__ float4 s_x[kStageMax];     // (mean x, a', 2b', q'_min)
  __shared__ float4 s_y[kStageMax];     // (-mean y, -mean y, c', c')
  __shared__ float4 s_o[kStageMax];     // (-o, -o, r, r)
  __shared__ float4 s_c[kStageMax];     // (g, g, b, b)
  __shared__ float4 s_co[kStageMax];    // (a, b, c, o): the conic for the gradient expansion
  __shared__ uint32_t s_max;
  const uint32_t* __restrict__ vals = ws.vals[ws.plan[kPlanFinal]];
  const int tw = b.cfg.tile_w;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int batch = min(b.cfg.batch, kStageMax);
  const float2 one2 = dup2(1.f);
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
    // per pixel pair: T, the upstream gradient g, and NP = -g . (colour behind the current
    // splat, background included), the only use of that colour in the chain rule
    float2 T[NP], G0[NP], G1[NP], G2[NP], NPb[NP], FY[NP];
    uint32_t last[PIX];
    uint32_t my_max = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      float t[2] = {0.f, 0.f}, g0[2] = {0.f, 0.f}, g1[2] = {0.f, 0.f}, g2[2] = {0.f, 0.f};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 2 * p + h;
        const int py = py0 + j;
        last[j] = 0;
        if (px < V.width && py < V.height) {
          const uint64_t i = (uint64_t)py * V.width + px;
          t[h] = fwd_T[V.pix_off + i];
          last[j] = fwd_nc[V.pix_off + i];
          g0[h] = dL[3 * V.pix_off + i];
          g1[h] = dL[3 * V.pix_off + npix + i];
          g2[h] = dL[3 * V.pix_off + 2 * npix + i];
        }
        my_max = max(my_max, last[j]);
        evals += last[j];
      }
      T[p] = make_float2(t[0], t[1]);
      G0[p] = make_float2(g0[0], g0[1]);
      G1[p] = make_float2(g1[0], g1[1]);
      G2[p] = make_float2(g2[0], g2[1]);
      FY[p] = make_float2((float)(py0 + 2 * p) + 0.5f, (float)(py0 + 2 * p + 1) + 0.5f);
      const float2 gb = fma2(G2[p], dup2(b.cfg.bg[2]),
                             fma2(G1[p], dup2(b.cfg.bg[1]), mul2(G0[p], dup2(b.cfg.bg[0]))));
      NPb[p] = mul2(dup2(-1.f), mul2(T[p], gb));
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
        const float2 m = ws.xy[id];
        const float4 co = ws.conic_o[id];
        const float4 cs = scale_conic(co);
        const float4 c = ws.rgb[id];
        s_x[k] = make_float4(m.x, cs.x, cs.y, splat_qmin(co.w));
        s_y[k] = make_float4(-m.y, -m.y, cs.z, cs.z);
        s_o[k] = make_float4(-co.w, -co.w, c.x, c.x);
        s_c[k] = make_float4(c.y, c.y, c.z, c.z);
        s_co[k] = co;
      }
      __syncthreads();
#pragma unroll 8
      for (int k = cnt - 1; k >= 0; --k) {
        const uint32_t pos = bstart - rg.x + (uint32_t)k + 1u;
        const float4 sx = s_x[k];
        const float4 sy = s_y[k];
        const float dx = fx - sx.x;
        const float2 t0 = dup2(__fmul_rn(__fmul_rn(sx.y, dx), dx));
        const float2 t1 = dup2(__fmul_rn(sx.z, dx));
        const float2 nmy = make_float2(sy.x, sy.y), cz = make_float2(sy.z, sy.w);
        // which of this thread's pixels blend the splat; a warp none of whose pixels does
        // skips it (one vote), the others take every pair, non-blending pixels with G = 0
        float2 dyv[NP], qv[NP];
        bool pav[NP], pbv[NP];
        bool any = false;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          dyv[p] = add2(FY[p], nmy);
          qv[p] = fma2(dyv[p], fma2(cz, dyv[p], t1), t0);
          pav[p] = pos <= last[2 * p] && !(qv[p].x < sx.w);      // alpha >= 1/255
          pbv[p] = pos <= last[2 * p + 1] && !(qv[p].y < sx.w);
          any = any || pav[p] || pbv[p];
        }
        if (!__any_sync(0xffffffffu, any)) continue;
        const float4 so = s_o[k];
        const float4 sc = s_c[k];
        // this thread's sums over its pixels (pairwise): colour gradient (negated), and the
        // moments E0 = sum e, E1 = sum e dy, E2 = sum e dy^2 of e = G dL/dalpha (unclamped)
        float2 nR0, nR1, nR2, E0, E1, E2;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float2 dy = dyv[p], q = qv[p];
          const bool pa = pav[p], pb = pbv[p];
          float2 g;                                   // G = 2^q' (0: pixel not blended)
          g.x = pa ? ex2_approx(q.x) : 0.f;
          g.y = pb ? ex2_approx(q.y) : 0.f;
          const float2 nog = mul2(make_float2(so.x, so.y), g);      // -o G
          const float2 na = make_float2(fmaxf(-kAlphaMax, nog.x), fmaxf(-kAlphaMax, nog.y));
          const float2 oma = add2(one2, na);                       // 1 - alpha
          const float2 ioma = make_float2(pa ? rcp_approx(oma.x) : 1.f,
                                          pb ? rcp_approx(oma.y) : 1.f);
          T[p] = mul2(T[p], ioma);                                 // T in front of this splat
          const float2 nw = mul2(na, T[p]);                        // -alpha T
          const float2 gc = fma2(G2[p], make_float2(sc.z, sc.w),
                                 fma2(G1[p], make_float2(sc.x, sc.y),
                                      mul2(G0[p], make_float2(so.z, so.w))));
          const float2 dal = fma2(ioma, NPb[p], mul2(T[p], gc));  // T (g.c) - P / (1 - alpha)
          NPb[p] = fma2(nw, gc, NPb[p]);                           // P += alpha T (g.c)
          const float2 ge = make_float2(nog.x > -kAlphaMax ? g.x : 0.f,
                                        nog.y > -kAlphaMax ? g.y : 0.f);
          const float2 e = mul2(ge, dal);
          const float2 ed = mul2(e, dy);
          if (p == 0) {
            nR0 = mul2(nw, G0[p]);
            nR1 = mul2(nw, G1[p]);
            nR2 = mul2(nw, G2[p]);
            E0 = e;
            E1 = ed;
            E2 = mul2(ed, dy);
          } else {
            nR0 = fma2(nw, G0[p], nR0);
            nR1 = fma2(nw, G1[p], nR1);
            nR2 = fma2(nw, G2[p], nR2);
            E0 = add2(E0, e);
            E1 = add2(E1, ed);
            E2 = fma2(ed, dy, E2);
          }
        }
        {
          // dL/dq = -o/2 e; q = a dx^2 + 2 b dx dy + c dy^2, dq/du = -2 (a dx + b dy), ...
          const float4 co = s_co[k];
          const float hq = -0.5f * co.w;
          const float e0 = E0.x + E0.y, e1 = E1.x + E1.y, e2 = E2.x + E2.y;
          const float Q0 = hq * e0, Q1 = hq * e1;
          float acc[9];
          acc[0] = -2.f * (co.x * dx * Q0 + co.y * Q1);
          acc[1] = -2.f * (co.y * dx * Q0 + co.z * Q1);
          acc[2] = e0;
          acc[3] = dx * dx * Q0;
          acc[4] = 2.f * dx * Q1;
          acc[5] = hq * e2;
          acc[6] = -(nR0.x + nR0.y);
          acc[7] = -(nR1.x + nR1.y);
          acc[8] = -(nR2.x + nR2.y);
          warp_reduce_add9(acc, ws.grad2d + 9ull * s_id[k]);
        }
      }
      bend = bstart;
    }
  }
  add_evals(ws.plan + kPlanEvalBwd, evals);
}

// Zero-fill of n 16-byte words, in stream order (the previous kernel may still read them).
__global__ void __launch_bounds__(256) k_zero16(uint4* __restrict__ p, size_t n) {
  pdl_entry();
  for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256)
    p[i] = make_uint4(0u, 0u, 0u, 0u);
}

// The device status word cleared, in stream order.
__global__ void k_clear_status(uint32_t* status) {
  pdl_entry();
  *status = 0u;
}

cudaError_t launch_zero16(void* p, size_t bytes, int grid, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  if (bytes % 16 || reinterpret_cast<uintptr_t>(p) % 16) return cudaErrorInvalidValue;
  return launch_k(k_zero16, dim3(grid), dim3(256), 0, st, reinterpret_cast<uint4*>(p), bytes / 16);
}

cudaError_t launch_clear_status(uint32_t* status, cudaStream_t st) {
  return launch_k(k_clear_status, dim3(1), dim3(1), 0, st, status);
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
    launch_k(k_render_fwd<MAXV, PIX, true>, dim3(grid), dim3(thr), 0, st, b, ws, out_rgb, out_T, out_nc);
  } else {
    launch_k(k_render_fwd<MAXV, PIX, false>, dim3(b.tiles), dim3(thr), 0, st, b, ws, out_rgb, out_T, out_nc);
  }
  return cudaGetLastError();
}

// The backward walk is launched after its predecessor (the 2D-gradient zero-fill) has
// finished, not scheduled while it drains: at 3M Gaussians / 1080p a training iteration took
// 2.27 ms this way against 2.37 ms with the overlapped launch (the other kernels gain or
// lose nothing either way).
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
    launch_k_full(k_render_bwd<MAXV, PIX, true>, dim3(grid), dim3(thr), 0, st, b, ws, dL, fwd_T,
                  fwd_nc);
  } else {
    launch_k_full(k_render_bwd<MAXV, PIX, false>, dim3(b.tiles), dim3(thr), 0, st, b, ws, dL,
                  fwd_T, fwd_nc);
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
