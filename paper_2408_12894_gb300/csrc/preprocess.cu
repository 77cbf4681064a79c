// Per-(view, Gaussian) preprocess (one thread per unit; a CTA's 128 Gaussians of one set
// have their geometry arrays copied into shared memory by asynchronous 16-byte copies when
// they form a whole aligned chunk): Eq. 4 constrained scale, Eq. 1 covariance, the
// local-affine projection of Eq. 2, conic, opacity, the opacity-aware extent, the tile set
// (rectangle, or ellipse rows) and the SH colour (geometry.cuh).
#include "geometry.cuh"
#include "kernels.h"

namespace flod {

// Staging of a CTA's kStageN consecutive Gaussians: every thread issues its share of 16-byte
// cp.async requests for each geometry array (means, rotations, scales, opacity logits), waits
// for its own requests and meets the others at a barrier; then each thread reads its
// Gaussian from shared memory. Nothing waits on a spin loop, and no copy outlives the barrier.
// The SH coefficients (192 of the 236 bytes at degree 3) are not staged: only a Gaussian that
// survives culling and touches a tile reads its row, as 12 float4 loads (a sixth of the level
// is culled at 3M / 1080p; 0.171 -> 0.169 ms against staging every row).
constexpr int kStageN = 128;
struct PreStage {
  float means[kStageN * 3];
  float4 quats[kStageN];
  float s_opt[kStageN * 3];
  float logit[kStageN];
};

template <int MAXV>
__global__ void __launch_bounds__(kStageN) k_preprocess(const __grid_constant__ Batch<MAXV> b, Ws ws) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char pre_smem[];
  PreStage& stg = *reinterpret_cast<PreStage*>(pre_smem);
  const uint32_t u = blockIdx.x * (uint32_t)kStageN + threadIdx.x;
  const bool in_range = u < b.units;   // always true (units are padded to 1024); kept for safety
  const ViewP& V = b.views[view_of_unit(b, in_range ? u : 0u)];
  // a selection longer than the view's units: reported once per view (its first CTA)
  if (V.sel && threadIdx.x == 0 && blockIdx.x * (uint32_t)kStageN == V.unit_off &&
      *V.sel_count > V.cap)
    set_status(ws.status, FLOD_DEV_SELECTION);
  // a whole chunk of one set (no selection, all kStageN Gaussians present): stage it (the
  // condition is the same for every thread of the CTA, whose units lie in one view)
  const uint32_t local0 = blockIdx.x * (uint32_t)kStageN - V.unit_off;
  const SetP& S0 = b.sets[V.sel ? 0 : V.set];
  const bool staged = !V.sel && S0.bulk_ok && local0 + kStageN <= V.cap &&
                      local0 + kStageN <= (uint32_t)S0.n;
  if (staged) {
    async_copy(stg.means, S0.means + 3ull * local0, kStageN * 12u);
    async_copy(stg.quats, S0.quats + 4ull * local0, kStageN * 16u);
    async_copy(stg.s_opt, S0.s_opt + 3ull * local0, kStageN * 12u);
    async_copy(stg.logit, S0.logit + local0, kStageN * 4u);
    async_copy_wait();
    __syncthreads();
  }
  int si = 0;
  uint32_t gi = 0;
  bool ok = in_range && unit_source(b, V, u - V.unit_off, si, gi);
  if (!ok) {   // padding, or past the view's selection: nothing reads it but its tile count
    if (in_range) ws.tiles_touched[u] = 0;
    return;
  }
  const uint32_t gl = staged ? threadIdx.x : gi;     // index into the parameter arrays used
  // the parameter arrays this unit reads: the staged chunk, or the set in global memory
  SetP S = b.sets[si];
  const int K3 = 3 * (S.deg + 1) * (S.deg + 1);
  const float* sh_row = S.sh + (size_t)K3 * gi;   // global memory (not staged)
  if (staged) {
    S.means = stg.means;
    S.quats = reinterpret_cast<const float*>(stg.quats);
    S.s_opt = stg.s_opt;
    S.logit = stg.logit;
  }
  float2 xy = make_float2(0.f, 0.f);
  float4 co = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 rgb = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 ext = make_float4(0.f, 0.f, 0.f, 0.f);
  float depth = 0.f, rad = 0.f, o = 0.f;
  uint32_t touched = 0;
  Geom G;
  UnitTiles t;
  if (ok) {
    geometry(S, gl, V, b.cfg, G);
    ok = G.t[2] > b.cfg.z_near && G.det > 0.f;
    o = 1.f / (1.f + expf(-S.logit[gl]));
    if (ok) {
      float lmax = 0.5f * (G.A + G.C) + sqrtf(fmaxf(0.25f * (G.A - G.C) * (G.A - G.C) + G.B * G.B, 0.f));
      const float tau = 2.f * logf(255.f * o);   // alpha >= 1/255 <=> q <= tau
      if (o >= kAlphaMin) {
        // support ellipse q <= tau (widened by 2^-10): row shear m, row scale h, box rx, ry
        const float tw = tau * kExtentMargin;
        ext = make_float4(G.B / G.C, sqrtf(G.det) / G.C, sqrtf(fmaxf(tw * G.A, 0.f)),
                          sqrtf(fmaxf(tw * G.C, 0.f)));
      }
      if (b.cfg.extent_rule != 1) {
        ok = o >= kAlphaMin;
        rad = sqrtf(fmaxf(tau * lmax, 0.f));
      } else {
        rad = 3.f * sqrtf(lmax);
      }
    }
    if (ok) {
      xy.x = V.fx * G.t[0] * G.itz + V.cx;
      xy.y = V.fy * G.t[1] * G.itz + V.cy;
      const bool rows = b.cfg.extent_rule == 2;
      ok = unit_tiles(xy.x, xy.y, rows ? ext : make_float4(0.f, 0.f, rad, rad), V.width,
                      V.height, b.cfg.tile_w, b.cfg.tile_h, rows, t);
    }
  }
  // tile count: the rows of the tile rectangle; the first rows also go to the tile record
  uint4 rec = make_uint4(0u, 0u, 0u, 0u);
  if (ok) {
    const int tx0 = t.px0 >> t.lw;
    const uint32_t nrows = (uint32_t)(t.ty1 - t.ty0 + 1);
    uint32_t mode = kRecTable;
    if (!t.rows) {
      touched = nrows * (uint32_t)((t.px1 >> t.lw) - tx0 + 1);
      mode = kRecUniform;
      rec.z = (uint32_t)((t.px1 >> t.lw) - tx0 + 1);
    } else {
      if (nrows > (uint32_t)kRecRows) mode = kRecCompute;
      for (int ty = t.ty0; ty <= t.ty1; ++ty) {
        int cx0, cx1;
        uint32_t off = 0, cnt = 0;
        if (unit_row(t, ty, cx0, cx1)) {
          cnt = (uint32_t)(cx1 - cx0 + 1);
          off = (uint32_t)(cx0 - tx0);
          touched += cnt;
        }
        const int r = ty - t.ty0;
        if (r < kRecRows) {
          if (off > 255u || cnt > 255u) mode = kRecCompute;
          const uint32_t h = (off & 0xffu) | (cnt & 0xffu) << 8;
          if (r < 2) rec.z |= h << (16 * r);
          else rec.w |= h << (16 * (r - 2));
        }
      }
    }
    rec.x = (uint32_t)tx0 | (uint32_t)t.ty0 << 16;
    rec.y = nrows | mode << 16;
  }
  ok = ok && touched > 0;
  if (ok) {
    float id = 1.f / G.det;
    co = make_float4(G.C * id, -G.B * id, G.A * id, o);
    depth = G.t[2];
    float Y[16], dir[3], dlen, raw[3];
    sh_colour(S, gl, sh_row, V, Y, dir, dlen, raw);
    rgb = make_float4(fmaxf(raw[0], 0.f), fmaxf(raw[1], 0.f), fmaxf(raw[2], 0.f), 0.f);
  } else {
    xy = make_float2(0.f, 0.f);
    rad = 0.f;
    ext = make_float4(0.f, 0.f, 0.f, 0.f);
    rec = make_uint4(0u, 0u, 0u, 0u);
    touched = 0;
  }
  if (in_range) {
    ws.xy[u] = xy;
    ws.depth[u] = depth;
    ws.conic_o[u] = co;
    ws.rgb[u] = rgb;
    ws.radius[u] = rad;
    ws.ext[u] = ext;
    ws.trec[u] = rec;
    ws.tiles_touched[u] = touched;
  }
}

// ---------------------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------------------
template <int MAXV>
cudaError_t launch_preprocess(const Batch<MAXV>& b, const Ws& ws, cudaStream_t st) {
  if (b.units == 0) return cudaSuccess;
  static bool attr = false;   // one opt-in per template instance
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_preprocess<MAXV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PreStage));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  launch_k(k_preprocess<MAXV>, dim3((b.units + kStageN - 1) / kStageN), dim3(kStageN), sizeof(PreStage), st, b, ws);
  return cudaGetLastError();
}

template cudaError_t launch_preprocess<kMaxViewsSmall>(const BatchS&, const Ws&, cudaStream_t);
template cudaError_t launch_preprocess<FLOD_MAX_VIEWS>(const BatchL&, const Ws&, cudaStream_t);

}  // namespace flod
