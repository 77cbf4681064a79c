// C ABI of the splatting path: argument checks, workspace layout, per-call parameter
// tables and kernel launches. See include/flod.h for the contract of every entry point.
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace flod {
uint32_t select_blocks(const int* ns, int n_levels);
}

using namespace flod;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

struct DevInfo {
  bool init = false;
  flod_status st = FLOD_OK;
  int sms = 0;
  int res_sort = 0;    // resident CTAs of the radix-sort pass kernel
  int res_small = 0;   // grid of the grid-stride helper kernels
};
DevInfo g_dev[64];
std::mutex g_mu;

flod_status device_info(DevInfo** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FLOD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  DevInfo& d = g_dev[dev];
  if (!d.init) {
    d.init = true;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (major != 10 || minor != 3) {
      d.st = FLOD_ERR_UNSUPPORTED;
    } else if (sort_kernel_prepare() != cudaSuccess) {
      d.st = FLOD_ERR_CUDA;
    } else {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sort_kernel_ptr(), kSortThreads,
                                                        sort_kernel_smem_bytes()) != cudaSuccess ||
          per_sm < 1)
        per_sm = 1;
      d.res_sort = per_sm * d.sms;
      d.res_small = 8 * d.sms;
      d.st = FLOD_OK;
    }
  }
  *out = &d;
  return d.st;
}

bool cfg_ok(const flod_raster_config* c) {
  if (!c) return false;
  const bool shape = (c->tile_w == 8 && c->tile_h == 8) || (c->tile_w == 16 && c->tile_h == 16) ||
                     (c->tile_w == 32 && c->tile_h == 8);
  const bool batch = c->batch == 32 || c->batch == 64 || c->batch == 128 || c->batch == 256;
  return shape && batch && c->dilation >= 0.f && c->z_near > 0.f &&
         (c->extent_rule >= 0 && c->extent_rule <= 2) && isfinite(c->dilation) &&
         isfinite(c->z_near);
}

struct Plan {
  flod_ws_layout L;
  uint64_t unit_off[FLOD_MAX_VIEWS + 1];
  uint64_t tile_off[FLOD_MAX_VIEWS + 1];
  uint64_t pix_off[FLOD_MAX_VIEWS + 1];
  uint32_t tiles_x[FLOD_MAX_VIEWS], tiles_y[FLOD_MAX_VIEWS], cap[FLOD_MAX_VIEWS];
  uint32_t max_parts;
  int n_passes;
  int tile_bits;
};

flod_status make_plan(const flod_gaussians* sets, int n_sets, const flod_view* views, int n_views,
                      uint64_t pair_capacity, const flod_raster_config* cfg, Plan& P) {
  if (!sets || !views || n_sets < 1 || n_sets > FLOD_MAX_SETS || n_views < 1 ||
      n_views > FLOD_MAX_VIEWS || pair_capacity > FLOD_MAX_PAIRS || !cfg_ok(cfg))
    return FLOD_ERR_INVALID_ARG;
  for (int s = 0; s < n_sets; ++s) {
    const flod_gaussians& g = sets[s];
    if (g.n < 0 || g.n >= (1 << FLOD_SEL_SHIFT) || g.sh_degree < 0 || g.sh_degree > 3 ||
        !(g.s_min >= 0.f) || !isfinite(g.s_min))
      return FLOD_ERR_INVALID_ARG;
    if (g.n > 0 && (!g.means || !g.quats || !g.s_opt || !g.opacity_logit || !g.sh))
      return FLOD_ERR_INVALID_ARG;
    if (g.n > 0 && (reinterpret_cast<uintptr_t>(g.quats) & 15u)) return FLOD_ERR_INVALID_ARG;
    if (g.n > 0 && g.sh_degree == 3 && (reinterpret_cast<uintptr_t>(g.sh) & 15u))
      return FLOD_ERR_INVALID_ARG;
  }
  uint64_t u = 0, t = 0, p = 0;
  for (int v = 0; v < n_views; ++v) {
    const flod_view& V = views[v];
    const flod_camera& C = V.cam;
    if (C.width <= 0 || C.height <= 0 || C.width > 16384 || C.height > 16384 || !(C.fx > 0.f) ||
        !(C.fy > 0.f))
      return FLOD_ERR_INVALID_ARG;
    for (int k = 0; k < 12; ++k)
      if (!isfinite(C.viewmat[k])) return FLOD_ERR_INVALID_ARG;
    uint64_t cap;
    if (V.sel) {
      if (!V.sel_count) return FLOD_ERR_INVALID_ARG;
      cap = V.sel_capacity;
    } else {
      if (V.set < 0 || V.set >= n_sets) return FLOD_ERR_INVALID_ARG;
      cap = (uint64_t)sets[V.set].n;
    }
    P.cap[v] = (uint32_t)cap;
    P.unit_off[v] = u;
    P.tile_off[v] = t;
    P.pix_off[v] = p;
    P.tiles_x[v] = (uint32_t)((C.width + cfg->tile_w - 1) / cfg->tile_w);
    P.tiles_y[v] = (uint32_t)((C.height + cfg->tile_h - 1) / cfg->tile_h);
    u += (cap + kScanBlock - 1) / kScanBlock * kScanBlock;
    t += (uint64_t)P.tiles_x[v] * P.tiles_y[v];
    p += (uint64_t)C.width * C.height;
  }
  P.unit_off[n_views] = u;
  P.tile_off[n_views] = t;
  P.pix_off[n_views] = p;
  if (u >= (1ull << 32) || t >= (1ull << 31)) return FLOD_ERR_INVALID_ARG;
  int tile_bits = 1;
  while (tile_bits < 31 && (1ull << tile_bits) < t) ++tile_bits;
  P.n_passes = (tile_bits + kRadixBits - 1) / kRadixBits;   // tile digits over the pairs
  P.tile_bits = tile_bits;
  const uint64_t parts_pairs = (pair_capacity + kSortPart - 1) / kSortPart;
  const uint64_t parts_units = (u + kSortPart - 1) / kSortPart;
  P.max_parts = (uint32_t)(parts_pairs > parts_units ? parts_pairs : parts_units);
  if (P.max_parts == 0) P.max_parts = 1;

  flod_ws_layout& L = P.L;
  memset(&L, 0, sizeof(L));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  L.status = take(4);
  L.pair_count = take(8);
  L.plan = take(64 * 4);
  L.xy = take(8 * u);
  L.depth = take(4 * u);
  L.conic_o = take(16 * u);
  L.rgb = take(16 * u);
  L.radius = take(4 * u);
  L.ext = take(16 * u);
  L.trec = take(16 * u);
  L.tiles_touched = take(4 * u);
  L.block_sums = take(8 * (u / kScanBlock + 1));
  L.slices = take(4 * (u / kScanBlock + 1));
  L.ukeys[0] = take(4 * u);
  L.ukeys[1] = take(4 * u);
  L.uvals[0] = take(4 * u);
  L.uvals[1] = take(4 * u);
  L.keys[0] = take(4 * pair_capacity);
  L.keys[1] = take(4 * pair_capacity);
  L.vals[0] = take(4 * pair_capacity);
  L.vals[1] = take(4 * pair_capacity);
  L.hist = take(4 * kPlanPasses * kRadixBins);
  L.counts = take(4ull * P.max_parts * kRadixBins);
  L.ranges = take(8 * t);
  L.grad2d = take(36 * u);
  L.queue = take(4 * (t + 128));
  L.total = off;
  L.units = u;
  L.tiles = t;
  L.pixels = p;
  L.pair_capacity = pair_capacity;
  return FLOD_OK;
}

Ws ws_ptrs(void* base, const Plan& P) {
  unsigned char* b = static_cast<unsigned char*>(base);
  const flod_ws_layout& L = P.L;
  Ws w;
  w.status = reinterpret_cast<uint32_t*>(b + L.status);
  w.pair_count = reinterpret_cast<unsigned long long*>(b + L.pair_count);
  w.plan = reinterpret_cast<uint32_t*>(b + L.plan);
  w.xy = reinterpret_cast<float2*>(b + L.xy);
  w.depth = reinterpret_cast<float*>(b + L.depth);
  w.conic_o = reinterpret_cast<float4*>(b + L.conic_o);
  w.rgb = reinterpret_cast<float4*>(b + L.rgb);
  w.radius = reinterpret_cast<float*>(b + L.radius);
  w.ext = reinterpret_cast<float4*>(b + L.ext);
  w.trec = reinterpret_cast<uint4*>(b + L.trec);
  w.tiles_touched = reinterpret_cast<uint32_t*>(b + L.tiles_touched);
  w.block_sums = reinterpret_cast<unsigned long long*>(b + L.block_sums);
  w.slices = reinterpret_cast<uint32_t*>(b + L.slices);
  for (int i = 0; i < 2; ++i) {
    w.ukeys[i] = reinterpret_cast<uint32_t*>(b + L.ukeys[i]);
    w.uvals[i] = reinterpret_cast<uint32_t*>(b + L.uvals[i]);
    w.keys[i] = reinterpret_cast<uint32_t*>(b + L.keys[i]);
    w.vals[i] = reinterpret_cast<uint32_t*>(b + L.vals[i]);
  }
  w.hist = reinterpret_cast<uint32_t*>(b + L.hist);
  w.counts = reinterpret_cast<uint32_t*>(b + L.counts);
  w.ranges = reinterpret_cast<uint2*>(b + L.ranges);
  w.grad2d = reinterpret_cast<float*>(b + L.grad2d);
  w.queue = reinterpret_cast<uint32_t*>(b + L.queue);
  w.pair_capacity = L.pair_capacity;
  w.max_parts = P.max_parts;
  w.units = (uint32_t)L.units;
  return w;
}

template <int MAXV>
void fill_batch(Batch<MAXV>& B, const flod_gaussians* sets, int n_sets, const flod_view* views,
                int n_views, const flod_raster_config* cfg, const Plan& P) {
  memset(&B, 0, sizeof(B));
  B.n_views = n_views;
  B.n_sets = n_sets;
  B.units = (uint32_t)P.L.units;
  B.tiles = (uint32_t)P.L.tiles;
  B.cfg.tile_w = cfg->tile_w;
  B.cfg.tile_h = cfg->tile_h;
  B.cfg.batch = cfg->batch;
  B.cfg.extent_rule = cfg->extent_rule;
  B.cfg.dilation = cfg->dilation;
  B.cfg.z_near = cfg->z_near;
  for (int c = 0; c < 3; ++c) B.cfg.bg[c] = cfg->bg[c];
  for (int s = 0; s < n_sets; ++s) {
    const flod_gaussians& g = sets[s];
    const bool al = !((reinterpret_cast<uintptr_t>(g.means) | reinterpret_cast<uintptr_t>(g.quats) |
                       reinterpret_cast<uintptr_t>(g.s_opt) |
                       reinterpret_cast<uintptr_t>(g.opacity_logit) |
                       reinterpret_cast<uintptr_t>(g.sh)) & 15u);
    B.sets[s] = SetP{g.means, g.quats, g.s_opt, g.opacity_logit, g.sh, g.n, g.sh_degree, g.s_min,
                     al ? 1 : 0};
  }
  for (int v = 0; v < n_views; ++v) {
    const flod_view& V = views[v];
    ViewP& O = B.views[v];
    memcpy(O.vm, V.cam.viewmat, sizeof(O.vm));
    O.fx = V.cam.fx;
    O.fy = V.cam.fy;
    O.cx = V.cam.cx;
    O.cy = V.cam.cy;
    O.width = V.cam.width;
    O.height = V.cam.height;
    O.cpx = V.cam.cam_pos[0];
    O.cpy = V.cam.cam_pos[1];
    O.cpz = V.cam.cam_pos[2];
    O.set = V.sel ? 0 : V.set;
    O.sel = V.sel;
    O.sel_count = V.sel_count;
    O.cap = P.cap[v];
    O.unit_off = (uint32_t)P.unit_off[v];
    O.tile_off = (uint32_t)P.tile_off[v];
    O.tiles_x = P.tiles_x[v];
    O.tiles_y = P.tiles_y[v];
    O.pix_off = P.pix_off[v];
    B.unit_end[v] = (uint32_t)P.unit_off[v + 1];
    B.tile_end[v] = (uint32_t)P.tile_off[v + 1];
  }
}

// The kernel parameter table is large for big batches; small batches use a small table.
template <typename F>
flod_status with_batch(const flod_gaussians* sets, int n_sets, const flod_view* views,
                       int n_views, const flod_raster_config* cfg, const Plan& P, F&& f) {
  cudaError_t e;
  if (n_views <= kMaxViewsSmall) {
    static thread_local BatchS B;
    fill_batch(B, sets, n_sets, views, n_views, cfg, P);
    e = f(B);
  } else {
    static thread_local BatchL B;
    fill_batch(B, sets, n_sets, views, n_views, cfg, P);
    e = f(B);
  }
  return e == cudaSuccess ? FLOD_OK : FLOD_ERR_CUDA;
}

flod_status common_checks(const flod_gaussians* sets, int n_sets, const flod_view* views,
                          int n_views, uint64_t cap, const flod_raster_config* cfg, void* ws,
                          size_t ws_bytes, Plan& P, DevInfo** dev) {
  flod_status s = make_plan(sets, n_sets, views, n_views, cap, cfg, P);
  if (s != FLOD_OK) return s;
  if (!ws) return FLOD_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) & 255u) return FLOD_ERR_INVALID_ARG;
  if (ws_bytes < P.L.total) return FLOD_ERR_WORKSPACE;
  return device_info(dev);
}

}  // namespace

extern "C" {

void flod_default_config(flod_raster_config* c) {
  if (!c) return;
  c->tile_w = 16;
  c->tile_h = 16;
  c->batch = 128;
  c->dilation = 0.3f;
  c->z_near = 0.2f;
  c->bg[0] = c->bg[1] = c->bg[2] = 0.f;
  c->extent_rule = 2;
  c->persistent = 0;
}

size_t flod_workspace_size(const flod_gaussians* sets, int n_sets, const flod_view* views,
                           int n_views, uint64_t pair_capacity, const flod_raster_config* cfg) {
  static thread_local Plan P;
  if (make_plan(sets, n_sets, views, n_views, pair_capacity, cfg, P) != FLOD_OK) return 0;
  return P.L.total;
}

flod_status flod_workspace_layout(const flod_gaussians* sets, int n_sets, const flod_view* views,
                                  int n_views, uint64_t pair_capacity,
                                  const flod_raster_config* cfg, flod_ws_layout* out,
                                  uint64_t* unit_offset, uint64_t* tile_offset,
                                  uint64_t* pixel_offset) {
  static thread_local Plan P;
  if (!out) return FLOD_ERR_INVALID_ARG;
  flod_status s = make_plan(sets, n_sets, views, n_views, pair_capacity, cfg, P);
  if (s != FLOD_OK) return s;
  *out = P.L;
  for (int v = 0; v <= n_views; ++v) {
    if (unit_offset) unit_offset[v] = P.unit_off[v];
    if (tile_offset) tile_offset[v] = P.tile_off[v];
    if (pixel_offset) pixel_offset[v] = P.pix_off[v];
  }
  return FLOD_OK;
}

flod_status flod_preprocess(const flod_gaussians* sets, int n_sets, const flod_view* views,
                            int n_views, const flod_raster_config* cfg, void* ws,
                            size_t ws_bytes, uint64_t pair_capacity, flod_stream stream) {
  static thread_local Plan P;
  DevInfo* dev = nullptr;
  flod_status s = common_checks(sets, n_sets, views, n_views, pair_capacity, cfg, ws, ws_bytes, P, &dev);
  if (s != FLOD_OK) return s;
  const Ws w = ws_ptrs(ws, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (launch_clear_status(w.status, st) != cudaSuccess) return FLOD_ERR_CUDA;
  return with_batch(sets, n_sets, views, n_views, cfg, P,
                    [&](const auto& B) { return launch_preprocess(B, w, st); });
}

flod_status flod_bin_sort_phase(const flod_gaussians* sets, int n_sets, const flod_view* views,
                                int n_views, const flod_raster_config* cfg, void* ws,
                                size_t ws_bytes, uint64_t pair_capacity, uint64_t* d_pair_count,
                                int phase, flod_stream stream) {
  static thread_local Plan P;
  DevInfo* dev = nullptr;
  if (phase < FLOD_BIN_ALL || phase > FLOD_BIN_PHASE_RANGES) return FLOD_ERR_INVALID_ARG;
  flod_status s = common_checks(sets, n_sets, views, n_views, pair_capacity, cfg, ws, ws_bytes, P, &dev);
  if (s != FLOD_OK) return s;
  const Ws w = ws_ptrs(ws, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n_passes = P.n_passes;
  return with_batch(sets, n_sets, views, n_views, cfg, P, [&](const auto& B) {
    return launch_binning(B, w, n_passes, P.tile_bits, dev->res_sort, dev->res_small,
                          reinterpret_cast<unsigned long long*>(d_pair_count),
                          cfg->persistent != 0, phase, st);
  });
}

flod_status flod_bin_sort(const flod_gaussians* sets, int n_sets, const flod_view* views,
                          int n_views, const flod_raster_config* cfg, void* ws, size_t ws_bytes,
                          uint64_t pair_capacity, uint64_t* d_pair_count, flod_stream stream) {
  return flod_bin_sort_phase(sets, n_sets, views, n_views, cfg, ws, ws_bytes, pair_capacity,
                             d_pair_count, FLOD_BIN_ALL, stream);
}

flod_status flod_render_fwd(const flod_gaussians* sets, int n_sets, const flod_view* views,
                            int n_views, const flod_raster_config* cfg, void* ws, size_t ws_bytes,
                            uint64_t pair_capacity, float* out_rgb, float* out_T, uint32_t* out_nc,
                            flod_stream stream) {
  static thread_local Plan P;
  DevInfo* dev = nullptr;
  if (!out_rgb || !out_T || !out_nc) return FLOD_ERR_INVALID_ARG;
  flod_status s = common_checks(sets, n_sets, views, n_views, pair_capacity, cfg, ws, ws_bytes, P, &dev);
  if (s != FLOD_OK) return s;
  const Ws w = ws_ptrs(ws, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool pers = cfg->persistent != 0;
  return with_batch(sets, n_sets, views, n_views, cfg, P, [&](const auto& B) {
    return launch_render_fwd(B, w, out_rgb, out_T, out_nc, dev->sms, pers, st);
  });
}

namespace {
// Per set: atomics when several units may hold one Gaussian (several views, or a selection
// list beside other views), plain read-modify-write otherwise, plain stores on request
// (overwrite 1); overwrite 2 zero-fills the set's buffers in the stream first.
bool grad_table(const flod_view* views, int n_views, int n_sets, const flod_grads* grads,
                GradTable& gt) {
  memset(&gt, 0, sizeof(gt));
  int direct[FLOD_MAX_SETS] = {0};
  int n_sel = 0;
  for (int v = 0; v < n_views; ++v) {
    if (views[v].sel) ++n_sel;
    else ++direct[views[v].set];
  }
  for (int k = 0; k < n_sets; ++k) {
    gt.g[k] = grads[k];
    // float4 gradient writes: quaternion rows, and SH rows at degree 3, 16-byte aligned
    if (reinterpret_cast<uintptr_t>(grads[k].quats) & 15u) return false;
    if (reinterpret_cast<uintptr_t>(grads[k].sh) & 15u) return false;
    const bool shared = (direct[k] + n_sel) > 1;
    if (grads[k].overwrite < 0 || grads[k].overwrite > 2) return false;
    if (grads[k].overwrite == 1) {
      if (direct[k] != 1 || n_sel != 0) return false;
      gt.mode[k] = kGradOverwrite;
    } else {
      gt.mode[k] = shared ? kGradAtomic : kGradAccumulate;
      gt.zero[k] = grads[k].overwrite == 2;
    }
  }
  return true;
}
}  // namespace

flod_status flod_blend_bwd(const flod_gaussians* sets, int n_sets, const flod_view* views,
                           int n_views, const flod_raster_config* cfg, void* ws, size_t ws_bytes,
                           uint64_t pair_capacity, const float* dL_drgb, const float* fwd_T,
                           const uint32_t* fwd_nc, flod_stream stream) {
  static thread_local Plan P;
  DevInfo* dev = nullptr;
  if (!dL_drgb || !fwd_T || !fwd_nc) return FLOD_ERR_INVALID_ARG;
  flod_status s = common_checks(sets, n_sets, views, n_views, pair_capacity, cfg, ws, ws_bytes, P, &dev);
  if (s != FLOD_OK) return s;
  const Ws w = ws_ptrs(ws, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (P.L.units && launch_zero16(w.grad2d, 36 * P.L.units, dev->res_small, st) != cudaSuccess)
    return FLOD_ERR_CUDA;
  const bool pers = cfg->persistent != 0;
  return with_batch(sets, n_sets, views, n_views, cfg, P, [&](const auto& B) {
    return launch_render_bwd(B, w, dL_drgb, fwd_T, fwd_nc, dev->sms, pers, st);
  });
}

flod_status flod_preprocess_bwd(const flod_gaussians* sets, int n_sets, const flod_view* views,
                                int n_views, const flod_raster_config* cfg, void* ws,
                                size_t ws_bytes, uint64_t pair_capacity, const flod_grads* grads,
                                flod_stream stream) {
  static thread_local Plan P;
  DevInfo* dev = nullptr;
  if (!grads) return FLOD_ERR_INVALID_ARG;
  flod_status s = common_checks(sets, n_sets, views, n_views, pair_capacity, cfg, ws, ws_bytes, P, &dev);
  if (s != FLOD_OK) return s;
  GradTable gt;
  if (!grad_table(views, n_views, n_sets, grads, gt)) return FLOD_ERR_INVALID_ARG;
  const Ws w = ws_ptrs(ws, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return with_batch(sets, n_sets, views, n_views, cfg, P, [&](const auto& B) {
    const cudaError_t e = launch_zero_grads(B, gt, dev->res_small, st);
    return e != cudaSuccess ? e : launch_preprocess_bwd(B, w, gt, st);
  });
}

flod_status flod_render_bwd(const flod_gaussians* sets, int n_sets, const flod_view* views,
                            int n_views, const flod_raster_config* cfg, void* ws,
                            size_t ws_bytes, uint64_t pair_capacity, const float* dL_drgb,
                            const float* fwd_T, const uint32_t* fwd_nc, const flod_grads* grads,
                            flod_stream stream) {
  if (!grads) return FLOD_ERR_INVALID_ARG;
  flod_status s = flod_blend_bwd(sets, n_sets, views, n_views, cfg, ws, ws_bytes, pair_capacity,
                                 dL_drgb, fwd_T, fwd_nc, stream);
  if (s != FLOD_OK) return s;
  return flod_preprocess_bwd(sets, n_sets, views, n_views, cfg, ws, ws_bytes, pair_capacity, grads,
                             stream);
}

namespace {
bool all_set(const flod_param_arrays* a) {
  return a && a->means && a->quats && a->s_opt && a->opacity_logit && a->sh;
}
bool aligned16(const void* p) { return !(reinterpret_cast<uintptr_t>(p) & 15u); }
bool adam_cfg_ok(const flod_adam_config* c) {
  return c && c->d_step && c->beta1 >= 0.0 && c->beta1 < 1.0 && c->beta2 >= 0.0 && c->beta2 < 1.0 &&
         c->eps >= 0.0 && isfinite(c->lr_means) && isfinite(c->lr_quats) && isfinite(c->lr_s_opt) &&
         isfinite(c->lr_opacity) && isfinite(c->lr_sh_dc) && isfinite(c->lr_sh_rest);
}
AdamHyper adam_hyper(const flod_adam_config* c) {
  AdamHyper h;
  h.lr[0] = c->lr_means;
  h.lr[1] = c->lr_quats;
  h.lr[2] = c->lr_s_opt;
  h.lr[3] = c->lr_opacity;
  h.lr[4] = c->lr_sh_dc;
  h.lr[5] = c->lr_sh_rest;
  h.beta1 = c->beta1;
  h.beta2 = c->beta2;
  h.b1 = (float)c->beta1;
  h.b2 = (float)c->beta2;
  h.omb1 = (float)(1.0 - c->beta1);
  h.omb2 = (float)(1.0 - c->beta2);
  h.eps = (float)c->eps;
  h.d_step = c->d_step;
  return h;
}
AdamArrays adam_arrays(const flod_param_arrays& in, const flod_param_arrays& out,
                       const flod_param_arrays& m, const flod_param_arrays& v) {
  AdamArrays a;
  const float* pi[5] = {in.means, in.quats, in.s_opt, in.opacity_logit, in.sh};
  float* po[5] = {out.means, out.quats, out.s_opt, out.opacity_logit, out.sh};
  float* pm[5] = {m.means, m.quats, m.s_opt, m.opacity_logit, m.sh};
  float* pv[5] = {v.means, v.quats, v.s_opt, v.opacity_logit, v.sh};
  for (int f = 0; f < 5; ++f) {
    a.in[f] = pi[f];
    a.out[f] = po[f];
    a.m[f] = pm[f];
    a.v[f] = pv[f];
  }
  return a;
}
}  // namespace

size_t flod_loss_scratch_size(const int* widths, const int* heights, int n_images) {
  if (!widths || !heights || n_images < 1 || n_images > FLOD_MAX_VIEWS) return 0;
  for (int i = 0; i < n_images; ++i)
    if (widths[i] <= 0 || heights[i] <= 0 || widths[i] > 16384 || heights[i] > 16384) return 0;
  return loss_scratch_bytes(widths, heights, n_images, nullptr, nullptr);
}

flod_status flod_loss(const float* img, const float* target, const int* widths, const int* heights,
                      int n_images, float lambda, float* d_loss, float* dL_dimg, void* scratch,
                      size_t scratch_bytes, flod_stream stream) {
  const size_t need = flod_loss_scratch_size(widths, heights, n_images);
  if (!need || !img || !target || !dL_dimg || !scratch || !(lambda >= 0.f && lambda <= 1.f))
    return FLOD_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(scratch) & 255u) return FLOD_ERR_INVALID_ARG;
  if (scratch_bytes < need) return FLOD_ERR_WORKSPACE;
  DevInfo* dev = nullptr;
  flod_status s = device_info(&dev);
  if (s != FLOD_OK) return s;
  return launch_loss(img, target, widths, heights, n_images, lambda, d_loss, dL_dimg, scratch,
                     reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FLOD_OK
             : FLOD_ERR_CUDA;
}

flod_status flod_adam_step(const flod_param_arrays* params, const flod_param_arrays* grads,
                           const flod_param_arrays* m, const flod_param_arrays* v, const int* n,
                           const int* sh_degree, int n_sets, const flod_adam_config* cfg,
                           flod_stream stream) {
  if (!params || !grads || !m || !v || !n || !sh_degree || n_sets < 1 || n_sets > FLOD_MAX_SETS ||
      !adam_cfg_ok(cfg))
    return FLOD_ERR_INVALID_ARG;
  AdamArrays a[FLOD_MAX_SETS];
  for (int k = 0; k < n_sets; ++k) {
    if (n[k] < 0 || n[k] >= (1 << FLOD_SEL_SHIFT) || sh_degree[k] < 0 || sh_degree[k] > 3)
      return FLOD_ERR_INVALID_ARG;
    if (n[k] > 0 && (!all_set(&params[k]) || !all_set(&grads[k]) || !all_set(&m[k]) ||
                     !all_set(&v[k])))
      return FLOD_ERR_INVALID_ARG;
    a[k] = adam_arrays(params[k], params[k], m[k], v[k]);
  }
  DevInfo* dev = nullptr;
  flod_status s = device_info(&dev);
  if (s != FLOD_OK) return s;
  return launch_adam(a, grads, n, sh_degree, n_sets, adam_hyper(cfg), dev->res_small,
                     reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FLOD_OK
             : FLOD_ERR_CUDA;
}

flod_status flod_preprocess_bwd_adam(const flod_gaussians* sets, int n_sets, const flod_view* views,
                                     int n_views, const flod_raster_config* cfg, void* ws,
                                     size_t ws_bytes, uint64_t pair_capacity,
                                     const flod_adam_state* states, const flod_adam_config* acfg,
                                     flod_stream stream) {
  static thread_local Plan P;
  DevInfo* dev = nullptr;
  if (!states || !adam_cfg_ok(acfg)) return FLOD_ERR_INVALID_ARG;
  flod_status s = common_checks(sets, n_sets, views, n_views, pair_capacity, cfg, ws, ws_bytes, P, &dev);
  if (s != FLOD_OK) return s;
  int direct[FLOD_MAX_SETS] = {0};
  for (int v = 0; v < n_views; ++v) {
    if (views[v].sel) return FLOD_ERR_INVALID_ARG;
    ++direct[views[v].set];
  }
  static thread_local AdamTable at;
  memset(&at, 0, sizeof(at));
  for (int k = 0; k < n_sets; ++k) {
    const flod_adam_state& S = states[k];
    if (direct[k] != 1 || !all_set(&S.params) || !all_set(&S.m) || !all_set(&S.v))
      return FLOD_ERR_INVALID_ARG;
    // the Adam pass moves each CTA's chunk of every array with 16-byte accesses
    const flod_param_arrays* arrs[3] = {&S.params, &S.m, &S.v};
    for (const flod_param_arrays* a : arrs)
      if (!aligned16(a->means) || !aligned16(a->quats) || !aligned16(a->s_opt) ||
          !aligned16(a->opacity_logit) || !aligned16(a->sh))
        return FLOD_ERR_INVALID_ARG;
    if (!aligned16(sets[k].means) || !aligned16(sets[k].s_opt) ||
        !aligned16(sets[k].opacity_logit) || !aligned16(sets[k].sh))
      return FLOD_ERR_INVALID_ARG;
    const flod_param_arrays in = {const_cast<float*>(sets[k].means), const_cast<float*>(sets[k].quats),
                                  const_cast<float*>(sets[k].s_opt),
                                  const_cast<float*>(sets[k].opacity_logit),
                                  const_cast<float*>(sets[k].sh)};
    at.a[k] = adam_arrays(in, S.params, S.m, S.v);
  }
  at.h = adam_hyper(acfg);
  const Ws w = ws_ptrs(ws, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return with_batch(sets, n_sets, views, n_views, cfg, P,
                    [&](const auto& B) { return launch_preprocess_bwd_adam(B, w, at, dev->sms, st); });
}

flod_status flod_gather(const flod_gaussians* sets, int n_sets, const uint32_t* entries,
                        const uint32_t* d_count, uint32_t capacity, const flod_param_arrays* out,
                        int out_sh_degree, int fold_s_min, float* out_s_min, flod_stream stream) {
  if (!sets || n_sets < 1 || n_sets > FLOD_MAX_SETS || !d_count || !out || out_sh_degree < 0 ||
      out_sh_degree > 3 || (fold_s_min != 0 && fold_s_min != 1))
    return FLOD_ERR_INVALID_ARG;
  if (capacity > 0 && (!all_set(out) || !aligned16(out->quats) ||
                       ((out_sh_degree == 1 || out_sh_degree == 3) && !aligned16(out->sh))))
    return FLOD_ERR_INVALID_ARG;
  static thread_local GatherP g;
  memset(&g, 0, sizeof(g));
  for (int k = 0; k < n_sets; ++k) {
    const flod_gaussians& S = sets[k];
    if (S.n < 0 || S.n >= (1 << FLOD_SEL_SHIFT) || S.sh_degree < 0 || S.sh_degree > 3 ||
        !(S.s_min >= 0.f))
      return FLOD_ERR_INVALID_ARG;
    if (S.n > 0 && (!S.means || !S.quats || !S.s_opt || !S.opacity_logit || !S.sh ||
                    !aligned16(S.quats) || ((S.sh_degree == 1 || S.sh_degree == 3) && !aligned16(S.sh))))
      return FLOD_ERR_INVALID_ARG;
    const float* src[5] = {S.means, S.quats, S.s_opt, S.opacity_logit, S.sh};
    if (S.n > 0) {
      // device memory, or host memory the device can address (pinned: its device address);
      // pageable host memory is refused here instead of faulting the kernel
      for (int f = 0; f < 5; ++f) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, src[f]) != cudaSuccess) {
          cudaGetLastError();
          return FLOD_ERR_INVALID_ARG;
        }
        if (at.type == cudaMemoryTypeUnregistered || !at.devicePointer) return FLOD_ERR_INVALID_ARG;
        src[f] = static_cast<const float*>(at.devicePointer);
      }
    }
    g.sets[k] = SetP{src[0], src[1], src[2], src[3], src[4], S.n, S.sh_degree, S.s_min, 0};
  }
  g.n_sets = n_sets;
  g.entries = entries;
  g.d_count = d_count;
  g.capacity = capacity;
  g.out = *out;
  g.out_s_min = out_s_min;
  g.out_K3 = 3 * (out_sh_degree + 1) * (out_sh_degree + 1);
  g.fold = fold_s_min;
  if (capacity == 0) return FLOD_OK;
  DevInfo* dev = nullptr;
  flod_status s = device_info(&dev);
  if (s != FLOD_OK) return s;
  const uint64_t want = (capacity + 255u) / 256u;
  const int grid = (int)(want < (uint64_t)dev->res_small ? want : (uint64_t)dev->res_small);
  return launch_gather(g, grid > 0 ? grid : 1, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FLOD_OK
             : FLOD_ERR_CUDA;
}

flod_status flod_densify_stats(const flod_gaussians* sets, int n_sets, const flod_view* views,
                               int n_views, const flod_raster_config* cfg, void* ws,
                               size_t ws_bytes, uint64_t pair_capacity, float* const* accum,
                               float* const* denom, flod_stream stream) {
  static thread_local Plan P;
  DevInfo* dev = nullptr;
  if (!accum || !denom) return FLOD_ERR_INVALID_ARG;
  flod_status s = common_checks(sets, n_sets, views, n_views, pair_capacity, cfg, ws, ws_bytes, P, &dev);
  if (s != FLOD_OK) return s;
  DensStatsP p;
  memset(&p, 0, sizeof(p));
  for (int k = 0; k < n_sets; ++k) {
    if (!accum[k] != !denom[k]) return FLOD_ERR_INVALID_ARG;
    p.accum[k] = accum[k];
    p.denom[k] = denom[k];
  }
  const Ws w = ws_ptrs(ws, P);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return with_batch(sets, n_sets, views, n_views, cfg, P,
                    [&](const auto& B) { return launch_dens_stats(B, w, p, st); });
}

size_t flod_densify_scratch_size(int n) {
  if (n < 0 || n >= (1 << FLOD_SEL_SHIFT)) return 0;
  return dens_scratch_bytes((uint32_t)n);
}

flod_status flod_densify(const flod_gaussians* set, const float* accum, const float* denom,
                         const float* normals, float tau, float max_clone_scale,
                         float min_opacity, const flod_param_arrays* m_in,
                         const flod_param_arrays* v_in, const flod_param_arrays* out,
                         const flod_param_arrays* m_out, const flod_param_arrays* v_out,
                         uint32_t capacity, uint32_t* d_count, uint32_t* d_counts3,
                         void* scratch, size_t scratch_bytes, flod_stream stream) {
  if (!set || set->n < 0 || set->n >= (1 << FLOD_SEL_SHIFT) || set->sh_degree < 0 ||
      set->sh_degree > 3 || !d_count || !scratch || !(tau >= 0.f) || !(max_clone_scale >= 0.f) ||
      !(min_opacity >= 0.f))
    return FLOD_ERR_INVALID_ARG;
  if (set->n > 0 && (!set->means || !set->quats || !set->s_opt || !set->opacity_logit ||
                     !set->sh || !accum || !denom || !normals || !aligned16(set->quats)))
    return FLOD_ERR_INVALID_ARG;
  if (capacity > 0 && (!all_set(out) || !aligned16(out->quats))) return FLOD_ERR_INVALID_ARG;
  const int nm = (m_in != nullptr) + (v_in != nullptr) + (m_out != nullptr) + (v_out != nullptr);
  if (nm != 0 && nm != 4) return FLOD_ERR_INVALID_ARG;
  if (nm == 4 && (!all_set(m_in) || !all_set(v_in) || (capacity > 0 && (!all_set(m_out) || !all_set(v_out)))))
    return FLOD_ERR_INVALID_ARG;
  if (scratch_bytes < dens_scratch_bytes((uint32_t)set->n)) return FLOD_ERR_WORKSPACE;
  DevInfo* dev = nullptr;
  flod_status s = device_info(&dev);
  if (s != FLOD_OK) return s;
  DensP p;
  memset(&p, 0, sizeof(p));
  p.in = SetP{set->means, set->quats, set->s_opt, set->opacity_logit, set->sh, set->n,
              set->sh_degree, set->s_min, 0};
  p.n = (uint32_t)set->n;
  p.s_min = set->s_min;
  p.K3 = 3 * (set->sh_degree + 1) * (set->sh_degree + 1);
  p.accum = accum;
  p.denom = denom;
  p.normals = normals;
  p.tau = tau;
  p.max_clone_scale = max_clone_scale;
  p.min_opacity = min_opacity;
  if (out) p.out = *out;
  if (nm == 4) {
    p.m_in = *m_in;
    p.v_in = *v_in;
    p.m_out = *m_out;
    p.v_out = *v_out;
    p.has_moments = 1;
  }
  p.capacity = capacity;
  p.d_count = d_count;
  p.d_counts3 = d_counts3;
  return launch_densify(p, scratch, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FLOD_OK
             : FLOD_ERR_CUDA;
}

size_t flod_prune_scratch_size(int n) {
  if (n < 0 || n >= (1 << FLOD_SEL_SHIFT)) return 0;
  return prune_scratch_bytes((uint32_t)n);
}

flod_status flod_overlap_prune(const flod_gaussians* set, float d_op, uint8_t* keep, float* d_avg,
                               uint32_t* out_kept, uint32_t* d_kept_count, uint32_t* d_status,
                               void* scratch, size_t scratch_bytes, flod_stream stream) {
  if (!set || set->n < 0 || set->n >= (1 << FLOD_SEL_SHIFT) || !(d_op > 0.f) || !isfinite(d_op) ||
      !d_kept_count || !scratch || (set->n > 0 && (!set->means || !keep)))
    return FLOD_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(scratch) & 255u) return FLOD_ERR_INVALID_ARG;
  if (scratch_bytes < prune_scratch_bytes((uint32_t)set->n)) return FLOD_ERR_WORKSPACE;
  DevInfo* dev = nullptr;
  flod_status s = device_info(&dev);
  if (s != FLOD_OK) return s;
  return launch_prune(set->means, (uint32_t)set->n, d_op, keep, d_avg, out_kept, d_kept_count,
                      d_status, scratch, dev->res_small, reinterpret_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? FLOD_OK
             : FLOD_ERR_CUDA;
}

size_t flod_select_scratch_size(const flod_gaussians* levels, int n_levels) {
  if (!levels || n_levels < 1 || n_levels > FLOD_MAX_SETS) return 0;
  int ns[FLOD_MAX_SETS];
  for (int l = 0; l < n_levels; ++l) ns[l] = levels[l].n < 0 ? 0 : levels[l].n;
  const size_t nb = select_blocks(ns, n_levels);
  return 4 * (nb + 1 + nb * select_mask_words());   // block counts, then keep bits
}

flod_status flod_select_levels(const flod_gaussians* levels, int n_levels, const float* d_thresh,
                               float gamma, float focal, const float origin[3], uint32_t* out_sel,
                               uint32_t sel_capacity, uint32_t* d_count, void* scratch,
                               size_t scratch_bytes, flod_stream stream) {
  if (!levels || n_levels < 1 || n_levels > FLOD_MAX_SETS || !origin || !d_count ||
      (!out_sel && sel_capacity > 0))
    return FLOD_ERR_INVALID_ARG;
  SetP lv[FLOD_MAX_SETS];
  int ns[FLOD_MAX_SETS];
  for (int l = 0; l < n_levels; ++l) {
    const flod_gaussians& g = levels[l];
    if (g.n < 0 || g.n >= (1 << FLOD_SEL_SHIFT) || (g.n > 0 && !g.means)) return FLOD_ERR_INVALID_ARG;
    lv[l] = SetP{g.means, g.quats, g.s_opt, g.opacity_logit, g.sh, g.n, g.sh_degree, g.s_min};
    ns[l] = g.n;
  }
  float th[FLOD_MAX_SETS];
  for (int l = 0; l + 1 < n_levels; ++l) {
    if (d_thresh) {
      th[l] = d_thresh[l];
    } else {
      if (!(gamma > 0.f) || !(focal > 0.f)) return FLOD_ERR_INVALID_ARG;
      th[l] = (float)((double)levels[l].s_min * (double)focal / (double)gamma);   // Eq. 7
    }
    if (!(th[l] >= 0.f)) return FLOD_ERR_INVALID_ARG;
    if (l > 0 && th[l] > th[l - 1]) return FLOD_ERR_INVALID_ARG;
  }
  float lo[FLOD_MAX_SETS], hi[FLOD_MAX_SETS];
  for (int l = 0; l < n_levels; ++l) {
    hi[l] = l == 0 ? INFINITY : th[l - 1];
    lo[l] = l == n_levels - 1 ? 0.f : th[l];
  }
  const uint32_t nb = select_blocks(ns, n_levels);
  if (nb && (!scratch || scratch_bytes < 4 * (size_t)(nb + 1))) return FLOD_ERR_WORKSPACE;
  DevInfo* dev = nullptr;
  flod_status s = device_info(&dev);
  if (s != FLOD_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the keep bits when the scratch holds them (else the write kernel decides again)
  uint32_t* counts = static_cast<uint32_t*>(scratch);
  uint32_t* masks = nb && scratch_bytes >= 4 * ((size_t)nb + 1 + (size_t)nb * select_mask_words())
                        ? counts + nb + 1 : nullptr;
  cudaError_t e = launch_select(lv, n_levels, lo, hi, origin, out_sel, sel_capacity, d_count,
                                counts, masks, nb, st);
  return e == cudaSuccess ? FLOD_OK : FLOD_ERR_CUDA;
}

flod_status flod_adjust_scale(float* s_opt, int64_t n, float s_min_cur, float s_min_next,
                              flod_stream stream) {
  if (n < 0 || (n > 0 && !s_opt) || !(s_min_cur >= s_min_next) || !(s_min_next >= 0.f))
    return FLOD_ERR_INVALID_ARG;
  DevInfo* dev = nullptr;
  flod_status s = device_info(&dev);
  if (s != FLOD_OK) return s;
  return launch_adjust_scale(s_opt, n, s_min_cur, s_min_next,
                             reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? FLOD_OK
             : FLOD_ERR_CUDA;
}

flod_status flod_read_status(const void* ws, uint32_t* out, flod_stream stream) {
  if (!ws || !out) return FLOD_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  if (cudaMemcpyAsync(&v, ws, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return FLOD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FLOD_ERR_CUDA;
  *out = v;
  return FLOD_OK;
}

const char* flod_status_string(flod_status s) {
  switch (s) {
    case FLOD_OK: return "ok";
    case FLOD_ERR_INVALID_ARG: return "invalid argument";
    case FLOD_ERR_CAPACITY: return "pair capacity exceeded";
    case FLOD_ERR_TIMEOUT: return "device wait timed out";
    case FLOD_ERR_CUDA: return "CUDA error";
    case FLOD_ERR_UNSUPPORTED: return "unsupported device (needs sm_103)";
    case FLOD_ERR_WORKSPACE: return "workspace too small";
  }
  return "unknown status";
}

}  // extern "C"
