// Density control of a level (the Densification and Pruning steps of Algorithm 1, with the
// backbone's rules, Sec. 5.1.4).
//
// k_dens_stats, after each blending backward: for every unit that touches a tile, the norm
// of its 2D-mean gradient in normalised device coordinates (the pixel-space gradient of the
// unit's record times (W/2, H/2)) is added to the Gaussian's accumulator and its count
// incremented (atomics: several views may render a Gaussian).
//
// The step (every densification interval), three launches without inter-CTA waits:
//   k_dens_count  per block of 1024 Gaussians, how many survive in place, are cloned, split;
//   k_dens_scan   one CTA: exclusive scans of the three counts and the new set's size;
//   k_dens_write  the new set in order: survivors (index order), then clones, then two
//                 children per split Gaussian (means mu + R (s * eps) from the caller's
//                 normal draws, the learnable part of the scale over 1.6), Adam moments
//                 carried for survivors and zero for the new Gaussians.
// Decisions in float32: g = accum / denom >= tau; max(exp(s_opt) + s_min) > max_clone_scale
// splits, else clones; sigmoid(logit) < min_opacity prunes (the Gaussian and its copies).
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace flod {

constexpr int kDensBlock = 1024;
constexpr float kSplitScale = 1.6f;

// ---------------------------------------------------------------------------------------
// statistics
// ---------------------------------------------------------------------------------------
template <int MAXV>
__global__ void __launch_bounds__(256) k_dens_stats(const __grid_constant__ Batch<MAXV> b, Ws ws,
                                                    const __grid_constant__ DensStatsP p) {
  pdl_entry();
  const uint32_t u = blockIdx.x * 256u + threadIdx.x;
  if (u >= b.units || ws.tiles_touched[u] == 0) return;
  const ViewP& V = b.views[view_of_unit(b, u)];
  const uint32_t local = u - V.unit_off;
  uint32_t si, gi;
  if (V.sel) {
    if (local >= *V.sel_count || local >= V.cap) return;
    const uint32_t e = V.sel[local];
    si = e >> FLOD_SEL_SHIFT;
    gi = e & ((1u << FLOD_SEL_SHIFT) - 1u);
  } else {
    si = (uint32_t)V.set;
    gi = local;
  }
  if (si >= (uint32_t)b.n_sets || gi >= (uint32_t)b.sets[si].n || !p.accum[si]) return;
  const float gx = ws.grad2d[9ull * u] * (0.5f * (float)V.width);
  const float gy = ws.grad2d[9ull * u + 1] * (0.5f * (float)V.height);
  atomicAdd(p.accum[si] + gi, sqrtf(gx * gx + gy * gy));
  atomicAdd(p.denom[si] + gi, 1.f);
}

// ---------------------------------------------------------------------------------------
// the step
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void dens_decide(const DensP& p, uint32_t i, bool& survive, bool& clone,
                                            bool& split) {
  const float den = p.denom[i];
  const float g = den > 0.f ? p.accum[i] / den : 0.f;
  const float* so = p.in.s_opt + 3ull * i;
  const float smax = fmaxf(fmaxf(expf(so[0]), expf(so[1])), expf(so[2])) + p.s_min;
  const bool big = smax > p.max_clone_scale;
  const float op = 1.f / (1.f + expf(-p.in.logit[i]));
  const bool low = op < p.min_opacity;
  const bool dens = g >= p.tau;
  clone = dens && !big && !low;
  split = dens && big && !low;
  survive = !(dens && big) && !low;
}

__global__ void __launch_bounds__(256) k_dens_count(const __grid_constant__ DensP p) {
  pdl_entry();
  __shared__ uint32_t red[3][8];
  uint32_t c[3] = {0u, 0u, 0u};
  for (int r = 0; r < kDensBlock / 256; ++r) {
    const uint32_t i = blockIdx.x * (uint32_t)kDensBlock + r * 256u + threadIdx.x;
    if (i >= p.n) break;
    bool s, cl, sp;
    dens_decide(p, i, s, cl, sp);
    c[0] += s;
    c[1] += cl;
    c[2] += sp;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = c[k];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += red[threadIdx.x][w];
    p.blocks[threadIdx.x * p.nb + blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_dens_scan(const __grid_constant__ DensP p) {
  pdl_entry();
  __shared__ uint32_t wt[32];
  __shared__ uint32_t carry_s;
  __shared__ uint32_t tot[3];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int k = 0; k < 3; ++k) {
    uint32_t* a = p.blocks + (size_t)k * p.nb;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (uint32_t base = 0; base < p.nb; base += 1024) {
      const uint32_t i = base + tid;
      const uint32_t v = i < p.nb ? a[i] : 0u;
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
      if (i < p.nb) a[i] = excl;
      __syncthreads();
      if (tid == 1023) carry_s = excl + v;
      __syncthreads();
    }
    if (tid == 0) tot[k] = carry_s;
    __syncthreads();
  }
  if (tid == 0) {
    p.blocks[3 * (size_t)p.nb] = tot[0];
    p.blocks[3 * (size_t)p.nb + 1] = tot[1];
    *p.d_count = tot[0] + tot[1] + 2u * tot[2];
    if (p.d_counts3) {
      p.d_counts3[0] = tot[0];
      p.d_counts3[1] = tot[1];
      p.d_counts3[2] = tot[2];
    }
  }
}

// Copies Gaussian i of the input into output slot k (parameters, and the moments or zeros).
__device__ __forceinline__ void dens_copy(const DensP& p, uint32_t i, uint32_t k, bool moments) {
  const int K3 = p.K3;
#pragma unroll
  for (int c = 0; c < 3; ++c) p.out.means[3ull * k + c] = p.in.means[3ull * i + c];
  reinterpret_cast<float4*>(p.out.quats)[k] = reinterpret_cast<const float4*>(p.in.quats)[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) p.out.s_opt[3ull * k + c] = p.in.s_opt[3ull * i + c];
  p.out.opacity_logit[k] = p.in.logit[i];
  for (int c = 0; c < K3; ++c) p.out.sh[(uint64_t)K3 * k + c] = p.in.sh[(uint64_t)K3 * i + c];
  if (!p.has_moments) return;
  for (int t = 0; t < 2; ++t) {
    const flod_param_arrays& src = t ? p.v_in : p.m_in;
    const flod_param_arrays& dst = t ? p.v_out : p.m_out;
    for (int c = 0; c < 3; ++c) dst.means[3ull * k + c] = moments ? src.means[3ull * i + c] : 0.f;
    for (int c = 0; c < 4; ++c) dst.quats[4ull * k + c] = moments ? src.quats[4ull * i + c] : 0.f;
    for (int c = 0; c < 3; ++c) dst.s_opt[3ull * k + c] = moments ? src.s_opt[3ull * i + c] : 0.f;
    dst.opacity_logit[k] = moments ? src.opacity_logit[i] : 0.f;
    for (int c = 0; c < K3; ++c)
      dst.sh[(uint64_t)K3 * k + c] = moments ? src.sh[(uint64_t)K3 * i + c] : 0.f;
  }
}

__device__ __forceinline__ void quat_rotate(const float4 q, const float v[3], float out[3]) {
  const float n = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x * n, x = q.y * n, y = q.z * n, z = q.w * n;
  const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                      2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                      2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
#pragma unroll
  for (int r = 0; r < 3; ++r) out[r] = R[3 * r] * v[0] + R[3 * r + 1] * v[1] + R[3 * r + 2] * v[2];
}

__global__ void __launch_bounds__(256) k_dens_write(const __grid_constant__ DensP p) {
  pdl_entry();
  __shared__ uint32_t wcnt[3][8];
  __shared__ uint32_t base_s[3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x < 3) base_s[threadIdx.x] = p.blocks[threadIdx.x * p.nb + blockIdx.x];
  const uint32_t S = p.blocks[3 * (size_t)p.nb], Cn = p.blocks[3 * (size_t)p.nb + 1];
  for (int r = 0; r < kDensBlock / 256; ++r) {
    const uint32_t i = blockIdx.x * (uint32_t)kDensBlock + r * 256u + threadIdx.x;
    bool f[3] = {false, false, false};
    if (i < p.n) dens_decide(p, i, f[0], f[1], f[2]);
    uint32_t pos[3];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const uint32_t bal = __ballot_sync(0xffffffffu, f[k]);
      if (lane == 0) wcnt[k][wid] = __popc(bal);
      pos[k] = __popc(bal & ((1u << lane) - 1u));
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 3; ++k)
      for (int w = 0; w < wid; ++w) pos[k] += wcnt[k][w];
    if (f[0]) {
      const uint32_t k = base_s[0] + pos[0];
      if (k < p.capacity) dens_copy(p, i, k, true);
    }
    if (f[1]) {
      const uint32_t k = S + base_s[1] + pos[1];
      if (k < p.capacity) dens_copy(p, i, k, false);
    }
    if (f[2]) {
      const float* so = p.in.s_opt + 3ull * i;
      const float s[3] = {expf(so[0]) + p.s_min, expf(so[1]) + p.s_min, expf(so[2]) + p.s_min};
      const float4 q = reinterpret_cast<const float4*>(p.in.quats)[i];
      for (int c = 0; c < 2; ++c) {
        const uint32_t k = S + Cn + 2u * (base_s[2] + pos[2]) + (uint32_t)c;
        if (k >= p.capacity) continue;
        dens_copy(p, i, k, false);
        const float* e = p.normals + 3ull * (2ull * i + c);
        const float v[3] = {s[0] * e[0], s[1] * e[1], s[2] * e[2]};
        float o[3];
        quat_rotate(q, v, o);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          p.out.means[3ull * k + a] = p.in.means[3ull * i + a] + o[a];
          p.out.s_opt[3ull * k + a] = so[a] - logf(kSplitScale);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      uint32_t t = 0;
      for (int w = 0; w < 8; ++w) t += wcnt[threadIdx.x][w];
      base_s[threadIdx.x] += t;
    }
  }
}

// ---------------------------------------------------------------------------------------
template <int MAXV>
cudaError_t launch_dens_stats(const Batch<MAXV>& b, const Ws& ws, const DensStatsP& p, cudaStream_t st) {
  if (!b.units) return cudaSuccess;
  launch_k(k_dens_stats<MAXV>, dim3((b.units + 255) / 256), dim3(256), 0, st, b, ws, p);
  return cudaGetLastError();
}
template cudaError_t launch_dens_stats<kMaxViewsSmall>(const BatchS&, const Ws&, const DensStatsP&, cudaStream_t);
template cudaError_t launch_dens_stats<FLOD_MAX_VIEWS>(const BatchL&, const Ws&, const DensStatsP&, cudaStream_t);

size_t dens_scratch_bytes(uint32_t n) { return 4 * (3 * (size_t)(n / kDensBlock + 1) + 2); }

cudaError_t launch_densify(DensP p, void* scratch, cudaStream_t st) {
  p.nb = (p.n + kDensBlock - 1) / kDensBlock;
  p.blocks = static_cast<uint32_t*>(scratch);
  if (p.nb) launch_k(k_dens_count, dim3(p.nb), dim3(256), 0, st, p);
  launch_k(k_dens_scan, dim3(1), dim3(1024), 0, st, p);
  if (p.nb) launch_k(k_dens_write, dim3(p.nb), dim3(256), 0, st, p);
  return cudaGetLastError();
}

}  // namespace flod
