// Gathers selected Gaussians of one or more sets into one compact set (structure of arrays):
// the predetermined selective set of Sec. 5.2 made resident on its own, level chunks streamed
// from host memory, pruned or densified sets. Entry k names (set << 28 | index); the output
// Gaussian k is a copy of that source Gaussian. With `fold`, the source set's minimum scale
// moves into the scale parameter, s_opt' = log(exp(s_opt) + s_min) (Eq. 4 with the output
// taken at s_min = 0, i.e. Eq. 5 towards 0), so Gaussians of different levels share one set
// whose rendering scale is exactly theirs.
//
// One warp per 32 output Gaussians: the per-Gaussian arrays move one entry per lane; the SH
// coefficients (3 K floats per Gaussian, contiguous in source and output) move as float4
// runs by the whole warp, Gaussian after Gaussian, so both sides are read and written in
// coalesced runs. Sources may be device memory or host memory the GPU can address (pinned
// and mapped): the copy then crosses the CPU-GPU link.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace flod {

__global__ void __launch_bounds__(256) k_gather(const __grid_constant__ GatherP g) {
  pdl_entry();
  const uint32_t n = min(*g.d_count, g.capacity);
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * 256u + threadIdx.x) >> 5;
  const uint32_t nwarps = gridDim.x * 8u;
  for (uint32_t base = warp * 32u; base < n; base += nwarps * 32u) {
    const uint32_t k = base + lane;
    const bool ok = k < n;
    uint32_t si = 0, gi = 0;
    if (ok) {
      const uint32_t e = g.entries ? g.entries[k] : k;
      si = e >> FLOD_SEL_SHIFT;
      gi = e & ((1u << FLOD_SEL_SHIFT) - 1u);
      if (si >= (uint32_t)g.n_sets || gi >= (uint32_t)g.sets[si].n) {
        si = 0xffffffffu;   // out of range: the output stays as it is
      }
    }
    if (ok && si != 0xffffffffu) {
      const SetP& S = g.sets[si];
#pragma unroll
      for (int c = 0; c < 3; ++c) g.out.means[3ull * k + c] = S.means[3ull * gi + c];
      reinterpret_cast<float4*>(g.out.quats)[k] = reinterpret_cast<const float4*>(S.quats)[gi];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float so = S.s_opt[3ull * gi + c];
        g.out.s_opt[3ull * k + c] = g.fold ? logf(expf(so) + S.s_min) : so;
      }
      g.out.opacity_logit[k] = S.logit[gi];
      if (g.out_s_min) g.out_s_min[k] = S.s_min;
    }
    // SH rows: the warp copies each of its (up to) 32 Gaussians' 3 K floats in turn
    const uint32_t cnt = min(32u, n - base);
    for (uint32_t j = 0; j < cnt; ++j) {
      const uint32_t sj = __shfl_sync(0xffffffffu, si, (int)j);
      const uint32_t gj = __shfl_sync(0xffffffffu, gi, (int)j);
      if (sj == 0xffffffffu) continue;
      const SetP& S = g.sets[sj];
      const int K3 = 3 * (S.deg + 1) * (S.deg + 1);
      const float* src = S.sh + (uint64_t)K3 * gj;
      float* dst = g.out.sh + (uint64_t)g.out_K3 * (base + j);
      if (K3 == g.out_K3 && K3 % 4 == 0) {
        for (int q = lane; q < K3 / 4; q += 32)
          reinterpret_cast<float4*>(dst)[q] = reinterpret_cast<const float4*>(src)[q];
      } else {
        // another degree: copy the common coefficients, zeros for the rest
        for (int q = lane; q < g.out_K3; q += 32) dst[q] = q < K3 ? src[q] : 0.f;
      }
    }
  }
}

cudaError_t launch_gather(const GatherP& g, int grid, cudaStream_t st) {
  launch_k(k_gather, dim3((unsigned)grid), dim3(256), 0, st, g);
  return cudaGetLastError();
}

}  // namespace flod
