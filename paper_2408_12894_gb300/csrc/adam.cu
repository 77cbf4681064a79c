// The Adam step of Algorithm 1 on the parameter arrays (means, rotations, s_opt, opacity
// logits, SH) of one or more Gaussian sets, one learning rate per group (the SH DC
// coefficient apart):
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
//   p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
// with t read from a device counter that k_adam_tick advances after the step (so a captured
// graph replays successive steps). One launch over a flat index of 4-entry chunks of every
// (set, array) segment (16-byte loads and stores when the segment's five arrays allow them).
#include "common.cuh"
#include "kernels.h"

namespace flod {

struct AdamLaunch {
  // one segment per (set, parameter array), in a flat index of 4-entry chunks
  const float* pin[5 * FLOD_MAX_SETS];
  float* pout[5 * FLOD_MAX_SETS];
  float* m[5 * FLOD_MAX_SETS];
  float* v[5 * FLOD_MAX_SETS];
  const float* g[5 * FLOD_MAX_SETS];
  uint64_t n[5 * FLOD_MAX_SETS];        // entries of the segment
  uint64_t chunk0[5 * FLOD_MAX_SETS + 1];   // first chunk of each segment (exclusive scan)
  int field[5 * FLOD_MAX_SETS];    // 0 means, 1 quats, 2 s_opt, 3 opacity logits, 4 sh
  int K3[5 * FLOD_MAX_SETS];       // SH entries per Gaussian of the segment's set
  int vec[5 * FLOD_MAX_SETS];      // the segment's five arrays are 16-byte aligned
  int nseg;
  AdamHyper h;
};

__device__ __forceinline__ int seg_of_chunk(const AdamLaunch& L, uint64_t q) {
  int lo = 0, hi = L.nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.chunk0[mid] <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One 4-entry chunk: its loads are issued before any store.
struct Chunk {
  float4 p, g, m, v;
  int sg;
  uint64_t i;   // first entry
  int cnt;      // entries (4 except at a segment's end)
};

__device__ __forceinline__ void chunk_load(const AdamLaunch& L, uint64_t q, Chunk& c) {
  c.sg = seg_of_chunk(L, q);
  c.i = 4 * (q - L.chunk0[c.sg]);
  const uint64_t n = L.n[c.sg];
  c.cnt = (int)min((uint64_t)4, n - c.i);
  if (c.cnt == 4 && L.vec[c.sg]) {
    c.p = *reinterpret_cast<const float4*>(L.pin[c.sg] + c.i);
    c.g = *reinterpret_cast<const float4*>(L.g[c.sg] + c.i);
    c.m = *reinterpret_cast<const float4*>(L.m[c.sg] + c.i);
    c.v = *reinterpret_cast<const float4*>(L.v[c.sg] + c.i);
  } else {
    float a[4][4] = {};
    for (int t = 0; t < c.cnt; ++t) {
      a[0][t] = L.pin[c.sg][c.i + t];
      a[1][t] = L.g[c.sg][c.i + t];
      a[2][t] = L.m[c.sg][c.i + t];
      a[3][t] = L.v[c.sg][c.i + t];
    }
    c.p = make_float4(a[0][0], a[0][1], a[0][2], a[0][3]);
    c.g = make_float4(a[1][0], a[1][1], a[1][2], a[1][3]);
    c.m = make_float4(a[2][0], a[2][1], a[2][2], a[2][3]);
    c.v = make_float4(a[3][0], a[3][1], a[3][2], a[3][3]);
  }
}

__device__ __forceinline__ void chunk_step(const AdamLaunch& L, const AdamCoef& k, Chunk& c) {
  const int f = L.field[c.sg];
  float lr[4];
  chunk_lr(L.h, f, c.i, L.K3[c.sg], lr);
  c.p.x = adam1(c.p.x, c.g.x, c.m.x, c.v.x, lr[0], k);
  c.p.y = adam1(c.p.y, c.g.y, c.m.y, c.v.y, lr[1], k);
  c.p.z = adam1(c.p.z, c.g.z, c.m.z, c.v.z, lr[2], k);
  c.p.w = adam1(c.p.w, c.g.w, c.m.w, c.v.w, lr[3], k);
  if (c.cnt == 4 && L.vec[c.sg]) {
    *reinterpret_cast<float4*>(L.pout[c.sg] + c.i) = c.p;
    *reinterpret_cast<float4*>(L.m[c.sg] + c.i) = c.m;
    *reinterpret_cast<float4*>(L.v[c.sg] + c.i) = c.v;
  } else {
    const float pp[4] = {c.p.x, c.p.y, c.p.z, c.p.w}, mm[4] = {c.m.x, c.m.y, c.m.z, c.m.w},
                vv[4] = {c.v.x, c.v.y, c.v.z, c.v.w};
    for (int t = 0; t < c.cnt; ++t) {
      L.pout[c.sg][c.i + t] = pp[t];
      L.m[c.sg][c.i + t] = mm[t];
      L.v[c.sg][c.i + t] = vv[t];
    }
  }
}

// Every thread takes two chunks per round (both loaded before either is stored), striding
// over the flat chunk index of all segments, so the work is spread evenly whatever the
// sizes of the arrays.
__global__ void __launch_bounds__(256) k_adam(const __grid_constant__ AdamLaunch L) {
  pdl_entry();
  __shared__ AdamCoef s_c;
  if (threadIdx.x == 0) s_c = adam_coef(L.h);
  __syncthreads();
  const AdamCoef k = s_c;
  const uint64_t total = L.chunk0[L.nseg];
  const uint64_t stride = (uint64_t)gridDim.x * 256u;
  for (uint64_t q = (uint64_t)blockIdx.x * 256u + threadIdx.x; q < total; q += 2 * stride) {
    Chunk a, b;
    chunk_load(L, q, a);
    const bool two = q + stride < total;
    if (two) chunk_load(L, q + stride, b);
    chunk_step(L, k, a);
    if (two) chunk_step(L, k, b);
  }
}

// Advances the step counter after the step's updates (in stream order).
__global__ void k_adam_tick(uint32_t* d_step) {
  pdl_entry();
  *d_step += 1u;
}

cudaError_t launch_adam(const AdamArrays* a, const flod_param_arrays* grads, const int* n,
                        const int* sh_degree, int n_sets, const AdamHyper& h, int grid,
                        cudaStream_t st) {
  static thread_local AdamLaunch L;
  int ns = 0;
  uint64_t chunks = 0;
  for (int k = 0; k < n_sets; ++k) {
    if (n[k] <= 0) continue;
    const int K = (sh_degree[k] + 1) * (sh_degree[k] + 1);
    const float* g[5] = {grads[k].means, grads[k].quats, grads[k].s_opt, grads[k].opacity_logit,
                         grads[k].sh};
    const uint64_t nn = (uint64_t)n[k];
    const uint64_t cnt[5] = {3 * nn, 4 * nn, 3 * nn, nn, 3 * (uint64_t)K * nn};
    for (int f = 0; f < 5; ++f) {
      L.pin[ns] = a[k].in[f];
      L.pout[ns] = a[k].out[f];
      L.m[ns] = a[k].m[f];
      L.v[ns] = a[k].v[f];
      L.g[ns] = g[f];
      L.n[ns] = cnt[f];
      L.chunk0[ns] = chunks;
      L.field[ns] = f;
      L.K3[ns] = 3 * K;
      L.vec[ns] = !((reinterpret_cast<uintptr_t>(a[k].in[f]) | reinterpret_cast<uintptr_t>(a[k].out[f]) |
                     reinterpret_cast<uintptr_t>(a[k].m[f]) | reinterpret_cast<uintptr_t>(a[k].v[f]) |
                     reinterpret_cast<uintptr_t>(g[f])) & 15u);
      chunks += (cnt[f] + 3) / 4;
      ++ns;
    }
  }
  if (ns) {
    L.chunk0[ns] = chunks;
    L.nseg = ns;
    L.h = h;
    const uint64_t want = (chunks + 511) / 512;   // two chunks per thread and round
    const unsigned blocks = (unsigned)min((uint64_t)grid, max((uint64_t)1, want));
    launch_k(k_adam, dim3(blocks), dim3(256), 0, st, L);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_adam_tick(const_cast<uint32_t*>(h.d_step), st);
}

cudaError_t launch_adam_tick(uint32_t* d_step, cudaStream_t st) {
  launch_k(k_adam_tick, dim3(1), dim3(1), 0, st, d_step);
  return cudaGetLastError();
}

}  // namespace flod
