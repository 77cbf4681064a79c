// The preprocess backward (one thread per unit): the chain rule of the preprocess steps
// (geometry.cuh), from the per-unit gradient of (u, v, conic, opacity, rgb) that the
// blending backward accumulated, to the parameters (means, quats, s_opt, opacity_logit, sh);
// and the same fused with the Adam step of Algorithm 1.
#include "geometry.cuh"
#include "kernels.h"

namespace flod {

// Writes v into one gradient slot: read-modify-write, atomic add or plain store.
__device__ __forceinline__ void put1(float* p, float v, int mode) {
  if (mode == kGradOverwrite) *p = v;
  else if (v != 0.f) {
    if (mode == kGradAtomic) atomicAdd(p, v);
    else *p += v;
  }
}
__device__ __forceinline__ void put4(float* p, float4 v, int mode) {   // p 16-byte aligned
  float4* q = reinterpret_cast<float4*>(p);
  if (mode == kGradOverwrite) {
    *q = v;
  } else if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) {
    if (mode == kGradAtomic) {
      atomicAdd(q, v);
    } else {
      float4 o = *q;
      *q = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
    }
  }
}

// Output policies of the preprocess backward. Entries are named by parameter array f
// (0 means, 1 quats, 2 s_opt, 3 opacity logits, 4 sh) and index into it; quats and, at SH
// degree 3, sh entries come four at a time from 16-byte aligned indices.
//   GradOut  writes the gradient (read-modify-write, atomic add or store, by mode);
struct GradOut {
  const flod_grads& G;
  int mode;
  __device__ __forceinline__ float* arr(int f) const {
    return f == 0 ? G.means : f == 1 ? G.quats : f == 2 ? G.s_opt : f == 3 ? G.opacity_logit : G.sh;
  }
  __device__ __forceinline__ bool has(int f) const { return arr(f) != nullptr; }
  __device__ __forceinline__ void one(int f, uint64_t i, float v) const { put1(arr(f) + i, v, mode); }
  __device__ __forceinline__ void four(int f, uint64_t i, float4 v) const { put4(arr(f) + i, v, mode); }
};

// Entries per Gaussian of each parameter array (means, quats, s_opt, opacity logits; the SH
// array has 3 K).
__device__ __forceinline__ int per_gauss(int f, int K3) {
  return f == 0 ? 3 : f == 1 ? 4 : f == 2 ? 3 : f == 3 ? 1 : K3;
}

// Gradients of a CTA's kBA consecutive Gaussians, laid out like their global chunk.
constexpr int kBA = 128;
struct BwdAdamSmem {
  float sh[kBA * 48];
  float4 quats[kBA];
  float means[kBA * 3];
  float s_opt[kBA * 3];
  float opacity[kBA];
};

//   SmemOut  puts the gradient in the CTA's shared chunk (entry index relative to the
//            CTA's first Gaussian), for the Adam pass that follows.
struct SmemOut {
  BwdAdamSmem& G;
  uint32_t g0;   // the CTA's first Gaussian
  int K3;
  __device__ __forceinline__ bool has(int) const { return true; }
  __device__ __forceinline__ float* arr(int f) const {
    return f == 0 ? G.means : f == 1 ? reinterpret_cast<float*>(G.quats) : f == 2 ? G.s_opt
         : f == 3 ? G.opacity : G.sh;
  }
  __device__ __forceinline__ uint64_t rel(int f, uint64_t i) const {
    return i - (uint64_t)per_gauss(f, K3) * g0;
  }
  __device__ __forceinline__ void one(int f, uint64_t i, float g) const { arr(f)[rel(f, i)] = g; }
  __device__ __forceinline__ void four(int f, uint64_t i, float4 g) const {
    *reinterpret_cast<float4*>(arr(f) + rel(f, i)) = g;
  }
};

// A zero gradient for every entry of Gaussian gi (one that touches no tile): stores zeros
// in overwrite mode (the other write modes skip zeros), an Adam step with g = 0 under Adam.
template <class O>
__device__ __forceinline__ void zero_entries(const O& out, uint32_t gi, int K, int deg) {
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (out.has(0)) for (int k = 0; k < 3; ++k) out.one(0, 3ull * gi + k, 0.f);
  if (out.has(1)) out.four(1, 4ull * gi, z4);
  if (out.has(2)) for (int k = 0; k < 3; ++k) out.one(2, 3ull * gi + k, 0.f);
  if (out.has(3)) out.one(3, gi, 0.f);
  if (out.has(4)) {
    const uint64_t b = 3ull * K * gi;
    if (deg == 3) {
      for (int i = 0; i < 12; ++i) out.four(4, b + 4 * i, z4);
    } else {
      for (int i = 0; i < 3 * K; ++i) out.one(4, b + i, 0.f);
    }
  }
}

// The chain rule of one unit from its 2D gradient record to the parameters of Gaussian gi,
// each entry handed to `out`.
template <int MAXV, class O>
__device__ __forceinline__ void unit_backward(const Batch<MAXV>& b, const Ws& ws, const ViewP& V,
                                              const SetP& S, uint32_t u, uint32_t gi,
                                              const O& out) {
  const int K = (S.deg + 1) * (S.deg + 1);
  if (ws.tiles_touched[u] == 0) {
    zero_entries(out, gi, K, S.deg);
    return;
  }
  const float* gr = ws.grad2d + 9ull * u;
  const float3 g0 = make_float3(gr[0], gr[1], gr[2]);   // du, dv, dopacity
  const float3 g1 = make_float3(gr[3], gr[4], gr[5]);   // da, db, dc
  const float3 g2 = make_float3(gr[6], gr[7], gr[8]);   // dr, dg, db
  Geom G;
  geometry(S, gi, V, b.cfg, G);

  // ---- colour -> SH coefficients and view direction. The forward stored max(raw, 0), so
  // a channel is clamped (no gradient) exactly where the stored colour is 0.
  const float4 rgb = ws.rgb[u];
  const float drgb[3] = {rgb.x > 0.f ? g2.x : 0.f, rgb.y > 0.f ? g2.y : 0.f,
                         rgb.z > 0.f ? g2.z : 0.f};
  float Y[16], dir[3], dlen;
  view_dir(S, gi, V, dir, dlen);
  sh_basis(S.deg, dir[0], dir[1], dir[2], Y);
  float dmu[3] = {0.f, 0.f, 0.f};
  if (drgb[0] != 0.f || drgb[1] != 0.f || drgb[2] != 0.f) {
    const float* c = S.sh + 3ull * K * gi;
    float wk[16];
    if (S.deg == 3) {
      const float4* c4 = reinterpret_cast<const float4*>(c);
      float cf[48];
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        const float4 v = __ldg(c4 + i);
        cf[4 * i] = v.x; cf[4 * i + 1] = v.y; cf[4 * i + 2] = v.z; cf[4 * i + 3] = v.w;
      }
#pragma unroll
      for (int k = 0; k < 16; ++k)
        wk[k] = cf[3 * k] * drgb[0] + cf[3 * k + 1] * drgb[1] + cf[3 * k + 2] * drgb[2];
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k)
        wk[k] = k < K ? __ldg(c + 3 * k) * drgb[0] + __ldg(c + 3 * k + 1) * drgb[1] +
                            __ldg(c + 3 * k + 2) * drgb[2]
                      : 0.f;
    }
    float gx, gy, gz;
    sh_grad_dir(S.deg, dir[0], dir[1], dir[2], wk, gx, gy, gz);
    const float proj = gx * dir[0] + gy * dir[1] + gz * dir[2];
    const float il = 1.f / dlen;
    dmu[0] += (gx - proj * dir[0]) * il;
    dmu[1] += (gy - proj * dir[1]) * il;
    dmu[2] += (gz - proj * dir[2]) * il;
  }
  if (out.has(4)) {
    const uint64_t gs = 3ull * K * gi;
    if (S.deg == 3) {
      // 48 values Y[k] * drgb[c] at index 3k + c, as 12 float4
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        float e[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int idx = 4 * q + t;
          e[t] = Y[idx / 3] * drgb[idx % 3];
        }
        out.four(4, gs + 4 * q, make_float4(e[0], e[1], e[2], e[3]));
      }
    } else {
      for (int k = 0; k < K; ++k)
        for (int c = 0; c < 3; ++c) out.one(4, gs + 3 * k + c, Y[k] * drgb[c]);
    }
  }

  // ---- opacity
  const float o = 1.f / (1.f + expf(-__ldg(S.logit + gi)));
  if (out.has(3)) out.one(3, gi, g0.z * o * (1.f - o));

  // ---- conic (a, b, c) -> Sigma' (A, B, C)
  const float A = G.A, B = G.B, C = G.C;
  const float id = 1.f / G.det, id2 = id * id;
  const float da = g1.x, db = g1.y, dc = g1.z;
  const float dA = (-C * C * da + B * C * db - B * B * dc) * id2;
  const float dB = (2.f * B * C * da - (A * C + B * B) * db + 2.f * A * B * dc) * id2;
  const float dC = (-B * B * da + A * B * db - A * A * dc) * id2;
  // ---- Sigma' = P P^T  ->  dP
  float dP[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dP[k] = 2.f * dA * G.P[k] + dB * G.P[3 + k];
    dP[3 + k] = dB * G.P[k] + 2.f * dC * G.P[3 + k];
  }
  // ---- P = T M -> dT, dM ; M = R diag(s)
  float dT[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float dM[9];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float Mjk = G.R[3 * j + k] * G.s[k];
      dT[j] += dP[k] * Mjk;
      dT[3 + j] += dP[3 + k] * Mjk;
      dM[3 * j + k] = G.T[j] * dP[k] + G.T[3 + j] * dP[3 + k];
    }
  float dR[9], ds[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dR[3 * j + k] = dM[3 * j + k] * G.s[k];
      ds[k] += dM[3 * j + k] * G.R[3 * j + k];
    }
  if (out.has(2)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) out.one(2, 3ull * gi + k, ds[k] * G.es[k]);
  }
  // ---- R(q_n) -> dq_n -> dq
  if (out.has(1)) {
    const float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
    const float dw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    const float dx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] +
                            z * dR[6] + w * dR[7] - 2.f * x * dR[8]);
    const float dy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] -
                            w * dR[6] + z * dR[7] - 2.f * y * dR[8]);
    const float dz = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] +
                            y * dR[5] + x * dR[6] + y * dR[7]);
    const float dot = w * dw + x * dx + y * dy + z * dz;
    out.four(1, 4ull * gi,
             make_float4((dw - w * dot) * G.qinv, (dx - x * dot) * G.qinv,
                         (dy - y * dot) * G.qinv, (dz - z * dot) * G.qinv));
  }
  // ---- T = J W -> dJ -> dt ; mean2d -> dt
  const float* W = V.vm;
  float dJ00 = 0.f, dJ02 = 0.f, dJ11 = 0.f, dJ12 = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dJ00 += dT[k] * W[k];
    dJ02 += dT[k] * W[8 + k];
    dJ11 += dT[3 + k] * W[4 + k];
    dJ12 += dT[3 + k] * W[8 + k];
  }
  const float itz = G.itz, itz2 = itz * itz;
  const float tx = G.t[0], ty = G.t[1];
  float dt0 = 0.f, dt1 = 0.f, dt2 = 0.f;
  dt2 += -V.fx * itz2 * dJ00 - V.fy * itz2 * dJ11;
  dt2 += dJ02 * V.fx * G.kx * itz2 + dJ12 * V.fy * G.ky * itz2;
  if (!G.ckx) {
    dt0 += -V.fx * itz2 * dJ02;
    dt2 += dJ02 * V.fx * tx * itz2 * itz;
  }
  if (!G.cky) {
    dt1 += -V.fy * itz2 * dJ12;
    dt2 += dJ12 * V.fy * ty * itz2 * itz;
  }
  dt0 += g0.x * V.fx * itz;
  dt1 += g0.y * V.fy * itz;
  dt2 += -(g0.x * V.fx * tx + g0.y * V.fy * ty) * itz2;
  dmu[0] += W[0] * dt0 + W[4] * dt1 + W[8] * dt2;
  dmu[1] += W[1] * dt0 + W[5] * dt1 + W[9] * dt2;
  dmu[2] += W[2] * dt0 + W[6] * dt1 + W[10] * dt2;
  if (out.has(0)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) out.one(0, 3ull * gi + k, dmu[k]);
  }
}

// Zero-fill of the gradient buffers of the sets marked in gt.zero, over a flat index of
// 16-byte chunks of every (set, parameter) buffer (so a 576 MB SH buffer gets its share of
// the grid like a 12 MB one), scalar stores for unaligned buffers and ragged ends.
struct ZeroSegs {
  float* p[5 * FLOD_MAX_SETS];
  uint64_t n[5 * FLOD_MAX_SETS];            // floats of the buffer
  uint64_t c0[5 * FLOD_MAX_SETS + 1];       // first chunk (4 floats) of each buffer
  int ns;
};

__global__ void __launch_bounds__(256) k_zero_grads(const __grid_constant__ ZeroSegs z) {
  pdl_entry();
  const uint64_t total = z.c0[z.ns];
  const uint64_t stride = (uint64_t)gridDim.x * 256u;
  for (uint64_t q = (uint64_t)blockIdx.x * 256u + threadIdx.x; q < total; q += stride) {
    int lo = 0, hi = z.ns - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (z.c0[mid] <= q) lo = mid; else hi = mid - 1;
    }
    float* p = z.p[lo];
    const uint64_t i = 4 * (q - z.c0[lo]);
    const uint64_t n = z.n[lo];
    if (i + 4 <= n && !(reinterpret_cast<uintptr_t>(p) & 15u)) {
      *reinterpret_cast<float4*>(p + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      for (uint64_t k = i; k < n && k < i + 4; ++k) p[k] = 0.f;
    }
  }
}

template <int MAXV>
__global__ void __launch_bounds__(128) k_preprocess_bwd(const __grid_constant__ Batch<MAXV> b,
                                                        Ws ws, GradTable gt) {
  pdl_entry();
  const uint32_t u = blockIdx.x * 128u + threadIdx.x;
  if (u >= b.units) return;
  const ViewP& V = b.views[view_of_unit(b, u)];
  int si = 0;
  uint32_t gi = 0;
  if (!unit_source(b, V, u - V.unit_off, si, gi)) return;
  unit_backward(b, ws, V, b.sets[si], u, gi, GradOut{gt.g[si], gt.mode[si]});
}

// The same with the Adam step applied to every parameter entry in place of storing its
// gradient. Each set is rendered by one view as a whole set, so a chunk of kBA consecutive
// units is kBA consecutive Gaussians of one set.
//
// Persistent CTAs (two per SM), two warp groups handing chunks over through two
// shared-memory buffers: the gradient group (kBA threads, one Gaussian each) writes a
// chunk's gradients, laid out like the set's arrays, into buffer k % 2 while the Adam group
// (eight warps) takes the Adam step of the previous chunk from the other buffer with
// coalesced 16-byte accesses over the chunk's five parameter arrays (one flat index over
// their 16-byte slots, kBAUnroll slots per thread and round, loads issued before stores).
// So the gradient work of one chunk runs under the memory traffic of another on every SM,
// instead of the two phases alternating within each CTA. Barriers: full[s] (the gradient
// group arrives, the Adam group waits) and empty[s] (the reverse, only before a buffer's
// reuse). At 3M Gaussians: 0.77 ms, against 0.87 ms for one CTA of 128 threads per chunk
// running both phases in turn (with the same Adam arithmetic).
constexpr int kBAAdam = 256;                    // Adam threads (eight warps)
constexpr int kBAThreads = kBA + kBAAdam;
constexpr int kBAUnroll = 2;                    // 16-byte slots per Adam thread and round
constexpr int kBACtasPerSM = 2;
constexpr int kBAStages = 2;                  // shared gradient buffers per CTA
constexpr int kBarFull = 1, kBarEmpty = 1 + kBAStages;   // named barrier ids (one per buffer each)

struct ChunkInfo {
  int set, K3;
  uint32_t g0, cnt;   // first Gaussian, Gaussians in the chunk
};

template <int MAXV>
__device__ __forceinline__ ChunkInfo chunk_info(const Batch<MAXV>& b, uint32_t c) {
  const uint32_t u0 = c * (uint32_t)kBA;
  const ViewP& V = b.views[view_of_unit(b, u0)];
  const SetP& S = b.sets[V.set];
  ChunkInfo ci;
  ci.set = V.set;
  ci.K3 = 3 * (S.deg + 1) * (S.deg + 1);
  ci.g0 = u0 - V.unit_off;
  ci.cnt = ci.g0 < (uint32_t)S.n ? min((uint32_t)kBA, (uint32_t)S.n - ci.g0) : 0u;
  return ci;
}

// Offset (floats) of parameter array f's gradients in BwdAdamSmem.
__device__ __forceinline__ uint32_t smem_field(int f) {
  constexpr uint32_t sh = 0, quats = kBA * 48, means = quats + 4 * kBA, s_opt = means + 3 * kBA,
                     opacity = s_opt + 3 * kBA;
  return f == 0 ? means : f == 1 ? quats : f == 2 ? s_opt : f == 3 ? opacity : sh;
}

// The Adam step of one chunk by the Adam group (thread t of kBAAdam), gradients from G.
__device__ __forceinline__ void adam_chunk(const AdamArrays& A, const AdamHyper& h,
                                           const AdamCoef& c, const BwdAdamSmem& G,
                                           const ChunkInfo& ci, int t) {
  const float* gsm = reinterpret_cast<const float*>(&G);
  // exclusive prefix of the five arrays' 16-byte slots in the chunk
  const uint32_t e0 = 3 * ci.cnt / 4, e1 = e0 + ci.cnt, e2 = e1 + 3 * ci.cnt / 4,
                 e3 = e2 + ci.cnt / 4, total = e3 + (uint32_t)ci.K3 * ci.cnt / 4;
  for (uint32_t q0 = t; q0 < total; q0 += kBAUnroll * kBAAdam) {
    float4 P[kBAUnroll], M[kBAUnroll], Vv[kBAUnroll], Gq[kBAUnroll];
    int F[kBAUnroll];
    uint32_t I[kBAUnroll];
#pragma unroll
    for (int r = 0; r < kBAUnroll; ++r) {
      const uint32_t q = q0 + r * kBAAdam;
      F[r] = (q >= e0) + (q >= e1) + (q >= e2) + (q >= e3);
      I[r] = q - (F[r] == 0 ? 0u : F[r] == 1 ? e0 : F[r] == 2 ? e1 : F[r] == 3 ? e2 : e3);
      if (q < total) {
        const uint64_t off = (uint64_t)per_gauss(F[r], ci.K3) * ci.g0 + 4ull * I[r];
        P[r] = *reinterpret_cast<const float4*>(A.in[F[r]] + off);
        M[r] = *reinterpret_cast<const float4*>(A.m[F[r]] + off);
        Vv[r] = *reinterpret_cast<const float4*>(A.v[F[r]] + off);
        Gq[r] = *reinterpret_cast<const float4*>(gsm + smem_field(F[r]) + 4 * I[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < kBAUnroll; ++r) {
      const uint32_t q = q0 + r * kBAAdam;
      if (q < total) {
        const uint64_t off = (uint64_t)per_gauss(F[r], ci.K3) * ci.g0 + 4ull * I[r];
        float lr[4];
        chunk_lr(h, F[r], 4ull * I[r], ci.K3, lr);   // chunks start on a Gaussian's row
        P[r].x = adam1(P[r].x, Gq[r].x, M[r].x, Vv[r].x, lr[0], c);
        P[r].y = adam1(P[r].y, Gq[r].y, M[r].y, Vv[r].y, lr[1], c);
        P[r].z = adam1(P[r].z, Gq[r].z, M[r].z, Vv[r].z, lr[2], c);
        P[r].w = adam1(P[r].w, Gq[r].w, M[r].w, Vv[r].w, lr[3], c);
        *reinterpret_cast<float4*>(A.out[F[r]] + off) = P[r];
        *reinterpret_cast<float4*>(A.m[F[r]] + off) = M[r];
        *reinterpret_cast<float4*>(A.v[F[r]] + off) = Vv[r];
      }
    }
  }
  if (!(ci.cnt & 3u)) return;
  // ragged ends (a set's last chunk, when its count is not a multiple of 4)
#pragma unroll 1
  for (int f = 0; f < 5; ++f) {
    const uint64_t base = (uint64_t)per_gauss(f, ci.K3) * ci.g0;
    const uint32_t n = (uint32_t)per_gauss(f, ci.K3) * ci.cnt;
    for (uint32_t i = n / 4 * 4 + t; i < n; i += kBAAdam) {
      const float lr = f == 4 ? sh_lr(h, (int)(i % (uint32_t)ci.K3)) : h.lr[f];
      float m = A.m[f][base + i], v = A.v[f][base + i];
      A.out[f][base + i] = adam1(A.in[f][base + i], gsm[smem_field(f) + i], m, v, lr, c);
      A.m[f][base + i] = m;
      A.v[f][base + i] = v;
    }
  }
}

template <int MAXV>
__global__ void __launch_bounds__(kBAThreads, kBACtasPerSM)
    k_preprocess_bwd_adam(const __grid_constant__ Batch<MAXV> b, Ws ws,
                          const __grid_constant__ AdamTable at, uint32_t n_chunks) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdAdamSmem* buf = reinterpret_cast<BwdAdamSmem*>(smem_raw);   // two buffers
  __shared__ AdamCoef s_c;
  if (threadIdx.x == 0) s_c = adam_coef(at.h);
  __syncthreads();
  if (threadIdx.x < kBA) {
    // gradient group: chunk k of this CTA into buffer k % 2
    uint32_t k = 0;
    for (uint32_t c = blockIdx.x; c < n_chunks; c += gridDim.x, ++k) {
      const int s = (int)(k % kBAStages);
      if (k >= (uint32_t)kBAStages) named_sync(kBarEmpty + s, kBAThreads);
      const uint32_t u = c * (uint32_t)kBA + threadIdx.x;
      const ViewP& V = b.views[view_of_unit(b, u)];
      const SetP& S = b.sets[V.set];
      const uint32_t g0 = c * (uint32_t)kBA - V.unit_off;
      int si = 0;
      uint32_t gi = 0;
      if (unit_source(b, V, u - V.unit_off, si, gi))
        unit_backward(b, ws, V, S, u, gi, SmemOut{buf[s], g0, 3 * (S.deg + 1) * (S.deg + 1)});
      named_arrive(kBarFull + s, kBAThreads);
    }
  } else {
    // Adam group: chunk k from buffer k % 2, then hand the buffer back if it is reused
    const AdamCoef c = s_c;
    const int t = threadIdx.x - kBA;
    uint32_t k = 0;
    for (uint32_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x, ++k) {
      const int s = (int)(k % kBAStages);
      named_sync(kBarFull + s, kBAThreads);
      const ChunkInfo ci = chunk_info(b, ch);
      if (ci.cnt) adam_chunk(at.a[ci.set], at.h, c, buf[s], ci, t);
      if (ch + kBAStages * gridDim.x < n_chunks) named_arrive(kBarEmpty + s, kBAThreads);
    }
  }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
template <int MAXV>
cudaError_t launch_zero_grads(const Batch<MAXV>& b, const GradTable& gt, int grid, cudaStream_t st) {
  ZeroSegs z;
  int ns = 0;
  uint64_t chunks = 0;
  for (int s = 0; s < b.n_sets; ++s) {
    if (!gt.zero[s] || b.sets[s].n == 0) continue;
    const uint64_t n = (uint64_t)b.sets[s].n;
    const uint64_t K = (uint64_t)(b.sets[s].deg + 1) * (b.sets[s].deg + 1);
    const flod_grads& g = gt.g[s];
    float* ptr[5] = {g.means, g.quats, g.s_opt, g.opacity_logit, g.sh};
    const uint64_t cnt[5] = {3 * n, 4 * n, 3 * n, n, 3 * K * n};
    for (int f = 0; f < 5; ++f) {
      if (!ptr[f]) continue;
      z.p[ns] = ptr[f];
      z.n[ns] = cnt[f];
      z.c0[ns] = chunks;
      chunks += (cnt[f] + 3) / 4;
      ++ns;
    }
  }
  if (!ns) return cudaSuccess;
  z.c0[ns] = chunks;
  z.ns = ns;
  const uint64_t want = (chunks + 2047) / 2048;   // about eight chunks per thread
  const unsigned blocks = (unsigned)(want < (uint64_t)grid ? (want ? want : 1) : (uint64_t)grid);
  launch_k(k_zero_grads, dim3(blocks), dim3(256), 0, st, z);
  return cudaGetLastError();
}

template <int MAXV>
cudaError_t launch_preprocess_bwd(const Batch<MAXV>& b, const Ws& ws, const GradTable& gt,
                                  cudaStream_t st) {
  if (b.units == 0) return cudaSuccess;
  launch_k(k_preprocess_bwd<MAXV>, dim3((b.units + 127) / 128), dim3(128), 0, st, b, ws, gt);
  return cudaGetLastError();
}

template <int MAXV>
cudaError_t launch_preprocess_bwd_adam(const Batch<MAXV>& b, const Ws& ws, const AdamTable& at,
                                       int sms, cudaStream_t st) {
  if (b.units) {
    constexpr int smem = kBAStages * (int)sizeof(BwdAdamSmem);
    static int per_sm = 0;   // resident CTAs per SM, once per template instance
    if (!per_sm) {
      cudaError_t e = cudaFuncSetAttribute(k_preprocess_bwd_adam<MAXV>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_preprocess_bwd_adam<MAXV>,
                                                          kBAThreads, smem);
      if (e != cudaSuccess) return e;
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
    }
    const uint32_t n_chunks = (uint32_t)((b.units + kBA - 1) / kBA);
    const uint32_t grid = min(n_chunks, (uint32_t)(per_sm * sms));
    launch_k(k_preprocess_bwd_adam<MAXV>, dim3(grid), dim3(kBAThreads), smem, st, b, ws, at,
             n_chunks);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_adam_tick(const_cast<uint32_t*>(at.h.d_step), st);
}

template cudaError_t launch_zero_grads<kMaxViewsSmall>(const BatchS&, const GradTable&, int, cudaStream_t);
template cudaError_t launch_zero_grads<FLOD_MAX_VIEWS>(const BatchL&, const GradTable&, int, cudaStream_t);
template cudaError_t launch_preprocess_bwd<kMaxViewsSmall>(const BatchS&, const Ws&, const GradTable&, cudaStream_t);
template cudaError_t launch_preprocess_bwd<FLOD_MAX_VIEWS>(const BatchL&, const Ws&, const GradTable&, cudaStream_t);
template cudaError_t launch_preprocess_bwd_adam<kMaxViewsSmall>(const BatchS&, const Ws&, const AdamTable&, int, cudaStream_t);
template cudaError_t launch_preprocess_bwd_adam<FLOD_MAX_VIEWS>(const BatchL&, const Ws&, const AdamTable&, int, cudaStream_t);

}  // namespace flod
