// Per-unit geometry shared by the preprocess and its backward: a unit's source Gaussian,
// the rotation of a unit quaternion, Eq. 4 constrained scale s = exp(s_opt) + s_min
// (Sec. 4.1), Eq. 1 covariance through M = R diag(s) (Sigma = M M^T, Sec. 3), the local-affine
// projection of Eq. 2 (Sigma' = (J W M)(J W M)^T + dilation I), the view direction and the
// SH colour.
#pragma once

#include "common.cuh"
#include "sh.cuh"

namespace flod {

template <int MAXV>
__device__ __forceinline__ bool unit_source(const Batch<MAXV>& b, const ViewP& V, uint32_t local,
                                            int& si, uint32_t& gi) {
  if (V.sel) {
    uint32_t cnt = *V.sel_count;
    if (local >= cnt || local >= V.cap) return false;
    uint32_t e = V.sel[local];
    si = (int)(e >> FLOD_SEL_SHIFT);
    gi = e & ((1u << FLOD_SEL_SHIFT) - 1u);
    return si < b.n_sets && gi < (uint32_t)b.sets[si].n;
  }
  if (local >= V.cap) return false;
  si = V.set;
  gi = local;
  return gi < (uint32_t)b.sets[si].n;
}

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float* R) {
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// Shared forward geometry of one unit (used by both passes).
struct Geom {
  float qn[4], qinv;          // normalised quaternion, 1 / |q|
  float R[9], s[3], es[3];    // rotation, constrained scale, exp(s_opt)
  float t[3], itz;            // view-space mean, 1 / t_z
  float kx, ky;               // clamped t_x/t_z, t_y/t_z used by the Jacobian
  bool ckx, cky;              // whether the clamps were active
  float T[6];                 // J W (2x3)
  float P[6];                 // J W M (2x3)
  float A, B, C, det;         // Sigma' entries (dilated) and determinant
};

__device__ __forceinline__ void geometry(const SetP& S, uint32_t gi, const ViewP& V,
                                         const CfgP& cfg, Geom& G) {
  const float* mu = S.means + 3ull * gi;
  const float4 q = reinterpret_cast<const float4*>(S.quats)[gi];
  const float* so = S.s_opt + 3ull * gi;
  float qq = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  G.qinv = 1.f / sqrtf(qq);
  G.qn[0] = q.x * G.qinv; G.qn[1] = q.y * G.qinv; G.qn[2] = q.z * G.qinv; G.qn[3] = q.w * G.qinv;
  quat_rot(G.qn[0], G.qn[1], G.qn[2], G.qn[3], G.R);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    G.es[k] = expf(so[k]);
    G.s[k] = G.es[k] + S.s_min;
  }
  const float mx = mu[0], my = mu[1], mz = mu[2];
  const float* W = V.vm;
  G.t[0] = W[0] * mx + W[1] * my + W[2] * mz + W[3];
  G.t[1] = W[4] * mx + W[5] * my + W[6] * mz + W[7];
  G.t[2] = W[8] * mx + W[9] * my + W[10] * mz + W[11];
  const float tz = G.t[2];
  G.itz = 1.f / tz;
  const float limx = kClampFov * 0.5f * (float)V.width / V.fx;
  const float limy = kClampFov * 0.5f * (float)V.height / V.fy;
  const float rx = G.t[0] * G.itz, ry = G.t[1] * G.itz;
  G.kx = fminf(fmaxf(rx, -limx), limx);
  G.ky = fminf(fmaxf(ry, -limy), limy);
  G.ckx = (rx < -limx) || (rx > limx);
  G.cky = (ry < -limy) || (ry > limy);
  // J = [[fx/tz, 0, -fx kx/tz], [0, fy/tz, -fy ky/tz]]; T = J W
  const float j00 = V.fx * G.itz, j02 = -V.fx * G.kx * G.itz;
  const float j11 = V.fy * G.itz, j12 = -V.fy * G.ky * G.itz;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    G.T[k] = j00 * W[k] + j02 * W[8 + k];
    G.T[3 + k] = j11 * W[4 + k] + j12 * W[8 + k];
  }
  // P = T M, M = R diag(s)
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      G.P[3 * r + k] = (G.T[3 * r] * G.R[k] + G.T[3 * r + 1] * G.R[3 + k] + G.T[3 * r + 2] * G.R[6 + k]) * G.s[k];
  G.A = G.P[0] * G.P[0] + G.P[1] * G.P[1] + G.P[2] * G.P[2] + cfg.dilation;
  G.B = G.P[0] * G.P[3] + G.P[1] * G.P[4] + G.P[2] * G.P[5];
  G.C = G.P[3] * G.P[3] + G.P[4] * G.P[4] + G.P[5] * G.P[5] + cfg.dilation;
  G.det = G.A * G.C - G.B * G.B;
}

// Unit view direction from the camera centre to the mean, and its length.
__device__ __forceinline__ void view_dir(const SetP& S, uint32_t gi, const ViewP& V, float dir[3],
                                         float& dlen) {
  const float* mu = S.means + 3ull * gi;
  float dx = mu[0] - V.cpx, dy = mu[1] - V.cpy, dz = mu[2] - V.cpz;
  dlen = sqrtf(dx * dx + dy * dy + dz * dz);
  float il = 1.f / dlen;
  dir[0] = dx * il; dir[1] = dy * il; dir[2] = dz * il;
}

// Colour of a unit (and the pre-clamp value), SH of degree deg.
// c: the Gaussian's SH coefficients (3 K floats).
__device__ __forceinline__ void sh_colour(const SetP& S, uint32_t gi, const float* c,
                                          const ViewP& V, float* Y, float dir[3], float& dlen,
                                          float raw[3]) {
  view_dir(S, gi, V, dir, dlen);
  const int K = (S.deg + 1) * (S.deg + 1);
  sh_basis(S.deg, dir[0], dir[1], dir[2], Y);
  raw[0] = raw[1] = raw[2] = 0.5f;
  if (S.deg == 3) {
    const float4* c4 = reinterpret_cast<const float4*>(c);
    float cf[48];
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      float4 v = c4[i];
      cf[4 * i] = v.x; cf[4 * i + 1] = v.y; cf[4 * i + 2] = v.z; cf[4 * i + 3] = v.w;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      raw[0] += Y[k] * cf[3 * k];
      raw[1] += Y[k] * cf[3 * k + 1];
      raw[2] += Y[k] * cf[3 * k + 2];
    }
  } else {
    for (int k = 0; k < K; ++k) {
      raw[0] += Y[k] * c[3 * k];
      raw[1] += Y[k] * c[3 * k + 1];
      raw[2] += Y[k] * c[3 * k + 2];
    }
  }
}

}  // namespace flod
