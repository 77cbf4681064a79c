// Real spherical harmonics to degree 3 (Condon-Shortley phase, index l*l + l + m) and their
// Cartesian gradients, for unit directions. The colour model of Sec. 3 ("spherical
// harmonic coefficients"): rgb = max(0, sum_k c_k Y_k(dir) + 0.5).
//
// Normalisation constants are K = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the
// polynomial factors of the associated Legendre functions; each literal below is given with
// its closed form. The polynomials use x^2 + y^2 + z^2 = 1 to stay low-order; the gradient
// of the colour with respect to the mean goes through the normalisation of the direction,
// which removes the radial part, so these forms give the same result as the unreduced ones.
#pragma once

namespace flod {

constexpr float kY0 = 0.28209479177387814f;    // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.4886025119029199f;     // sqrt(3 / (4 pi))
constexpr float kY2a = 1.0925484305920792f;    // sqrt(15 / (4 pi))
constexpr float kY2b = 0.31539156525252005f;   // sqrt(5 / (16 pi))
constexpr float kY2c = 0.5462742152960396f;    // sqrt(15 / (16 pi))
constexpr float kY3a = 0.5900435899266435f;    // sqrt(35 / (32 pi))
constexpr float kY3b = 2.890611442640554f;     // sqrt(105 / (4 pi))
constexpr float kY3c = 0.4570457994644658f;    // sqrt(21 / (32 pi))
constexpr float kY3d = 0.3731763325901154f;    // sqrt(7 / (16 pi))
constexpr float kY3e = 1.445305721320277f;     // sqrt(105 / (16 pi))

// Y[k] for k < (deg+1)^2.
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
  Y[0] = kY0;
  if (deg < 1) return;
  Y[1] = -kY1 * y;
  Y[2] = kY1 * z;
  Y[3] = -kY1 * x;
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kY2a * x * y;
  Y[5] = -kY2a * y * z;
  Y[6] = kY2b * (2.f * zz - xx - yy);
  Y[7] = -kY2a * x * z;
  Y[8] = kY2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -kY3a * y * (3.f * xx - yy);
  Y[10] = kY3b * x * y * z;
  Y[11] = -kY3c * y * (4.f * zz - xx - yy);
  Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kY3c * x * (4.f * zz - xx - yy);
  Y[14] = kY3e * z * (xx - yy);
  Y[15] = -kY3a * x * (xx - 3.f * yy);
}

// Gradient of sum_k w[k] Y_k with respect to the (unit) direction, for weights w[k].
__device__ __forceinline__ void sh_grad_dir(int deg, float x, float y, float z, const float* w,
                                            float& gx, float& gy, float& gz) {
  gx = gy = gz = 0.f;
  if (deg < 1) return;
  gx += -kY1 * w[3];
  gy += -kY1 * w[1];
  gz += kY1 * w[2];
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  gx += kY2a * y * w[4];
  gy += kY2a * x * w[4];
  gy += -kY2a * z * w[5];
  gz += -kY2a * y * w[5];
  gx += -2.f * kY2b * x * w[6];
  gy += -2.f * kY2b * y * w[6];
  gz += 4.f * kY2b * z * w[6];
  gx += -kY2a * z * w[7];
  gz += -kY2a * x * w[7];
  gx += 2.f * kY2c * x * w[8];
  gy += -2.f * kY2c * y * w[8];
  if (deg < 3) return;
  gx += -kY3a * 6.f * x * y * w[9];
  gy += -kY3a * 3.f * (xx - yy) * w[9];
  gx += kY3b * y * z * w[10];
  gy += kY3b * x * z * w[10];
  gz += kY3b * x * y * w[10];
  gx += -kY3c * (-2.f * x * y) * w[11];
  gy += -kY3c * (4.f * zz - xx - 3.f * yy) * w[11];
  gz += -kY3c * 8.f * y * z * w[11];
  gx += kY3d * (-6.f * x * z) * w[12];
  gy += kY3d * (-6.f * y * z) * w[12];
  gz += kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
  gx += -kY3c * (4.f * zz - 3.f * xx - yy) * w[13];
  gy += -kY3c * (-2.f * x * y) * w[13];
  gz += -kY3c * 8.f * x * z * w[13];
  gx += kY3e * 2.f * x * z * w[14];
  gy += kY3e * (-2.f * y * z) * w[14];
  gz += kY3e * (xx - yy) * w[14];
  gx += -kY3a * 3.f * (xx - yy) * w[15];
  gy += -kY3a * (-6.f * x * y) * w[15];
}

}  // namespace flod
