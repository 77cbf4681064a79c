// The training loss of a level and its gradient: L = (1 - lambda) L1 + lambda (1 - SSIM)
// per image (Sec. 5.1.4: the backbone's L1 and SSIM losses; the Loss step of Algorithm 1),
// SSIM with an 11 x 11 Gaussian window (sigma 1.5, zero outside the image), C1 = 0.01^2,
// C2 = 0.03^2, means over the image's channels and pixels.
//
// The SSIM of pixel p is a function S(mx, my, exx, eyy, exy) of five window sums around p.
// Its gradient to the image x at pixel q is
//   sum_p w(q - p) [dS/dmx(p) + 2 x(q) dS/dexx(p) + y(q) dS/dexy(p)],
// i.e. the same window applied to three per-pixel maps. Two kernels, one CTA per 32 x 32
// output tile of one channel (tiles staged by 4-byte asynchronous copies, zero-filled off the
// image, all in flight at once):
//   k_ssim_maps   stages x and y with a 5-pixel halo, takes the five window sums (rows,
//                 then columns, in shared memory), evaluates S and writes the three maps
//                 (already scaled by -lambda / N) and the CTA's sums of |x - y| and S;
//   k_ssim_grad   stages the three maps with the halo, applies the window to them and
//                 writes dL/dx = the three terms + (1 - lambda) / N sign(x - y); the first
//                 CTA of each image also reduces that image's partial sums into its loss.
// Threads take four output rows of one column in the column pass (14 staged rows in
// registers for 4 x 11 taps) and four adjacent columns in the row pass; outputs are summed
// two at a time with packed float32 FMAs.
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace flod {

constexpr int kLT = 32;                 // output tile edge
constexpr int kLR = 5;                  // window radius (11 taps)
constexpr int kLH = kLT + 2 * kLR;      // staged tile edge with halo (42)
constexpr int kLS = kLH + 1;            // row stride of staged tiles (43: no bank conflicts)
constexpr int kLThreads = 256;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct LossImg {
  uint64_t pix_off;    // first pixel of the image in the concatenated planar layout
  int width, height;
  int tiles_x, tiles_y;
  uint32_t cta_off;    // first CTA (3 channels x tiles) of the image
  float inv_n;         // 1 / (3 W H)
};

struct LossBatch {
  int n_images;
  float lambda;
  uint32_t ctas;
  float win[2 * kLR + 1];   // normalised 1-D Gaussian weights of the window
  LossImg img[FLOD_MAX_VIEWS];
};

__device__ __forceinline__ int image_of_cta(const LossBatch& B, uint32_t c) {
  int lo = 0, hi = B.n_images - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.img[mid].cta_off <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Stages a kLH x kLH region of plane `src` (origin x0 - kLR, y0 - kLR) into `dst`, zeros
// outside the image: one 4-byte cp.async per element (a source size of 0 writes the zero),
// so every element of the region is in flight at once; the caller waits (async_copy_wait)
// and synchronises the CTA.
__device__ __forceinline__ void stage_plane(float* dst, const float* __restrict__ src, int W, int H,
                                            int x0, int y0) {
  // rows by warps, columns by lanes (no division per element)
  const int lane = threadIdx.x & 31;
  for (int r = threadIdx.x >> 5; r < kLH; r += kLThreads / 32) {
    const int gy = y0 - kLR + r;
    const bool rok = gy >= 0 && gy < H;
    const float* row = src + (size_t)(rok ? gy : 0) * W;
    const uint32_t d = smem_addr(dst + r * kLS);
    for (int c = lane; c < kLH; c += 32) {
      const int gx = x0 - kLR + c;
      const bool in = rok && gx >= 0 && gx < W;
      const float* a = in ? row + gx : src;   // a valid address either way
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d + 4u * c), "l"(a),
                   "r"(in ? 4 : 0) : "memory");
    }
  }
}

// Both passes sum 11 taps for outputs taken two at a time as float32 pairs: output pairs
// (2p, 2p + 1) take input j with the weights (w[j - 2p], w[j - 2p - 1]), zero outside the
// window, in one packed FMA. W2[m] = (w[m], w[m - 1]) for m = 0 .. 11.
struct Win2 {
  float2 w[2 * kLR + 2];
};

__device__ __forceinline__ Win2 win_pairs(const float (&win)[2 * kLR + 1]) {
  Win2 W;
#pragma unroll
  for (int m = 0; m < 2 * kLR + 2; ++m)
    W.w[m] = make_float2(m <= 2 * kLR ? win[m] : 0.f, m >= 1 ? win[m - 1] : 0.f);
  return W;
}

// Row pass: for every staged row and every output column, the window sum along the row of
// NV values produced by `val(j)` from the staged arrays. out[v][row * kLT + col]. Items are
// (staged row, kRowCols output columns).
constexpr int kRowCols = 4;
template <int NV, typename F>
__device__ __forceinline__ void row_pass(const Win2& W, float (*out)[kLH * kLT], F&& val) {
  constexpr int NP = kRowCols / 2;   // output pairs per item
  for (int it = threadIdx.x; it < kLH * (kLT / kRowCols); it += kLThreads) {
    const int r = it / (kLT / kRowCols), c0 = (it % (kLT / kRowCols)) * kRowCols;
    float2 acc[NV][NP];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int p = 0; p < NP; ++p) acc[v][p] = dup2(0.f);
#pragma unroll
    for (int j = 0; j < 2 * kLR + 2 + kRowCols - 2; ++j) {
      float e[NV];
      val(r * kLS + c0 + j, e);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const int m = j - 2 * p;
        if (m >= 0 && m <= 2 * kLR + 1) {
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v][p] = fma2(W.w[m], dup2(e[v]), acc[v][p]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float* o = out[v] + r * kLT + c0;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        o[2 * p] = acc[v][p].x;
        o[2 * p + 1] = acc[v][p].y;
      }
    }
  }
}

// Column pass: thread (column tx, row group ty) sums 4 output rows of NV row-pass planes.
template <int NV>
__device__ __forceinline__ void col_pass(const Win2& W, const float (*in)[kLH * kLT],
                                         float (&res)[NV][4]) {
  const int tx = threadIdx.x % kLT, r0 = (threadIdx.x / kLT) * 4;
  float2 acc[NV][2];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v][0] = acc[v][1] = dup2(0.f);
#pragma unroll
  for (int j = 0; j < 2 * kLR + 4; ++j) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float2 e = dup2(in[v][(r0 + j) * kLT + tx]);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int m = j - 2 * p;
        if (m >= 0 && m <= 2 * kLR + 1) acc[v][p] = fma2(W.w[m], e, acc[v][p]);
      }
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    res[v][0] = acc[v][0].x;
    res[v][1] = acc[v][0].y;
    res[v][2] = acc[v][1].x;
    res[v][3] = acc[v][1].y;
  }
}

__device__ __forceinline__ void cta_image(const LossBatch& B, int& im, int& ch, int& x0, int& y0) {
  const uint32_t c = blockIdx.x;
  im = image_of_cta(B, c);
  const LossImg& I = B.img[im];
  const uint32_t local = c - I.cta_off;
  const uint32_t per_ch = (uint32_t)(I.tiles_x * I.tiles_y);
  ch = (int)(local / per_ch);
  const uint32_t t = local % per_ch;
  x0 = (int)(t % I.tiles_x) * kLT;
  y0 = (int)(t / I.tiles_x) * kLT;
}

struct SsimSmem {
  float x[kLH * kLS];
  float y[kLH * kLS];
  float h[5][kLH * kLT];
  float red[2][kLThreads / 32];
};

__global__ void __launch_bounds__(kLThreads) k_ssim_maps(const __grid_constant__ LossBatch B,
                                                         const float* __restrict__ img,
                                                         const float* __restrict__ tgt,
                                                         float* __restrict__ maps,
                                                         float2* __restrict__ partial,
                                                         uint64_t plane_total) {
  pdl_entry();
  __shared__ SsimSmem S;
  float win[2 * kLR + 1];   // the window in registers (not read through a pointer per tap)
#pragma unroll
  for (int k = 0; k < 2 * kLR + 1; ++k) win[k] = B.win[k];
  const Win2 W = win_pairs(win);
  int im, ch, x0, y0;
  cta_image(B, im, ch, x0, y0);
  const LossImg& I = B.img[im];
  const size_t base = 3 * I.pix_off + (size_t)ch * I.width * I.height;
  stage_plane(S.x, img + base, I.width, I.height, x0, y0);
  stage_plane(S.y, tgt + base, I.width, I.height, x0, y0);
  async_copy_wait();
  __syncthreads();
  row_pass<5>(W, S.h, [&](int a, float (&e)[5]) {
    const float xv = S.x[a], yv = S.y[a];
    e[0] = xv;
    e[1] = yv;
    e[2] = xv * xv;
    e[3] = yv * yv;
    e[4] = xv * yv;
  });
  __syncthreads();
  float m[5][4];
  col_pass<5>(W, S.h, m);
  const int tx = threadIdx.x % kLT, r0 = (threadIdx.x / kLT) * 4;
  const float kS = -B.lambda * I.inv_n;     // dL/dS per pixel
  float sum_l1 = 0.f, sum_s = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gx = x0 + tx, gy = y0 + r0 + q;
    if (gx >= I.width || gy >= I.height) continue;
    const float mx = m[0][q], my = m[1][q];
    const float sxx = m[2][q] - mx * mx, syy = m[3][q] - my * my, sxy = m[4][q] - mx * my;
    const float A = 2.f * mx * my + kC1, Bv = 2.f * sxy + kC2;
    const float Cv = mx * mx + my * my + kC1, D = sxx + syy + kC2;
    // C >= C1 and D >= C2 > 0: the only divisions (no division by A or B, which may vanish)
    const float iC = 1.f / Cv, iD = 1.f / D;
    const float iCD = iC * iD;
    const float s = A * Bv * iCD;
    const float dmx = 2.f * my * (Bv - A) * iCD + 2.f * mx * s * (iD - iC);
    const float dexx = -s * iD;
    const float dexy = 2.f * A * iCD;
    const size_t p = base + (size_t)gy * I.width + gx;
    maps[p] = kS * dmx;
    maps[plane_total + p] = kS * dexx;
    maps[2 * plane_total + p] = kS * dexy;
    sum_s += s;
    sum_l1 += fabsf(S.x[(r0 + q + kLR) * kLS + tx + kLR] - S.y[(r0 + q + kLR) * kLS + tx + kLR]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum_l1 += __shfl_xor_sync(0xffffffffu, sum_l1, o);
    sum_s += __shfl_xor_sync(0xffffffffu, sum_s, o);
  }
  if ((threadIdx.x & 31) == 0) {
    S.red[0][threadIdx.x >> 5] = sum_l1;
    S.red[1][threadIdx.x >> 5] = sum_s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f;
    for (int w = 0; w < kLThreads / 32; ++w) {
      a += S.red[0][w];
      b += S.red[1][w];
    }
    partial[blockIdx.x] = make_float2(a, b);
  }
}

struct GradSmem {
  float f[3][kLH * kLS];
  float h[3][kLH * kLT];
  double red[2][kLThreads / 32];
};

__global__ void __launch_bounds__(kLThreads) k_ssim_grad(const __grid_constant__ LossBatch B,
                                                         const float* __restrict__ img,
                                                         const float* __restrict__ tgt,
                                                         const float* __restrict__ maps,
                                                         const float2* __restrict__ partial,
                                                         uint64_t plane_total,
                                                         float* __restrict__ dL,
                                                         float* __restrict__ loss) {
  pdl_entry();
  __shared__ GradSmem S;
  float win[2 * kLR + 1];
#pragma unroll
  for (int k = 0; k < 2 * kLR + 1; ++k) win[k] = B.win[k];
  const Win2 W = win_pairs(win);
  int im, ch, x0, y0;
  cta_image(B, im, ch, x0, y0);
  const LossImg& I = B.img[im];
  const size_t base = 3 * I.pix_off + (size_t)ch * I.width * I.height;
  const int tx = threadIdx.x % kLT, r0 = (threadIdx.x / kLT) * 4;
  // this thread's four outputs' image and target values, requested first so that their
  // latency passes under the staging and the window sums
  float xv[4], yv[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gx = x0 + tx, gy = y0 + r0 + q;
    const bool in = gx < I.width && gy < I.height;
    const size_t p = base + (size_t)(in ? gy : 0) * I.width + (in ? gx : 0);
    xv[q] = img[p];
    yv[q] = tgt[p];
  }
#pragma unroll
  for (int v = 0; v < 3; ++v)
    stage_plane(S.f[v], maps + v * plane_total + base, I.width, I.height, x0, y0);
  async_copy_wait();
  __syncthreads();
  row_pass<3>(W, S.h, [&](int a, float (&e)[3]) {
    e[0] = S.f[0][a];
    e[1] = S.f[1][a];
    e[2] = S.f[2][a];
  });
  __syncthreads();
  float g[3][4];
  col_pass<3>(W, S.h, g);
  const float kL1 = (1.f - B.lambda) * I.inv_n;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gx = x0 + tx, gy = y0 + r0 + q;
    if (gx >= I.width || gy >= I.height) continue;
    const size_t p = base + (size_t)gy * I.width + gx;
    const float d = xv[q] - yv[q];
    const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    dL[p] = g[0][q] + 2.f * xv[q] * g[1][q] + yv[q] * g[2][q] + kL1 * sg;
  }
  // the image's loss, by its first CTA: (1 - lambda) sum|x - y| / N + lambda (1 - sum S / N)
  if (loss && blockIdx.x == I.cta_off) {
    const uint32_t n = (im + 1 < B.n_images ? B.img[im + 1].cta_off : B.ctas) - I.cta_off;
    double a = 0.0, b = 0.0;
    for (uint32_t i = threadIdx.x; i < n; i += kLThreads) {
      const float2 v = partial[I.cta_off + i];
      a += v.x;
      b += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
      S.red[0][threadIdx.x >> 5] = a;
      S.red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sa = 0.0, sb = 0.0;
      for (int w = 0; w < kLThreads / 32; ++w) {
        sa += S.red[0][w];
        sb += S.red[1][w];
      }
      const double inv_n = 1.0 / (3.0 * I.width * (double)I.height);
      loss[im] = (float)((1.0 - B.lambda) * sa * inv_n + B.lambda * (1.0 - sb * inv_n));
    }
  }
}

// ---------------------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------------------
size_t loss_scratch_bytes(const int* widths, const int* heights, int n, uint32_t* ctas_out,
                          uint64_t* pixels_out) {
  uint64_t pix = 0;
  uint32_t ctas = 0;
  for (int i = 0; i < n; ++i) {
    pix += (uint64_t)widths[i] * heights[i];
    ctas += 3u * (uint32_t)((widths[i] + kLT - 1) / kLT) * (uint32_t)((heights[i] + kLT - 1) / kLT);
  }
  if (ctas_out) *ctas_out = ctas;
  if (pixels_out) *pixels_out = pix;
  // three maps per pixel and channel, then one float2 per CTA (256-byte aligned)
  return (3 * 3 * pix * sizeof(float) + 255) / 256 * 256 + (size_t)ctas * sizeof(float2);
}

cudaError_t launch_loss(const float* img, const float* tgt, const int* widths, const int* heights,
                        int n, float lambda, float* loss, float* dL, void* scratch,
                        cudaStream_t st) {
  static thread_local LossBatch B;
  double wd[2 * kLR + 1], ws = 0.0;
  for (int k = -kLR; k <= kLR; ++k) {
    wd[k + kLR] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
    ws += wd[k + kLR];
  }
  for (int k = 0; k < 2 * kLR + 1; ++k) B.win[k] = (float)(wd[k] / ws);
  uint32_t ctas = 0;
  uint64_t pix = 0;
  loss_scratch_bytes(widths, heights, n, &ctas, &pix);
  if (ctas == 0) return cudaSuccess;
  B.n_images = n;
  B.lambda = lambda;
  B.ctas = ctas;
  uint64_t po = 0;
  uint32_t co = 0;
  for (int i = 0; i < n; ++i) {
    LossImg& I = B.img[i];
    I.pix_off = po;
    I.width = widths[i];
    I.height = heights[i];
    I.tiles_x = (widths[i] + kLT - 1) / kLT;
    I.tiles_y = (heights[i] + kLT - 1) / kLT;
    I.cta_off = co;
    I.inv_n = (float)(1.0 / (3.0 * widths[i] * (double)heights[i]));
    po += (uint64_t)widths[i] * heights[i];
    co += 3u * (uint32_t)(I.tiles_x * I.tiles_y);
  }
  const uint64_t plane_total = 3 * pix;   // floats of one map over all images
  float* maps = static_cast<float*>(scratch);
  float2* partial = reinterpret_cast<float2*>(static_cast<unsigned char*>(scratch) +
                                              (3 * plane_total * sizeof(float) + 255) / 256 * 256);
  launch_k(k_ssim_maps, dim3(ctas), dim3(kLThreads), 0, st, B, img, tgt, maps, partial,
           plane_total);
  launch_k(k_ssim_grad, dim3(ctas), dim3(kLThreads), 0, st, B, img, tgt,
           (const float*)maps, (const float2*)partial, plane_total, dL, loss);
  return cudaGetLastError();
}

}  // namespace flod
