// Launchers of the kernels, one group per translation unit; called by the C-ABI layer.
#pragma once

#include "common.cuh"

namespace flod {

// Launches a kernel (which starts with pdl_entry) with programmatic stream serialization:
// it may be scheduled while the stream's previous kernel finishes. launch_k_full waits for
// the previous kernel to finish first (an ordinary launch; pdl_entry's wait is then a no-op).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kx(bool overlap, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                             size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = overlap ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, Args... args) {
  return launch_kx(true, kernel, grid, block, smem, st, args...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k_full(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                 cudaStream_t st, Args... args) {
  return launch_kx(false, kernel, grid, block, smem, st, args...);
}

// How the preprocess backward writes a set's gradients.
enum GradMode : int { kGradAccumulate = 0, kGradAtomic = 1, kGradOverwrite = 2 };

struct GradTable {
  flod_grads g[FLOD_MAX_SETS];
  int mode[FLOD_MAX_SETS];   // GradMode: RMW (one unit per Gaussian), atomics, or store
  int zero[FLOD_MAX_SETS];   // 1: the set's buffers are zero-filled first (flod_grads.overwrite 2)
};

// ---------------------------------------------------------------------------------------
// Adam (the Adam step of Algorithm 1) on the parameter arrays of a set
// ---------------------------------------------------------------------------------------
struct AdamArrays {
  const float* in[5];   // current parameters: means, quats, s_opt, opacity logits, sh
  float* out[5];        // where the updated parameters go (may alias in)
  float* m[5];          // first moments
  float* v[5];          // second moments
};

struct AdamHyper {
  float lr[6];          // means, quats, s_opt, opacity logits, SH coefficient 0, SH 1..K-1
  double beta1, beta2;  // exact, for the bias corrections
  float b1, b2, omb1, omb2, eps;   // beta and 1 - beta rounded from double, eps
  const uint32_t* d_step;   // steps taken so far: this step is t = *d_step + 1
};

struct AdamTable {
  AdamArrays a[FLOD_MAX_SETS];
  AdamHyper h;
};

// Bias corrections of step t: 1 / (1 - beta1^t) and 1 / sqrt(1 - beta2^t), in double.
struct AdamCoef {
  float b1, b2, omb1, omb2, eps, bc1, bc2s;
};

__device__ __forceinline__ AdamCoef adam_coef(const AdamHyper& h) {
  const double t = (double)(*h.d_step) + 1.0;
  AdamCoef c;
  c.b1 = h.b1;
  c.b2 = h.b2;
  c.omb1 = h.omb1;
  c.omb2 = h.omb2;
  c.eps = h.eps;
  c.bc1 = (float)(1.0 / (1.0 - pow(h.beta1, t)));
  c.bc2s = (float)(1.0 / sqrt(1.0 - pow(h.beta2, t)));
  return c;
}

// One Adam step of one entry: m, v updated in place, the new parameter returned. The
// square root and the division are the hardware approximations (sqrt.approx, __fdividef),
// a few float32 ulp on the step instead of the correctly rounded instruction sequences,
// which made the Adam passes issue-bound (standalone Adam at 3M Gaussians 0.93 -> 0.75 ms).
__device__ __forceinline__ float adam1(float p, float g, float& m, float& v, float lr,
                                       const AdamCoef& c) {
  m = fmaf(c.b1, m, c.omb1 * g);
  v = fmaf(c.b2, v, c.omb2 * (g * g));
  float sq;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(sq) : "f"(v));
  return fmaf(-lr, __fdividef(m * c.bc1, fmaf(sq, c.bc2s, c.eps)), p);
}

// Learning rate of entry e (0 .. 3K-1) of a Gaussian's SH coefficients: coefficient 0 (the
// DC term) has its own rate.
__device__ __forceinline__ float sh_lr(const AdamHyper& h, int e) { return e < 3 ? h.lr[4] : h.lr[5]; }

// Learning rates of the four entries i .. i+3 of parameter array f (one modulo per chunk).
__device__ __forceinline__ void chunk_lr(const AdamHyper& h, int f, uint64_t i, int K3,
                                         float (&lr)[4]) {
  if (f != 4) {
    lr[0] = lr[1] = lr[2] = lr[3] = h.lr[f];
    return;
  }
  // the entry's place in its Gaussian's SH row: 32-bit arithmetic below 2^32 entries, a
  // constant divisor at degree 3 (a 64-bit modulo is a long instruction sequence)
  const uint32_t i32 = (uint32_t)i;
  const int e0 = i >> 32 ? (int)(i % (uint64_t)K3)
               : K3 == 48 ? (int)(i32 % 48u) : (int)(i32 % (uint32_t)K3);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int e = e0 + t;
    e = e >= K3 ? e - K3 : e;
    lr[t] = sh_lr(h, e);
  }
}

// adam.cu
cudaError_t launch_adam(const AdamArrays* a, const flod_param_arrays* grads, const int* n,
                        const int* sh_degree, int n_sets, const AdamHyper& h, int grid,
                        cudaStream_t st);
cudaError_t launch_adam_tick(uint32_t* d_step, cudaStream_t st);

// gather.cu
struct GatherP {
  SetP sets[FLOD_MAX_SETS];
  int n_sets;
  const uint32_t* entries;   // (set << FLOD_SEL_SHIFT) | index, or NULL: index k of set 0
  const uint32_t* d_count;   // entries to copy (device)
  uint32_t capacity;         // at most this many
  flod_param_arrays out;
  float* out_s_min;          // optional: the source set's s_min of every output Gaussian
  int out_K3;                // SH floats per output Gaussian
  int fold;                  // 1: s_opt' = log(exp(s_opt) + s_min) (output at s_min = 0)
};
cudaError_t launch_gather(const GatherP& g, int grid, cudaStream_t st);

// densify.cu
struct DensStatsP {
  float* accum[FLOD_MAX_SETS];   // per set (NULL: skipped)
  float* denom[FLOD_MAX_SETS];
};
struct DensP {
  SetP in;
  uint32_t n;
  float s_min;
  int K3;
  const float* accum;
  const float* denom;
  const float* normals;          // [2n, 3] standard normal draws for the split children
  float tau, max_clone_scale, min_opacity;
  flod_param_arrays out, m_in, v_in, m_out, v_out;
  int has_moments;
  uint32_t capacity;
  uint32_t* d_count;
  uint32_t* d_counts3;
  uint32_t* blocks;
  uint32_t nb;
};
template <int MAXV>
cudaError_t launch_dens_stats(const Batch<MAXV>& b, const Ws& ws, const DensStatsP& p, cudaStream_t st);
size_t dens_scratch_bytes(uint32_t n);
cudaError_t launch_densify(DensP p, void* scratch, cudaStream_t st);

// prune.cu
size_t prune_scratch_bytes(uint32_t n);
cudaError_t launch_prune(const float* means, uint32_t n, float d_op, uint8_t* keep, float* d_avg,
                         uint32_t* out_kept, uint32_t* d_kept, uint32_t* d_status, void* scratch,
                         int grid, cudaStream_t st);

// loss.cu
size_t loss_scratch_bytes(const int* widths, const int* heights, int n, uint32_t* ctas,
                          uint64_t* pixels);
cudaError_t launch_loss(const float* img, const float* tgt, const int* widths, const int* heights,
                        int n, float lambda, float* loss, float* dL, void* scratch,
                        cudaStream_t st);

// preprocess.cu
template <int MAXV>
cudaError_t launch_preprocess(const Batch<MAXV>& b, const Ws& ws, cudaStream_t st);
template <int MAXV>
cudaError_t launch_preprocess_bwd(const Batch<MAXV>& b, const Ws& ws, const GradTable& gt,
                                  cudaStream_t st);
// the preprocess backward with an Adam step on each entry in place of writing its gradient
template <int MAXV>
cudaError_t launch_preprocess_bwd_adam(const Batch<MAXV>& b, const Ws& ws, const AdamTable& at,
                                       int sms, cudaStream_t st);
// zero-fills the gradient buffers of the sets with gt.zero set (one launch, in stream order)
template <int MAXV>
cudaError_t launch_zero_grads(const Batch<MAXV>& b, const GradTable& gt, int grid, cudaStream_t st);

// binning.cu: unit sort -> block sums -> scan -> emit -> pair sort -> ranges. phase 0 runs
// everything; phases 1..4 one part each (FLOD_BIN_PHASE_*), in that order
template <int MAXV>
cudaError_t launch_binning(const Batch<MAXV>& b, const Ws& ws, int n_passes, int tile_bits,
                           int resident_sort,
                           int resident_small, unsigned long long* d_pair_count, bool build_queue,
                           int phase, cudaStream_t st);

// sort.cu
// launch_unit_sort also clears the n_tiles tile ranges (when there are units)
cudaError_t launch_unit_sort(const Ws& ws, uint32_t n_tiles, int resident_small, int resident_sort,
                             cudaStream_t st);
cudaError_t launch_pair_sort(const Ws& ws, int n_digits, int tile_bits, int resident_small,
                             int resident_sort, cudaStream_t st);
int sort_kernel_smem_bytes();
cudaError_t sort_kernel_prepare();           // opt-in shared memory size
const void* sort_kernel_ptr();

// render.cu
template <int MAXV>
cudaError_t launch_render_fwd(const Batch<MAXV>& b, const Ws& ws, float* out_rgb, float* out_T,
                              uint32_t* out_nc, int resident, bool persistent, cudaStream_t st);
template <int MAXV>
cudaError_t launch_render_bwd(const Batch<MAXV>& b, const Ws& ws, const float* dL,
                              const float* fwd_T, const uint32_t* fwd_nc, int resident,
                              bool persistent, cudaStream_t st);

// render.cu: helpers in stream order
cudaError_t launch_zero16(void* p, size_t bytes, int grid, cudaStream_t st);   // 16-B aligned
cudaError_t launch_clear_status(uint32_t* status, cudaStream_t st);

// select.cu
cudaError_t launch_select(const SetP* levels, int n_levels, const float* thresh_lo,
                          const float* thresh_hi, const float origin[3], uint32_t* out,
                          uint32_t cap, uint32_t* d_count, uint32_t* scratch, uint32_t* masks,
                          uint32_t n_blocks, cudaStream_t st);
uint32_t select_blocks(const int* ns, int n_levels);
uint32_t select_mask_words();   // keep-bit words per selection block
cudaError_t launch_adjust_scale(float* s_opt, int64_t n, float s_cur, float s_next,
                                cudaStream_t st);

}  // namespace flod
