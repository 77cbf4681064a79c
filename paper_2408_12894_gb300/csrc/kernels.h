// Launchers of the kernels, one group per translation unit; called by the C-ABI layer.
#pragma once

#include "common.cuh"

namespace flod {

// Launches a kernel (which starts with pdl_entry) with programmatic stream serialization:
// it may be scheduled while the stream's previous kernel finishes.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// How the preprocess backward writes a set's gradients.
enum GradMode : int { kGradAccumulate = 0, kGradAtomic = 1, kGradOverwrite = 2 };

struct GradTable {
  flod_grads g[FLOD_MAX_SETS];
  int mode[FLOD_MAX_SETS];   // GradMode: RMW (one unit per Gaussian), atomics, or store
  int zero[FLOD_MAX_SETS];   // 1: the set's buffers are zero-filled first (flod_grads.overwrite 2)
};

// preprocess.cu
template <int MAXV>
cudaError_t launch_preprocess(const Batch<MAXV>& b, const Ws& ws, cudaStream_t st);
template <int MAXV>
cudaError_t launch_preprocess_bwd(const Batch<MAXV>& b, const Ws& ws, const GradTable& gt,
                                  cudaStream_t st);
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
                          uint32_t cap, uint32_t* d_count, uint32_t* scratch, uint32_t n_blocks,
                          cudaStream_t st);
uint32_t select_blocks(const int* ns, int n_levels);
cudaError_t launch_adjust_scale(float* s_opt, int64_t n, float s_cur, float s_next,
                                cudaStream_t st);

}  // namespace flod
