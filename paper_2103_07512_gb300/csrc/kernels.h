// kernels.h -- host-side launchers of the device kernels.
#pragma once
#include <cuda_runtime.h>

#include "tgp_ir.h"

namespace tgp {

// Fused interpreter: K in {1, 2, 4, 8, 16}; pheno selects phenotype stores
// instead of fitness partials at tree roots; ext selects the variant that also
// runs the rest of Table 1 (a plan without those operators uses the smaller
// kernel).  threads <= 128.
cudaError_t launch_eval(const EvalParams& p, int K, bool pheno, bool ext, int grid, int threads, size_t smem,
                        cudaStream_t s);
cudaError_t eval_occupancy(int K, bool pheno, bool ext, int threads, size_t smem, int* blocks_per_sm);

// Dynamic shared memory of one interpreter CTA: target values and value
// slots, K points per thread.
size_t eval_smem_bytes(int K, int threads, int n_slots);

// The x part of Eq. 1, x^4 / (1 + x^4) in binary32, at the n_out first columns
// of a grid of W columns on [xlo, xhi] (columns past W - 1 take column W - 1).
cudaError_t launch_pagie_columns(int32_t W, float xlo, float xhi, float* out, int32_t n_out, cudaStream_t s);

// Per-tree binary64 reduction of the fitness partials and sqrt(sum / N).
cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t s);

// Straight-line chains of one operator (0 add, 1 div, 2 sin, 3 cos, 4 mul, 5 min,
// 6 exp, 7 log, 8 pow, 9 tan, 10 sqrt, 11 mod, 12 fused multiply-add).
cudaError_t launch_calib(int opk, const float* in, float* out, int iters, int grid, int threads, cudaStream_t s);

}  // namespace tgp
