// Internal launch interface between the C-ABI layer (lbmrv_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "d2q9.cuh"

namespace lbmrv {

enum { kStoreF32 = 0, kStoreF16 = 1, kStoreBF16 = 2 };

constexpr int kReduceThreads = 256;
constexpr int kReduceMaxBlocks = 152 * 8;

// Widest vector pack (nodes per thread) the fused step can use for this row length.
int step_vector_width(int storage, int nx);

// One fused step src -> dst. um: UM_* of d2q9.cuh; nv: 1 (scalar kernel) or a vector
// width returned by step_vector_width (or any smaller power of two dividing nx).
cudaError_t launch_step(int storage, int um, int nv, const void* src, void* dst,
                        const StepArgs& a, cudaStream_t st);

cudaError_t launch_init_eq(int storage, void* dst, const float* rho, const float* u, int64_t n,
                           float rho_ref, float inv_lambda, cudaStream_t st);

cudaError_t launch_moments(int storage, const void* src, float* rho, float* u, int64_t n,
                           float rho_ref, float lambda, cudaStream_t st);

int conserved_blocks(int64_t n);

// partials: 4 * nblk doubles of scratch; out: 4 doubles (device).
cudaError_t launch_conserved(int storage, const void* src, int64_t n, double rho_ref,
                             double lambda, double* partials, int nblk, double* out,
                             cudaStream_t st);

}  // namespace lbmrv
