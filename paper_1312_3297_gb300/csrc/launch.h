// Internal launch interface between the C-ABI layer (lbmrv_api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "d2q9.cuh"
#include "d3q19.cuh"

namespace lbmrv {

enum { kStoreF32 = 0, kStoreF16 = 1, kStoreBF16 = 2 };

constexpr int kReduceThreads = 256;
// Most partial sums of a reduction (8 blocks per SM of a 152-SM GB300; any GPU works with
// it). A compile-time constant because it sizes the fixed scratch of
// lbmrv_conserved_noalloc.
constexpr int kReduceMaxBlocks = 152 * 8;
// Blocks of the reduction kernels resident on one SM, at least (their launch bounds).
constexpr int kReduceMinBlocks = 4;

// Blocks of a grid-stride kernel over n items with `threads` per block: enough for every
// item, at most 16 per SM of the current device (found once per device).
int grid_stride_blocks(int64_t n, int threads);

// Widest vector pack (nodes per thread) the fused step can use for this row length.
int step_vector_width(int storage, int nx);

// One fused step src -> dst. um: UM_* of d2q9.cuh; nv: 1 (scalar kernel) or a vector
// width returned by step_vector_width (or any smaller power of two dividing nx); basis 0:
// the orthogonal moments of the paper's D2Q9 example, 1: Geier's (cascaded) basis.
cudaError_t launch_step(int storage, int um, int nv, const void* src, void* dst,
                        const StepArgs& a, cudaStream_t st, int basis = 0);

// The same step (nv >= 2) with the FP64 conserved sums of dst fused in, written to out[4]
// as launch_conserved does; partials: step_sum_scratch(nx, ny, nv) doubles of scratch.
int64_t step_sum_blocks(int nx, int ny, int nv);
int64_t step_sum_scratch(int nx, int ny, int nv);
cudaError_t launch_step_conserved(int storage, int um, int nv, const void* src, void* dst,
                                  const StepArgs& a, cudaStream_t st, int basis, double rho_ref,
                                  double jx_ref, double jy_ref, double lambda,
                                  double* partials, double* out);

cudaError_t launch_init_eq(int storage, void* dst, const float* rho, const float* u, int64_t n,
                           const StoreRef& ref, float inv_lambda, cudaStream_t st,
                           int basis = 0);

cudaError_t launch_moments(int storage, const void* src, float* rho, float* u, int64_t n,
                           const StoreRef& ref, float lambda, cudaStream_t st);

int conserved_blocks(int64_t n);

// Sums over nodes 0 .. n-1 of src, whose planes are `plane` >= n elements apart.
// partials: 4 * nblk doubles of scratch; out: 4 doubles (device). rho_ref, jx_ref, jy_ref:
// the stored reference state (jx_ref = rho_ref U_x / lambda).
cudaError_t launch_conserved(int storage, const void* src, int64_t n, int64_t plane,
                             double rho_ref, double jx_ref, double jy_ref, double lambda,
                             double* partials, int nblk, double* out, cudaStream_t st);

// Sums {rho, rho u_x, rho u_y, rho u_z} over nodes 0 .. n-1 of initial fields (rho NULL:
// 1; u: dim planes `plane` floats apart) into out[4] (device); partials: 4 * nblk doubles.
cudaError_t launch_mean_flow(const float* rho, const float* u, int64_t n, int64_t plane,
                             int dim, double* partials, int nblk, double* out, cudaStream_t st);

// ---------------------------------------------------------------- D3Q19
int step3_vector_width(int storage, int nx);
cudaError_t launch_step3(int storage, int um, int nv, const void* src, void* dst,
                         const StepArgs3& a, cudaStream_t st);
cudaError_t launch_init_eq3(int storage, void* dst, const float* rho, const float* u, int64_t n,
                            const StoreRef3& ref, float inv_lambda, cudaStream_t st);
cudaError_t launch_moments3(int storage, const void* src, float* rho, float* u, int64_t n,
                            const StoreRef3& ref, float lambda, cudaStream_t st);
// The step with the FP64 conserved sums of dst fused in (FP32 with 4-node packs, 16-bit with
// 8-node packs), written to out[5] as launch_conserved3 does; partials: scratch of
// step3_sum_scratch(...) doubles (-1 on a CUDA error).
bool step3_fuses_sums(int storage, int nv, int ny, int nz);
int64_t step3_sum_scratch(int storage, int nv, const StepArgs3& a);
cudaError_t launch_step3_conserved(int storage, int um, int nv, const void* src, void* dst,
                                   const StepArgs3& a, cudaStream_t st, double lambda,
                                   double* partials, int64_t scratch, double* out);
// partials: 8 * nblk doubles; out: 5 doubles (sum rho, sum q (3), non-finite nodes) over
// nodes 0 .. n-1 of src, whose planes are `plane` >= n elements apart.
cudaError_t launch_conserved3(int storage, const void* src, int64_t n, int64_t plane,
                              const StoreRef3& ref, double lambda, double* partials, int nblk,
                              double* out, cudaStream_t st);

// ---------------------------------------------------------------- adjoint (FP32 adjoint
// vectors; forward states in the handle's storage type)
struct AdjointArgs {
    StepArgs step;     // step arguments of the relaxation being reversed (time k)
    float da_factor;   // d(u~/lambda)/dA = cos(2 pi k / P) / lambda for dL/dA
    float* dut0;       // optional [2][n]: accumulates amp_t * dL/d(u~/lambda) per node
    double* acc;       // per-block FP64 accumulators, 8 per block (6 rates, dL/dA, unused)
    int y0 = 0, y1 = 0;  // rows reversed: [y0, y1) (a slab's own rows; else 0 .. ny)
};

dim3 adjoint_grid(int nx, int ny, int nv);
int64_t adjoint_blocks(int nx, int ny, int nv);

// mu_out = J_C(P s_prev)^T a, a = (gather ? P^T a_in : a_in); accumulates into aa.acc;
// nv nodes per thread (1, 2 or 4, dividing nx unless 1); s_prev in the storage type.
cudaError_t launch_adjoint_step(int storage, int um, int nv, const void* s_prev,
                                const float* a_in, bool gather, float* mu_out,
                                const AdjointArgs& aa, cudaStream_t st);
// The same for FP16 / BF16 forward states (d2q9_adjoint16.cu).
cudaError_t launch_adjoint_step16(int storage, int um, int nv, const void* s_prev,
                                  const float* a_in, bool gather, float* mu_out,
                                  const AdjointArgs& aa, cudaStream_t st);
cudaError_t launch_gather(const float* src, float* dst, int nx, int ny, cudaStream_t st);
cudaError_t launch_acc_final(const double* acc, int64_t nblk, double* out, cudaStream_t st);
cudaError_t launch_equilibrium_vjp(const float* rho, const float* u, const float* a, float* drho,
                                   float* du, int64_t n, float inv_lambda, cudaStream_t st);
cudaError_t launch_moments_vjp(int storage, const void* g, const float* drho, const float* du,
                               float* out, int64_t n, const StoreRef& ref, float lambda,
                               cudaStream_t st);
// partials: 4 * nblk doubles of scratch (slot 0 of each used); out: 1 double (device).
// Over nodes 0 .. n-1 of g (and grad), planes `plane` elements apart.
cudaError_t launch_kinetic_energy(int storage, const void* g, float* grad, int64_t n,
                                  int64_t plane, const StoreRef& ref, float lambda,
                                  double* partials, int nblk, double* out, cudaStream_t st);

}  // namespace lbmrv
