// Adjoint kernels of the D2Q9 relative-velocity step: the reverse step with FP32 forward
// states (the kernel itself is in d2q9_adjoint_step.cuh; the 16-bit instances are in
// d2q9_adjoint16.cu), the final gather, the accumulator sum, and the adjoints of the
// equilibrium initialisation, the moments and the kinetic energy.
#include <cuda_runtime.h>

#include "d2q9.cuh"
#include "d2q9_adjoint.cuh"
#include "d2q9_adjoint_step.cuh"
#include "launch.h"
#include "pull.cuh"

namespace lbmrv {

namespace {

// dst = P^T src (gather), used once for dL/dS_0 = P^T mu_1.
template <int NV>
__global__ void __launch_bounds__(kAdjThreads) k_gather(const float* __restrict__ src,
                                                        float* __restrict__ dst, int nx, int ny) {
    const int64_t n = (int64_t)nx * ny;
    const PackLane p = pack_lane<NV>(nx);
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        const int ym = y == 0 ? ny - 1 : y - 1;
        const int yp = y == ny - 1 ? 0 : y + 1;
        const int64_t r0 = (int64_t)y * nx, rm = (int64_t)ym * nx, rp = (int64_t)yp * nx;
        float v[9][NV];
        gather_pack<float, NV>(src, n, r0, rm, rp, p, v);
        if (p.act) {
#pragma unroll
            for (int j = 0; j < 9; ++j) store_pack<float, NV>(dst + j * n + r0 + p.x0, v[j]);
        }
    }
}

// Sum of the per-block accumulators, fixed order: out[c] = sum_b acc[b * 8 + c].
__global__ void __launch_bounds__(256) k_acc_final(const double* __restrict__ acc, int64_t nblk,
                                                   double* __restrict__ out) {
    __shared__ double sh[256];
    for (int c = 0; c < 8; ++c) {
        double s = 0.0;
        for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) s += acc[b * 8 + c];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int st = 128; st > 0; st >>= 1) {
            if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = sh[0];
        __syncthreads();
    }
}

// Adjoint of the equilibrium initialisation g_j = f_eq,j(rho, u) - f_eq,j(rho_ref, U):
// dL/drho = sum_j a_j w_j (1 + 3 cu + 9/2 cu^2 - 3/2 |u|^2),
// dL/du   = sum_j a_j w_j rho (3 c + 9 cu c - 3 u) / lambda, with u in units of lambda.
__global__ void k_equilibrium_vjp(const float* __restrict__ rho, const float* __restrict__ u,
                                  const float* __restrict__ a, float* __restrict__ drho,
                                  float* __restrict__ du, int64_t n, float inv_lambda) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float r = rho ? rho[i] : 1.0f;
        const float ux = u[i] * inv_lambda, uy = u[n + i] * inv_lambda;
        const float uu = ux * ux + uy * uy;
        float gr = 0.f, gx = 0.f, gy = 0.f;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const float cx = (float)((j == 1 || j == 5 || j == 8) - (j == 3 || j == 6 || j == 7));
            const float cy = (float)((j == 2 || j == 5 || j == 6) - (j == 4 || j == 7 || j == 8));
            const float cu = cx * ux + cy * uy;
            const float wa = wgt(j) * a[j * n + i];
            gr += wa * (1.0f + 3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
            gx += wa * r * (3.0f * cx + 9.0f * cu * cx - 3.0f * ux);
            gy += wa * r * (3.0f * cy + 9.0f * cu * cy - 3.0f * uy);
        }
        if (drho) drho[i] = gr;
        if (du) {
            du[i] = gx * inv_lambda;
            du[n + i] = gy * inv_lambda;
        }
    }
}

// Adjoint of the moments (rho, u = lambda j / rho) of a stored state (storage type T):
// dL/dg_j = dL/drho + (lambda / rho) (dL/du . (c_j - j / rho)).
template <typename T>
__global__ void k_moments_vjp(const T* __restrict__ g, const float* __restrict__ drho,
                              const float* __restrict__ du, float* __restrict__ out, int64_t n,
                              StoreRef ref, float lambda) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float h[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) h[j] = to_f(g[j * n + i]);
        const NodeMoments m = node_moments(h);
        const float ir = recip(ref.rho + m.drho);
        const float ux = (ref.jx + m.jx) * ir, uy = (ref.jy + m.jy) * ir;
        const float br = drho ? drho[i] : 0.0f;
        const float bx = du ? du[i] * lambda * ir : 0.0f;
        const float by = du ? du[n + i] * lambda * ir : 0.0f;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const float cx = (float)((j == 1 || j == 5 || j == 8) - (j == 3 || j == 6 || j == 7));
            const float cy = (float)((j == 2 || j == 5 || j == 6) - (j == 4 || j == 7 || j == 8));
            out[j * n + i] = br + bx * (cx - ux) + by * (cy - uy);
        }
    }
}

// Kinetic energy L = 1/2 sum lambda^2 |j|^2 / rho of nodes 0 .. n-1 of a stored state
// (storage type T, planes `plane` elements apart; per-block FP64 partials in part[b*4]), and
// optionally dL/dg_j = lambda^2 (c_j . j / rho - 1/2 |j|^2 / rho^2) at those nodes.
template <typename T>
__global__ void __launch_bounds__(kReduceThreads) k_kinetic_energy(const T* __restrict__ g,
                                                                   float* __restrict__ grad,
                                                                   int64_t n, int64_t plane,
                                                                   StoreRef ref,
                                                                   float lambda,
                                                                   double* __restrict__ part) {
    float ke = 0.0f;
    const float l2 = lambda * lambda;
    double acc = 0.0;
    int cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float h[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) h[j] = to_f(g[j * plane + i]);
        const NodeMoments m = node_moments(h);
        const float ir = recip(ref.rho + m.drho);
        const float jx = ref.jx + m.jx, jy = ref.jy + m.jy;
        const float jj = jx * jx + jy * jy;
        ke += 0.5f * l2 * jj * ir;
        if (++cnt == 64) {  // keep the FP32 run short, accumulate in FP64
            acc += (double)ke;
            ke = 0.0f;
            cnt = 0;
        }
        if (grad) {
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const float cx = (float)((j == 1 || j == 5 || j == 8) - (j == 3 || j == 6 || j == 7));
                const float cy = (float)((j == 2 || j == 5 || j == 6) - (j == 4 || j == 7 || j == 8));
                grad[j * plane + i] = l2 * ((cx * jx + cy * jy) * ir - 0.5f * jj * ir * ir);
            }
        }
    }
    acc += (double)ke;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFullMask, acc, o);
    __shared__ double sh[kReduceThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) s += sh[w];
        part[4 * (int64_t)blockIdx.x] = s;
    }
}

__global__ void k_partials_final(const double* __restrict__ part, int nblk,
                                 double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[4 * b];
        out[0] = s;
    }
}


}  // namespace

dim3 adjoint_grid(int nx, int ny, int nv) {
    const int threads_x = (nx / nv + (nx % nv ? 1 : 0));
    return dim3((threads_x + kAdjThreads - 1) / kAdjThreads, ny < 65535 ? ny : 65535);
}

int64_t adjoint_blocks(int nx, int ny, int nv) {
    const dim3 g = adjoint_grid(nx, ny, nv);
    return (int64_t)g.x * g.y;
}

cudaError_t launch_adjoint_step(int storage, int um, int nv, const void* s_prev,
                                const float* a_in, bool gather, float* mu_out,
                                const AdjointArgs& aa, cudaStream_t st) {
    if (storage == kStoreF32)
        return launch_adjoint_step_t<float>(um, nv, s_prev, a_in, gather, mu_out, aa, st);
    return launch_adjoint_step16(storage, um, nv, s_prev, a_in, gather, mu_out, aa, st);
}

cudaError_t launch_gather(const float* src, float* dst, int nx, int ny, cudaStream_t st) {
    const int nv = (nx % 4 == 0) ? 4 : 1;
    const dim3 grid = adjoint_grid(nx, ny, nv);
    if (nv == 4)
        k_gather<4><<<grid, kAdjThreads, 0, st>>>(src, dst, nx, ny);
    else
        k_gather<1><<<grid, kAdjThreads, 0, st>>>(src, dst, nx, ny);
    return cudaGetLastError();
}

cudaError_t launch_acc_final(const double* acc, int64_t nblk, double* out, cudaStream_t st) {
    k_acc_final<<<1, 256, 0, st>>>(acc, nblk, out);
    return cudaGetLastError();
}

cudaError_t launch_equilibrium_vjp(const float* rho, const float* u, const float* a, float* drho,
                                   float* du, int64_t n, float inv_lambda, cudaStream_t st) {
    k_equilibrium_vjp<<<grid_stride_blocks(n, 256), 256, 0, st>>>(rho, u, a, drho, du, n, inv_lambda);
    return cudaGetLastError();
}

cudaError_t launch_moments_vjp(int storage, const void* g, const float* drho, const float* du,
                               float* out, int64_t n, const StoreRef& ref, float lambda,
                               cudaStream_t st) {
    const int b = grid_stride_blocks(n, 256);
    switch (storage) {
        case kStoreF32:
            k_moments_vjp<<<b, 256, 0, st>>>(static_cast<const float*>(g), drho, du, out, n, ref,
                                             lambda);
            break;
        case kStoreF16:
            k_moments_vjp<<<b, 256, 0, st>>>(static_cast<const __half*>(g), drho, du, out, n,
                                             ref, lambda);
            break;
        case kStoreBF16:
            k_moments_vjp<<<b, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(g), drho, du, out,
                                             n, ref, lambda);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_kinetic_energy(int storage, const void* g, float* grad, int64_t n,
                                  int64_t plane, const StoreRef& ref, float lambda,
                                  double* partials, int nblk, double* out, cudaStream_t st) {
    switch (storage) {
        case kStoreF32:
            k_kinetic_energy<<<nblk, kReduceThreads, 0, st>>>(static_cast<const float*>(g), grad,
                                                              n, plane, ref, lambda, partials);
            break;
        case kStoreF16:
            k_kinetic_energy<<<nblk, kReduceThreads, 0, st>>>(static_cast<const __half*>(g), grad,
                                                              n, plane, ref, lambda, partials);
            break;
        case kStoreBF16:
            k_kinetic_energy<<<nblk, kReduceThreads, 0, st>>>(
                static_cast<const __nv_bfloat16*>(g), grad, n, plane, ref, lambda, partials);
            break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_partials_final<<<1, 32, 0, st>>>(partials, nblk, out);
    return cudaGetLastError();
}

}  // namespace lbmrv
