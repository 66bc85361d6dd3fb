// D3Q19 kernels: fused pull transport + relative-velocity relaxation, equilibrium
// initialisation, moments and FP64 conserved sums. Layout: 19 planes of nx*ny*nz, index
// (z*ny + y)*nx + x.
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "launch.h"
#include "pull.cuh"

namespace lbmrv {

namespace {

constexpr int kThreads3 = 128;

template <int UM>
__device__ __forceinline__ void relative_velocity3(const float g[19], int64_t i, int64_t n,
                                                   const StepArgs3& a, float& ux, float& uy,
                                                   float& uz) {
    if (UM == UM_ZERO) {
        ux = uy = uz = 0.0f;
    } else if (UM == UM_FLUID) {
        const NodeMoments3 m = node_moments3(g);
        const float ir = recip(a.ref.rho + m.drho);
        ux = (a.ref.jx + m.jx) * ir;
        uy = (a.ref.jy + m.jy) * ir;
        uz = (a.ref.jz + m.jz) * ir;
    } else {
        ux = a.amp_t * __ldg(a.ut0 + i);
        uy = a.amp_t * __ldg(a.ut0 + n + i);
        uz = a.amp_t * __ldg(a.ut0 + 2 * n + i);
    }
}

// One thread: NV consecutive nodes of the row (y, z). Population j is pulled from
// (x, y, z) - c_j, periodic (relation (transport)).
template <typename T, int NV, int UM>
__global__ void __launch_bounds__(kThreads3) k_step3(const T* __restrict__ src,
                                                     T* __restrict__ dst, StepArgs3 a) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t n = (int64_t)nx * ny * nz;
    const PackLane p = pack_lane<NV>(nx);
    for (int z = blockIdx.z; z < nz; z += gridDim.z) {
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        for (int y = blockIdx.y; y < ny; y += gridDim.y) {
            const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            auto row = [&](int yy, int zz) { return ((int64_t)zz * ny + yy) * nx; };
            const int64_t r00 = row(y, z), rm0 = row(ym, z), rp0 = row(yp, z);
            const int64_t r0m = row(y, zm), r0p = row(y, zp);
            const int64_t rmm = row(ym, zm), rpp = row(yp, zp), rmp = row(ym, zp), rpm = row(yp, zm);
            float g[19][NV];
            const T* s = src;
            load_pack<T, NV>(s + r00 + p.x0, p.act, g[0]);
            load_from_left<T, NV>(s + 1 * n + r00, p.x0, p.xprev, p.act, p.left_edge, g[1]);
            load_from_right<T, NV>(s + 2 * n + r00, p.x0, p.xnext, p.act, p.right_edge, g[2]);
            load_pack<T, NV>(s + 3 * n + rm0 + p.x0, p.act, g[3]);
            load_pack<T, NV>(s + 4 * n + rp0 + p.x0, p.act, g[4]);
            load_pack<T, NV>(s + 5 * n + r0m + p.x0, p.act, g[5]);
            load_pack<T, NV>(s + 6 * n + r0p + p.x0, p.act, g[6]);
            load_from_left<T, NV>(s + 7 * n + rm0, p.x0, p.xprev, p.act, p.left_edge, g[7]);
            load_from_right<T, NV>(s + 8 * n + rp0, p.x0, p.xnext, p.act, p.right_edge, g[8]);
            load_from_left<T, NV>(s + 9 * n + rp0, p.x0, p.xprev, p.act, p.left_edge, g[9]);
            load_from_right<T, NV>(s + 10 * n + rm0, p.x0, p.xnext, p.act, p.right_edge, g[10]);
            load_from_left<T, NV>(s + 11 * n + r0m, p.x0, p.xprev, p.act, p.left_edge, g[11]);
            load_from_right<T, NV>(s + 12 * n + r0p, p.x0, p.xnext, p.act, p.right_edge, g[12]);
            load_from_left<T, NV>(s + 13 * n + r0p, p.x0, p.xprev, p.act, p.left_edge, g[13]);
            load_from_right<T, NV>(s + 14 * n + r0m, p.x0, p.xnext, p.act, p.right_edge, g[14]);
            load_pack<T, NV>(s + 15 * n + rmm + p.x0, p.act, g[15]);
            load_pack<T, NV>(s + 16 * n + rpp + p.x0, p.act, g[16]);
            load_pack<T, NV>(s + 17 * n + rmp + p.x0, p.act, g[17]);
            load_pack<T, NV>(s + 18 * n + rpm + p.x0, p.act, g[18]);
            if (p.act) {
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    float h[19];
#pragma unroll
                    for (int j = 0; j < 19; ++j) h[j] = g[j][k];
                    float ux = 0.0f, uy = 0.0f, uz = 0.0f;
                    if constexpr (UM != UM_ZERO && UM != UM_FLUID)
                        relative_velocity3<UM>(h, r00 + p.x0 + k, n, a, ux, uy, uz);
                    relax_node3<UM>(h, ux, uy, uz, a.s, a.ref);
#pragma unroll
                    for (int j = 0; j < 19; ++j) g[j][k] = h[j];
                }
#pragma unroll
                for (int j = 0; j < 19; ++j) store_pack<T, NV>(dst + j * n + r00 + p.x0, g[j]);
            }
        }
    }
}

__constant__ int kC3X[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__constant__ int kC3Y[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__constant__ int kC3Z[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

// g_j = f_eq,j(rho, u) - f_eq,j(rho_ref, U), difference form as in the D2Q9 kernel.
template <typename T>
__global__ void k_init_eq3(T* __restrict__ dst, const float* __restrict__ rho,
                           const float* __restrict__ u, int64_t n, StoreRef3 ref,
                           float inv_lambda) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float r = rho ? rho[i] : 1.0f;
        const float ux = u[i] * inv_lambda, uy = u[n + i] * inv_lambda, uz = u[2 * n + i] * inv_lambda;
        const float uu = ux * ux + uy * uy + uz * uz;
        const float UU = ref.ux * ref.ux + ref.uy * ref.uy + ref.uz * ref.uz;
#pragma unroll
        for (int j = 0; j < 19; ++j) {
            const float cx = (float)kC3X[j], cy = (float)kC3Y[j], cz = (float)kC3Z[j];
            const float cu = cx * ux + cy * uy + cz * uz;
            const float cU = cx * ref.ux + cy * ref.uy + cz * ref.uz;
            const float w = wgt3(j);
            const float pu = 3.0f * cu + 4.5f * cu * cu - 1.5f * uu;
            const float pU = 3.0f * cU + 4.5f * cU * cU - 1.5f * UU;
            dst[j * n + i] = from_f<T>(w * (r - ref.rho) + w * (r * pu - ref.rho * pU));
        }
    }
}

template <typename T>
__global__ void k_moments3(const T* __restrict__ src, float* __restrict__ rho,
                           float* __restrict__ u, int64_t n, StoreRef3 ref, float lambda) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float g[19];
#pragma unroll
        for (int j = 0; j < 19; ++j) g[j] = to_f(src[j * n + i]);
        const NodeMoments3 m = node_moments3(g);
        const float r = ref.rho + m.drho;
        if (rho) rho[i] = r;
        if (u) {
            u[i] = lambda * (ref.jx + m.jx) / r;
            u[n + i] = lambda * (ref.jy + m.jy) / r;
            u[2 * n + i] = lambda * (ref.jz + m.jz) / r;
        }
    }
}

// FP64 sums of (sum g, sum c g (3), non-finite nodes), 8 doubles per block (5 used).
template <typename T>
__global__ void __launch_bounds__(kReduceThreads) k_conserved3_partial(const T* __restrict__ src,
                                                                       int64_t n,
                                                                       double* __restrict__ part) {
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    float r[4] = {0.f, 0.f, 0.f, 0.f};
    int run = 0, bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float g[19];
#pragma unroll
        for (int j = 0; j < 19; ++j) g[j] = to_f(src[j * n + i]);
        const NodeMoments3 m = node_moments3(g);
        r[0] += m.drho;
        r[1] += m.jx;
        r[2] += m.jy;
        r[3] += m.jz;
        bad += (isfinite(m.drho) && isfinite(m.jx) && isfinite(m.jy) && isfinite(m.jz)) ? 0 : 1;
        if (++run == 32) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                v[c] += (double)r[c];
                r[c] = 0.f;
            }
            run = 0;
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] += (double)r[c];
    v[4] = (double)bad;
    __shared__ double sh[kReduceThreads / 32][5];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        double t = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFullMask, t, o);
        if (l == 0) sh[w][c] = t;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0.0;
        for (int k = 0; k < kReduceThreads / 32; ++k) t += sh[k][threadIdx.x];
        part[8 * (int64_t)blockIdx.x + threadIdx.x] = t;
    }
}

__global__ void k_conserved3_final(const double* __restrict__ part, int nblk, double rho_ref_n,
                                   double jx_n, double jy_n, double jz_n, double lambda,
                                   double* __restrict__ out) {
    __shared__ double sh[256];
    double res[5];
    for (int c = 0; c < 5; ++c) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[8 * b + c];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int st = 128; st > 0; st >>= 1) {
            if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
            __syncthreads();
        }
        res[c] = sh[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = res[0] + rho_ref_n;
        out[1] = lambda * (res[1] + jx_n);
        out[2] = lambda * (res[2] + jy_n);
        out[3] = lambda * (res[3] + jz_n);
        out[4] = res[4];
    }
}

int grid1d3(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = 152LL * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T, int UM>
cudaError_t step3_nv(const void* src, void* dst, const StepArgs3& a, cudaStream_t st, int nv) {
    const dim3 grid = dim3(1, a.ny < 65535 ? a.ny : 65535, a.nz < 65535 ? a.nz : 65535);
    const T* s = static_cast<const T*>(src);
    T* d = static_cast<T*>(dst);
    if (nv == 1) {
        dim3 g = grid;
        g.x = (a.nx + kThreads3 - 1) / kThreads3;
        k_step3<T, 1, UM><<<g, kThreads3, 0, st>>>(s, d, a);
    } else if (nv == 2) {
        dim3 g = grid;
        g.x = (a.nx / 2 + kThreads3 - 1) / kThreads3;
        k_step3<T, 2, UM><<<g, kThreads3, 0, st>>>(s, d, a);
    } else if (nv == 4) {
        dim3 g = grid;
        g.x = (a.nx / 4 + kThreads3 - 1) / kThreads3;
        k_step3<T, 4, UM><<<g, kThreads3, 0, st>>>(s, d, a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t step3_um(const void* src, void* dst, const StepArgs3& a, cudaStream_t st, int um,
                     int nv) {
    switch (um) {
        case UM_ZERO: return step3_nv<T, UM_ZERO>(src, dst, a, st, nv);
        case UM_FLUID: return step3_nv<T, UM_FLUID>(src, dst, a, st, nv);
        case UM_FIELD: return step3_nv<T, UM_FIELD>(src, dst, a, st, nv);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int step3_vector_width(int storage, int nx) {
    // Measured fastest on GB300 at 256^3: 4-node packs for FP32, 2-node packs for 16-bit.
    const int widest = storage == kStoreF32 ? 4 : 2;
    for (int nv = widest; nv > 1; nv >>= 1)
        if (nx % nv == 0) return nv;
    return 1;
}

cudaError_t launch_step3(int storage, int um, int nv, const void* src, void* dst,
                         const StepArgs3& a, cudaStream_t st) {
    switch (storage) {
        case kStoreF32: return step3_um<float>(src, dst, a, st, um, nv);
        case kStoreF16: return step3_um<__half>(src, dst, a, st, um, nv);
        case kStoreBF16: return step3_um<__nv_bfloat16>(src, dst, a, st, um, nv);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_init_eq3(int storage, void* dst, const float* rho, const float* u, int64_t n,
                            const StoreRef3& ref, float inv_lambda, cudaStream_t st) {
    const int g = grid1d3(n);
    switch (storage) {
        case kStoreF32:
            k_init_eq3<float><<<g, 256, 0, st>>>(static_cast<float*>(dst), rho, u, n, ref, inv_lambda);
            break;
        case kStoreF16:
            k_init_eq3<__half><<<g, 256, 0, st>>>(static_cast<__half*>(dst), rho, u, n, ref, inv_lambda);
            break;
        case kStoreBF16:
            k_init_eq3<__nv_bfloat16><<<g, 256, 0, st>>>(static_cast<__nv_bfloat16*>(dst), rho, u, n,
                                                        ref, inv_lambda);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_moments3(int storage, const void* src, float* rho, float* u, int64_t n,
                            const StoreRef3& ref, float lambda, cudaStream_t st) {
    const int g = grid1d3(n);
    switch (storage) {
        case kStoreF32:
            k_moments3<float><<<g, 256, 0, st>>>(static_cast<const float*>(src), rho, u, n, ref, lambda);
            break;
        case kStoreF16:
            k_moments3<__half><<<g, 256, 0, st>>>(static_cast<const __half*>(src), rho, u, n, ref, lambda);
            break;
        case kStoreBF16:
            k_moments3<__nv_bfloat16><<<g, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(src), rho, u,
                                                        n, ref, lambda);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_conserved3(int storage, const void* src, int64_t n, const StoreRef3& ref,
                              double lambda, double* partials, int nblk, double* out,
                              cudaStream_t st) {
    switch (storage) {
        case kStoreF32:
            k_conserved3_partial<float><<<nblk, kReduceThreads, 0, st>>>(static_cast<const float*>(src), n,
                                                                         partials);
            break;
        case kStoreF16:
            k_conserved3_partial<__half><<<nblk, kReduceThreads, 0, st>>>(static_cast<const __half*>(src), n,
                                                                          partials);
            break;
        case kStoreBF16:
            k_conserved3_partial<__nv_bfloat16><<<nblk, kReduceThreads, 0, st>>>(
                static_cast<const __nv_bfloat16*>(src), n, partials);
            break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double dn = (double)n;
    k_conserved3_final<<<1, 256, 0, st>>>(partials, nblk, (double)ref.rho * dn,
                                          (double)ref.jx * dn, (double)ref.jy * dn,
                                          (double)ref.jz * dn, lambda, out);
    return cudaGetLastError();
}

}  // namespace lbmrv
