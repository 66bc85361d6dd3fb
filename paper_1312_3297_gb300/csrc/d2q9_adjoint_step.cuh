// The reverse step kernel of the D2Q9 adjoint, templated on the storage type T of the
// forward states it reads (FP32, FP16 or BF16; the adjoint vectors are FP32). Included by
// d2q9_adjoint.cu (FP32) and d2q9_adjoint16.cu (16-bit), which instantiate it.
//
// Forward, as stored by the library: S_k = C_k(P S_{k-1}), P the pull transport of
// relation (transport), C_k the relaxation at time k (relax_node). For a loss L(S_N):
//   mu_k = J_{C_k}(P S_{k-1})^T a_k,   a_N = dL/dS_N,   a_k = P^T mu_{k+1} (k < N),
//   dL/dS_0 = P^T mu_1,
// where P^T (a push) is read here as a gather: (P^T mu)_j(x) = mu_j(x + c_j). One launch
// of k_adjoint_step_bal computes mu_k from S_{k-1} (pulled) and mu_{k+1} (gathered) or
// dL/dS_N (aligned), adds the node contributions to dL/ds (six non-conserved rates) and to
// dL/dA (amplitude of a prescribed u~) into per-block FP64 accumulators, and optionally
// adds alpha_k * dL/du~ to a per-node field gradient. With 16-bit storage the forward
// states are the rounded ones the 16-bit step produced; J_C is the derivative of the FP32
// relaxation at them (the rounding to the storage type is taken as the identity).
#pragma once

#include <cuda_runtime.h>

#include "d2q9.cuh"
#include "d2q9_adjoint.cuh"
#include "launch.h"
#include "pdl.cuh"
#include "pull.cuh"

namespace lbmrv {
namespace {

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

// Add the block's sums of v[0..6] to acc[block * 8 + c] in FP64 (the block owns its slot).
template <int NT>
__device__ __forceinline__ void block_accumulate7(float v[7], double* __restrict__ acc) {
    __shared__ float sh[NT / 32][7];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        const float t = warp_sum_f(v[c]);
        if (l == 0) sh[w][c] = t;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) s += (double)sh[k][threadIdx.x];
        const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
        acc[blk * 8 + threadIdx.x] += s;
    }
}

constexpr int kAdjThreads = 128;

// Form of 1/rho in the reverse relaxation's forward recomputation (measured: the
// approximation 1.5 % faster than the correctly rounded form at 1024^2, equal at 4096^2;
// the gradients' 1e-4 agreement is unaffected).
constexpr int kAdjointRcp = RCP_APPROX;

// Prescribed mode: dL/dA and the optional field gradient of one node from a^T dg*/du.
template <int UM>
__device__ __forceinline__ void prescribed_grads(float ubx, float uby, float bx, float by,
                                                 int64_t i, const AdjointArgs& aa,
                                                 float acc[7]) {
    if constexpr (UM == UM_ANALYTIC || UM == UM_FIELD) {
        acc[6] += aa.da_factor * (ubx * bx + uby * by);
        if (aa.dut0) {
            const int64_t n = (int64_t)aa.step.nx * aa.step.ny;
            aa.dut0[i] += aa.step.amp_t * ubx;
            aa.dut0[n + i] += aa.step.amp_t * uby;
        }
    }
}

// The reverse relaxation of one pack from its pulled state g and adjoint input adj; stores
// mu_k.
template <int NV, int UM>
__device__ __forceinline__ void adjoint_pack_relax(float g[9][NV], const float adj[9][NV],
                                                   float* __restrict__ mu_out,
                                                   const AdjointArgs& aa, int y,
                                                   const PackLane& p, float acc[7]) {
    const StepArgs& a = aa.step;
    const int64_t n = (int64_t)a.nx * a.ny;
    const int64_t r0 = (int64_t)y * a.nx;
    const float cy = UM == UM_ANALYTIC ? cospif(a.two_over_ny * (float)(y + a.y_off)) : 0.0f;
    constexpr bool kPrescribed = UM == UM_ANALYTIC || UM == UM_FIELD;
    if constexpr (NV >= 2) {
        F2 sb[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) sb[c] = F2(0.0f);
#pragma unroll
        for (int k = 0; k < NV; k += 2) {
            const int x = p.x0 + k;
            const int64_t i = r0 + x;
            F2 h[9], ah[9], o[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                h[j] = pack2(g[j][k], g[j][k + 1]);
                ah[j] = pack2(adj[j][k], adj[j][k + 1]);
            }
            float bx0 = 0.f, bx1 = 0.f, by0 = 0.f, by1 = 0.f;
            F2 ux(0.0f), uy(0.0f);
            if constexpr (UM == UM_ANALYTIC) {
                bx0 = bx1 = cy;
                by0 = __ldg(a.sin_x + x);
                by1 = __ldg(a.sin_x + x + 1);
            } else if constexpr (UM == UM_FIELD) {
                bx0 = __ldg(a.ut0 + i);
                bx1 = __ldg(a.ut0 + i + 1);
                by0 = __ldg(a.ut0 + n + i);
                by1 = __ldg(a.ut0 + n + i + 1);
            }
            if constexpr (kPrescribed) {
                ux = F2(a.amp_t) * pack2(bx0, bx1);
                uy = F2(a.amp_t) * pack2(by0, by1);
            }
            F2 ubx, uby;
            relax_node_vjp<UM, kAdjointRcp>(h, ah, ux, uy, a.s, a.ref, o, sb, ubx, uby);
#pragma unroll
            for (int j = 0; j < 9; ++j) unpack2(o[j], g[j][k], g[j][k + 1]);
            if constexpr (kPrescribed) {
                float u0, u1, v0, v1;
                unpack2(ubx, u0, u1);
                unpack2(uby, v0, v1);
                prescribed_grads<UM>(u0, v0, bx0, by0, i, aa, acc);
                prescribed_grads<UM>(u1, v1, bx1, by1, i + 1, aa, acc);
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float s0, s1;
            unpack2(sb[c], s0, s1);
            acc[c] += s0 + s1;
        }
    } else {
        const int x = p.x0;
        const int64_t i = r0 + x;
        F1 h[9], ah[9], o[9], sb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            h[j] = g[j][0];
            ah[j] = adj[j][0];
        }
        float bx = 0.f, by = 0.f, ux = 0.f, uy = 0.f;
        if constexpr (UM == UM_ANALYTIC) {
            bx = cy;
            by = __ldg(a.sin_x + x);
        } else if constexpr (UM == UM_FIELD) {
            bx = __ldg(a.ut0 + i);
            by = __ldg(a.ut0 + n + i);
        }
        if constexpr (kPrescribed) {
            ux = a.amp_t * bx;
            uy = a.amp_t * by;
        }
        F1 ubx, uby;
        relax_node_vjp<UM, kAdjointRcp>(h, ah, F1(ux), F1(uy), a.s, a.ref, o, sb, ubx, uby);
#pragma unroll
        for (int j = 0; j < 9; ++j) g[j][0] = o[j].v;
        prescribed_grads<UM>(ubx.v, uby.v, bx, by, i, aa, acc);
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += sb[c].v;
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) store_pack<float, NV>(mu_out + j * n + r0 + p.x0, g[j]);
}

// The adjoint input of a pack: mu_{k+1} gathered (the transpose of the pull), or dL/dS_N
// read in place.
template <int NV, bool GATHER>
__device__ __forceinline__ void load_adjoint(const float* __restrict__ a_in, int64_t n,
                                             int64_t r0, int64_t rm, int64_t rp,
                                             const PackLane& p, float adj[9][NV]) {
    if constexpr (GATHER) {
        gather_pack<float, NV>(a_in, n, r0, rm, rp, p, adj);
    } else {
#pragma unroll
        for (int j = 0; j < 9; ++j) load_pack<float, NV>(a_in + j * n + r0 + p.x0, p.act, adj[j]);
    }
}

// The reverse step on one pack of row y (lane geometry p): pull S_{k-1} (stored as T: FP32,
// or 16-bit values widened to FP32), gather mu_{k+1} (or read dL/dS_N aligned), reverse each
// node's relaxation, store mu_k. Packs of two or more nodes reverse node pairs with packed
// FP32 instructions (two nodes per instruction), so 2- and 4-node packs give the same bits;
// one-node packs use the scalar form (F1) of the same arithmetic, which agrees with them to
// rounding.
template <typename T, int NV, int UM, bool GATHER>
__device__ __forceinline__ void adjoint_pack(const T* __restrict__ s_prev,
                                             const float* __restrict__ a_in,
                                             float* __restrict__ mu_out, const AdjointArgs& aa,
                                             int y, const PackLane& p, float acc[7]) {
    const StepArgs& a = aa.step;
    const int nx = a.nx, ny = a.ny;
    const int64_t n = (int64_t)nx * ny;
    const int ym = y == 0 ? ny - 1 : y - 1;
    const int yp = y == ny - 1 ? 0 : y + 1;
    const int64_t r0 = (int64_t)y * nx, rm = (int64_t)ym * nx, rp = (int64_t)yp * nx;
    float g[9][NV], adj[9][NV];
    pull_pack<T, NV>(s_prev, n, r0, rm, rp, p, g);
    load_adjoint<NV, GATHER>(a_in, n, r0, rm, rp, p, adj);
    if (!p.act) return;
    adjoint_pack_relax<NV, UM>(g, adj, mu_out, aa, y, p, acc);
}

// One reverse step, persistent, with the work balanced across the resident warps. A warp
// item is 32 consecutive packs of one row (`chunks` items per row); warp w of W takes items
// [w I / W, (w + 1) I / W) of the I = chunks * (y1 - y0) of rows [y0, y1) (all rows, or a
// slab's own rows) in row order, so every warp holds the same
// number of items to within one and the grid (every block resident at once) ends nearly
// together. A grid of whole rows per block leaves its last wave part-empty when the rows
// do not fill a whole number of waves (1024^2: 3.4 waves).
template <typename T, int NV, int UM, bool GATHER>
__global__ void __launch_bounds__(kAdjThreads, NV >= 4 ? 3 : 4)
    k_adjoint_step_bal(const T* __restrict__ s_prev, const float* __restrict__ a_in,
                       float* __restrict__ mu_out, AdjointArgs aa, int chunks) {
    pdl_wait_prior();
    pdl_allow_next();
    const int nx = aa.step.nx;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kAdjThreads / 32);
    const int64_t w = (int64_t)blockIdx.x * (kAdjThreads / 32) + (threadIdx.x >> 5);
    const int64_t items = (int64_t)chunks * (aa.y1 - aa.y0);
    const int64_t i0 = w * items / warps, i1 = (w + 1) * items / warps;
    int y = (int)(i0 / chunks), c = (int)(i0 - (int64_t)y * chunks);
    y += aa.y0;
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t it = i0; it < i1; ++it) {  // warp-uniform bounds: shuffles stay full-mask
        PackLane p;
        p.x0 = (c * 32 + lane) * NV;
        p.act = p.x0 < nx;
        p.left_edge = lane == 0;
        p.right_edge = lane == 31 || p.x0 + NV >= nx;
        p.xprev = p.x0 == 0 ? nx - 1 : p.x0 - 1;
        p.xnext = p.x0 + NV >= nx ? 0 : p.x0 + NV;
        adjoint_pack<T, NV, UM, GATHER>(s_prev, a_in, mu_out, aa, y, p, acc);
        if (++c == chunks) {
            c = 0;
            ++y;
        }
    }
    block_accumulate7<kAdjThreads>(acc, aa.acc);
}

// Blocks of the balanced kernel: as many as are resident at once on the device (found once
// per kernel instance and device), at most one per 4 items.
template <typename K>
int64_t balanced_blocks(K kernel, int64_t items) {
    constexpr int kMaxDevices = 64;
    static int per_sm[kMaxDevices] = {0};
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    if (per_sm[dev] == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kAdjThreads, 0) !=
                cudaSuccess || b < 1)
            return -1;
        per_sm[dev] = b;
    }
    const int64_t need = (items + kAdjThreads / 32 - 1) / (kAdjThreads / 32);
    const int64_t res = (int64_t)per_sm[dev] * sms;
    return need < res ? need : res;
}

template <typename T, int NV, int UM, bool GATHER>
cudaError_t adjoint_launch(const T* s_prev, const float* a_in, float* mu_out,
                           const AdjointArgs& aa, cudaStream_t st) {
    const int chunks = (aa.step.nx + 32 * NV - 1) / (32 * NV);
    const int64_t items = (int64_t)chunks * (aa.y1 - aa.y0);
    if (items <= 0) return cudaErrorInvalidValue;
    // the accumulators hold one slot per block of adjoint_grid, never fewer than nb
    const int64_t nb = balanced_blocks(k_adjoint_step_bal<T, NV, UM, GATHER>, items);
    if (nb < 1) return cudaErrorInvalidConfiguration;
    return launch_pdl(k_adjoint_step_bal<T, NV, UM, GATHER>, dim3((unsigned)nb), dim3(kAdjThreads),
                      st, s_prev, a_in, mu_out, aa, chunks);
}

template <typename T, int NV, int UM>
cudaError_t adjoint_nv_um(const T* s_prev, const float* a_in, bool gather, float* mu_out,
                          const AdjointArgs& aa, cudaStream_t st) {
    const cudaError_t e = gather ? adjoint_launch<T, NV, UM, true>(s_prev, a_in, mu_out, aa, st)
                                 : adjoint_launch<T, NV, UM, false>(s_prev, a_in, mu_out, aa, st);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T, int NV>
cudaError_t adjoint_nv(int um, const T* s_prev, const float* a_in, bool gather,
                       float* mu_out, const AdjointArgs& aa, cudaStream_t st) {
    switch (um) {
        case UM_ZERO: return adjoint_nv_um<T, NV, UM_ZERO>(s_prev, a_in, gather, mu_out, aa, st);
        case UM_FLUID: return adjoint_nv_um<T, NV, UM_FLUID>(s_prev, a_in, gather, mu_out, aa, st);
        case UM_ANALYTIC:
            return adjoint_nv_um<T, NV, UM_ANALYTIC>(s_prev, a_in, gather, mu_out, aa, st);
        case UM_FIELD: return adjoint_nv_um<T, NV, UM_FIELD>(s_prev, a_in, gather, mu_out, aa, st);
        default: return cudaErrorInvalidValue;
    }
}


// One reverse step with forward states of type T; nv nodes per thread (1, 2 or 4).
template <typename T>
cudaError_t launch_adjoint_step_t(int um, int nv, const void* s_prev, const float* a_in,
                                  bool gather, float* mu_out, const AdjointArgs& aa,
                                  cudaStream_t st) {
    const T* s = static_cast<const T*>(s_prev);
    switch (nv) {
        case 4: return adjoint_nv<T, 4>(um, s, a_in, gather, mu_out, aa, st);
        case 2: return adjoint_nv<T, 2>(um, s, a_in, gather, mu_out, aa, st);
        case 1: return adjoint_nv<T, 1>(um, s, a_in, gather, mu_out, aa, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace lbmrv
