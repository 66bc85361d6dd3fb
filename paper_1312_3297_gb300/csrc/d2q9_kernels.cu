// D2Q9 kernels: fused pull-transport + relative-velocity relaxation, equilibrium
// initialisation, moments and FP64 conserved-quantity reductions.
#include <cuda_runtime.h>

#include <atomic>

#include "d2q9.cuh"
#include "launch.h"
#include "occupancy.cuh"
#include "pdl.cuh"
#include "pull.cuh"

namespace lbmrv {

namespace {

// --------------------------------------------------------------------------------------
// Fused step, one node per thread. Works for every lattice size (ragged rows, nx or
// ny equal to 1 or 2). Relation (transport) in pull form: node (x, y) reads population
// j from (x - cx_j, y - cy_j), periodic.
// BASIS 0: the orthogonal moments of relation (mom); 1: Geier's basis (relax_node_geier).
// For BASIS 0 the relaxation takes u~ = q / rho itself (UM_FLUID) and ignores u~ for
// UM_ZERO, so only the prescribed modes evaluate relative_velocity first.
template <int BASIS, int UM, int RCP>
__device__ __forceinline__ void relax_basis(float g[9], float ux, float uy, const Rates& s,
                                            const StoreRef& ref) {
    if constexpr (BASIS == 0)
        relax_node<UM, RCP>(g, ux, uy, s, ref);
    else
        relax_node_geier(g, ux, uy, s, ref);
}

// Two nodes per call (R = F2) for the paired packs of 16-bit storage (step_vec_pairs).
template <int BASIS, int UM, int RCP>
__device__ __forceinline__ void relax_basis2(F2 g[9], F2 ux, F2 uy, const Rates& s,
                                             const StoreRef& ref) {
    if constexpr (BASIS == 0)
        relax_node<UM, RCP>(g, ux, uy, s, ref);
    else
        relax_node_geier_r<UM, RCP>(g, ux, uy, s, ref);
}

template <int BASIS, int UM>
constexpr bool needs_utilde() {
    return BASIS != 0 || UM == UM_ANALYTIC || UM == UM_FIELD;
}

// Form of 1/rho per kernel variant, measured fastest on GB300 (see recip): the
// approximation for FP32 storage, the correctly rounded one for 16-bit storage with one
// node per relaxation call; for paired packs the fast division, except without a shift
// (u~ = 0).
template <typename T>
constexpr int scalar_rcp() {
    return sizeof(T) == 4 ? RCP_APPROX : RCP_RN;
}
template <int UM>
constexpr int paired_rcp() {
    return UM == UM_ZERO ? RCP_RN : RCP_DIV;
}

// --------------------------------------------------------------------------------------
// FP64 sums of the deviations (sum g, sum c g, non-finite nodes): per-node
// FP32 moments accumulated in FP64 per thread, warp-shuffle and shared-memory tree per
// block, one partial per block; a second one-block kernel adds the partials in a fixed
// order, so the result is deterministic.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFullMask, v, o);
    return v;
}

template <int NT>
__device__ __forceinline__ void block_sum4(double v[4], double* out) {
    __shared__ double sh[NT / 32][4];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        v[c] = warp_sum(v[c]);
        if (l == 0) sh[w][c] = v[c];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double t = l < NT / 32 ? sh[l][c] : 0.0;
            t = warp_sum(t);
            if (l == 0) out[c] = t;
        }
    }
}

template <typename T, int UM, int BASIS>
__global__ void __launch_bounds__(256) k_step_scalar(const T* __restrict__ src,
                                                     T* __restrict__ dst, StepArgs a) {
    pdl_wait_prior();
    pdl_allow_next();
    const int nx = a.nx, ny = a.ny;
    const int64_t n = (int64_t)nx * ny;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;
    for (int y = blockIdx.y; y < ny; y += gridDim.y) {
        const int ym = y == 0 ? ny - 1 : y - 1;
        const int yp = y == ny - 1 ? 0 : y + 1;
        const int64_t r0 = (int64_t)y * nx, rm = (int64_t)ym * nx, rp = (int64_t)yp * nx;
        float g[9];
        g[0] = to_f(src[r0 + x]);
        g[1] = to_f(src[n + r0 + xm]);
        g[2] = to_f(src[2 * n + rm + x]);
        g[3] = to_f(src[3 * n + r0 + xp]);
        g[4] = to_f(src[4 * n + rp + x]);
        g[5] = to_f(src[5 * n + rm + xm]);
        g[6] = to_f(src[6 * n + rm + xp]);
        g[7] = to_f(src[7 * n + rp + xp]);
        g[8] = to_f(src[8 * n + rp + xm]);
        float ux = 0.0f, uy = 0.0f;
        if constexpr (needs_utilde<BASIS, UM>())
            relative_velocity<UM>(g, a.ref, x, y, r0 + x, a, ux, uy);
        relax_basis<BASIS, UM, scalar_rcp<T>()>(g, ux, uy, a.s, a.ref);
#pragma unroll
        for (int j = 0; j < 9; ++j) dst[j * n + r0 + x] = from_f<T>(g[j]);
    }
}

// --------------------------------------------------------------------------------------
// Fused step, NV consecutive nodes of a row per thread with aligned vector loads and
// stores (requires nx % NV == 0 and 16-byte aligned planes); row loads in pull.cuh.
//
// SUMS: also add up the conserved moments of the stored result (the values as rounded to
// the storage type) in the block's slot part[4 * block] (sum g, sum c_x g, sum c_y g,
// non-finite nodes), as k_conserved_partial does for a stored state; k_conserved_final then
// adds the slots in a fixed order. The launcher then sizes the grid to the blocks resident
// at once, so each block walks many rows and its FP64 reduction runs once.
// The paired cascaded relaxation (Geier's basis, 8-node packs) is held to five blocks per
// SM (96 registers, a few spilled), four with a stored u~ field: with the registers left to
// the compiler it takes 126, runs four blocks and, for u~ = q / rho, reaches 0.88 of copy
// bandwidth instead of 0.98 (measured at 8192^2; the stored field runs faster with four).
// A minimum of 0 blocks leaves every other instance's register budget as without one (same
// allocation); a minimum of 1 lets the orthogonal-basis 8-node packs grow to 194 registers.
// With 16-bit 4-node packs Geier's basis also relaxes node pairs, at eight blocks per SM,
// except with a stored reference field (FP16 / BF16 at 4100^2, of copy bandwidth, paired
// against node by node: u~ = 0 0.95 / 0.95 against 0.86 / 0.81, u~ = q/rho 0.87 / 0.88
// against 0.81 / 0.77, the analytic field 0.83 / 0.83 against 0.74 / 0.73, a stored field
// 0.59 / 0.59 against 0.64 / 0.64). The orthogonal basis is faster node by node there
// (0.86 against 0.70 with u~ = q/rho).
// The instances with fused sums (not the timed step) keep the compiler's choice, and with
// 4-node packs relax node by node.
template <typename T, int BASIS, int NV, int UM, bool SUMS>
constexpr bool step_vec_pairs4 =
    !SUMS && BASIS == 1 && NV == 4 && sizeof(T) == 2 && UM != UM_FIELD;
template <typename T, int BASIS, int NV, int UM, bool SUMS>
constexpr bool step_vec_pairs = NV >= 8 || step_vec_pairs4<T, BASIS, NV, UM, SUMS>;
template <typename T, int BASIS, int NV, int UM, bool SUMS>
constexpr int step_vec_min_blocks =
    SUMS ? 0
    : (BASIS == 1 && NV >= 8) ? (UM == UM_FIELD ? 4 : 5)
    : step_vec_pairs4<T, BASIS, NV, UM, SUMS> ? 8
                                              : 0;

template <typename T, int NV, int UM, int BASIS, bool SUMS = false>
__global__ void __launch_bounds__(128, (step_vec_min_blocks<T, BASIS, NV, UM, SUMS>))
    k_step_vec(const T* __restrict__ src, T* __restrict__ dst, StepArgs a,
               double* __restrict__ part) {
    pdl_wait_prior();
    pdl_allow_next();
    const int nx = a.nx, ny = a.ny;
    const int64_t n = (int64_t)nx * ny;
    const PackLane p = pack_lane<NV>(nx);
    // SUMS: node moments in FP32 runs of kRun packs (32 nodes), each run added in FP64 (FP64
    // adds are scarce on this GPU; a run of 32 loses < 1e-6 relative)
    constexpr int kRun = NV >= 32 ? 1 : 32 / NV;
    double sums[3] = {0.0, 0.0, 0.0};
    float run_r[3] = {0.f, 0.f, 0.f};
    int bad = 0;
    auto row = [&](int y) {
        const int ym = y == 0 ? ny - 1 : y - 1;
        const int yp = y == ny - 1 ? 0 : y + 1;
        const int64_t r0 = (int64_t)y * nx, rm = (int64_t)ym * nx, rp = (int64_t)yp * nx;
        float g[9][NV];
        pull_pack<T, NV>(src, n, r0, rm, rp, p, g);
        if (p.act) {
            // analytic prescribed field: cos 2 pi y/ny once per row, sin 2 pi x/nx from a
            // per-column table (one vector load per pack, served by L1/L2)
            float ux_row = 0.0f, sx[NV];
            if (UM == UM_ANALYTIC) {
                ux_row = a.amp_t * cospif(a.two_over_ny * (float)(y + a.y_off));
                load_pack<float, NV>(a.sin_x + p.x0, true, sx);
            }
            if constexpr (step_vec_pairs<T, BASIS, NV, UM, SUMS>) {
                // Two nodes per packed FP32 instruction. With 8-node packs (16-bit storage)
                // the step is issue-bound and pairing removes about a third of its
                // instructions. With 4 or fewer nodes per thread the broadcast constants'
                // registers cost more than pairing saves, but for Geier's 16-bit 4-node packs.
#pragma unroll
                for (int k = 0; k < NV; k += 2) {
                    F2 h[9];
#pragma unroll
                    for (int j = 0; j < 9; ++j) h[j] = pack2(g[j][k], g[j][k + 1]);
                    F2 ux(0.0f), uy(0.0f);
                    if constexpr (UM == UM_ANALYTIC) {
                        ux = F2(ux_row);
                        uy = F2(a.amp_t) * pack2(sx[k], sx[k + 1]);
                    } else if constexpr (UM == UM_FIELD) {
                        const int64_t i = r0 + p.x0 + k;
                        ux = F2(a.amp_t) * pack2(__ldg(a.ut0 + i), __ldg(a.ut0 + i + 1));
                        uy = F2(a.amp_t) * pack2(__ldg(a.ut0 + n + i), __ldg(a.ut0 + n + i + 1));
                    }
                    relax_basis2<BASIS, UM, paired_rcp<UM>()>(h, ux, uy, a.s, a.ref);
#pragma unroll
                    for (int j = 0; j < 9; ++j) unpack2(h[j], g[j][k], g[j][k + 1]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    float h[9];
#pragma unroll
                    for (int j = 0; j < 9; ++j) h[j] = g[j][k];
                    float ux = 0.0f, uy = 0.0f;
                    if constexpr (UM == UM_ANALYTIC) {
                        ux = ux_row;
                        uy = a.amp_t * sx[k];
                    } else if constexpr (needs_utilde<BASIS, UM>()) {
                        relative_velocity<UM>(h, a.ref, p.x0 + k, y, r0 + p.x0 + k, a, ux, uy);
                    }
                    relax_basis<BASIS, UM, scalar_rcp<T>()>(h, ux, uy, a.s, a.ref);
#pragma unroll
                    for (int j = 0; j < 9; ++j) g[j][k] = h[j];
                }
            }
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                if constexpr (SUMS) {  // keep the stored (rounded) values for the sums
                    Pack<T, NV> pk;
                    PackCvt<T, NV>::out(g[j], pk);
                    *reinterpret_cast<Pack<T, NV>*>(dst + j * n + r0 + p.x0) = pk;
                    PackCvt<T, NV>::in(pk, g[j]);
                } else {
                    store_pack<T, NV>(dst + j * n + r0 + p.x0, g[j]);
                }
            }
            if constexpr (SUMS) {
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    float h[9];
#pragma unroll
                    for (int j = 0; j < 9; ++j) h[j] = g[j][k];
                    const NodeMoments m = node_moments(h);
                    run_r[0] += m.drho;
                    run_r[1] += m.jx;
                    run_r[2] += m.jy;
                    bad += (finite_f(m.drho) && finite_f(m.jx) && finite_f(m.jy)) ? 0 : 1;
                }
            }
        }
    };
    if constexpr (!SUMS) {
        for (int y = blockIdx.y; y < ny; y += gridDim.y) row(y);
    } else {
        // rows in chunks of kRun (one pack per thread and row); a chunk's FP32 run is added
        // in FP64 after it, outside the rows' loop (FP64 issues at 2 operations per clock
        // per SM on this GPU, and predicated adds inside the loop would hold that pipe)
        for (int y0 = blockIdx.y; y0 < ny; y0 += kRun * gridDim.y) {
            for (int t = 0, y = y0; t < kRun && y < ny; ++t, y += gridDim.y) row(y);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sums[c] += (double)run_r[c];
                run_r[c] = 0.f;
            }
        }
    }
    if constexpr (SUMS) {
        double v[4];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = sums[c] + (double)run_r[c];
        v[3] = (double)bad;
        block_sum4<128>(v, part + 4 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x));
    }
}

// --------------------------------------------------------------------------------------
// Equilibrium initialisation: g_j = f_eq,j(rho, u) - f_eq,j(rho_ref, U), written as
// w_j (rho - rho_ref) + w_j (rho P_j(u) - rho_ref P_j(U)), P_j(v) = 3 c.v + 9/2 (c.v)^2
// - 3/2 |v|^2, velocities in units of lambda.
__constant__ int kCX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kCY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Product-form factor of Geier's equilibrium: phi(0, a) = 2/3 - a^2,
// phi(+-1, a) = (1/3 + a^2 +- a) / 2 (a in units of lambda).
__device__ __forceinline__ float phi1(int c, float a) {
    return c == 0 ? (2.0f / 3.0f - a * a) : 0.5f * ((1.0f / 3.0f + a * a) + (float)c * a);
}

template <typename T>
__global__ void k_init_eq_product(T* __restrict__ dst, const float* __restrict__ rho,
                                  const float* __restrict__ u, int64_t n, StoreRef ref,
                                  float inv_lambda) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float r = rho ? rho[i] : 1.0f;
        const float ux = u ? u[i] * inv_lambda : 0.0f;
        const float uy = u ? u[n + i] * inv_lambda : 0.0f;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const int cx = kCX[j], cy = kCY[j];
            dst[j * n + i] = from_f<T>(r * phi1(cx, ux) * phi1(cy, uy) -
                                       ref.rho * phi1(cx, ref.ux) * phi1(cy, ref.uy));
        }
    }
}

template <typename T>
__global__ void k_init_eq(T* __restrict__ dst, const float* __restrict__ rho,
                          const float* __restrict__ u, int64_t n, StoreRef ref,
                          float inv_lambda) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float r = rho ? rho[i] : 1.0f;
        const float ux = u ? u[i] * inv_lambda : 0.0f;
        const float uy = u ? u[n + i] * inv_lambda : 0.0f;
        const float uu = ux * ux + uy * uy;
        const float UU = ref.ux * ref.ux + ref.uy * ref.uy;
        const float dr = r - ref.rho;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const float cu = (float)kCX[j] * ux + (float)kCY[j] * uy;
            const float cU = (float)kCX[j] * ref.ux + (float)kCY[j] * ref.uy;
            const float w = wgt(j);
            const float pu = 3.0f * cu + 4.5f * cu * cu - 1.5f * uu;
            const float pU = 3.0f * cU + 4.5f * cU * cU - 1.5f * UU;
            dst[j * n + i] = from_f<T>(w * dr + w * (r * pu - ref.rho * pU));
        }
    }
}

// Density and velocity (relation (rhoq)) of the stored state.
template <typename T>
__global__ void k_moments(const T* __restrict__ src, float* __restrict__ rho,
                          float* __restrict__ u, int64_t n, StoreRef ref, float lambda) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float g[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) g[j] = to_f(src[j * n + i]);
        const NodeMoments m = node_moments(g);
        const float r = ref.rho + m.drho;
        if (rho) rho[i] = r;
        if (u) {
            u[i] = lambda * (ref.jx + m.jx) / r;
            u[n + i] = lambda * (ref.jy + m.jy) / r;
        }
    }
}

// Nodes 0 .. n-1 of a state whose planes are `plane` elements apart (plane = n for a whole
// lattice; larger for the interior layers of a slab), NV consecutive nodes per thread and
// pack (one vector load per plane; n and plane multiples of NV, planes NV-aligned). At
// least kReduceMinBlocks blocks fit on an SM, the count conserved_blocks launches.
template <typename T, int NV>
__global__ void __launch_bounds__(kReduceThreads, kReduceMinBlocks)
    k_conserved_partial(const T* __restrict__ src, int64_t n, int64_t plane,
                        double* __restrict__ part) {
    // Node moments are FP32; each thread adds runs of up to 32 of them in FP32 and the
    // runs in FP64 (a run of 32 loses < 1e-6 relative). The FP64 adds sit after the run's
    // loop rather than under a condition inside it: FP64 issues at 2 operations per clock
    // per SM on this GPU, and a predicated add inside the loop held that pipe every node.
    constexpr int kRunPacks = NV >= 32 ? 1 : 32 / NV;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    int bad = 0;
    const int64_t packs = n / NV;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // pack index
    while (i < packs) {
        float r[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < kRunPacks && i < packs; ++k, i += stride) {
            float g[9][NV];
#pragma unroll
            for (int j = 0; j < 9; ++j)
                PackCvt<T, NV>::in(*reinterpret_cast<const Pack<T, NV>*>(src + j * plane + i * NV),
                                   g[j]);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                float h[9];
#pragma unroll
                for (int j = 0; j < 9; ++j) h[j] = g[j][q];
                const NodeMoments m = node_moments(h);
                r[0] += m.drho;
                r[1] += m.jx;
                r[2] += m.jy;
                bad += (finite_f(m.drho) && finite_f(m.jx) && finite_f(m.jy)) ? 0 : 1;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] += (double)r[c];
    }
    v[3] = (double)bad;
    block_sum4<kReduceThreads>(v, part + 4 * (int64_t)blockIdx.x);
}

__global__ void __launch_bounds__(kReduceThreads) k_conserved_final(const double* __restrict__ part,
                                                                    int nblk, double rho_ref_n,
                                                                    double jx_ref_n,
                                                                    double jy_ref_n,
                                                                    double lambda,
                                                                    double* __restrict__ out) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] += part[4 * b + c];
    }
    __shared__ double res[4];
    block_sum4<kReduceThreads>(v, res);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = res[0] + rho_ref_n;
        out[1] = lambda * (res[1] + jx_ref_n);
        out[2] = lambda * (res[2] + jy_ref_n);
        out[3] = res[3];
    }
}

// FP64 sums of rho, rho u_x, rho u_y and rho u_z (0 when dim = 2) over initial fields:
// the total mass and momentum of the equilibrium state built from them (relation (rhoq)
// summed over the lattice; sum_j v_j f_eq,j = rho u at every node). rho may be NULL
// (rho = 1); u holds dim planes of n values.
__global__ void __launch_bounds__(kReduceThreads) k_mean_flow_partial(
    const float* __restrict__ rho, const float* __restrict__ u, int64_t n, int64_t plane,
    int dim, double* __restrict__ part) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double r = rho ? (double)rho[i] : 1.0;
        v[0] += r;
        v[1] += r * (double)u[i];
        v[2] += r * (double)u[plane + i];
        if (dim == 3) v[3] += r * (double)u[2 * plane + i];
    }
    block_sum4<kReduceThreads>(v, part + 4 * (int64_t)blockIdx.x);
}

// Block b adds partials [256 b, 256 b + 256) of 4 doubles each into out[4 b].
__global__ void __launch_bounds__(kReduceThreads) k_sum_partials(const double* __restrict__ part,
                                                                 int64_t nblk,
                                                                 double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * kReduceThreads + threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < nblk) {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = part[4 * i + c];
    }
    block_sum4<kReduceThreads>(v, out + 4 * (int64_t)blockIdx.x);
}


// With the sums (part != nullptr) the grid has as many blocks as are resident at once
// (rows strided over blocks), and *nblk receives the number of block slots written: with
// one row per block the FP64 block reductions of a 4096^2 step took longer than the step.
template <typename T, int NV, int UM, int BASIS>
cudaError_t launch_vec(const T* s, T* d, const StepArgs& a, cudaStream_t st, double* part,
                       int64_t* nblk) {
    const int gx = ((a.nx / NV) + 127) / 128;
    const int rows = a.ny < 65535 ? a.ny : 65535;
    // successive steps overlap their launch with the previous step's tail (pdl.cuh)
    if (!part)
        return launch_pdl(k_step_vec<T, NV, UM, BASIS, false>, dim3(gx, rows), dim3(128), st, s,
                          d, a, static_cast<double*>(nullptr));
    auto kernel = k_step_vec<T, NV, UM, BASIS, true>;
    static std::atomic<int> resident[kMaxDevicesOcc];
    int full = 0;
    const cudaError_t e = resident_blocks(kernel, resident, 128, 0, 32, &full);
    if (e != cudaSuccess) return e;
    const int per_x = full / gx;
    const int gy = per_x < 1 ? 1 : (per_x < rows ? per_x : rows);
    if (nblk) *nblk = (int64_t)gx * gy;
    return launch_pdl(kernel, dim3(gx, gy), dim3(128), st, s, d, a, part);
}

template <typename T, int UM, int BASIS>
cudaError_t step_dispatch_nv(const void* src, void* dst, const StepArgs& a, cudaStream_t st,
                             int nv, double* part, int64_t* nblk) {
    const T* s = static_cast<const T*>(src);
    T* d = static_cast<T*>(dst);
    const int gy = a.ny < 65535 ? a.ny : 65535;
    cudaError_t e;
    if (nv == 1) {
        if (part) return cudaErrorInvalidValue;  // sums are fused into the vector kernel only
        e = launch_pdl(k_step_scalar<T, UM, BASIS>, dim3((a.nx + 255) / 256, gy), dim3(256), st,
                       s, d, a);
    } else if (nv == 2) {
        e = launch_vec<T, 2, UM, BASIS>(s, d, a, st, part, nblk);
    } else if (nv == 4) {
        e = launch_vec<T, 4, UM, BASIS>(s, d, a, st, part, nblk);
    } else if (nv == 8) {
        if constexpr (sizeof(T) == 2) {
            e = launch_vec<T, 8, UM, BASIS>(s, d, a, st, part, nblk);
        } else {
            return cudaErrorInvalidValue;
        }
    } else {
        return cudaErrorInvalidValue;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T, int BASIS>
cudaError_t step_dispatch_um(const void* src, void* dst, const StepArgs& a, cudaStream_t st,
                             int um, int nv, double* part, int64_t* nblk) {
    switch (um) {
        case UM_ZERO:
            return step_dispatch_nv<T, UM_ZERO, BASIS>(src, dst, a, st, nv, part, nblk);
        case UM_FLUID:
            return step_dispatch_nv<T, UM_FLUID, BASIS>(src, dst, a, st, nv, part, nblk);
        case UM_ANALYTIC:
            return step_dispatch_nv<T, UM_ANALYTIC, BASIS>(src, dst, a, st, nv, part, nblk);
        case UM_FIELD:
            return step_dispatch_nv<T, UM_FIELD, BASIS>(src, dst, a, st, nv, part, nblk);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t step_dispatch_basis(const void* src, void* dst, const StepArgs& a, cudaStream_t st,
                                int um, int nv, int basis, double* part, int64_t* nblk) {
    return basis == 0 ? step_dispatch_um<T, 0>(src, dst, a, st, um, nv, part, nblk)
                      : step_dispatch_um<T, 1>(src, dst, a, st, um, nv, part, nblk);
}

}  // namespace

int grid_stride_blocks(int64_t n, int threads) {
    constexpr int kMaxDevices = 64;
    static std::atomic<int> sms_of[kMaxDevices];
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        sms = dev < kMaxDevices ? sms_of[dev].load(std::memory_order_relaxed) : 0;
        if (sms == 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ==
                            cudaSuccess && dev < kMaxDevices)
            sms_of[dev].store(sms, std::memory_order_relaxed);
    }
    if (sms <= 0) sms = 152;  // no answer from the runtime: the GB300's count
    const int64_t b = (n + threads - 1) / threads, cap = 16LL * sms;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

int step_vector_width(int storage, int nx) {
    // Widest pack that divides nx, up to the width measured fastest on GB300 (8192^2 sweep):
    // 4 nodes for FP32 (16-byte packs), 8 for FP16 and BF16 (16-byte packs, relaxed in
    // pairs).
    const int widest = storage == kStoreF32 ? 4 : 8;
    for (int nv = widest; nv > 1; nv >>= 1)
        if (nx % nv == 0 && nx >= nv) return nv;
    return 1;
}

namespace {

cudaError_t step_storage(int storage, int um, int nv, const void* src, void* dst,
                         const StepArgs& a, cudaStream_t st, int basis, double* part,
                         int64_t* nblk = nullptr) {
    switch (storage) {
        case kStoreF32:
            return step_dispatch_basis<float>(src, dst, a, st, um, nv, basis, part, nblk);
        case kStoreF16:
            return step_dispatch_basis<__half>(src, dst, a, st, um, nv, basis, part, nblk);
        case kStoreBF16:
            return step_dispatch_basis<__nv_bfloat16>(src, dst, a, st, um, nv, basis, part,
                                                      nblk);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_step(int storage, int um, int nv, const void* src, void* dst,
                        const StepArgs& a, cudaStream_t st, int basis) {
    return step_storage(storage, um, nv, src, dst, a, st, basis, nullptr);
}

int64_t step_sum_blocks(int nx, int ny, int nv) {
    return (int64_t)(((nx / nv) + 127) / 128) * (ny < 65535 ? ny : 65535);
}

int64_t step_sum_scratch(int nx, int ny, int nv) {
    const int64_t nblk = step_sum_blocks(nx, ny, nv);
    return 4 * nblk + 4 * ((nblk + kReduceThreads - 1) / kReduceThreads);
}

cudaError_t launch_step_conserved(int storage, int um, int nv, const void* src, void* dst,
                                  const StepArgs& a, cudaStream_t st, int basis, double rho_ref,
                                  double jx_ref, double jy_ref, double lambda,
                                  double* partials, double* out) {
    if (nv < 2 || !partials || !out) return cudaErrorInvalidValue;
    int64_t nblk = 0;  // block slots the step writes (at most step_sum_blocks)
    cudaError_t e = step_storage(storage, um, nv, src, dst, a, st, basis, partials, &nblk);
    if (e != cudaSuccess) return e;
    // the step's block partials, a fixed 256 per block of a middle level, then one block
    const int64_t mid = (nblk + kReduceThreads - 1) / kReduceThreads;
    double* mids = partials + 4 * nblk;
    k_sum_partials<<<(unsigned)mid, kReduceThreads, 0, st>>>(partials, nblk, mids);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double n = (double)a.nx * (double)a.ny;
    k_conserved_final<<<1, kReduceThreads, 0, st>>>(mids, (int)mid, rho_ref * n, jx_ref * n,
                                                    jy_ref * n, lambda, out);
    return cudaGetLastError();
}

cudaError_t launch_init_eq(int storage, void* dst, const float* rho, const float* u, int64_t n,
                           const StoreRef& rho_ref, float inv_lambda, cudaStream_t st,
                           int basis) {
    const int g = grid_stride_blocks(n, 256);
    if (basis == 1) {
        switch (storage) {
            case kStoreF32:
                k_init_eq_product<float><<<g, 256, 0, st>>>(static_cast<float*>(dst), rho, u, n,
                                                            rho_ref, inv_lambda);
                break;
            case kStoreF16:
                k_init_eq_product<__half><<<g, 256, 0, st>>>(static_cast<__half*>(dst), rho, u, n,
                                                             rho_ref, inv_lambda);
                break;
            case kStoreBF16:
                k_init_eq_product<__nv_bfloat16><<<g, 256, 0, st>>>(
                    static_cast<__nv_bfloat16*>(dst), rho, u, n, rho_ref, inv_lambda);
                break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (storage) {
        case kStoreF32:
            k_init_eq<float><<<g, 256, 0, st>>>(static_cast<float*>(dst), rho, u, n, rho_ref,
                                                inv_lambda);
            break;
        case kStoreF16:
            k_init_eq<__half><<<g, 256, 0, st>>>(static_cast<__half*>(dst), rho, u, n, rho_ref,
                                                 inv_lambda);
            break;
        case kStoreBF16:
            k_init_eq<__nv_bfloat16><<<g, 256, 0, st>>>(static_cast<__nv_bfloat16*>(dst), rho, u,
                                                        n, rho_ref, inv_lambda);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_moments(int storage, const void* src, float* rho, float* u, int64_t n,
                           const StoreRef& rho_ref, float lambda, cudaStream_t st) {
    const int g = grid_stride_blocks(n, 256);
    switch (storage) {
        case kStoreF32:
            k_moments<float><<<g, 256, 0, st>>>(static_cast<const float*>(src), rho, u, n,
                                                rho_ref, lambda);
            break;
        case kStoreF16:
            k_moments<__half><<<g, 256, 0, st>>>(static_cast<const __half*>(src), rho, u, n,
                                                 rho_ref, lambda);
            break;
        case kStoreBF16:
            k_moments<__nv_bfloat16><<<g, 256, 0, st>>>(
                static_cast<const __nv_bfloat16*>(src), rho, u, n, rho_ref, lambda);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int conserved_blocks(int64_t n) {
    // kReduceMinBlocks per SM, which every reduction kernel's launch bounds guarantee: no
    // partial second wave (one ran at a third of the occupancy)
    static std::atomic<int> sms_of[kMaxDevicesOcc];
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        sms = dev < kMaxDevicesOcc ? sms_of[dev].load(std::memory_order_relaxed) : 0;
        if (sms == 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ==
                            cudaSuccess && dev < kMaxDevicesOcc)
            sms_of[dev].store(sms, std::memory_order_relaxed);
    }
    int64_t full = (int64_t)(sms > 0 ? sms : 152) * kReduceMinBlocks;
    if (full > kReduceMaxBlocks) full = kReduceMaxBlocks;
    const int64_t b = (n + kReduceThreads - 1) / kReduceThreads;
    return (int)(b < 1 ? 1 : (b > full ? full : b));
}

cudaError_t launch_mean_flow(const float* rho, const float* u, int64_t n, int64_t plane,
                             int dim, double* partials, int nblk, double* out, cudaStream_t st) {
    k_mean_flow_partial<<<nblk, kReduceThreads, 0, st>>>(rho, u, n, plane, dim, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_conserved_final<<<1, kReduceThreads, 0, st>>>(partials, nblk, 0.0, 0.0, 0.0, 1.0, out);
    return cudaGetLastError();
}

namespace {

// The widest pack (up to 16 bytes) that n, plane and the base address allow.
template <typename T>
int reduce_width(const void* src, int64_t n, int64_t plane, int widest) {
    for (int nv = widest; nv > 1; nv >>= 1)
        if (n % nv == 0 && plane % nv == 0 &&
            reinterpret_cast<uintptr_t>(src) % (nv * sizeof(T)) == 0)
            return nv;
    return 1;
}

template <typename T>
void launch_conserved_t(const void* src, int64_t n, int64_t plane, double* partials, int nblk,
                        cudaStream_t st) {
    const T* s = static_cast<const T*>(src);
    const int nv = reduce_width<T>(src, n, plane, sizeof(T) == 4 ? 4 : 8);
    auto run = [&](auto kernel) { kernel<<<nblk, kReduceThreads, 0, st>>>(s, n, plane, partials); };
    if constexpr (sizeof(T) == 2) {
        if (nv == 8) return run(k_conserved_partial<T, 8>);
    }
    if (nv >= 4) return run(k_conserved_partial<T, 4>);
    if (nv == 2) return run(k_conserved_partial<T, 2>);
    run(k_conserved_partial<T, 1>);
}

}  // namespace

cudaError_t launch_conserved(int storage, const void* src, int64_t n, int64_t plane,
                             double rho_ref, double jx_ref, double jy_ref, double lambda,
                             double* partials, int nblk, double* out, cudaStream_t st) {
    switch (storage) {
        case kStoreF32: launch_conserved_t<float>(src, n, plane, partials, nblk, st); break;
        case kStoreF16: launch_conserved_t<__half>(src, n, plane, partials, nblk, st); break;
        case kStoreBF16:
            launch_conserved_t<__nv_bfloat16>(src, n, plane, partials, nblk, st);
            break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_conserved_final<<<1, kReduceThreads, 0, st>>>(partials, nblk, rho_ref * (double)n,
                                                    jx_ref * (double)n, jy_ref * (double)n,
                                                    lambda, out);
    return cudaGetLastError();
}

}  // namespace lbmrv
