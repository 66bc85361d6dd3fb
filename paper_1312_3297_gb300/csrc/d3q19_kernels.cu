// D3Q19 kernels: fused pull transport + relative-velocity relaxation, equilibrium
// initialisation, moments and FP64 conserved sums. Layout: 19 planes of nx*ny*nz, index
// (z*ny + y)*nx + x.
#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>

#include "async_copy.cuh"
#include "d3q19.cuh"
#include "launch.h"
#include "occupancy.cuh"
#include "pdl.cuh"
#include "pull.cuh"

namespace lbmrv {

namespace {

constexpr int kThreads3 = 128;

// Element type of a step kernel's state arguments.
template <typename K>
struct KernelArg;
template <typename T>
struct KernelArg<void (*)(const T*, T*, StepArgs3, double*)> {
    using type = T;
};

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

// Rows of the 3x3 (y, z) neighbourhood of row (y, z): offsets of rows (y + dy, z + dz),
// periodic.
struct Rows3 {
    int64_t r00, rm0, rp0, r0m, r0p, rmm, rpp, rmp, rpm;
    __device__ __forceinline__ Rows3(int y, int z, int nx, int ny, int nz) {
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        auto row = [&](int yy, int zz) { return ((int64_t)zz * ny + yy) * nx; };
        r00 = row(y, z), rm0 = row(ym, z), rp0 = row(yp, z);
        r0m = row(y, zm), r0p = row(y, zp);
        rmm = row(ym, zm), rpp = row(yp, zp), rmp = row(ym, zp), rpm = row(yp, zm);
    }
};

// Stored pair w plus the increments inc, rounded once to storage form. The 16-bit values
// enter FP32 additions directly (add.f32.f16 / add.f32.bf16, sm_100 and later): the same
// exact widening and single rounding as converting first, in one instruction per value.
template <typename T>
struct MixedAdd;
template <>
struct MixedAdd<__half> {
    __device__ __forceinline__ static float add(unsigned short v, float c) {
        float d;
        asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(v), "f"(c));
        return d;
    }
};
template <>
struct MixedAdd<__nv_bfloat16> {
    __device__ __forceinline__ static float add(unsigned short v, float c) {
        float d;
        asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(v), "f"(c));
        return d;
    }
};
template <typename T>
__device__ __forceinline__ uint32_t add_to_pair(uint32_t w, F2 inc) {
    unsigned short lo, hi;
    asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(w));
    float a, b;
    unpack2(inc, a, b);
    return Cvt16<T>::pack(MixedAdd<T>::add(lo, a), MixedAdd<T>::add(hi, b));
}

// Conserved moments of one stored node (values as rounded to the storage type) added to
// r[0..3] (sum g, sum c g), and its non-finite flag to bad.
template <typename T>
__device__ __forceinline__ void add_node_sums3(const float g[19], float r[4], int& bad) {
    float h[19];
#pragma unroll
    for (int j = 0; j < 19; ++j) h[j] = to_f(from_f<T>(g[j]));
    const NodeMoments3 m = node_moments3(h);
    r[0] += m.drho;
    r[1] += m.jx;
    r[2] += m.jy;
    r[3] += m.jz;
    bad += (finite_f(m.drho) && finite_f(m.jx) && finite_f(m.jy) && finite_f(m.jz)) ? 0 : 1;
}

// Sums of v[0..4] over the block (a multiple of 32 threads, at most 1024) into
// slot[0..4]; every thread of the block must call it.
__device__ __forceinline__ void block_sum5(const double v[5], double* __restrict__ slot) {
    __shared__ double sh[32][5];
    const int t = threadIdx.x + blockDim.x * threadIdx.y;
    const int nw = (blockDim.x * blockDim.y) >> 5, w = t >> 5, l = t & 31;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        double x = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFullMask, x, o);
        if (l == 0) sh[w][c] = x;
    }
    __syncthreads();
    if (t < 5) {
        double x = 0.0;
        for (int k = 0; k < nw; ++k) x += sh[k][t];
        slot[t] = x;
    }
}

// Thread blocks of 32 to kThreads3 threads (a multiple of 32) along one row, each thread
// owning NV consecutive nodes, sized to the row so that short rows leave no warp idle; the
// row index stays uniform across the block (its offsets are computed once per warp, in
// uniform registers).
//
// One thread: NV consecutive nodes of the row (y, z). Population j is pulled from
// (x, y, z) - c_j, periodic (relation (transport)).
//
// SUMS: also add up the conserved moments of the stored result in the block's slot
// part[8 * block] (sum g, sum c g, non-finite nodes), as k_conserved3_partial does for a
// stored state.
template <typename T, int NV, int UM, bool SUMS = false>
__global__ void __launch_bounds__(kThreads3) k_step3(const T* __restrict__ src,
                                                     T* __restrict__ dst, StepArgs3 a,
                                                     double* __restrict__ part) {
    pdl_wait_prior();
    pdl_allow_next();
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t n = (int64_t)nx * ny * nz;
    const PackLane p = pack_lane<NV>(nx);
    // SUMS: node moments in FP32 runs of kRun packs (32 nodes), each run added in FP64
    constexpr int kRun = NV >= 32 ? 1 : 32 / NV;
    double sums[4] = {0.0, 0.0, 0.0, 0.0};
    float run_r[4] = {0.f, 0.f, 0.f, 0.f};
    int bad = 0;
    auto row = [&](int y, int z) {
        const Rows3 r(y, z, nx, ny, nz);
        float g[19][NV];
        const T* s = src;
        load_pack<T, NV>(s + r.r00 + p.x0, p.act, g[0]);
        load_from_left<T, NV>(s + 1 * n + r.r00, p.x0, p.xprev, p.act, p.left_edge, g[1]);
        load_from_right<T, NV>(s + 2 * n + r.r00, p.x0, p.xnext, p.act, p.right_edge, g[2]);
        load_pack<T, NV>(s + 3 * n + r.rm0 + p.x0, p.act, g[3]);
        load_pack<T, NV>(s + 4 * n + r.rp0 + p.x0, p.act, g[4]);
        load_pack<T, NV>(s + 5 * n + r.r0m + p.x0, p.act, g[5]);
        load_pack<T, NV>(s + 6 * n + r.r0p + p.x0, p.act, g[6]);
        load_from_left<T, NV>(s + 7 * n + r.rm0, p.x0, p.xprev, p.act, p.left_edge, g[7]);
        load_from_right<T, NV>(s + 8 * n + r.rp0, p.x0, p.xnext, p.act, p.right_edge, g[8]);
        load_from_left<T, NV>(s + 9 * n + r.rp0, p.x0, p.xprev, p.act, p.left_edge, g[9]);
        load_from_right<T, NV>(s + 10 * n + r.rm0, p.x0, p.xnext, p.act, p.right_edge, g[10]);
        load_from_left<T, NV>(s + 11 * n + r.r0m, p.x0, p.xprev, p.act, p.left_edge, g[11]);
        load_from_right<T, NV>(s + 12 * n + r.r0p, p.x0, p.xnext, p.act, p.right_edge, g[12]);
        load_from_left<T, NV>(s + 13 * n + r.r0p, p.x0, p.xprev, p.act, p.left_edge, g[13]);
        load_from_right<T, NV>(s + 14 * n + r.r0m, p.x0, p.xnext, p.act, p.right_edge, g[14]);
        load_pack<T, NV>(s + 15 * n + r.rmm + p.x0, p.act, g[15]);
        load_pack<T, NV>(s + 16 * n + r.rpp + p.x0, p.act, g[16]);
        load_pack<T, NV>(s + 17 * n + r.rmp + p.x0, p.act, g[17]);
        load_pack<T, NV>(s + 18 * n + r.rpm + p.x0, p.act, g[18]);
        if (p.act) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                float h[19];
#pragma unroll
                for (int j = 0; j < 19; ++j) h[j] = g[j][k];
                float ux = 0.0f, uy = 0.0f, uz = 0.0f;
                if constexpr (UM != UM_ZERO && UM != UM_FLUID)
                    relative_velocity3<UM>(h, r.r00 + p.x0 + k, n, a, ux, uy, uz);
                relax_node3<UM>(h, ux, uy, uz, a.s, a.ref);
#pragma unroll
                for (int j = 0; j < 19; ++j) g[j][k] = h[j];
            }
#pragma unroll
            for (int j = 0; j < 19; ++j) store_pack<T, NV>(dst + j * n + r.r00 + p.x0, g[j]);
            if constexpr (SUMS) {
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    float h[19];
#pragma unroll
                    for (int j = 0; j < 19; ++j) h[j] = g[j][k];
                    add_node_sums3<T>(h, run_r, bad);
                }
            }
        }
    };
    if constexpr (!SUMS) {
        for (int z = blockIdx.z; z < nz; z += gridDim.z)
            for (int y = blockIdx.y; y < ny; y += gridDim.y) row(y, z);
    } else {
        // the block's rows (y fastest, then z) in chunks of kRun; a chunk's FP32 run is
        // added in FP64 after it, outside the rows' loop (FP64 issues at 2 operations per
        // clock per SM on this GPU, and predicated adds inside the loop would hold that pipe)
        int y = blockIdx.y, z = blockIdx.z;
        while (z < nz) {
            for (int t = 0; t < kRun && z < nz; ++t) {
                row(y, z);
                y += gridDim.y;
                if (y >= ny) {
                    y = blockIdx.y;
                    z += gridDim.z;
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                sums[c] += (double)run_r[c];
                run_r[c] = 0.f;
            }
        }
    }
    if constexpr (SUMS) {
        double v[5];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = sums[c] + (double)run_r[c];
        v[4] = (double)bad;
        block_sum5(v, part + 8 * (((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x +
                                  blockIdx.x));
    }
}

// ---------------------------------------------------------------------------------------
// 16-bit D3Q19 step with the next row staged in shared memory. Each warp owns a sequence of
// row segments of 256 nodes (32 lanes x 8-node packs); while it relaxes one, asynchronous
// copies (cp.async) bring the next one's 19 plane segments, plus for every x-moving plane
// the 4-byte word that holds the element across the pack boundary, into the other half of
// its double buffer, in plane groups spread over the relaxation (pipe_plane_groups).
// Memory parallelism then no longer depends on registers, and the kernel runs two 4-warp
// blocks per SM with up to 255 registers per thread (measured on
// GB300: more warps with fewer registers spill, and deeper rings with fewer warps issue
// too slowly).
constexpr int kPipeNpl = 8;  // nodes per lane (4: 168 registers, 3 blocks per SM, slower)
constexpr int kPipeSeg = 32 * kPipeNpl;                         // nodes per row segment
constexpr int kPipeData = 19 * 32 * 2 * kPipeNpl;               // packs of one stage
constexpr int kPipeStage = kPipeData + 10 * 32 * 4;            // + halo words
constexpr int kPipeBlocksPerSm = kPipeNpl == 8 ? 2 : 3;

constexpr int kPipeWarps = 4;                                   // per block, 2 blocks per SM
constexpr int kPipeStages = 2;                                  // segments per warp
constexpr int kPipeSmem = kPipeWarps * kPipeStages * kPipeStage;  // bytes per block


// x shift of plane j: 0 none, 1 from the left (x - 1), 2 from the right (x + 1); relation
// (transport) in pull form. hslot: the plane's halo slot (x-moving planes only).
__host__ __device__ constexpr int plane_shift(int j) {
    return (j == 1 || j == 7 || j == 9 || j == 11 || j == 13) ? 1
         : (j == 2 || j == 8 || j == 10 || j == 12 || j == 14) ? 2 : 0;
}
__host__ __device__ constexpr int plane_hslot(int j) {
    return j == 1 ? 0 : j == 7 ? 1 : j == 9 ? 2 : j == 11 ? 3 : j == 13 ? 4
         : j == 2 ? 5 : j == 8 ? 6 : j == 10 ? 7 : j == 12 ? 8 : j == 14 ? 9 : -1;
}

// Rows of the (y, z) neighbourhood as row numbers z * ny + y (the launcher checks that
// ny * nz fits in 31 bits), periodic.
struct RowNums3 {
    int r00, rm0, rp0, r0m, r0p, rmm, rpp, rmp, rpm;
    __device__ __forceinline__ RowNums3(int y, int z, int ny, int nz) {
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const int zr = z * ny, zmr = (z == 0 ? nz - 1 : z - 1) * ny;
        const int zpr = (z == nz - 1 ? 0 : z + 1) * ny;
        r00 = zr + y, rm0 = zr + ym, rp0 = zr + yp;
        r0m = zmr + y, r0p = zpr + y;
        rmm = zmr + ym, rpp = zpr + yp, rmp = zpr + ym, rpm = zmr + yp;
    }
};
// Source row of plane j among the nine rows of the (y, z) neighbourhood.
__device__ __forceinline__ int plane_rownum(const RowNums3& r, int j) {
    switch (j) {
        case 0: case 1: case 2: return r.r00;
        case 3: case 7: case 10: return r.rm0;
        case 4: case 8: case 9: return r.rp0;
        case 5: case 11: case 14: return r.r0m;
        case 6: case 12: case 13: return r.r0p;
        case 15: return r.rmm;
        case 16: return r.rpp;
        case 17: return r.rmp;
        default: return r.rpm;
    }
}

// The next item's copies go out in this many plane groups, interleaved with the relaxation
// of the current item's node pairs (group 0 before it, the others before pairs 1-3 or 2),
// so that the warps' loads and stores do not reach memory in bursts. Measured on GB300 at
// 256^3 (fraction of copy bandwidth for 1, 2 and 4 groups): u~ = 0 FP16 0.84 / 0.91 / 0.97,
// BF16 0.84 / 0.90 / 0.94; u~ = q/rho FP16 0.94 / 0.71 / 0.73, BF16 0.92 / 0.95 / 0.92.
template <typename T, int UM>
constexpr int pipe_plane_groups() {
    return UM == UM_ZERO ? 4 : std::is_same<T, __nv_bfloat16>::value ? 2 : 1;
}

// A stored pair widened to FP32 for the relaxation. BF16 with u~ = 0 widens by
// mixed-precision adds of -0 (exact for every value, as the shifts are): they run on the
// FMA pipe, like FP16's conversions, and space out the copies of the next segment. Measured
// at 256^3, of copy bandwidth: BF16 u~ = 0 0.952 against 0.938 with shifts; with u~ = q/rho
// the shifts are faster (0.947 against 0.918).
template <typename T, int UM>
__device__ __forceinline__ float2 unpack_widen(uint32_t w) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value && UM == UM_ZERO) {
        unsigned short lo, hi;
        asm("mov.b32 {%0, %1}, %2;" : "=h"(lo), "=h"(hi) : "r"(w));
        float x, y;
        asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(x) : "h"(lo), "f"(-0.0f));
        asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(y) : "h"(hi), "f"(-0.0f));
        return make_float2(x, y);
    } else {
        return Cvt16<T>::unpack(w);
    }
}

template <typename T, int UM, int RCP, bool SUMS = false, bool TAILS = false>
__global__ void __launch_bounds__(kPipeWarps * 32, kPipeBlocksPerSm) k_step3_pipe(const T* __restrict__ src,
                                                                   T* __restrict__ dst,
                                                                   StepArgs3 a,
                                                                   double* __restrict__ part) {
    constexpr int S = kPipeStages;
    constexpr int NPL = kPipeNpl, P = NPL / 2;  // nodes and node pairs per lane
    // SUMS: the stored result's moments, in FP32 runs of 4 items (32 nodes), each run added
    // in FP64
    double sums[4] = {0.0, 0.0, 0.0, 0.0};
    float run_r[4] = {0.f, 0.f, 0.f, 0.f};
    int bad = 0;
    pdl_wait_prior();
    pdl_allow_next();
    extern __shared__ __align__(16) unsigned char pipe_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t n = (int64_t)nx * ny * nz;
    // TAILS (nx not a multiple of kPipeSeg): `segs` counts a row's full segments, and the
    // rows' short last segments (tail_lanes lanes each) are packed rows_per_tail rows to an
    // item after all full segments, lane l of such an item taking row base + l / tail_lanes
    // (with one row per item they left most lanes idle). Without TAILS a row has segs
    // segments.
    const int segs = TAILS ? nx / kPipeSeg : (nx + kPipeSeg - 1) / kPipeSeg;
    const int tail_lanes = TAILS ? (nx % kPipeSeg) / NPL : 1;
    const int rows_per_tail = 32 / tail_lanes;
    const int64_t nrows = (int64_t)ny * nz, nfull = nrows * segs;
    const int64_t ntail = TAILS ? (nrows + rows_per_tail - 1) / rows_per_tail : 0;
    unsigned char* wbuf = pipe_smem + warp * S * kPipeStage;

    // Warp w takes work items (row segments, x fastest, then y, z) w, w + W, w + 2W, ...
    // (W warps in the grid), so that the warps in flight read neighbouring rows. A cursor
    // (seg, y, z) steps by W in mixed radix (segs, ny, nz), so no item index is divided.
    const int64_t nwarps = (int64_t)gridDim.x * kPipeWarps;
    struct Cursor {
        int seg, y, z;
    };
    auto split = [&](int64_t it) {
        const int64_t row = it / segs;
        Cursor c;
        c.seg = (int)(it - row * segs);
        c.z = (int)(row / ny);
        c.y = (int)(row - (int64_t)c.z * ny);
        return c;
    };
    // (TAILS without full segments: a cursor that starts past the last plane)
    const Cursor step = (TAILS && segs == 0) ? Cursor{0, 0, 0} : split(nwarps);
    auto advance = [&](Cursor c) {
        c.seg += step.seg;
        int carry = c.seg >= segs;
        c.seg -= carry ? segs : 0;
        c.y += step.y + carry;
        carry = c.y >= ny;
        c.y -= carry ? ny : 0;
        c.z += step.z + carry;
        return c;
    };
    // TAILS: this lane's row and first node in tail item it - nfull
    auto tail_work = [&](int64_t it, int& y, int& z, int& x0, bool& ok) {
        const int64_t t = it - nfull;
        const int64_t row = t * rows_per_tail + lane / tail_lanes;
        ok = t < ntail && lane < rows_per_tail * tail_lanes && row < nrows;
        const int r = ok ? (int)row : 0;  // rows are numbered in 32 bits (launcher)
        z = r / ny;
        y = r - z * ny;
        x0 = segs * kPipeSeg + (lane % tail_lanes) * NPL;
    };
    // queue the copies of planes [LO, HI) of the item at `c` (TAILS: at index it) into
    // buffer `stage`
    auto copy = [&](const Cursor& c, int64_t it, int stage, auto lo, auto hi) {
        constexpr int LO = decltype(lo)::value, HI = decltype(hi)::value;
        int y = c.y, z = c.z, x0 = c.seg * kPipeSeg + lane * NPL;
        bool ok = c.z < nz && x0 < nx;
        if constexpr (TAILS) {
            if (c.z >= nz) tail_work(it, y, z, x0, ok);
        }
        if (ok) {
            const RowNums3 r(y, z, ny, nz);
            unsigned char* sb = wbuf + stage * kPipeStage;
            const int xl = (x0 == 0 ? nx : x0) - 2;       // word (x0-2, x0-1), periodic
            const int xr = x0 + NPL >= nx ? 0 : x0 + NPL;  // word after the pack, periodic
#pragma unroll
            for (int j = LO; j < HI; ++j) {
                const T* row = src + j * n + (int64_t)plane_rownum(r, j) * nx;
                if constexpr (NPL == 8)
                    cp_async16(sb + (j * 32 + lane) * 16, row + x0);
                else
                    cp_async8(sb + (j * 32 + lane) * 8, row + x0);
                if (plane_hslot(j) >= 0)
                    cp_async4(sb + kPipeData + (plane_hslot(j) * 32 + lane) * 4,
                              row + (plane_shift(j) == 1 ? xl : xr));
            }
        }
    };
    constexpr int Q = S != 2 ? 1 : pipe_plane_groups<T, UM>() < P ? pipe_plane_groups<T, UM>() : P;
    using I0 = std::integral_constant<int, 0>;
    using I19 = std::integral_constant<int, 19>;
    auto copy_group = [&](const Cursor& c, int64_t it, int stage, auto q) {
        constexpr int G = decltype(q)::value;
        copy(c, it, stage, std::integral_constant<int, (19 * G + Q - 1) / Q>(),
             std::integral_constant<int, (19 * (G + 1) + Q - 1) / Q>());
    };

    // S-stage ring: the copies of the next S - 1 items are in flight while one is relaxed.
    // TAILS: icur / iahead are the items' indexes (the cursor's position while it is inside
    // the full segments).
    const int64_t first = (int64_t)blockIdx.x * kPipeWarps + warp;
    Cursor cur = (TAILS && segs == 0) ? Cursor{0, 0, nz} : split(first), ahead = cur;
    int64_t icur = first, iahead = first;
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        copy(ahead, iahead, s, I0(), I19());
        cp_async_commit();  // (empty groups keep the count of groups uniform)
        ahead = advance(ahead);
        if constexpr (TAILS) iahead += nwarps;
    }
    auto more = [&]() {
        if constexpr (TAILS) return icur < nfull + ntail;
        else return cur.z < nz;
    };
    int stage = 0, fill = S - 1;
    // the groups of the next item issued before node pair k of the current one (k > 0);
    // group 0 goes before the wait for the current item
    auto issue_groups_before = [&](int k) {
        if constexpr (Q == 4) {
            if (k == 1) copy_group(ahead, iahead, fill, std::integral_constant<int, 1>());
            if (k == 2) copy_group(ahead, iahead, fill, std::integral_constant<int, 2>());
            if (k == 3) copy_group(ahead, iahead, fill, std::integral_constant<int, 3>());
        } else if constexpr (Q == 2) {
            if (k == P / 2) copy_group(ahead, iahead, fill, std::integral_constant<int, 1>());
        }
    };
    auto item = [&]() {
        if constexpr (Q > 1) {
            copy_group(ahead, iahead, fill, I0());  // committed with the other groups, below
            cp_async_wait_all_but<0>();             // every committed group: the item at `cur`
        } else {
            copy(ahead, iahead, fill, I0(), I19());
            cp_async_commit();
            cp_async_wait_all_but<S - 1>();  // the oldest group: the item at `cur`
        }
        __syncwarp();
        int y = cur.y, z = cur.z, x0 = cur.seg * kPipeSeg + lane * NPL;
        bool ok = x0 < nx;
        if constexpr (TAILS) {
            if (cur.z >= nz) tail_work(icur, y, z, x0, ok);
        }
        if (ok) {
            const unsigned char* sb = wbuf + stage * kPipeStage;
            const int64_t r00 = (int64_t)(z * ny + y) * nx;
            // pair k of an x-moving plane straddles words k and k + 1 of (left halo, pack)
            // or (pack, right halo)
            uint32_t w[19][P];
#pragma unroll
            for (int j = 0; j < 19; ++j) {
                uint32_t e[P + 2];
                const uint32_t hw = plane_hslot(j) >= 0
                    ? *reinterpret_cast<const uint32_t*>(sb + kPipeData +
                                                         (plane_hslot(j) * 32 + lane) * 4)
                    : 0u;
                e[0] = hw;
                e[P + 1] = hw;
                if constexpr (NPL == 8) {
                    const uint4 v = *reinterpret_cast<const uint4*>(sb + (j * 32 + lane) * 16);
                    e[1] = v.x;
                    e[2] = v.y;
                    e[3] = v.z;
                    e[4] = v.w;
                } else {
                    const uint2 v = *reinterpret_cast<const uint2*>(sb + (j * 32 + lane) * 8);
                    e[1] = v.x;
                    e[2] = v.y;
                }
#pragma unroll
                for (int k = 0; k < P; ++k)
                    w[j][k] = plane_shift(j) == 1 ? __byte_perm(e[k], e[k + 1], 0x5432)
                            : plane_shift(j) == 2 ? __byte_perm(e[k + 1], e[k + 2], 0x5432)
                                                  : e[k + 1];
            }
#pragma unroll
            for (int k = 0; k < P; ++k) {
                if constexpr (Q > 1) issue_groups_before(k);
                const int64_t i = r00 + x0 + 2 * k;  // first node of the pair
                F2 h[19];
#pragma unroll
                for (int j = 0; j < 19; ++j) {
                    const float2 f = unpack_widen<T, UM>(w[j][k]);
                    h[j] = pack2(f.x, f.y);
                }
                F2 ux(0.0f), uy(0.0f), uz(0.0f);
                if constexpr (UM != UM_ZERO && UM != UM_FLUID) {
                    const F2 amp(a.amp_t);
                    ux = amp * pack2(__ldg(a.ut0 + i), __ldg(a.ut0 + i + 1));
                    uy = amp * pack2(__ldg(a.ut0 + n + i), __ldg(a.ut0 + n + i + 1));
                    uz = amp * pack2(__ldg(a.ut0 + 2 * n + i), __ldg(a.ut0 + 2 * n + i + 1));
                }
                // the same arithmetic as k_step3_pipe_pairs (increments added to the
                // stored pair), so that both kernels give the same bits
                relax_node3<UM, RCP, true>(h, ux, uy, uz, a.s, a.ref);
#pragma unroll
                for (int j = 0; j < 19; ++j) w[j][k] = add_to_pair<T>(w[j][k], h[j]);
            }
#pragma unroll
            for (int j = 0; j < 19; ++j) store_raw16<NPL>(dst + j * n + r00 + x0, w[j]);
            if constexpr (SUMS) {
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    float lo[19], hi[19];
#pragma unroll
                    for (int j = 0; j < 19; ++j) {
                        const float2 f = Cvt16<T>::unpack(w[j][k]);
                        lo[j] = f.x;
                        hi[j] = f.y;
                    }
                    add_node_sums3<float>(lo, run_r, bad);
                    add_node_sums3<float>(hi, run_r, bad);
                }
            }
        } else if constexpr (Q > 1) {
#pragma unroll
            for (int k = 1; k < P; ++k) issue_groups_before(k);  // as the relaxation would
        }
        if constexpr (Q > 1) cp_async_commit();
        __syncwarp();  // every lane is done with `stage` before it is refilled
        ahead = advance(ahead);
        fill = fill == S - 1 ? 0 : fill + 1;
        cur = advance(cur);
        if constexpr (TAILS) {
            iahead += nwarps;
            icur += nwarps;
        }
        stage = stage == S - 1 ? 0 : stage + 1;
    };
    if constexpr (!SUMS) {
        while (more()) item();
    } else {
        // items in chunks of 32 / NPL (32 nodes per lane); a chunk's FP32 run is added in
        // FP64 after it, outside the items' loop (FP64 issues at 2 operations per clock per
        // SM on this GPU, and predicated adds inside the loop would hold that pipe)
        while (more()) {
            for (int t = 0; t < 32 / NPL && more(); ++t) item();
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                sums[c] += (double)run_r[c];
                run_r[c] = 0.f;
            }
        }
    }
    if constexpr (SUMS) {
        double v[5];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = sums[c] + (double)run_r[c];
        v[4] = (double)bad;
        block_sum5(v, part + 8 * (int64_t)blockIdx.x);
    }
}

// ---------------------------------------------------------------------------------------
// 16-bit D3Q19 step for rows of 4-node packs (nx a multiple of 4, not of 8), staged in
// shared memory with lanes interleaved by node pair. A warp owns a sequence of row
// segments of 128 nodes; their 19 plane segments arrive by cp.async (lane l copies nodes
// [4 l, 4 l + 4) of each) into a two-stage ring while the warp relaxes the previous
// segment. Lane l relaxes the node pairs 2 l and 2 l + 64: it reads each pair's word from
// shared memory just before relaxing it (the x-moving planes by a byte permute of two
// neighbouring words, conflict-free across the warp) and stores the relaxed pair straight
// to global memory, where the warp's 32 words fill one 128-byte line. The arithmetic is
// that of k_step3_pipe (increments added to the stored pair), so that both give the same
// bits. Measured on GB300 at 256^3 with 4-node packs, of copy bandwidth: FP16 / BF16 0.847 /
// 0.842 with u~ = q/rho, against 0.72 / 0.73 for 4-node packs held in registers (16 warps
// per SM at 128 registers). With 8-node packs (256-node segments, 8-10 warps per SM) it
// was slower than k_step3_pipe: 0.76-0.86 against 0.92-0.97, at 12 % more instructions
// per node (the per-pair stores and shared loads) and a lower issue rate.
// Shared layout of one plane segment, in 32-bit words: word 3 the word left of the segment
// (planes pulling from x - 1), words 4 .. 3 + nv / 2 the nv nodes of the segment, word
// 4 + nv / 2 the word right of it (planes pulling from x + 1); periodic in x.
struct PipePairs {
    static constexpr int kNpl = 4;                       // nodes per lane and segment
    static constexpr int kSeg = 32 * kNpl;               // nodes per row segment
    static constexpr int kPlaneWords = kSeg / 2 + 8;     // head, segment, right word, pad
    static constexpr int kStageWords = 19 * kPlaneWords;
    static constexpr int kWarps = 8;                     // per block
    static constexpr int kBlocksPerSm = 2;
    static constexpr int kStages = 2;
    static constexpr int kSmem = kWarps * kStages * kStageWords * 4;  // bytes per block
};

template <typename T, int UM, int RCP>
__global__ void __launch_bounds__(PipePairs::kWarps * 32, PipePairs::kBlocksPerSm)
    k_step3_pipe_pairs(const T* __restrict__ src, T* __restrict__ dst, StepArgs3 a) {
    using C = PipePairs;
    constexpr int S = C::kStages, P = C::kNpl / 2, PW = C::kPlaneWords, SEG = C::kSeg;
    static_assert(sizeof(T) == 2, "16-bit storage");
    pdl_wait_prior();
    pdl_allow_next();
    extern __shared__ __align__(16) uint32_t pairs_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int64_t n = (int64_t)nx * ny * nz;
    const int segs = (nx + SEG - 1) / SEG;
    uint32_t* wbuf = pairs_smem + warp * S * C::kStageWords;

    // Warp w takes work items (row segments, x fastest, then y, z) w, w + W, w + 2W, ...
    // (W warps in the grid); a cursor (seg, y, z) steps by W in mixed radix (segs, ny, nz).
    const int64_t nwarps = (int64_t)gridDim.x * C::kWarps;
    struct Cursor {
        int seg, y, z;
    };
    auto split = [&](int64_t it) {
        const int64_t row = it / segs;
        Cursor c;
        c.seg = (int)(it - row * segs);
        c.z = (int)(row / ny);
        c.y = (int)(row - (int64_t)c.z * ny);
        return c;
    };
    const Cursor step = split(nwarps);
    auto advance = [&](Cursor c) {
        c.seg += step.seg;
        int carry = c.seg >= segs;
        c.seg -= carry ? segs : 0;
        c.y += step.y + carry;
        carry = c.y >= ny;
        c.y -= carry ? ny : 0;
        c.z += step.z + carry;
        return c;
    };
    // queue the copies of the item at `c` into buffer `stg`
    auto copy = [&](const Cursor& c, int stg) {
        if (c.z < nz) {
            const RowNums3 r(c.y, c.z, ny, nz);
            uint32_t* sb = wbuf + stg * C::kStageWords;
            const int xs = c.seg * SEG;
            const int nv = nx - xs < SEG ? nx - xs : SEG;  // nodes in this segment
            const int xl = xs + lane * C::kNpl;             // this lane's copy
            const int x_left = (xs == 0 ? nx : xs) - 2;     // word left of the segment
            const int x_right = xs + nv == nx ? 0 : xs + nv;  // word right of it
#pragma unroll
            for (int j = 0; j < 19; ++j) {
                const T* row = src + j * n + (int64_t)plane_rownum(r, j) * nx;
                uint32_t* pl = sb + j * PW;
                if (xl < nx) cp_async8(pl + 4 + lane * 2, row + xl);
                if (lane == 0 && plane_shift(j) == 1) cp_async4(pl + 3, row + x_left);
                if (lane == 0 && plane_shift(j) == 2) cp_async4(pl + 4 + nv / 2, row + x_right);
            }
        }
    };

    Cursor cur = split((int64_t)blockIdx.x * C::kWarps + warp), ahead = cur;
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        copy(ahead, s);
        cp_async_commit();
        ahead = advance(ahead);
    }
    int stage = 0, fill = S - 1;
    while (cur.z < nz) {
        copy(ahead, fill);
        cp_async_commit();
        cp_async_wait_all_but<S - 1>();  // the oldest group: the item at `cur`
        __syncwarp();                    // the other lanes' copies are visible
        const uint32_t* sb = wbuf + stage * C::kStageWords;
        const int xs = cur.seg * SEG;
        const int nv = nx - xs < SEG ? nx - xs : SEG;
        const int64_t r0 = (int64_t)(cur.z * ny + cur.y) * nx + xs;  // first node
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const int q = lane + 32 * k;  // node pair of the segment
            if (2 * q < nv) {
                uint32_t w[19];
                F2 h[19];
#pragma unroll
                for (int j = 0; j < 19; ++j) {
                    const uint32_t* pl = sb + j * PW + 4 + q;
                    w[j] = plane_shift(j) == 1 ? __byte_perm(pl[-1], pl[0], 0x5432)
                         : plane_shift(j) == 2 ? __byte_perm(pl[0], pl[1], 0x5432)
                                               : pl[0];
                    const float2 f = Cvt16<T>::unpack(w[j]);
                    h[j] = pack2(f.x, f.y);
                }
                const int64_t i = r0 + 2 * q;  // first node of the pair
                F2 ux(0.0f), uy(0.0f), uz(0.0f);
                if constexpr (UM != UM_ZERO && UM != UM_FLUID) {
                    const F2 amp(a.amp_t);
                    ux = amp * pack2(__ldg(a.ut0 + i), __ldg(a.ut0 + i + 1));
                    uy = amp * pack2(__ldg(a.ut0 + n + i), __ldg(a.ut0 + n + i + 1));
                    uz = amp * pack2(__ldg(a.ut0 + 2 * n + i), __ldg(a.ut0 + 2 * n + i + 1));
                }
                relax_node3<UM, RCP, true>(h, ux, uy, uz, a.s, a.ref);
#pragma unroll
                for (int j = 0; j < 19; ++j)
                    *reinterpret_cast<uint32_t*>(dst + j * n + i) = add_to_pair<T>(w[j], h[j]);
            }
        }
        __syncwarp();  // every lane is done with `stage` before it is refilled
        ahead = advance(ahead);
        fill = fill == S - 1 ? 0 : fill + 1;
        cur = advance(cur);
        stage = stage == S - 1 ? 0 : stage + 1;
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

// FP64 sums of (sum g, sum c g (3), non-finite nodes), 8 doubles per block (5 used), NV
// consecutive nodes per thread and pack (n and plane multiples of NV, planes NV-aligned).
// At least kReduceMinBlocks blocks fit on an SM, the count conserved_blocks launches.
template <typename T, int NV>
__global__ void __launch_bounds__(kReduceThreads, kReduceMinBlocks)
    k_conserved3_partial(const T* __restrict__ src, int64_t n, int64_t plane,
                         double* __restrict__ part) {
    // FP32 runs of up to 32 nodes, each run added in FP64 after its loop (as in the D2Q9
    // reduction)
    constexpr int kRunPacks = NV >= 32 ? 1 : 32 / NV;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int bad = 0;
    const int64_t packs = n / NV;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // pack index
    while (i < packs) {
        float r[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < kRunPacks && i < packs; ++k, i += stride) {
            float g[19][NV];
#pragma unroll
            for (int j = 0; j < 19; ++j)
                PackCvt<T, NV>::in(*reinterpret_cast<const Pack<T, NV>*>(src + j * plane + i * NV),
                                   g[j]);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                float h[19];
#pragma unroll
                for (int j = 0; j < 19; ++j) h[j] = g[j][q];
                const NodeMoments3 m = node_moments3(h);
                r[0] += m.drho;
                r[1] += m.jx;
                r[2] += m.jy;
                r[3] += m.jz;
                bad += (finite_f(m.drho) && finite_f(m.jx) && finite_f(m.jy) && finite_f(m.jz))
                           ? 0
                           : 1;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] += (double)r[c];
    }
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


// Block shape for NV-node packs on rows of nx nodes: 32 to kThreads3 threads along x (a
// multiple of 32), and, for kernels that take it, the rest of the block on further rows.
inline dim3 step3_block(int nx, int nv, bool multi_row) {
    const int packs = (nx + nv - 1) / nv;
    int tx = ((packs + 31) / 32) * 32;
    if (tx > kThreads3) tx = kThreads3;
    return dim3(tx, multi_row ? kThreads3 / tx : 1, 1);
}

dim3 step3_grid(const StepArgs3& a, int nv, bool multi_row) {
    const dim3 b = step3_block(a.nx, nv, multi_row);
    const int packs = (a.nx + nv - 1) / nv;
    const int gy = (a.ny + (int)b.y - 1) / (int)b.y;
    return dim3((packs + b.x - 1) / b.x, gy < 65535 ? gy : 65535, a.nz < 65535 ? a.nz : 65535);
}

template <typename K>
cudaError_t launch3(K kernel, const void* src, void* dst, const StepArgs3& a, cudaStream_t st,
                    int nv, bool multi_row = false, double* part = nullptr) {
    const dim3 b = step3_block(a.nx, nv, multi_row);
    using TT = typename KernelArg<K>::type;
    const cudaError_t e = launch_pdl(kernel, step3_grid(a, nv, multi_row), b, st,
                                     static_cast<const TT*>(src), static_cast<TT*>(dst), a, part);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// 16-bit packs of 4 and 8 nodes run in storage form, relaxed in pairs by packed FP32
// instructions, by the shared-memory pipelines: 8-node packs by k_step3_pipe, 4-node packs by
// k_step3_pipe_pairs. Both number rows in 32 bits (ny * nz < 2^31, which any 16-bit
// lattice of 4 or more nodes per row that fits in device memory meets); beyond that
// 2-node packs run.

// Form of 1/rho in the 16-bit pipelines, measured on GB300 at 256^3 (8-node packs, of copy
// bandwidth): FP16 with u~ = q/rho takes the fast division (0.938, against 0.934 with the
// approximation and 0.921 correctly rounded); the other kernels keep the correctly rounded
// reciprocal, which the fast division slows to 0.86 (FP16 u~ = 0), 0.72 (BF16 u~ = q/rho)
// and 0.87 (BF16 u~ = 0). Both pipelines take the same form, so they give the same bits.
template <typename T, int UM>
constexpr int rcp3() {
    return (std::is_same<T, __half>::value && UM == UM_FLUID) ? RCP_DIV : RCP_RN;
}

// Blocks of a persistent pipeline over the lattice's row segments: no more than are
// resident at once (work is split between warps up front), no more than there is work.
inline int pipeline_blocks(const StepArgs3& a, int seg, int warps, int full) {
    const int64_t segs = (a.nx + seg - 1) / seg;
    const int64_t items = (int64_t)a.ny * a.nz * segs;
    const int64_t need = (items + warps - 1) / warps;
    return (int)(need < full ? need : full);
}

// The 8-node pipeline. Rows whose last segment is short enough for two or more to share an
// item (16 lanes or fewer) run the instance that packs them (TAILS). Measured at
// 264^3 (tails of 1 lane), FP16 u~ = q/rho / BF16 u~ = q/rho / FP16 u~ = 0: 0.66 / 0.71 /
// 0.71 of copy bandwidth against 0.52 / 0.52 / 0.60 with one row per item; at 384^3 (16
// lanes) 0.82 / 0.85 / 0.90 against 0.76 / 0.76 / 0.83. At 200^3 (25 lanes, one row per
// item either way) the packing instance was slower (0.56-0.59 against 0.71-0.80).
template <typename T, int UM, bool SUMS, bool TAILS>
cudaError_t launch_pipe3_t(const void* src, void* dst, const StepArgs3& a, cudaStream_t st,
                           double* part, int64_t* slots) {
    auto kernel = k_step3_pipe<T, UM, rcp3<T, UM>(), SUMS, TAILS>;
    static std::atomic<int> resident[kMaxDevicesOcc];
    int full = 0;
    cudaError_t e = resident_blocks(kernel, resident, kPipeWarps * 32, kPipeSmem,
                                    kPipeBlocksPerSm, &full);
    if (e != cudaSuccess) return e;
    const int64_t rows = (int64_t)a.ny * a.nz;  // the kernel's item count:
    int64_t items = rows * ((a.nx + kPipeSeg - 1) / kPipeSeg);
    if constexpr (TAILS) {
        const int rows_per_tail = 32 / ((a.nx % kPipeSeg) / kPipeNpl);
        items = rows * (a.nx / kPipeSeg) + (rows + rows_per_tail - 1) / rows_per_tail;
    }
    const int64_t need = (items + kPipeWarps - 1) / kPipeWarps;
    const int blocks = (int)(need < full ? need : full);
    if (slots) *slots = blocks;
    e = launch_pdl_smem(kernel, dim3(blocks), dim3(kPipeWarps * 32), kPipeSmem, st,
                        static_cast<const T*>(src), static_cast<T*>(dst), a, part);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T, int UM, bool SUMS = false>
cudaError_t launch_pipe3(const void* src, void* dst, const StepArgs3& a, cudaStream_t st,
                         double* part = nullptr, int64_t* slots = nullptr) {
    const int tail_lanes = (a.nx % kPipeSeg) / kPipeNpl;
    return tail_lanes == 0 || tail_lanes > 16
               ? launch_pipe3_t<T, UM, SUMS, false>(src, dst, a, st, part, slots)
               : launch_pipe3_t<T, UM, SUMS, true>(src, dst, a, st, part, slots);
}

template <typename T, int UM>
cudaError_t launch_pipe_pairs(const void* src, void* dst, const StepArgs3& a,
                              cudaStream_t st) {
    using C = PipePairs;
    auto kernel = k_step3_pipe_pairs<T, UM, rcp3<T, UM>()>;
    static std::atomic<int> resident[kMaxDevicesOcc];
    int full = 0;
    cudaError_t e = resident_blocks(kernel, resident, C::kWarps * 32, C::kSmem,
                                    C::kBlocksPerSm, &full);
    if (e != cudaSuccess) return e;
    const int blocks = pipeline_blocks(a, C::kSeg, C::kWarps, full);
    e = launch_pdl_smem(kernel, dim3(blocks), dim3(C::kWarps * 32), C::kSmem, st,
                        static_cast<const T*>(src), static_cast<T*>(dst), a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

inline bool rows_fit_31_bits(const StepArgs3& a) { return (int64_t)a.ny * a.nz < (1LL << 31); }

// The step with the conserved sums fused in: the FP32 4-node kernel or the 16-bit
// 8-node pipeline; *slots receives the number of block slots written.
template <typename T, int UM>
cudaError_t step3_sums(const void* src, void* dst, const StepArgs3& a, cudaStream_t st,
                       int nv, double* part, int64_t* slots) {
    if constexpr (sizeof(T) == 2) {
        if (nv == 8 && rows_fit_31_bits(a))
            return launch_pipe3<T, UM, true>(src, dst, a, st, part, slots);
    } else {
        if (nv == 4) {
            // as many blocks as are resident at once, planes (then rows) strided over them,
            // so that each block's FP64 reduction runs once (one row per block spent longer
            // in the reductions than in the step)
            auto kernel = k_step3<T, 4, UM, true>;
            const dim3 b = step3_block(a.nx, 4, false);
            static std::atomic<int> resident[kMaxDevicesOcc];
            int full = 0;
            cudaError_t e = resident_blocks(kernel, resident, (int)(b.x * b.y), 0, 32, &full);
            if (e != cudaSuccess) return e;
            dim3 g = step3_grid(a, 4, false);
            const int64_t plane_blocks = (int64_t)g.x * g.y;
            if (plane_blocks >= full) {
                const int64_t gy = full / g.x;
                g.y = (unsigned)(gy < 1 ? 1 : (gy < g.y ? gy : g.y));
                g.z = 1;
            } else {
                const int64_t gz = full / plane_blocks;
                g.z = (unsigned)(gz < g.z ? gz : g.z);
            }
            *slots = (int64_t)g.x * g.y * g.z;
            e = launch_pdl(kernel, g, b, st, static_cast<const T*>(src), static_cast<T*>(dst), a,
                           part);
            return e != cudaSuccess ? e : cudaGetLastError();
        }
    }
    return cudaErrorNotSupported;
}

template <typename T, int UM>
cudaError_t step3_nv(const void* src, void* dst, const StepArgs3& a, cudaStream_t st, int nv) {
    if constexpr (sizeof(T) == 2) {
        if (nv == 8 && rows_fit_31_bits(a)) return launch_pipe3<T, UM>(src, dst, a, st);
        if (nv == 4 && rows_fit_31_bits(a)) return launch_pipe_pairs<T, UM>(src, dst, a, st);
        if (nv == 4 || nv == 8) nv = 2;
    } else {
        if (nv == 4) return launch3(k_step3<T, 4, UM>, src, dst, a, st, nv);
    }
    if (nv == 1) return launch3(k_step3<T, 1, UM>, src, dst, a, st, nv);
    if (nv == 2) return launch3(k_step3<T, 2, UM>, src, dst, a, st, nv);
    return cudaErrorInvalidValue;
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

template <typename T>
cudaError_t step3_sums_um(const void* src, void* dst, const StepArgs3& a, cudaStream_t st,
                          int um, int nv, double* part, int64_t* slots) {
    switch (um) {
        case UM_ZERO: return step3_sums<T, UM_ZERO>(src, dst, a, st, nv, part, slots);
        case UM_FLUID: return step3_sums<T, UM_FLUID>(src, dst, a, st, nv, part, slots);
        case UM_FIELD: return step3_sums<T, UM_FIELD>(src, dst, a, st, nv, part, slots);
        default: return cudaErrorInvalidValue;
    }
}

// Block b adds slots [256 b, 256 b + 256) (8 doubles each, 5 used) into out[8 b].
__global__ void __launch_bounds__(kReduceThreads) k_sum_slots5(const double* __restrict__ part,
                                                               int64_t nslots,
                                                               double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * kReduceThreads + threadIdx.x;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < nslots) {
#pragma unroll
        for (int c = 0; c < 5; ++c) v[c] = part[8 * i + c];
    }
    block_sum5(v, out + 8 * (int64_t)blockIdx.x);
}

}  // namespace

bool step3_fuses_sums(int storage, int nv, int ny, int nz) {
    return storage == kStoreF32 ? nv == 4 : nv == 8 && (int64_t)ny * nz < (1LL << 31);
}

int64_t step3_sum_scratch(int storage, int nv, const StepArgs3& a) {
    int64_t slots = 0;
    if (storage == kStoreF32) {
        const dim3 g = step3_grid(a, nv, false);
        slots = (int64_t)g.x * g.y * g.z;
    } else {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return -1;
        slots = (int64_t)kPipeBlocksPerSm * sms;  // the pipeline's persistent grid
    }
    return 8 * slots + 8 * ((slots + kReduceThreads - 1) / kReduceThreads);
}

cudaError_t launch_step3_conserved(int storage, int um, int nv, const void* src, void* dst,
                                   const StepArgs3& a, cudaStream_t st, double lambda,
                                   double* partials, int64_t scratch, double* out) {
    if (!partials || !out || !step3_fuses_sums(storage, nv, a.ny, a.nz))
        return cudaErrorInvalidValue;
    int64_t slots = 0;
    cudaError_t e;
    switch (storage) {
        case kStoreF32: e = step3_sums_um<float>(src, dst, a, st, um, nv, partials, &slots); break;
        case kStoreF16: e = step3_sums_um<__half>(src, dst, a, st, um, nv, partials, &slots); break;
        case kStoreBF16:
            e = step3_sums_um<__nv_bfloat16>(src, dst, a, st, um, nv, partials, &slots);
            break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const int64_t mid = (slots + kReduceThreads - 1) / kReduceThreads;
    if (8 * slots + 8 * mid > scratch) return cudaErrorInvalidValue;  // cannot happen
    double* mids = partials + 8 * slots;
    k_sum_slots5<<<(unsigned)mid, kReduceThreads, 0, st>>>(partials, slots, mids);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double dn = (double)a.nx * (double)a.ny * (double)a.nz;
    k_conserved3_final<<<1, 256, 0, st>>>(mids, (int)mid, (double)a.ref.rho * dn,
                                          (double)a.ref.jx * dn, (double)a.ref.jy * dn,
                                          (double)a.ref.jz * dn, lambda, out);
    return cudaGetLastError();
}

int step3_vector_width(int storage, int nx) {
    // Measured fastest on GB300 at 256^3: 4-node packs for FP32, 8-node packs for 16-bit.
    const int widest = storage == kStoreF32 ? 4 : 8;
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
    const int g = grid_stride_blocks(n, 256);
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
    const int g = grid_stride_blocks(n, 256);
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

namespace {

// Packs of up to 8 bytes per plane, 4 bytes for BF16 (wider packs of 19 planes spill at the
// reduction's register budget), as wide as n, plane and the base address allow.
template <typename T>
void launch_conserved3_t(const void* src, int64_t n, int64_t plane, double* partials,
                         int nblk, cudaStream_t st) {
    const T* s = static_cast<const T*>(src);
    int nv = std::is_same<T, __nv_bfloat16>::value ? 2 : 8 / (int)sizeof(T);
    while (nv > 1 && !(n % nv == 0 && plane % nv == 0 &&
                       reinterpret_cast<uintptr_t>(src) % (nv * sizeof(T)) == 0))
        nv >>= 1;
    auto run = [&](auto kernel) { kernel<<<nblk, kReduceThreads, 0, st>>>(s, n, plane, partials); };
    if constexpr (std::is_same<T, __half>::value) {
        if (nv == 4) return run(k_conserved3_partial<T, 4>);
    }
    if (nv >= 2) return run(k_conserved3_partial<T, 2>);
    run(k_conserved3_partial<T, 1>);
}

}  // namespace

cudaError_t launch_conserved3(int storage, const void* src, int64_t n, int64_t plane,
                              const StoreRef3& ref, double lambda, double* partials, int nblk,
                              double* out, cudaStream_t st) {
    switch (storage) {
        case kStoreF32: launch_conserved3_t<float>(src, n, plane, partials, nblk, st); break;
        case kStoreF16: launch_conserved3_t<__half>(src, n, plane, partials, nblk, st); break;
        case kStoreBF16:
            launch_conserved3_t<__nv_bfloat16>(src, n, plane, partials, nblk, st);
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
