// Row loads for pull transport with vector packs (shared by the step and adjoint kernels).
//
// A thread owns NV consecutive nodes x0 .. x0+NV-1 of a row (x0 a multiple of NV). A plane
// whose population moved along +x (or is gathered from x-1) needs the element just left of
// the pack; one moving along -x needs the element just right of it. Those come from the
// neighbouring lane with a warp shuffle; lanes at a warp edge or at the end of the row load
// them directly, with the periodic wrap. Every lane of the warp must call these helpers
// (they shuffle with a full mask); inactive lanes (x0 >= nx) load nothing.
#pragma once

#include <cstring>

#include "d2q9.cuh"

namespace lbmrv {

constexpr unsigned kFullMask = 0xffffffffu;

template <typename T, int NV>
struct alignas(sizeof(T) * NV) Pack {
    T v[NV];
};

// Conversions between a pack and FP32 registers; 16-bit types go two at a time.
template <typename T, int NV>
struct PackCvt {
    __device__ __forceinline__ static void in(const Pack<T, NV>& pk, float out[NV]) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = to_f(pk.v[k]);
    }
    __device__ __forceinline__ static void out(const float v[NV], Pack<T, NV>& pk) {
#pragma unroll
        for (int k = 0; k < NV; ++k) pk.v[k] = from_f<T>(v[k]);
    }
};

template <int NV>
struct PackCvt<__half, NV> {
    static_assert(NV == 1 || NV % 2 == 0, "16-bit packs convert in pairs");
    __device__ __forceinline__ static void in(const Pack<__half, NV>& pk, float out[NV]) {
        if constexpr (NV == 1) {
            out[0] = __half2float(pk.v[0]);
        } else {
#pragma unroll
            for (int k = 0; k < NV; k += 2) {
                const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&pk.v[k]));
                out[k] = f.x;
                out[k + 1] = f.y;
            }
        }
    }
    __device__ __forceinline__ static void out(const float v[NV], Pack<__half, NV>& pk) {
        if constexpr (NV == 1) {
            pk.v[0] = __float2half_rn(v[0]);
        } else {
#pragma unroll
            for (int k = 0; k < NV; k += 2)
                *reinterpret_cast<__half2*>(&pk.v[k]) = __floats2half2_rn(v[k], v[k + 1]);
        }
    }
};

template <int NV>
struct PackCvt<__nv_bfloat16, NV> {
    static_assert(NV == 1 || NV % 2 == 0, "16-bit packs convert in pairs");
    __device__ __forceinline__ static void in(const Pack<__nv_bfloat16, NV>& pk, float out[NV]) {
        if constexpr (NV == 1) {
            out[0] = __uint_as_float((uint32_t)__bfloat16_as_ushort(pk.v[0]) << 16);
        } else {
#pragma unroll
            for (int k = 0; k < NV; k += 2) {
                // a BF16 value is the upper half of the FP32 value: two integer operations
                // (measured faster at 8192^2 than the conversion intrinsic, same bits)
                uint32_t w;
                memcpy(&w, &pk.v[k], 4);
                out[k] = __uint_as_float(w << 16);
                out[k + 1] = __uint_as_float(w & 0xffff0000u);
            }
        }
    }
    __device__ __forceinline__ static void out(const float v[NV], Pack<__nv_bfloat16, NV>& pk) {
        if constexpr (NV == 1) {
            pk.v[0] = __float2bfloat16_rn(v[0]);
        } else {
#pragma unroll
            for (int k = 0; k < NV; k += 2)
                *reinterpret_cast<__nv_bfloat162*>(&pk.v[k]) = __floats2bfloat162_rn(v[k], v[k + 1]);
        }
    }
};

template <typename T, int NV>
__device__ __forceinline__ void load_pack(const T* __restrict__ p, bool act, float out[NV]) {
    if (act) {
        const Pack<T, NV> pk = *reinterpret_cast<const Pack<T, NV>*>(p);
        PackCvt<T, NV>::in(pk, out);
    } else {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = 0.0f;
    }
}

// Row segment starting one element left of the pack: (prev, v0, ..., v_{NV-2}).
template <typename T, int NV>
__device__ __forceinline__ void load_from_left(const T* __restrict__ row, int x0, int xprev,
                                               bool act, bool edge, float out[NV]) {
    float v[NV];
    load_pack<T, NV>(row + x0, act, v);
    float prev = __shfl_up_sync(kFullMask, v[NV - 1], 1);
    if (edge && act) prev = to_f(row[xprev]);
    out[0] = prev;
#pragma unroll
    for (int k = 1; k < NV; ++k) out[k] = v[k - 1];
}

// Row segment starting one element right of the pack start: (v1, ..., v_{NV-1}, next).
template <typename T, int NV>
__device__ __forceinline__ void load_from_right(const T* __restrict__ row, int x0, int xnext,
                                                bool act, bool edge, float out[NV]) {
    float v[NV];
    load_pack<T, NV>(row + x0, act, v);
    float next = __shfl_down_sync(kFullMask, v[0], 1);
    if (edge && act) next = to_f(row[xnext]);
#pragma unroll
    for (int k = 0; k < NV - 1; ++k) out[k] = v[k + 1];
    out[NV - 1] = next;
}

// Lane geometry of a pack-per-thread row sweep.
struct PackLane {
    int x0, xprev, xnext;
    bool act, left_edge, right_edge;
};

template <int NV>
__device__ __forceinline__ PackLane pack_lane(int nx) {
    PackLane p;
    const int lane = threadIdx.x & 31;
    p.x0 = (blockIdx.x * blockDim.x + threadIdx.x) * NV;
    p.act = p.x0 < nx;
    p.left_edge = lane == 0;  // otherwise lane - 1 exists and is active
    p.right_edge = lane == 31 || p.x0 + NV >= nx;
    p.xprev = p.x0 == 0 ? nx - 1 : p.x0 - 1;
    p.xnext = p.x0 + NV >= nx ? 0 : p.x0 + NV;
    return p;
}

// Pre-relaxation populations of the pack: population j pulled from x - c_j (periodic),
// relation (transport). r0, rm, rp: offsets of rows y, y-1, y+1.
template <typename T, int NV>
__device__ __forceinline__ void pull_pack(const T* __restrict__ src, int64_t n, int64_t r0,
                                          int64_t rm, int64_t rp, const PackLane& p,
                                          float g[9][NV]) {
    load_pack<T, NV>(src + r0 + p.x0, p.act, g[0]);
    load_from_left<T, NV>(src + n + r0, p.x0, p.xprev, p.act, p.left_edge, g[1]);
    load_pack<T, NV>(src + 2 * n + rm + p.x0, p.act, g[2]);
    load_from_right<T, NV>(src + 3 * n + r0, p.x0, p.xnext, p.act, p.right_edge, g[3]);
    load_pack<T, NV>(src + 4 * n + rp + p.x0, p.act, g[4]);
    load_from_left<T, NV>(src + 5 * n + rm, p.x0, p.xprev, p.act, p.left_edge, g[5]);
    load_from_right<T, NV>(src + 6 * n + rm, p.x0, p.xnext, p.act, p.right_edge, g[6]);
    load_from_right<T, NV>(src + 7 * n + rp, p.x0, p.xnext, p.act, p.right_edge, g[7]);
    load_from_left<T, NV>(src + 8 * n + rp, p.x0, p.xprev, p.act, p.left_edge, g[8]);
}

// Transpose of the pull (a push read as a gather): element j of node x is taken from
// node x + c_j. Used by the adjoint.
template <typename T, int NV>
__device__ __forceinline__ void gather_pack(const T* __restrict__ src, int64_t n, int64_t r0,
                                            int64_t rm, int64_t rp, const PackLane& p,
                                            float g[9][NV]) {
    load_pack<T, NV>(src + r0 + p.x0, p.act, g[0]);
    load_from_right<T, NV>(src + n + r0, p.x0, p.xnext, p.act, p.right_edge, g[1]);
    load_pack<T, NV>(src + 2 * n + rp + p.x0, p.act, g[2]);
    load_from_left<T, NV>(src + 3 * n + r0, p.x0, p.xprev, p.act, p.left_edge, g[3]);
    load_pack<T, NV>(src + 4 * n + rm + p.x0, p.act, g[4]);
    load_from_right<T, NV>(src + 5 * n + rp, p.x0, p.xnext, p.act, p.right_edge, g[5]);
    load_from_left<T, NV>(src + 6 * n + rp, p.x0, p.xprev, p.act, p.left_edge, g[6]);
    load_from_left<T, NV>(src + 7 * n + rm, p.x0, p.xprev, p.act, p.left_edge, g[7]);
    load_from_right<T, NV>(src + 8 * n + rm, p.x0, p.xnext, p.act, p.right_edge, g[8]);
}

// ---- 16-bit packs kept in storage form: NV elements in NV/2 32-bit words, element 2i in
// the low half of word i. The one-element shifts of the x-moving planes are byte permutes;
// values are converted to FP32 only when a node pair is relaxed.
template <int NV>
struct alignas(2 * NV) Raw16 {
    uint32_t w[NV / 2];
};

template <int NV>
__device__ __forceinline__ void load_raw16(const void* p, bool act, uint32_t out[NV / 2]) {
    if (act) {
        const Raw16<NV> r = *reinterpret_cast<const Raw16<NV>*>(p);
#pragma unroll
        for (int i = 0; i < NV / 2; ++i) out[i] = r.w[i];
    } else {
#pragma unroll
        for (int i = 0; i < NV / 2; ++i) out[i] = 0u;
    }
}

__device__ __forceinline__ uint32_t load_elem16(const void* p) {
    return *reinterpret_cast<const unsigned short*>(p);
}

// Elements (prev, v0, ..., v_{NV-2}) of a row, in storage form.
template <typename T, int NV>
__device__ __forceinline__ void load_raw16_from_left(const T* __restrict__ row, int x0, int xprev,
                                                     bool act, bool edge, uint32_t out[NV / 2]) {
    uint32_t v[NV / 2];
    load_raw16<NV>(row + x0, act, v);
    uint32_t prev = __shfl_up_sync(kFullMask, v[NV / 2 - 1], 1) >> 16;
    if (edge && act) prev = load_elem16(row + xprev);
    out[0] = __byte_perm(prev, v[0], 0x5410);
#pragma unroll
    for (int i = 1; i < NV / 2; ++i) out[i] = __byte_perm(v[i - 1], v[i], 0x5432);
}

// Elements (v1, ..., v_{NV-1}, next) of a row, in storage form.
template <typename T, int NV>
__device__ __forceinline__ void load_raw16_from_right(const T* __restrict__ row, int x0, int xnext,
                                                      bool act, bool edge, uint32_t out[NV / 2]) {
    uint32_t v[NV / 2];
    load_raw16<NV>(row + x0, act, v);
    uint32_t next = __shfl_down_sync(kFullMask, v[0], 1);
    if (edge && act) next = load_elem16(row + xnext);
#pragma unroll
    for (int i = 0; i < NV / 2 - 1; ++i) out[i] = __byte_perm(v[i], v[i + 1], 0x5432);
    out[NV / 2 - 1] = __byte_perm(v[NV / 2 - 1], next, 0x5432);
}

template <int NV>
__device__ __forceinline__ void store_raw16(void* p, const uint32_t w[NV / 2]) {
    Raw16<NV> r;
#pragma unroll
    for (int i = 0; i < NV / 2; ++i) r.w[i] = w[i];
    *reinterpret_cast<Raw16<NV>*>(p) = r;
}

// A word of two 16-bit values <-> two floats (low half first).
template <typename T>
struct Cvt16;

template <>
struct Cvt16<__half> {
    __device__ __forceinline__ static float2 unpack(uint32_t w) {
        __half2 h;
        memcpy(&h, &w, 4);
        return __half22float2(h);
    }
    // element `hi` (0: low half, 1: high half) of a word, and the word with it replaced
    __device__ __forceinline__ static float get(uint32_t w, int hi) {
        const unsigned short b = (unsigned short)(hi ? w >> 16 : w & 0xffffu);
        return __half2float(__ushort_as_half(b));
    }
    __device__ __forceinline__ static uint32_t put(uint32_t w, int hi, float v) {
        const uint32_t b = __half_as_ushort(__float2half_rn(v));
        return hi ? __byte_perm(w, b, 0x5410) : __byte_perm(w, b, 0x3254);
    }
    __device__ __forceinline__ static uint32_t pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};

template <>
struct Cvt16<__nv_bfloat16> {
    __device__ __forceinline__ static float2 unpack(uint32_t w) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    __device__ __forceinline__ static float get(uint32_t w, int hi) {
        return __uint_as_float(hi ? (w & 0xffff0000u) : (w << 16));
    }
    __device__ __forceinline__ static uint32_t put(uint32_t w, int hi, float v) {
        const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        return hi ? __byte_perm(w, b, 0x5410) : __byte_perm(w, b, 0x3254);
    }
    __device__ __forceinline__ static uint32_t pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        uint32_t w;
        memcpy(&w, &h, 4);
        return w;
    }
};

template <typename T, int NV>
__device__ __forceinline__ void store_pack(T* __restrict__ p, const float v[NV]) {
    Pack<T, NV> pk;
    PackCvt<T, NV>::out(v, pk);
    *reinterpret_cast<Pack<T, NV>*>(p) = pk;
}

}  // namespace lbmrv
