// Two FP32 values in one 64-bit register pair, operated on by the packed FP32 instructions
// of sm_100-family GPUs (add / sub / mul / fma .rn .f32x2). Each lane is rounded exactly as
// the scalar .rn instruction would round it, so a formula evaluated on F2 gives, lane by
// lane, the bits of the same formula evaluated on float with the same operation order and
// the same explicit fused multiply-adds. Used to relax two nodes per instruction.
#pragma once

#include <cuda_runtime.h>

namespace lbmrv {

struct F2 {
    unsigned long long v;
    __device__ __forceinline__ F2() {}
    // Both lanes equal to a.
    __device__ __forceinline__ F2(float a) { asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(a)); }
};

__device__ __forceinline__ F2 pack2(float a, float b) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void unpack2(F2 x, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}

__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

// a * b + c with one rounding per lane.
__device__ __forceinline__ F2 fma_(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// One FP32 value whose arithmetic the compiler never contracts into fused multiply-adds
// (each operator is a single .rn operation): the scalar counterpart of F2 for code written
// once for both.
struct F1 {
    float v;
    __device__ __forceinline__ F1() {}
    __device__ __forceinline__ F1(float a) : v(a) {}
};

__device__ __forceinline__ F1 operator+(F1 a, F1 b) { return F1(__fadd_rn(a.v, b.v)); }
__device__ __forceinline__ F1 operator-(F1 a, F1 b) { return F1(__fsub_rn(a.v, b.v)); }
__device__ __forceinline__ F1 operator*(F1 a, F1 b) { return F1(__fmul_rn(a.v, b.v)); }
__device__ __forceinline__ F1 fma_(F1 a, F1 b, F1 c) { return F1(__fmaf_rn(a.v, b.v, c.v)); }

}  // namespace lbmrv
