// Internal: the handle behind lbmrv_t and helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "launch.h"
#include "lbmrv.h"

struct lbmrv_s {
    int lattice = LBMRV_D2Q9;
    int umode = LBMRV_UT_ZERO;
    int storage = LBMRV_FP32;
    int device = 0;
    int width = 0;  // 0: automatic kernel choice; else nodes per thread of the fused step
    int64_t nx = 0, ny = 0, n = 0;
    double lambda = 1.0, rho_ref = 0.0;
    double s[9] = {0};
    cudaStream_t stream = nullptr;
    void* f[2] = {nullptr, nullptr};
    bool owns_f = false;
    int cur = 0;
    int64_t t = 0;
    const float* ut0 = nullptr;
    double amp = 0.0, period = 0.0;
    double* red = nullptr;  // reduction scratch: 4 * red_blocks partials + 4 results
    int red_blocks = 0;
    // last lbmrv_forward_checkpointed: the adjoint must match it
    bool ckpt_valid = false;
    int64_t ckpt_n = 0, ckpt_seg = 0, ckpt_t0 = 0;
    const void* ckpt_ws = nullptr;
    char err[320] = {0};
};

namespace lbmrv {

int fail(lbmrv_t h, int code, const char* fmt, ...);
const char* last_create_error();

inline int cuda_fail(lbmrv_t h, cudaError_t e, const char* what) {
    return fail(h, LBMRV_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

inline int64_t elem_size(int storage) {
    switch (storage) {
        case LBMRV_FP32: return 4;
        case LBMRV_FP16:
        case LBMRV_BF16: return 2;
        default: return -1;
    }
}

// Make the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

// Time factor of the prescribed field at time index t: cos(2 pi t / P), or 1 if P <= 0.
inline double time_factor(const lbmrv_s* h, int64_t t) {
    return h->period > 0.0 ? std::cos(2.0 * M_PI * (double)t / h->period) : 1.0;
}

// Arguments of the relaxation at time index t.
inline StepArgs make_args(const lbmrv_s* h, int64_t t) {
    StepArgs a;
    a.nx = (int)h->nx;
    a.ny = (int)h->ny;
    a.s = Rates{(float)h->s[3], (float)h->s[4], (float)h->s[5],
                (float)h->s[6], (float)h->s[7], (float)h->s[8]};
    a.rho_ref = (float)h->rho_ref;
    a.amp_t = (float)(h->amp * time_factor(h, t) / h->lambda);
    a.two_over_nx = (float)(2.0 / (double)h->nx);
    a.two_over_ny = (float)(2.0 / (double)h->ny);
    a.ut0 = h->ut0;
    for (int k = 0; k < 8; ++k) {
        a.sin_k[k] = (float)std::sin(2.0 * M_PI * (double)k / (double)h->nx);
        a.cos_k[k] = (float)std::cos(2.0 * M_PI * (double)k / (double)h->nx);
    }
    return a;
}

inline int kernel_mode(const lbmrv_s* h) {
    if (h->umode == LBMRV_UT_ZERO) return UM_ZERO;
    if (h->umode == LBMRV_UT_FLUID) return UM_FLUID;
    return h->ut0 ? UM_FIELD : UM_ANALYTIC;
}

// Widest usable pack for the fused step on buffers a, b (1: one node per thread).
int choose_width(const lbmrv_s* h, const void* a, const void* b);

}  // namespace lbmrv
