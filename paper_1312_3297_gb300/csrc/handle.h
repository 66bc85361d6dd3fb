// Internal: the handle behind lbmrv_t and helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "d3q19.cuh"
#include "launch.h"
#include "lbmrv.h"

struct lbmrv_s {
    int lattice = LBMRV_D2Q9;
    int q = 9;       // populations per node
    int dim = 2;     // spatial dimensions
    int basis = 0;   // D2Q9 moment basis: 0 orthogonal set of relation (mom), 1 Geier's set
    int umode = LBMRV_UT_ZERO;
    int storage = LBMRV_FP32;
    int device = 0;
    int width = 0;  // 0: automatic kernel choice; else nodes per thread of the fused step
    int64_t nx = 0, ny = 0, nz = 1, n = 0;
    double lambda = 1.0, rho_ref = 0.0;
    double u_ref[3] = {0.0, 0.0, 0.0};  // reference velocity of the stored deviations
    bool ref_auto = true;  // u_ref := mean flow of the fields of each init_equilibrium
    // Slab of a larger periodic lattice (lbmrv_set_slab): layers (D2Q9 rows, D3Q19 z-planes)
    // 1 .. m-2 are the global layers slab_first .. slab_first + m - 3 of slab_extent; layers
    // 0 and m-1 are halo copies of the neighbouring slabs' edge layers.
    bool slab = false;
    int64_t slab_first = 0, slab_extent = 0;
    double s[19] = {0};
    cudaStream_t stream = nullptr;
    void* f[2] = {nullptr, nullptr};
    bool owns_f = false;
    int cur = 0;
    int64_t t = 0;
    const float* ut0 = nullptr;
    double amp = 0.0, period = 0.0;
    double* red = nullptr;   // reduction scratch: 8 * red_blocks partials + 8 results
    int red_blocks = 0;
    double* fused = nullptr;  // partials of the step with fused sums, + 4 results (lazy)
    int64_t fused_doubles = 0;
    float* sin_x = nullptr;  // sin(2 pi x / nx) table of the analytic prescribed field
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

inline size_t state_bytes(const lbmrv_s* h) {
    return (size_t)(h->q * h->n * elem_size(h->storage));
}

// Nodes of one layer (the unit a slab is cut into) and the number of layers.
inline int64_t layer_size(const lbmrv_s* h) { return h->dim == 2 ? h->nx : h->nx * h->ny; }
inline int64_t layer_count(const lbmrv_s* h) { return h->dim == 2 ? h->ny : h->nz; }

// The nodes the handle owns: the whole lattice, or a slab's interior layers (first node and
// count; the state's planes stay h->n elements apart).
inline int64_t owned_first(const lbmrv_s* h) { return h->slab ? layer_size(h) : 0; }
inline int64_t owned_count(const lbmrv_s* h) {
    return h->slab ? h->n - 2 * layer_size(h) : h->n;
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

// Reference state of the stored deviations, lattice units (see StoreRef in d2q9.cuh).
inline StoreRef store_ref(const lbmrv_s* h) {
    const double r = h->rho_ref;
    const double ux = h->u_ref[0] / h->lambda, uy = h->u_ref[1] / h->lambda;
    const double uu = ux * ux + uy * uy;
    StoreRef ref;
    ref.rho = (float)r;
    ref.jx = (float)(r * ux);
    ref.jy = (float)(r * uy);
    ref.ux = (float)ux;
    ref.uy = (float)uy;
    if (h->basis == 0) {
        ref.c[0] = (float)(3.0 * r * uu);             // e
        ref.c[1] = (float)(r * (ux * ux - uy * uy));  // p_xx
        ref.c[2] = (float)(r * ux * uy);              // p_xy
        ref.c[3] = (float)(-r * ux);                  // q_x (3rd order)
        ref.c[4] = (float)(-r * uy);                  // q_y (3rd order)
        ref.c[5] = (float)(-3.0 * r * uu);            // eps
    } else {  // Geier basis, product equilibrium: monomials XX, YY, XY, XYY, YXX, XXYY
        ref.c[0] = (float)(r * ux * ux);
        ref.c[1] = (float)(r * uy * uy);
        ref.c[2] = (float)(r * ux * uy);
        ref.c[3] = (float)(r * ux * uy * uy);
        ref.c[4] = (float)(r * uy * ux * ux);
        ref.c[5] = (float)(r * uu / 3.0 + r * ux * ux * uy * uy);
    }
    return ref;
}

// D3Q19 reference state: q terms are Q_k(j_ref)/rho_ref of the equilibrium moments.
inline StoreRef3 store_ref3(const lbmrv_s* h) {
    const double r = h->rho_ref;
    const double ux = h->u_ref[0] / h->lambda, uy = h->u_ref[1] / h->lambda,
                 uz = h->u_ref[2] / h->lambda;
    StoreRef3 ref;
    ref.rho = (float)r;
    ref.jx = (float)(r * ux);
    ref.jy = (float)(r * uy);
    ref.jz = (float)(r * uz);
    ref.ux = (float)ux;
    ref.uy = (float)uy;
    ref.uz = (float)uz;
    ref.qxx = (float)(r * ux * ux);
    ref.qyy = (float)(r * uy * uy);
    ref.qzz = (float)(r * uz * uz);
    ref.qxy = (float)(r * ux * uy);
    ref.qxz = (float)(r * ux * uz);
    ref.qyz = (float)(r * uy * uz);
    ref.qxxyy = (float)(r * ((ux * ux + uy * uy) / 3.0 - uz * uz / 6.0));
    ref.qxxzz = (float)(r * ((ux * ux + uz * uz) / 3.0 - uy * uy / 6.0));
    ref.qyyzz = (float)(r * ((uy * uy + uz * uz) / 3.0 - ux * ux / 6.0));
    return ref;
}

// Arguments of the D2Q9 relaxation at time index t.
inline StepArgs make_args(const lbmrv_s* h, int64_t t) {
    StepArgs a;
    a.nx = (int)h->nx;
    a.ny = (int)h->ny;
    a.s = Rates{(float)h->s[3], (float)h->s[4], (float)h->s[5],
                (float)h->s[6], (float)h->s[7], (float)h->s[8]};
    a.ref = store_ref(h);
    a.amp_t = (float)(h->amp * time_factor(h, t) / h->lambda);
    a.two_over_nx = (float)(2.0 / (double)h->nx);
    // a slab evaluates the analytic field at the global row: y + y_off of slab_extent rows
    a.two_over_ny = (float)(2.0 / (double)(h->slab ? h->slab_extent : h->ny));
    a.y_off = h->slab ? (int)(h->slab_first - 1) : 0;
    a.ut0 = h->ut0;
    a.sin_x = h->sin_x;
    return a;
}

// Arguments of the D3Q19 relaxation at time index t.
inline StepArgs3 make_args3(const lbmrv_s* h, int64_t t) {
    StepArgs3 a;
    a.nx = (int)h->nx;
    a.ny = (int)h->ny;
    a.nz = (int)h->nz;
    const double* s = h->s;
    a.s = Rates3{(float)s[4],  (float)s[5],  (float)s[6],  (float)s[7],  (float)s[8],
                 (float)s[9],  (float)s[10], (float)s[11], (float)s[12], (float)s[13],
                 (float)s[14], (float)s[15], (float)s[16], (float)s[17], (float)s[18]};
    a.ref = store_ref3(h);
    a.amp_t = (float)(h->amp * time_factor(h, t) / h->lambda);
    a.ut0 = h->ut0;
    return a;
}

inline int kernel_mode(const lbmrv_s* h) {
    if (h->umode == LBMRV_UT_ZERO) return UM_ZERO;
    if (h->umode == LBMRV_UT_FLUID) return UM_FLUID;
    return h->ut0 ? UM_FIELD : UM_ANALYTIC;
}

// Widest usable pack for the fused step on buffers a, b (1: one node per thread).
int choose_width(const lbmrv_s* h, const void* a, const void* b);

// One fused step src -> dst at time index t, for the handle's lattice.
cudaError_t launch_handle_step(const lbmrv_s* h, int nv, const void* src, void* dst, int64_t t);

}  // namespace lbmrv
