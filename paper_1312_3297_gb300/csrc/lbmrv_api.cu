// C ABI of the lbmrv library (declarations and contracts in include/lbmrv.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "handle.h"
#include "launch.h"
#include "lbmrv.h"

using namespace lbmrv;

namespace lbmrv {

namespace {
thread_local char g_create_err[320] = {0};
}  // namespace

int fail(lbmrv_t h, int code, const char* fmt, ...) {
    char* buf = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 320, fmt, ap);
    va_end(ap);
    return code;
}

int choose_width(const lbmrv_s* h, const void* a, const void* b) {
    if (h->width > 0) return h->width;
    const int nv = step_vector_width(h->storage, (int)h->nx);
    const size_t align = (size_t)(nv * elem_size(h->storage));
    if (nv > 1 && ((reinterpret_cast<uintptr_t>(a) % align) != 0 ||
                   (reinterpret_cast<uintptr_t>(b) % align) != 0))
        return 1;
    return nv;
}

const char* last_create_error() { return g_create_err; }

}  // namespace lbmrv

extern "C" {

int lbmrv_version(void) { return LBMRV_VERSION; }

int64_t lbmrv_state_bytes(int lattice, const int64_t dims[3], int storage) {
    if (lattice != LBMRV_D2Q9 || !dims || dims[0] < 1 || dims[1] < 1) return -1;
    const int64_t es = elem_size(storage);
    if (es < 0) return -1;
    return 9 * dims[0] * dims[1] * es;
}

int lbmrv_create(lbmrv_t* out, int lattice, const int64_t dims[3], double lambda,
                 const double* s, int umode, int storage, double rho_ref, void* stream,
                 void* f_a_dev, void* f_b_dev) {
    if (!out) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: out is NULL");
    *out = nullptr;
    if (lattice == LBMRV_D3Q19)
        return fail(nullptr, LBMRV_E_UNSUPPORTED, "lbmrv_create: D3Q19 is not built");
    if (lattice != LBMRV_D2Q9) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: bad lattice");
    if (!dims || dims[0] < 1 || dims[1] < 1 || (dims[2] != 1 && dims[2] != 0))
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: dims must be {nx>=1, ny>=1, 1}");
    if (dims[0] * dims[1] >= (int64_t(1) << 31) || dims[0] > (1 << 30) || dims[1] > (1 << 30))
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: nx*ny must be below 2^31");
    if (!(lambda > 0.0) || !std::isfinite(lambda))
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: lambda must be finite and > 0");
    if (!s) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: s is NULL");
    for (int k = 0; k < 3; ++k)
        if (s[k] != 0.0)
            return fail(nullptr, LBMRV_E_INVAL,
                        "lbmrv_create: s[%d] must be 0 (conserved moment)", k);
    for (int k = 3; k < 9; ++k)
        if (!std::isfinite(s[k]))
            return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: s[%d] is not finite", k);
    if (umode < LBMRV_UT_ZERO || umode > LBMRV_UT_PRESCRIBED)
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: bad u~ mode %d", umode);
    if (elem_size(storage) < 0)
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: bad storage %d", storage);
    if (!std::isfinite(rho_ref))
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: rho_ref is not finite");
    if ((f_a_dev == nullptr) != (f_b_dev == nullptr) || (f_a_dev && f_a_dev == f_b_dev))
        return fail(nullptr, LBMRV_E_INVAL,
                    "lbmrv_create: pass two distinct state buffers or none");
    if ((f_a_dev && reinterpret_cast<uintptr_t>(f_a_dev) % 16) ||
        (f_b_dev && reinterpret_cast<uintptr_t>(f_b_dev) % 16))
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: state buffers must be 16-byte aligned");

    lbmrv_s* h = new (std::nothrow) lbmrv_s();
    if (!h) return fail(nullptr, LBMRV_E_NOMEM, "lbmrv_create: host allocation failed");
    h->lattice = lattice;
    h->umode = umode;
    h->storage = storage;
    h->nx = dims[0];
    h->ny = dims[1];
    h->n = dims[0] * dims[1];
    h->lambda = lambda;
    h->rho_ref = rho_ref;
    for (int k = 0; k < 9; ++k) h->s[k] = s[k];
    h->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, LBMRV_E_CUDA, "lbmrv_create: cudaGetDevice: %s",
                    cudaGetErrorString(e));
    }
    const size_t bytes = (size_t)lbmrv_state_bytes(lattice, dims, storage);
    if (f_a_dev) {
        h->f[0] = f_a_dev;
        h->f[1] = f_b_dev;
    } else {
        h->owns_f = true;
        if (cudaMalloc(&h->f[0], bytes) != cudaSuccess ||
            cudaMalloc(&h->f[1], bytes) != cudaSuccess) {
            cudaGetLastError();
            if (h->f[0]) cudaFree(h->f[0]);
            delete h;
            return fail(nullptr, LBMRV_E_NOMEM, "lbmrv_create: cudaMalloc of 2 x %zu bytes failed",
                        bytes);
        }
    }
    h->red_blocks = conserved_blocks(h->n);
    if (cudaMalloc(&h->red, sizeof(double) * (4 * (size_t)h->red_blocks + 4)) != cudaSuccess) {
        cudaGetLastError();
        if (h->owns_f) {
            cudaFree(h->f[0]);
            cudaFree(h->f[1]);
        }
        delete h;
        return fail(nullptr, LBMRV_E_NOMEM, "lbmrv_create: reduction buffer allocation failed");
    }
    *out = h;
    return LBMRV_OK;
}

int lbmrv_destroy(lbmrv_t h) {
    if (!h) return LBMRV_OK;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->owns_f) {
        cudaFree(h->f[0]);
        cudaFree(h->f[1]);
    }
    cudaFree(h->red);
    delete h;
    return LBMRV_OK;
}

const char* lbmrv_last_error(lbmrv_t h) { return h ? h->err : last_create_error(); }

int lbmrv_set_stream(lbmrv_t h, void* stream) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_set_stream: NULL handle");
    h->stream = static_cast<cudaStream_t>(stream);
    return LBMRV_OK;
}

int lbmrv_set_kernel_width(lbmrv_t h, int nodes_per_thread) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_set_kernel_width: NULL handle");
    const int w = nodes_per_thread;
    if (w == 0 || w == 1) {
        h->width = w;
        return LBMRV_OK;
    }
    const int widest = h->storage == LBMRV_FP32 ? 4 : 8;
    if ((w != 2 && w != 4 && w != 8) || w > widest || h->nx % w != 0)
        return fail(h, LBMRV_E_INVAL,
                    "lbmrv_set_kernel_width: %d must be 0, 1 or a pack width (<= %d) dividing nx",
                    w, widest);
    const size_t align = (size_t)(w * elem_size(h->storage));
    if (reinterpret_cast<uintptr_t>(h->f[0]) % align || reinterpret_cast<uintptr_t>(h->f[1]) % align)
        return fail(h, LBMRV_E_INVAL, "lbmrv_set_kernel_width: buffers not aligned for %d", w);
    h->width = w;
    return LBMRV_OK;
}

int lbmrv_set_rates(lbmrv_t h, const double* s) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_set_rates: NULL handle");
    if (!s) return fail(h, LBMRV_E_INVAL, "lbmrv_set_rates: s is NULL");
    for (int k = 0; k < 3; ++k)
        if (s[k] != 0.0)
            return fail(h, LBMRV_E_INVAL, "lbmrv_set_rates: s[%d] must be 0 (conserved moment)", k);
    for (int k = 3; k < 9; ++k)
        if (!std::isfinite(s[k]))
            return fail(h, LBMRV_E_INVAL, "lbmrv_set_rates: s[%d] is not finite", k);
    for (int k = 0; k < 9; ++k) h->s[k] = s[k];
    return LBMRV_OK;
}

int lbmrv_set_utilde(lbmrv_t h, const float* ut0_dev, double amplitude, double period) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_set_utilde: NULL handle");
    if (!std::isfinite(amplitude) || !std::isfinite(period))
        return fail(h, LBMRV_E_INVAL, "lbmrv_set_utilde: amplitude and period must be finite");
    h->ut0 = ut0_dev;
    h->amp = amplitude;
    h->period = period;
    return LBMRV_OK;
}

int lbmrv_init_equilibrium(lbmrv_t h, const float* rho_dev, const float* u_dev) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_init_equilibrium: NULL handle");
    if (!u_dev) return fail(h, LBMRV_E_INVAL, "lbmrv_init_equilibrium: u is NULL");
    DeviceGuard g(h->device);
    cudaError_t e = launch_init_eq(h->storage, h->f[h->cur], rho_dev, u_dev, h->n,
                                   (float)h->rho_ref, (float)(1.0 / h->lambda), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_init_equilibrium");
    h->t = 0;
    return LBMRV_OK;
}

int lbmrv_init_equilibrium_host(lbmrv_t h, const float* rho_host, const float* u_host) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_init_equilibrium_host: NULL handle");
    if (!u_host) return fail(h, LBMRV_E_INVAL, "lbmrv_init_equilibrium_host: u is NULL");
    DeviceGuard g(h->device);
    // Staging: 3 floats per node fit in the non-current state buffer (>= 18 bytes per node).
    float* stage = static_cast<float*>(h->f[1 - h->cur]);
    const size_t nb = sizeof(float) * (size_t)h->n;
    cudaError_t e = cudaSuccess;
    if (rho_host) e = cudaMemcpyAsync(stage, rho_host, nb, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(stage + h->n, u_host, 2 * nb, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_init_equilibrium_host: copy");
    e = launch_init_eq(h->storage, h->f[h->cur], rho_host ? stage : nullptr, stage + h->n, h->n,
                       (float)h->rho_ref, (float)(1.0 / h->lambda), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_init_equilibrium_host");
    h->t = 0;
    return LBMRV_OK;
}

int lbmrv_step(lbmrv_t h, int64_t n) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_step: NULL handle");
    if (n < 0) return fail(h, LBMRV_E_INVAL, "lbmrv_step: n < 0");
    DeviceGuard g(h->device);
    const int um = kernel_mode(h);
    const int nv = choose_width(h, h->f[0], h->f[1]);
    for (int64_t k = 0; k < n; ++k) {
        const StepArgs a = make_args(h, h->t + 1);
        cudaError_t e = launch_step(h->storage, um, nv, h->f[h->cur], h->f[1 - h->cur], a,
                                    h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_step");
        h->cur = 1 - h->cur;
        h->t += 1;
    }
    return LBMRV_OK;
}

int lbmrv_moments(lbmrv_t h, float* rho_dev, float* u_dev) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_moments: NULL handle");
    DeviceGuard g(h->device);
    cudaError_t e = launch_moments(h->storage, h->f[h->cur], rho_dev, u_dev, h->n,
                                   (float)h->rho_ref, (float)h->lambda, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_moments");
    return LBMRV_OK;
}

int lbmrv_moments_host(lbmrv_t h, float* rho_host, float* u_host) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_moments_host: NULL handle");
    DeviceGuard g(h->device);
    float* stage = static_cast<float*>(h->f[1 - h->cur]);
    const size_t nb = sizeof(float) * (size_t)h->n;
    cudaError_t e = launch_moments(h->storage, h->f[h->cur], stage, stage + h->n, h->n,
                                   (float)h->rho_ref, (float)h->lambda, h->stream);
    if (e == cudaSuccess && rho_host)
        e = cudaMemcpyAsync(rho_host, stage, nb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && u_host)
        e = cudaMemcpyAsync(u_host, stage + h->n, 2 * nb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_moments_host");
    return LBMRV_OK;
}

int lbmrv_conserved(lbmrv_t h, double out_host[4]) {
    if (!h || !out_host) return fail(h, LBMRV_E_INVAL, "lbmrv_conserved: NULL argument");
    DeviceGuard g(h->device);
    double* res = h->red + 4 * (size_t)h->red_blocks;
    cudaError_t e = launch_conserved(h->storage, h->f[h->cur], h->n, h->rho_ref, h->lambda,
                                     h->red, h->red_blocks, res, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out_host, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_conserved");
    if (out_host[3] > 0.0)
        return fail(h, LBMRV_E_NONFINITE, "lbmrv_conserved: %.0f nodes hold non-finite values",
                    out_host[3]);
    return LBMRV_OK;
}

int lbmrv_get_state(lbmrv_t h, void* dst_dev) {
    if (!h || !dst_dev) return fail(h, LBMRV_E_INVAL, "lbmrv_get_state: NULL argument");
    DeviceGuard g(h->device);
    const size_t bytes = (size_t)(9 * h->n * elem_size(h->storage));
    cudaError_t e = cudaMemcpyAsync(dst_dev, h->f[h->cur], bytes, cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_get_state");
    return LBMRV_OK;
}

int lbmrv_set_state(lbmrv_t h, const void* src_dev, int64_t t) {
    if (!h || !src_dev) return fail(h, LBMRV_E_INVAL, "lbmrv_set_state: NULL argument");
    if (t < 0) return fail(h, LBMRV_E_INVAL, "lbmrv_set_state: t < 0");
    DeviceGuard g(h->device);
    const size_t bytes = (size_t)(9 * h->n * elem_size(h->storage));
    cudaError_t e = cudaMemcpyAsync(h->f[h->cur], src_dev, bytes, cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_set_state");
    h->t = t;
    return LBMRV_OK;
}

int lbmrv_state_ptr(lbmrv_t h, void** ptr_out) {
    if (!h || !ptr_out) return fail(h, LBMRV_E_INVAL, "lbmrv_state_ptr: NULL argument");
    *ptr_out = h->f[h->cur];
    return LBMRV_OK;
}

int64_t lbmrv_time(lbmrv_t h) { return h ? h->t : -1; }

}  // extern "C"
