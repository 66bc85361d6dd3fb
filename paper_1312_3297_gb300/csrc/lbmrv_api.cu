// C ABI of the lbmrv library (declarations and contracts in include/lbmrv.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "handle.h"
#include "launch.h"
#include "lbmrv.h"
#include "trace.h"

using namespace lbmrv;

namespace lbmrv {

namespace {
thread_local char g_create_err[320] = {0};

int lattice_q(int lattice) {
    if (lattice == LBMRV_D2Q9 || lattice == LBMRV_D2Q9_CASCADED) return 9;
    return lattice == LBMRV_D3Q19 ? 19 : -1;
}
int lattice_dim(int lattice) { return lattice == LBMRV_D3Q19 ? 3 : 2; }

// Validation shared by lbmrv_create and lbmrv_set_rates: conserved rates are 0 (Section
// 1.1: 1 + d conserved moments), the others finite.
int check_rates(lbmrv_t h, int lattice, const double* s, const char* who) {
    const int q = lattice_q(lattice), nc = 1 + lattice_dim(lattice);
    if (!s) return fail(h, LBMRV_E_INVAL, "%s: s is NULL", who);
    for (int k = 0; k < nc; ++k)
        if (s[k] != 0.0)
            return fail(h, LBMRV_E_INVAL, "%s: s[%d] must be 0 (conserved moment)", who, k);
    for (int k = nc; k < q; ++k)
        if (!std::isfinite(s[k])) return fail(h, LBMRV_E_INVAL, "%s: s[%d] is not finite", who, k);
    return LBMRV_OK;
}

// A rate outside (0, 2) is accepted, with a warning in the last-error message: the
// relaxation multiplies a moment's distance to equilibrium by 1 - s per step, so s = 0 or
// 2 leaves that moment undamped and s < 0 or s > 2 amplifies it (Section 1.1).
void warn_rates(lbmrv_t h, int lattice, const double* s, const char* who) {
    const int q = lattice_q(lattice), nc = 1 + lattice_dim(lattice);
    for (int k = nc; k < q; ++k)
        if (!(s[k] > 0.0 && s[k] < 2.0)) {
            fail(h, LBMRV_OK, "%s: warning: s[%d] = %g is outside (0, 2); that moment is %s",
                 who, k, s[k], (s[k] == 0.0 || s[k] == 2.0) ? "not damped" : "amplified");
            return;
        }
}
}  // namespace

// The automatic reference velocity: U_ref = sum rho u / sum rho over the fields an
// equilibrium is about to be built from (an FP64 device reduction, read back on the host).
// Total mass and momentum are invariants of the periodic scheme (relation (rhoq) summed
// over the lattice: relaxation conserves them at every node, transport moves them), so
// U_ref stays the mean flow of the whole run. Synchronises the handle's stream.
int apply_auto_reference(lbmrv_t h, const float* rho, const float* u, const char* who) {
    if (!h->ref_auto) return LBMRV_OK;
    if (h->slab)
        return fail(h, LBMRV_E_INVAL,
                    "%s: a slab needs the reference shared by all slabs (lbmrv_set_reference)",
                    who);
    double* res = h->red + 8 * (size_t)h->red_blocks;
    double sums[4] = {0.0, 0.0, 0.0, 0.0};
    cudaError_t e = launch_mean_flow(rho, u, h->n, h->n, h->dim, h->red, h->red_blocks, res,
                                     h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sums, res, sizeof(sums), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, who);
    for (int c = 0; c < 4; ++c)
        if (!std::isfinite(sums[c]))
            return fail(h, LBMRV_E_NONFINITE, "%s: the fields hold non-finite values", who);
    if (!(sums[0] > 0.0))
        return fail(h, LBMRV_E_INVAL, "%s: the total mass must be positive", who);
    for (int a = 0; a < 3; ++a) h->u_ref[a] = a < h->dim ? sums[1 + a] / sums[0] : 0.0;
    return LBMRV_OK;
}

int fail(lbmrv_t h, int code, const char* fmt, ...) {
    char* buf = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 320, fmt, ap);
    va_end(ap);
    return code;
}

const char* last_create_error() { return g_create_err; }

int choose_width(const lbmrv_s* h, const void* a, const void* b) {
    if (h->width > 0) return h->width;
    const int nv = h->dim == 2 ? step_vector_width(h->storage, (int)h->nx)
                               : step3_vector_width(h->storage, (int)h->nx);
    const size_t align = (size_t)(nv * elem_size(h->storage));
    if (nv > 1 && ((reinterpret_cast<uintptr_t>(a) % align) != 0 ||
                   (reinterpret_cast<uintptr_t>(b) % align) != 0))
        return 1;
    return nv;
}

cudaError_t launch_handle_step(const lbmrv_s* h, int nv, const void* src, void* dst, int64_t t) {
    if (h->dim == 2)
        return launch_step(h->storage, kernel_mode(h), nv, src, dst, make_args(h, t), h->stream,
                           h->basis);
    return launch_step3(h->storage, kernel_mode(h), nv, src, dst, make_args3(h, t), h->stream);
}

}  // namespace lbmrv

extern "C" {

int lbmrv_version(void) { return LBMRV_VERSION; }

int64_t lbmrv_state_bytes(int lattice, const int64_t dims[3], int storage) {
    const int q = lattice_q(lattice);
    if (q < 0 || !dims || dims[0] < 1 || dims[1] < 1) return -1;
    const int64_t nz = lattice == LBMRV_D3Q19 ? dims[2] : 1;
    if (nz < 1) return -1;
    const int64_t es = elem_size(storage);
    if (es < 0) return -1;
    return q * dims[0] * dims[1] * nz * es;
}

int lbmrv_create(lbmrv_t* out, int lattice, const int64_t dims[3], double lambda,
                 const double* s, int umode, int storage, double rho_ref, void* stream,
                 void* f_a_dev, void* f_b_dev) {
    if (!out) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: out is NULL");
    *out = nullptr;
    const int q = lattice_q(lattice);
    if (q < 0) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: bad lattice");
    if (!dims || dims[0] < 1 || dims[1] < 1)
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: dims must be >= 1");
    if (lattice != LBMRV_D3Q19 && dims[2] != 1 && dims[2] != 0)
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: D2Q9 dims must be {nx>=1, ny>=1, 1}");
    if (lattice == LBMRV_D3Q19 && dims[2] < 1)
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: D3Q19 dims must be >= 1");
    const int64_t nz = lattice == LBMRV_D3Q19 ? dims[2] : 1;
    if (dims[0] > (1 << 30) || dims[1] > (1 << 30) || nz > (1 << 30) ||
        dims[0] * dims[1] * nz >= (int64_t(1) << 31))
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: the node count must be below 2^31");
    if (!(lambda > 0.0) || !std::isfinite(lambda))
        return fail(nullptr, LBMRV_E_INVAL, "lbmrv_create: lambda must be finite and > 0");
    int rc = check_rates(nullptr, lattice, s, "lbmrv_create");
    if (rc != LBMRV_OK) return rc;
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
    h->q = q;
    h->dim = lattice_dim(lattice);
    h->basis = lattice == LBMRV_D2Q9_CASCADED ? 1 : 0;
    h->umode = umode;
    h->storage = storage;
    h->nx = dims[0];
    h->ny = dims[1];
    h->nz = nz;
    h->n = dims[0] * dims[1] * nz;
    h->lambda = lambda;
    h->rho_ref = rho_ref;
    for (int k = 0; k < q; ++k) h->s[k] = s[k];
    h->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, LBMRV_E_CUDA, "lbmrv_create: cudaGetDevice: %s",
                    cudaGetErrorString(e));
    }
    const size_t bytes = state_bytes(h);
    bool ok = true;
    if (f_a_dev) {
        h->f[0] = f_a_dev;
        h->f[1] = f_b_dev;
    } else {
        h->owns_f = true;
        ok = cudaMalloc(&h->f[0], bytes) == cudaSuccess && cudaMalloc(&h->f[1], bytes) == cudaSuccess;
    }
    h->red_blocks = conserved_blocks(h->n);
    ok = ok && cudaMalloc(&h->red, sizeof(double) * (8 * (size_t)h->red_blocks + 8)) == cudaSuccess;
    ok = ok && cudaMalloc(&h->sin_x, sizeof(float) * (size_t)h->nx) == cudaSuccess;
    if (ok) {
        std::vector<float> tab((size_t)h->nx);
        for (int64_t x = 0; x < h->nx; ++x)
            tab[(size_t)x] = (float)std::sin(2.0 * M_PI * (double)x / (double)h->nx);
        ok = cudaMemcpy(h->sin_x, tab.data(), sizeof(float) * tab.size(),
                        cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        if (h->owns_f) {
            cudaFree(h->f[0]);
            cudaFree(h->f[1]);
        }
        cudaFree(h->red);
        cudaFree(h->sin_x);
        delete h;
        return fail(nullptr, LBMRV_E_NOMEM, "lbmrv_create: device allocation of %zu bytes failed",
                    2 * bytes);
    }
    warn_rates(h, lattice, s, "lbmrv_create");
    warn_rates(nullptr, lattice, s, "lbmrv_create");
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
    cudaFree(h->sin_x);
    cudaFree(h->fused);
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
    int rc = check_rates(h, h->lattice, s, "lbmrv_set_rates");
    if (rc != LBMRV_OK) return rc;
    warn_rates(h, h->lattice, s, "lbmrv_set_rates");
    for (int k = 0; k < h->q; ++k) h->s[k] = s[k];
    return LBMRV_OK;
}

int lbmrv_set_reference(lbmrv_t h, double rho_ref, const double* u_ref) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_set_reference: NULL handle");
    double u[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < h->dim && u_ref; ++a) u[a] = u_ref[a];
    if (!std::isfinite(rho_ref) || !std::isfinite(u[0]) || !std::isfinite(u[1]) ||
        !std::isfinite(u[2]))
        return fail(h, LBMRV_E_INVAL, "lbmrv_set_reference: values must be finite");
    h->rho_ref = rho_ref;
    for (int a = 0; a < 3; ++a) h->u_ref[a] = u[a];
    h->ref_auto = false;
    return LBMRV_OK;
}

int lbmrv_set_reference_auto(lbmrv_t h, double rho_ref) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_set_reference_auto: NULL handle");
    if (!std::isfinite(rho_ref))
        return fail(h, LBMRV_E_INVAL, "lbmrv_set_reference_auto: rho_ref is not finite");
    h->rho_ref = rho_ref;
    h->ref_auto = true;
    return LBMRV_OK;
}

int lbmrv_get_reference(lbmrv_t h, double* rho_ref, double* u_ref) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_get_reference: NULL handle");
    if (rho_ref) *rho_ref = h->rho_ref;
    if (u_ref)
        for (int a = 0; a < 3; ++a) u_ref[a] = h->u_ref[a];
    return h->ref_auto ? 1 : 0;
}

int lbmrv_set_utilde(lbmrv_t h, const float* ut0_dev, double amplitude, double period) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_set_utilde: NULL handle");
    if (!std::isfinite(amplitude) || !std::isfinite(period))
        return fail(h, LBMRV_E_INVAL, "lbmrv_set_utilde: amplitude and period must be finite");
    if (h->lattice == LBMRV_D3Q19 && h->umode == LBMRV_UT_PRESCRIBED && !ut0_dev)
        return fail(h, LBMRV_E_UNSUPPORTED, "lbmrv_set_utilde: D3Q19 needs a u~0 field");
    h->ut0 = ut0_dev;
    h->amp = amplitude;
    h->period = period;
    return LBMRV_OK;
}

int lbmrv_init_equilibrium(lbmrv_t h, const float* rho_dev, const float* u_dev) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_init_equilibrium: NULL handle");
    if (!u_dev) return fail(h, LBMRV_E_INVAL, "lbmrv_init_equilibrium: u is NULL");
    DeviceGuard g(h->device);
    int rc = apply_auto_reference(h, rho_dev, u_dev, "lbmrv_init_equilibrium");
    if (rc != LBMRV_OK) return rc;
    cudaError_t e;
    if (h->dim == 2)
        e = launch_init_eq(h->storage, h->f[h->cur], rho_dev, u_dev, h->n, store_ref(h),
                           (float)(1.0 / h->lambda), h->stream, h->basis);
    else
        e = launch_init_eq3(h->storage, h->f[h->cur], rho_dev, u_dev, h->n, store_ref3(h),
                            (float)(1.0 / h->lambda), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_init_equilibrium");
    h->t = 0;
    return LBMRV_OK;
}

int lbmrv_init_equilibrium_host(lbmrv_t h, const float* rho_host, const float* u_host) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_init_equilibrium_host: NULL handle");
    if (!u_host) return fail(h, LBMRV_E_INVAL, "lbmrv_init_equilibrium_host: u is NULL");
    DeviceGuard g(h->device);
    // Staging: 1 + d floats per node fit in the non-current state buffer (>= 18 bytes/node).
    float* stage = static_cast<float*>(h->f[1 - h->cur]);
    const size_t nb = sizeof(float) * (size_t)h->n;
    cudaError_t e = cudaSuccess;
    if (rho_host) e = cudaMemcpyAsync(stage, rho_host, nb, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(stage + h->n, u_host, h->dim * nb, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_init_equilibrium_host: copy");
    const float* rho = rho_host ? stage : nullptr;
    int rc = apply_auto_reference(h, rho, stage + h->n, "lbmrv_init_equilibrium_host");
    if (rc != LBMRV_OK) return rc;
    if (h->dim == 2)
        e = launch_init_eq(h->storage, h->f[h->cur], rho, stage + h->n, h->n, store_ref(h),
                           (float)(1.0 / h->lambda), h->stream, h->basis);
    else
        e = launch_init_eq3(h->storage, h->f[h->cur], rho, stage + h->n, h->n, store_ref3(h),
                            (float)(1.0 / h->lambda), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_init_equilibrium_host");
    h->t = 0;
    return LBMRV_OK;
}

int lbmrv_step(lbmrv_t h, int64_t n) {
    lbmrv::TraceRange trace("lbmrv_step");
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_step: NULL handle");
    if (n < 0) return fail(h, LBMRV_E_INVAL, "lbmrv_step: n < 0");
    if (h->lattice == LBMRV_D3Q19 && h->umode == LBMRV_UT_PRESCRIBED && !h->ut0)
        return fail(h, LBMRV_E_INVAL, "lbmrv_step: D3Q19 prescribed mode needs a u~0 field");
    DeviceGuard g(h->device);
    const int nv = choose_width(h, h->f[0], h->f[1]);
    for (int64_t k = 0; k < n; ++k) {
        cudaError_t e = launch_handle_step(h, nv, h->f[h->cur], h->f[1 - h->cur], h->t + 1);
        if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_step");
        h->cur = 1 - h->cur;
        h->t += 1;
    }
    return LBMRV_OK;
}

static cudaError_t moments_into(lbmrv_t h, float* rho, float* u) {
    if (h->dim == 2)
        return launch_moments(h->storage, h->f[h->cur], rho, u, h->n, store_ref(h),
                              (float)h->lambda, h->stream);
    return launch_moments3(h->storage, h->f[h->cur], rho, u, h->n, store_ref3(h),
                           (float)h->lambda, h->stream);
}

int lbmrv_moments(lbmrv_t h, float* rho_dev, float* u_dev) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_moments: NULL handle");
    DeviceGuard g(h->device);
    cudaError_t e = moments_into(h, rho_dev, u_dev);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_moments");
    return LBMRV_OK;
}

int lbmrv_moments_host(lbmrv_t h, float* rho_host, float* u_host) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_moments_host: NULL handle");
    DeviceGuard g(h->device);
    float* stage = static_cast<float*>(h->f[1 - h->cur]);
    const size_t nb = sizeof(float) * (size_t)h->n;
    cudaError_t e = moments_into(h, stage, stage + h->n);
    if (e == cudaSuccess && rho_host)
        e = cudaMemcpyAsync(rho_host, stage, nb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && u_host)
        e = cudaMemcpyAsync(u_host, stage + h->n, h->dim * nb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_moments_host");
    return LBMRV_OK;
}

int lbmrv_conserved3(lbmrv_t h, double out_host[5]) {
    lbmrv::TraceRange trace("lbmrv_conserved");
    if (!h || !out_host) return fail(h, LBMRV_E_INVAL, "lbmrv_conserved3: NULL argument");
    DeviceGuard g(h->device);
    double* res = h->red + 8 * (size_t)h->red_blocks;
    cudaError_t e;
    double tmp[5] = {0, 0, 0, 0, 0};
    // a slab sums its interior layers only
    const void* src = static_cast<const char*>(h->f[h->cur]) +
                      owned_first(h) * elem_size(h->storage);
    const int64_t count = owned_count(h);
    if (h->dim == 2) {
        double four[4] = {0, 0, 0, 0};
        e = launch_conserved(h->storage, src, count, h->n, h->rho_ref,
                             h->rho_ref * h->u_ref[0] / h->lambda,
                             h->rho_ref * h->u_ref[1] / h->lambda, h->lambda, h->red,
                             h->red_blocks, res, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(four, res, sizeof(four), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        tmp[0] = four[0];
        tmp[1] = four[1];
        tmp[2] = four[2];
        tmp[4] = four[3];
    } else {
        e = launch_conserved3(h->storage, src, count, h->n, store_ref3(h), h->lambda, h->red,
                              h->red_blocks, res, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp, res, sizeof(tmp), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_conserved");
    for (int k = 0; k < 5; ++k) out_host[k] = tmp[k];
    if (out_host[4] > 0.0)
        return fail(h, LBMRV_E_NONFINITE, "lbmrv_conserved: %.0f nodes hold non-finite values",
                    out_host[4]);
    return LBMRV_OK;
}

int lbmrv_step_conserved(lbmrv_t h, int64_t n, double out_host[5]) {
    lbmrv::TraceRange trace("lbmrv_step_conserved");
    if (!h || !out_host) return fail(h, LBMRV_E_INVAL, "lbmrv_step_conserved: NULL argument");
    if (n < 1) return fail(h, LBMRV_E_INVAL, "lbmrv_step_conserved: n < 1");
    int rc = lbmrv_step(h, n - 1);
    if (rc != LBMRV_OK) return rc;
    DeviceGuard g(h->device);
    const int nv = choose_width(h, h->f[0], h->f[1]);
    const bool fused = !h->slab && (h->dim == 2 ? nv >= 2
                                                : step3_fuses_sums(h->storage, nv, (int)h->ny,
                                                                   (int)h->nz));
    if (!fused) {  // no fused form for this kernel: the step, then the sums' own pass
        rc = lbmrv_step(h, 1);
        return rc != LBMRV_OK ? rc : lbmrv_conserved3(h, out_host);
    }
    if (h->dim == 3 && h->umode == LBMRV_UT_PRESCRIBED && !h->ut0)
        return fail(h, LBMRV_E_INVAL, "lbmrv_step_conserved: D3Q19 prescribed mode needs a u~0 field");
    const int64_t scratch = h->dim == 2
        ? step_sum_scratch((int)h->nx, (int)h->ny, nv)
        : step3_sum_scratch(h->storage, nv, make_args3(h, h->t + 1));
    if (scratch < 0) return cuda_fail(h, cudaGetLastError(), "lbmrv_step_conserved");
    const int64_t need = scratch + 8;  // + the results
    if (need > h->fused_doubles) {
        cudaError_t e = cudaStreamSynchronize(h->stream);  // the old scratch may be in use
        if (e == cudaSuccess) e = cudaFree(h->fused);
        h->fused = nullptr;
        h->fused_doubles = 0;
        if (e == cudaSuccess)
            e = cudaMalloc(reinterpret_cast<void**>(&h->fused), sizeof(double) * need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->fused = nullptr;
            return fail(h, LBMRV_E_NOMEM, "lbmrv_step_conserved: scratch of %lld doubles: %s",
                        (long long)need, cudaGetErrorString(e));
        }
        h->fused_doubles = need;
    }
    double* res = h->fused + scratch;
    cudaError_t e;
    if (h->dim == 2)
        e = launch_step_conserved(h->storage, kernel_mode(h), nv, h->f[h->cur], h->f[1 - h->cur],
                                  make_args(h, h->t + 1), h->stream, h->basis, h->rho_ref,
                                  h->rho_ref * h->u_ref[0] / h->lambda,
                                  h->rho_ref * h->u_ref[1] / h->lambda, h->lambda, h->fused, res);
    else
        e = launch_step3_conserved(h->storage, kernel_mode(h), nv, h->f[h->cur],
                                   h->f[1 - h->cur], make_args3(h, h->t + 1), h->stream,
                                   h->lambda, h->fused, scratch, res);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_step_conserved");
    h->cur = 1 - h->cur;
    h->t += 1;
    double five[5] = {0, 0, 0, 0, 0};
    e = cudaMemcpyAsync(five, res, sizeof(double) * (h->dim == 2 ? 4 : 5),
                        cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_step_conserved");
    if (h->dim == 2) {  // {rho, q_x, q_y, non-finite} -> the lbmrv_conserved3 layout
        five[4] = five[3];
        five[3] = 0.0;
    }
    for (int k = 0; k < 5; ++k) out_host[k] = five[k];
    if (out_host[4] > 0.0)
        return fail(h, LBMRV_E_NONFINITE,
                    "lbmrv_step_conserved: %.0f nodes hold non-finite values", out_host[4]);
    return LBMRV_OK;
}

int lbmrv_conserved(lbmrv_t h, double out_host[4]) {
    if (!h || !out_host) return fail(h, LBMRV_E_INVAL, "lbmrv_conserved: NULL argument");
    double five[5];
    const int rc = lbmrv_conserved3(h, five);
    if (rc != LBMRV_OK && rc != LBMRV_E_NONFINITE) return rc;
    out_host[0] = five[0];
    out_host[1] = five[1];
    out_host[2] = five[2];
    out_host[3] = five[4];
    return rc;
}

int lbmrv_get_state(lbmrv_t h, void* dst_dev) {
    if (!h || !dst_dev) return fail(h, LBMRV_E_INVAL, "lbmrv_get_state: NULL argument");
    DeviceGuard g(h->device);
    cudaError_t e = cudaMemcpyAsync(dst_dev, h->f[h->cur], state_bytes(h), cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_get_state");
    return LBMRV_OK;
}

int lbmrv_set_state(lbmrv_t h, const void* src_dev, int64_t t) {
    if (!h || !src_dev) return fail(h, LBMRV_E_INVAL, "lbmrv_set_state: NULL argument");
    if (t < 0) return fail(h, LBMRV_E_INVAL, "lbmrv_set_state: t < 0");
    DeviceGuard g(h->device);
    cudaError_t e = cudaMemcpyAsync(h->f[h->cur], src_dev, state_bytes(h), cudaMemcpyDeviceToDevice,
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
