// C ABI of the discrete adjoint: checkpointed forward, reverse sweep, and the adjoints
// of the equilibrium initialisation, of the moments and of the kinetic energy.
#include <cuda_runtime.h>

#include "handle.h"
#include "launch.h"
#include "lbmrv.h"
#include "trace.h"

using namespace lbmrv;

namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Workspace: C checkpoints S_{t0 + c seg} (c = 0 .. C-1) and seg - 1 recomputed states of the
// current segment, in the handle's storage type; two FP32 adjoint states; then 8 FP64
// accumulators per adjoint block and 8 results.
struct WsLayout {
    int64_t C = 0, seg = 0, nblk = 0;
    size_t state = 0, mu = 0, off_seg = 0, off_mu = 0, off_acc = 0, total = 0;
};

// Nodes per thread of the adjoint kernel: the handle's kernel width when it is 1, 2 or 4,
// else 4 when it divides nx, else 1.
int adjoint_nv(const lbmrv_s* h) {
    if (h->width == 1 || h->width == 2 || h->width == 4) return h->width;
    return h->nx % 4 == 0 ? 4 : 1;
}

WsLayout layout(const lbmrv_s* h, int64_t n, int64_t seg) {
    WsLayout L;
    L.seg = seg;
    L.C = (n + seg - 1) / seg;
    L.state = round_up(state_bytes(h));
    L.mu = round_up((size_t)(9 * h->n) * sizeof(float));
    L.nblk = adjoint_blocks((int)h->nx, (int)h->ny, adjoint_nv(h));
    L.off_seg = (size_t)L.C * L.state;
    L.off_mu = L.off_seg + (size_t)(seg - 1) * L.state;
    L.off_acc = L.off_mu + 2 * L.mu;
    L.total = L.off_acc + round_up((size_t)(L.nblk + 1) * 8 * sizeof(double));
    return L;
}

int check_common(lbmrv_t h, int64_t n, int64_t seg, const void* ws, size_t ws_bytes,
                 const char* who, WsLayout* out) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "%s: NULL handle", who);
    if (h->lattice != LBMRV_D2Q9)
        return fail(h, LBMRV_E_UNSUPPORTED, "%s: the adjoint needs a D2Q9 handle", who);
    if (h->slab) return fail(h, LBMRV_E_UNSUPPORTED, "%s: no adjoint for a slab", who);
    if (n < 1 || seg < 1 || seg > n)
        return fail(h, LBMRV_E_INVAL, "%s: need n >= 1 and 1 <= seg <= n", who);
    if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign)
        return fail(h, LBMRV_E_INVAL, "%s: workspace must be a 256-byte aligned device buffer",
                    who);
    *out = layout(h, n, seg);
    if (ws_bytes < out->total)
        return fail(h, LBMRV_E_NOMEM, "%s: workspace of %zu bytes, %zu needed", who, ws_bytes,
                    out->total);
    return LBMRV_OK;
}

char* at(void* ws, size_t off) { return static_cast<char*>(ws) + off; }

}  // namespace

extern "C" {

int64_t lbmrv_adjoint_workspace_bytes(lbmrv_t h, int64_t n, int64_t seg) {
    if (!h || n < 1 || seg < 1 || seg > n || h->lattice != LBMRV_D2Q9) return -1;
    return (int64_t)layout(h, n, seg).total;
}

int lbmrv_forward_checkpointed(lbmrv_t h, int64_t n, int64_t seg, void* ws_dev,
                               size_t ws_bytes) {
    lbmrv::TraceRange trace("lbmrv_forward_checkpointed");
    WsLayout L;
    int rc = check_common(h, n, seg, ws_dev, ws_bytes, "lbmrv_forward_checkpointed", &L);
    if (rc != LBMRV_OK) return rc;
    DeviceGuard g(h->device);
    const size_t bytes = state_bytes(h);
    // the pack width must suit both the handle's buffers and the checkpoint slots
    const int nv_f = choose_width(h, h->f[0], h->f[1]), nv_w = choose_width(h, ws_dev, ws_dev);
    const int nv = nv_f < nv_w ? nv_f : nv_w;
    const int64_t t0 = h->t;
    cudaError_t e = cudaMemcpyAsync(at(ws_dev, 0), h->f[h->cur], bytes, cudaMemcpyDeviceToDevice,
                                    h->stream);
    // Checkpointed states are written by their step straight into their slot (no copy); the
    // next step reads them there. The final state ends in the handle's buffers.
    const void* src = h->f[h->cur];
    int cur = h->cur;
    for (int64_t k = 1; k <= n && e == cudaSuccess; ++k) {
        void* dst;
        if (k % seg == 0 && k < n)
            dst = at(ws_dev, (size_t)(k / seg) * L.state);
        else
            dst = src == h->f[cur] ? h->f[1 - cur] : h->f[cur];
        e = launch_handle_step(h, nv, src, dst, t0 + k);
        if (dst == h->f[0]) cur = 0;
        if (dst == h->f[1]) cur = 1;
        src = dst;
        h->t = t0 + k;
    }
    h->cur = cur;
    if (e != cudaSuccess) {
        h->ckpt_valid = false;
        return cuda_fail(h, e, "lbmrv_forward_checkpointed");
    }
    h->ckpt_valid = true;
    h->ckpt_n = n;
    h->ckpt_seg = seg;
    h->ckpt_t0 = t0;
    h->ckpt_ws = ws_dev;
    return LBMRV_OK;
}

int lbmrv_adjoint(lbmrv_t h, int64_t n, int64_t seg, void* ws_dev, size_t ws_bytes,
                  const float* dL_dS_dev, float* dL_dS0_dev, double* dL_ds_host,
                  double* dL_damp_host, float* dL_dut0_dev) {
    lbmrv::TraceRange trace("lbmrv_adjoint");
    WsLayout L;
    int rc = check_common(h, n, seg, ws_dev, ws_bytes, "lbmrv_adjoint", &L);
    if (rc != LBMRV_OK) return rc;
    if (!dL_dS_dev || !dL_dS0_dev)
        return fail(h, LBMRV_E_INVAL, "lbmrv_adjoint: dL/dS_N and dL/dS_0 buffers are required");
    // the reverse step reads dL/dS_N, and the final gather writes dL/dS_0, in 16-byte packs
    if (reinterpret_cast<uintptr_t>(dL_dS_dev) % 16 || reinterpret_cast<uintptr_t>(dL_dS0_dev) % 16)
        return fail(h, LBMRV_E_INVAL,
                    "lbmrv_adjoint: dL/dS_N and dL/dS_0 must be 16-byte aligned device buffers");
    if (!h->ckpt_valid || h->ckpt_n != n || h->ckpt_seg != seg || h->ckpt_ws != ws_dev)
        return fail(h, LBMRV_E_INVAL,
                    "lbmrv_adjoint: no matching lbmrv_forward_checkpointed(n, seg, ws) before");
    DeviceGuard g(h->device);
    const int64_t t0 = h->ckpt_t0;
    const int um = kernel_mode(h);
    const int nv = choose_width(h, ws_dev, ws_dev);
    const int anv = adjoint_nv(h);
    double* acc = reinterpret_cast<double*>(at(ws_dev, L.off_acc));
    double* res = acc + 8 * L.nblk;
    float* mu[2] = {reinterpret_cast<float*>(at(ws_dev, L.off_mu)),
                    reinterpret_cast<float*>(at(ws_dev, L.off_mu + L.mu))};
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)L.nblk * 8 * sizeof(double), h->stream);
    if (e == cudaSuccess && dL_dut0_dev)
        e = cudaMemsetAsync(dL_dut0_dev, 0, (size_t)(2 * h->n) * sizeof(float), h->stream);
    const float* a = dL_dS_dev;
    bool gather = false;
    int pp = 0;
    for (int64_t c = L.C - 1; c >= 0 && e == cudaSuccess; --c) {
        const int64_t base = c * seg;
        const int64_t khi = base + seg < n ? base + seg : n;
        const void* ck = at(ws_dev, (size_t)c * L.state);
        auto seg_state = [&](int64_t k) {  // S_k for base < k < khi
            return static_cast<void*>(at(ws_dev, L.off_seg + (size_t)(k - base - 1) * L.state));
        };
        const void* src = ck;
        for (int64_t k = base + 1; k < khi && e == cudaSuccess; ++k) {
            e = launch_step(h->storage, um, nv, src, seg_state(k), make_args(h, t0 + k),
                            h->stream);
            src = seg_state(k);
        }
        for (int64_t k = khi; k > base && e == cudaSuccess; --k) {
            const void* s_prev = (k - 1 == base) ? ck : seg_state(k - 1);
            AdjointArgs aa;
            aa.step = make_args(h, t0 + k);
            aa.da_factor = (float)(time_factor(h, t0 + k) / h->lambda);
            aa.dut0 = dL_dut0_dev;
            aa.acc = acc;
            aa.y0 = 0;
            aa.y1 = (int)h->ny;
            e = launch_adjoint_step(h->storage, um, anv, s_prev, a, gather, mu[pp], aa,
                                    h->stream);
            a = mu[pp];
            gather = true;
            pp ^= 1;
        }
    }
    if (e == cudaSuccess) e = launch_gather(a, dL_dS0_dev, (int)h->nx, (int)h->ny, h->stream);
    if (e == cudaSuccess) e = launch_acc_final(acc, L.nblk, res, h->stream);
    double out[8] = {0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, res, sizeof(out), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_adjoint");
    if (dL_ds_host) {
        dL_ds_host[0] = dL_ds_host[1] = dL_ds_host[2] = 0.0;
        for (int k = 0; k < 6; ++k) dL_ds_host[3 + k] = out[k];
    }
    if (dL_damp_host) *dL_damp_host = out[6];
    return LBMRV_OK;
}

int64_t lbmrv_adjoint_acc_doubles(lbmrv_t h) {
    if (!h || h->lattice != LBMRV_D2Q9) return -1;
    return 8 * (adjoint_blocks((int)h->nx, (int)h->ny, adjoint_nv(h)) + 1);
}

int lbmrv_adjoint_step(lbmrv_t h, const void* s_prev_dev, int64_t t, const float* a_dev,
                       int gather, float* mu_dev, double* acc_dev, float* dL_dut0_dev) {
    if (!h) return fail(nullptr, LBMRV_E_INVAL, "lbmrv_adjoint_step: NULL handle");
    if (h->lattice != LBMRV_D2Q9)
        return fail(h, LBMRV_E_UNSUPPORTED, "lbmrv_adjoint_step: needs a D2Q9 handle");
    if (!s_prev_dev || !a_dev || !mu_dev || !acc_dev || t < 1)
        return fail(h, LBMRV_E_INVAL, "lbmrv_adjoint_step: NULL buffer or t < 1");
    // the kernel reads and writes the adjoint vectors, and reads the state, in 16-byte packs
    if (reinterpret_cast<uintptr_t>(a_dev) % 16 || reinterpret_cast<uintptr_t>(mu_dev) % 16 ||
        reinterpret_cast<uintptr_t>(s_prev_dev) % 16 || a_dev == mu_dev)
        return fail(h, LBMRV_E_INVAL,
                    "lbmrv_adjoint_step: buffers must be distinct and 16-byte aligned");
    DeviceGuard g(h->device);
    AdjointArgs aa;
    aa.step = make_args(h, t);
    aa.da_factor = (float)(time_factor(h, t) / h->lambda);
    aa.dut0 = dL_dut0_dev;
    aa.acc = acc_dev;
    aa.y0 = h->slab ? 1 : 0;  // a slab reverses its own rows only
    aa.y1 = h->slab ? (int)h->ny - 1 : (int)h->ny;
    const cudaError_t e = launch_adjoint_step(h->storage, kernel_mode(h), adjoint_nv(h),
                                              s_prev_dev, a_dev, gather != 0, mu_dev, aa,
                                              h->stream);
    return e == cudaSuccess ? LBMRV_OK : cuda_fail(h, e, "lbmrv_adjoint_step");
}

int lbmrv_adjoint_acc_sum(lbmrv_t h, const double* acc_dev, double* dL_ds_host,
                          double* dL_damp_host) {
    if (!h || !acc_dev) return fail(h, LBMRV_E_INVAL, "lbmrv_adjoint_acc_sum: NULL argument");
    if (h->lattice != LBMRV_D2Q9)
        return fail(h, LBMRV_E_UNSUPPORTED, "lbmrv_adjoint_acc_sum: needs a D2Q9 handle");
    DeviceGuard g(h->device);
    double* res = h->red + 8 * (size_t)h->red_blocks;
    double out[8] = {0};
    cudaError_t e = launch_acc_final(acc_dev, lbmrv_adjoint_acc_doubles(h) / 8 - 1, res,
                                     h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, res, sizeof(out), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_adjoint_acc_sum");
    if (dL_ds_host) {
        dL_ds_host[0] = dL_ds_host[1] = dL_ds_host[2] = 0.0;
        for (int k = 0; k < 6; ++k) dL_ds_host[3 + k] = out[k];
    }
    if (dL_damp_host) *dL_damp_host = out[6];
    return LBMRV_OK;
}

int lbmrv_adjoint_gather(lbmrv_t h, const float* mu_dev, float* out_dev) {
    if (!h || !mu_dev || !out_dev || mu_dev == out_dev)
        return fail(h, LBMRV_E_INVAL, "lbmrv_adjoint_gather: NULL or aliased buffers");
    if (reinterpret_cast<uintptr_t>(mu_dev) % 16 || reinterpret_cast<uintptr_t>(out_dev) % 16)
        return fail(h, LBMRV_E_INVAL, "lbmrv_adjoint_gather: buffers must be 16-byte aligned");
    DeviceGuard g(h->device);
    const cudaError_t e = launch_gather(mu_dev, out_dev, (int)h->nx, (int)h->ny, h->stream);
    return e == cudaSuccess ? LBMRV_OK : cuda_fail(h, e, "lbmrv_adjoint_gather");
}

int lbmrv_kinetic_energy(lbmrv_t h, double* ke_host, float* dL_dS_dev) {
    if (!h || !ke_host) return fail(h, LBMRV_E_INVAL, "lbmrv_kinetic_energy: NULL argument");
    if (h->lattice != LBMRV_D2Q9)
        return fail(h, LBMRV_E_UNSUPPORTED, "lbmrv_kinetic_energy: needs a D2Q9 handle");
    DeviceGuard g(h->device);
    double* res = h->red + 8 * (size_t)h->red_blocks;
    cudaError_t e = cudaSuccess;
    if (h->slab && dL_dS_dev)  // the halo layers are not part of the loss
        e = cudaMemsetAsync(dL_dS_dev, 0, sizeof(float) * 9 * (size_t)h->n, h->stream);
    const int64_t o = owned_first(h);
    if (e == cudaSuccess)
        e = launch_kinetic_energy(h->storage,
                                  static_cast<const char*>(h->f[h->cur]) + o * elem_size(h->storage),
                                  dL_dS_dev ? dL_dS_dev + o : nullptr, owned_count(h), h->n,
                                  store_ref(h), (float)h->lambda, h->red, h->red_blocks, res,
                                  h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ke_host, res, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_kinetic_energy");
    return LBMRV_OK;
}

int lbmrv_moments_vjp(lbmrv_t h, const float* dL_drho_dev, const float* dL_du_dev,
                      float* dL_dS_dev) {
    if (!h || !dL_dS_dev) return fail(h, LBMRV_E_INVAL, "lbmrv_moments_vjp: NULL argument");
    if (h->lattice != LBMRV_D2Q9)
        return fail(h, LBMRV_E_UNSUPPORTED, "lbmrv_moments_vjp: needs a D2Q9 handle");
    DeviceGuard g(h->device);
    cudaError_t e = launch_moments_vjp(h->storage, h->f[h->cur], dL_drho_dev,
                                       dL_du_dev, dL_dS_dev, h->n, store_ref(h),
                                       (float)h->lambda, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_moments_vjp");
    return LBMRV_OK;
}

int lbmrv_equilibrium_vjp(lbmrv_t h, const float* rho_dev, const float* u_dev,
                          const float* dL_dS0_dev, float* dL_drho_dev, float* dL_du_dev) {
    if (!h || !u_dev || !dL_dS0_dev)
        return fail(h, LBMRV_E_INVAL, "lbmrv_equilibrium_vjp: NULL argument");
    if (h->lattice != LBMRV_D2Q9)
        return fail(h, LBMRV_E_UNSUPPORTED, "lbmrv_equilibrium_vjp: needs a D2Q9 handle");
    DeviceGuard g(h->device);
    cudaError_t e = launch_equilibrium_vjp(rho_dev, u_dev, dL_dS0_dev, dL_drho_dev, dL_du_dev, h->n,
                                           (float)(1.0 / h->lambda), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmrv_equilibrium_vjp");
    return LBMRV_OK;
}

}  // extern "C"
