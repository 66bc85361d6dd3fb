// Allocation-free variant of the conserved-quantity reduction (lbmrv_conserved_noalloc).
//
// Some callers cannot allocate device memory at the moment they want the check: a host
// framework whose allocator owns every byte of the device, code running in a
// latency-critical loop where cudaMalloc would synchronise the device, or a monitor
// that inspects a state buffer it did not create and has no lbmrv handle for (creating
// a handle allocates). This entry point reduces a caller-owned state into a
// caller-owned output and takes its scratch from a fixed array that lives in the
// library's device image instead of from cudaMalloc.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "launch.h"
#include "lbmrv.h"

using namespace lbmrv;

namespace {

// One FP64 partial (4 sums) per reduction block, for at most kReduceMaxBlocks blocks:
// 4 * 1216 doubles = 38,912 bytes. Every GPU that loads the library holds this array
// until the process exits. Each call overwrites every slot it later reads, so nothing
// has to be cleared between calls.
constexpr int kSlots = 4 * kReduceMaxBlocks;
static __device__ __align__(256) double g_noalloc_partials[kSlots];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;

// The scratch address found for a device, and the context it belongs to: a device reset
// (cudaDeviceReset, or a new primary context) makes the old address meaningless, so the
// address is looked up again whenever the current context is not the one it was found in.
struct ScratchAddress {
    bool valid = false;
    unsigned long long ctx_id = 0;
    double* ptr = nullptr;
};
ScratchAddress g_scratch[kMaxDevices];

// cuCtxGetCurrent and cuCtxGetId through the runtime's driver entry points (no link
// against the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

cudaError_t load_context_queries() {
    if (g_ctx_get_current && g_ctx_get_id) return cudaSuccess;
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                     cudaEnableDefault, &q1);
    if (e == cudaSuccess)
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
        return cudaErrorNotSupported;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    return cudaSuccess;
}

// Identity of the calling thread's current context; *has = false when there is none yet.
cudaError_t current_context(bool* has, unsigned long long* id) {
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorUnknown;
    *has = ctx != nullptr;
    if (*has && g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorUnknown;
    return cudaSuccess;
}

// Device address of the scratch array on the current device and context. In host code
// g_noalloc_partials names a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with that device current; it is looked up once per device and
// context and kept.
cudaError_t scratch_for_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    e = load_context_queries();
    if (e != cudaSuccess) return e;
    bool has = false;
    unsigned long long id = 0;
    e = current_context(&has, &id);
    if (e != cudaSuccess) return e;
    ScratchAddress& c = g_scratch[dev];
    if (!has || !c.valid || c.ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);  // creates the context if needed
        if (e != cudaSuccess) return e;
        e = current_context(&has, &id);
        if (e != cudaSuccess) return e;
        if (!has) return cudaErrorInvalidDevice;
        c.valid = true;
        c.ctx_id = id;
        c.ptr = static_cast<double*>(p);
    }
    *out = c.ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" int lbmrv_conserved_noalloc(const void* state_dev, int storage, const int64_t dims[3],
                                       double lambda, double rho_ref, double* out_dev,
                                       void* stream) {
    if (!state_dev || !out_dev || !dims) return LBMRV_E_INVAL;
    if (storage != LBMRV_FP32 && storage != LBMRV_FP16 && storage != LBMRV_BF16)
        return LBMRV_E_INVAL;
    if (dims[0] < 1 || dims[1] < 1 || dims[2] != 1) return LBMRV_E_INVAL;
    const int64_t n = dims[0] * dims[1];
    if (dims[0] > (1 << 30) || dims[1] > (1 << 30) || n >= (int64_t(1) << 31))
        return LBMRV_E_INVAL;
    if (!(lambda > 0.0)) return LBMRV_E_INVAL;
    double* partials = nullptr;
    if (scratch_for_current_device(&partials) != cudaSuccess) return LBMRV_E_CUDA;
    const int nblk = conserved_blocks(n);  // never more than kReduceMaxBlocks
    if (4 * nblk > kSlots) return LBMRV_E_INVAL;
    const cudaError_t e = launch_conserved(storage, state_dev, n, n, rho_ref, 0.0, 0.0, lambda,
                                           partials, nblk, out_dev,
                                           static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LBMRV_OK : LBMRV_E_CUDA;
}
