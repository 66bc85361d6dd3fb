// Allocation-free variant of the conserved-quantity reduction (lbmrv_conserved_noalloc).
//
// Some callers cannot allocate device memory at the moment they want the check: a host
// framework whose allocator owns every byte of the device, code running in a
// latency-critical loop where cudaMalloc would synchronise the device, or a monitor
// that inspects a state buffer it did not create and has no lbmrv handle for (creating
// a handle allocates). This entry point reduces a caller-owned state into a
// caller-owned output and takes its scratch from a fixed array that lives in the
// library's device image instead of from cudaMalloc.
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
double* g_partials_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
// In host code g_noalloc_partials names a host-side stand-in, so the address must come
// from cudaGetSymbolAddress with that device current.
cudaError_t scratch_for_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_partials_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int lbmrv_conserved_noalloc(const void* state_dev, int storage, const int64_t dims[3],
                                       double lambda, double rho_ref, double* out_dev,
                                       void* stream) {
    if (!state_dev || !out_dev || !dims) return LBMRV_E_INVAL;
    if (storage != LBMRV_FP32 && storage != LBMRV_FP16 && storage != LBMRV_BF16)
        return LBMRV_E_INVAL;
    if (dims[0] < 1 || dims[1] < 1 || (dims[2] != 1 && dims[2] != 0)) return LBMRV_E_INVAL;
    const int64_t n = dims[0] * dims[1];
    if (dims[0] > (1 << 30) || dims[1] > (1 << 30) || n >= (int64_t(1) << 31))
        return LBMRV_E_INVAL;
    if (!(lambda > 0.0)) return LBMRV_E_INVAL;
    double* partials = nullptr;
    if (scratch_for_current_device(&partials) != cudaSuccess) return LBMRV_E_CUDA;
    const int nblk = conserved_blocks(n);  // never more than kReduceMaxBlocks
    if (4 * nblk > kSlots) return LBMRV_E_INVAL;
    const cudaError_t e = launch_conserved(storage, state_dev, n, rho_ref, 0.0, 0.0, lambda,
                                           partials, nblk, out_dev,
                                           static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? LBMRV_OK : LBMRV_E_CUDA;
}
