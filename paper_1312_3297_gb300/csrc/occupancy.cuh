// Resident blocks of a kernel on the current device, for grids sized to what runs at once
// (persistent kernels, and reductions whose block count is set by occupancy rather than by
// the data).
#pragma once

#include <cuda_runtime.h>

#include <atomic>

namespace lbmrv {

constexpr int kMaxDevicesOcc = 64;

// SMs x blocks per SM of `kernel` at `threads` threads and `smem` bytes of dynamic shared
// memory (at most max_per_sm per SM, at least one), found once per device and kept in
// cache[device] (0 = not yet known). The shared-memory attribute is set first when smem
// is non-zero.
template <typename... KArgs>
cudaError_t resident_blocks(void (*kernel)(KArgs...), std::atomic<int>* cache, int threads,
                            int smem, int max_per_sm, int* full) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    *full = dev < kMaxDevicesOcc ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (*full != 0) return cudaSuccess;
    int sms = 0, per_sm = 0;
    if (smem > 0)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : (per_sm > max_per_sm ? max_per_sm : per_sm);
    *full = per_sm * sms;
    if (dev < kMaxDevicesOcc) cache[dev].store(*full, std::memory_order_relaxed);
    return cudaSuccess;
}

}  // namespace lbmrv
