// Programmatic dependent launch (sm_90 and later) for kernels issued back to back in one
// stream, such as successive time steps. A kernel launched with launch_pdl may be scheduled
// while its predecessor in the stream finishes; before touching global memory it waits,
// with griddepcontrol.wait, until the predecessor has completed and its writes are
// visible. Each step kernel also signals at its start that its successor may be launched,
// which the hardware acts on once every block of the grid has started, so the successor's
// blocks never hold resources that the current grid still needs. Without the launch
// attribute the wait returns at once.
#pragma once

#include <cuda_runtime.h>

namespace lbmrv {

__device__ __forceinline__ void pdl_wait_prior() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void pdl_allow_next() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                       Args... args) {
    return launch_pdl_smem(kernel, grid, block, 0, st, args...);
}

}  // namespace lbmrv
