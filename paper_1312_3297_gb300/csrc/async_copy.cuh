// Asynchronous global -> shared copies (cp.async, sm_80 and later) for kernels that stage
// the next work item while they compute the current one. A thread's copies are grouped by
// commit; wait_group returns once the thread's older groups have landed (a hardware wait,
// not a spin). Other lanes' copies become visible after the wait and a __syncwarp.
#pragma once

#include <cuda_runtime.h>

namespace lbmrv {

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {  // L2 only
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_all_but() {  // all but the latest N groups
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace lbmrv
