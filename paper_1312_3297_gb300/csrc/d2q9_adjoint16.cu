// The reverse step of the D2Q9 adjoint with forward states stored in FP16 or BF16 (the
// adjoint vectors stay FP32): instances of the kernel in d2q9_adjoint_step.cuh, in a
// translation unit of their own so that they compile beside the FP32 ones.
#include <cuda_runtime.h>

#include "d2q9_adjoint_step.cuh"
#include "launch.h"

namespace lbmrv {

cudaError_t launch_adjoint_step16(int storage, int um, int nv, const void* s_prev,
                                  const float* a_in, bool gather, float* mu_out,
                                  const AdjointArgs& aa, cudaStream_t st) {
    if (storage == kStoreF16)
        return launch_adjoint_step_t<__half>(um, nv, s_prev, a_in, gather, mu_out, aa, st);
    if (storage == kStoreBF16)
        return launch_adjoint_step_t<__nv_bfloat16>(um, nv, s_prev, a_in, gather, mu_out, aa,
                                                    st);
    return cudaErrorInvalidValue;
}

}  // namespace lbmrv
