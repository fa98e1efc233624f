// Small-face pass kernels for FP16 tensors (scheme in small.cu).
#include "small_kernel.cuh"

namespace hoscf {

cudaError_t launch_small_f16(const SmallPlanInfo& sp, const SmallArgs& a, bool vec, cudaStream_t st,
                             const KernelEvents* kev) {
    return vec ? launch_small_bm<f16_t, true>(sp, a, st, kev) : launch_small_bm<f16_t, false>(sp, a, st, kev);
}

}  // namespace hoscf
