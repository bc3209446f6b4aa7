// Fused FP32 refine + scalar-step kernel (MR_VEL_FUSED).
#include "mr_internal.cuh"

namespace mr {

bool fused_supported(const mr_config& cfg, std::string* why)
{
    (void)cfg;
    *why = "MR_VEL_FUSED is not available in this build";
    return false;
}

cudaError_t launch_step_fused_f32(const Grid<float>&, const float*, const float*, const float*, const float*,
                                  const float*, float*, StepCoef, cudaStream_t)
{
    return cudaErrorNotSupported;
}

cudaError_t launch_maxdiv_fused_f32(const Grid<float>&, const float*, const float*, const float*, double*, int,
                                    cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace mr
