// swe_fused_f32_0.cu -- instantiation of the fused step for FP32 without dissipation.
#include "swe_fused.cuh"

namespace swe {
namespace fz {

cudaError_t launch_f32_0(swe_ctx* c, const Plan& pl, int s, long long k) {
    return launch_dir<float, CPT_F32, false>(c, pl, s, k);
}

}  // namespace fz
}  // namespace swe
