// swe_fused_f32_k.cu -- instantiation of the fused step for FP32 with dissipation.
#include "swe_fused.cuh"

namespace swe {
namespace fz {

cudaError_t launch_f32_k(swe_ctx* c, const Plan& pl, int s, long long k) {
    return launch_dir<float, CPT_F32, true>(c, pl, s, k);
}

int occupancy_f32(swe_ctx*) {
    int nb = 0;
    auto kern = k_fused<float, CPT_F32, 1, 1, true>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cpt_smem<float, CPT_F32>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NWARP * 32, cpt_smem<float, CPT_F32>());
    return nb < 1 ? 1 : nb;
}

}  // namespace fz
}  // namespace swe
