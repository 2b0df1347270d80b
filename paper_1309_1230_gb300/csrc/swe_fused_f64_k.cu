// swe_fused_f64_k.cu -- instantiation of the fused step for FP64 with dissipation.
#include "swe_fused.cuh"

namespace swe {
namespace fz {

cudaError_t launch_f64_k(swe_ctx* c, const Plan& pl, int s, long long k) {
    return launch_dir<double, 2, true>(c, pl, s, k);
}

int occupancy_f64(swe_ctx*) {
    int nb = 0;
    auto kern = k_fused<double, 2, 1, 1, true>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cpt_smem<double, 2>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NWARP * 32, cpt_smem<double, 2>());
    return nb < 1 ? 1 : nb;
}

}  // namespace fz
}  // namespace swe
