// placeholder, replaced by the fused sweep
#include "swe_internal.cuh"
cudaError_t swe_fused_prepare(swe_ctx*) { return cudaSuccess; }
cudaError_t swe_fused_run(swe_ctx*, int) { return cudaErrorNotSupported; }
