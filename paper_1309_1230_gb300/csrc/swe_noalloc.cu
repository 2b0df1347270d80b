// swe_noalloc.cu -- the no-allocation FP32 step (swe_step_plain_f32_noalloc).
//
// For callers that must not allocate device memory: code running while a
// CUDA stream is being captured into a graph (an allocation there breaks the
// capture), engines whose device memory is all handed out by their own pool,
// and loops with hard latency limits that cannot wait on the allocator.
// Such a caller owns the state buffers; the step's own scratch (the predicted
// planes, the reduction control block and the step size) lives in one
// file-scope __device__ array that every GPU loading this library keeps until
// the process exits.
#include <cstring>
#include <mutex>

#include "swe_internal.cuh"

cudaError_t swe_plain_step_f32_raw(const swe_params* p, int pitch, const float* z, const float* e, const float* u,
                                   const float* v, float* e1, float* u1, float* v1, float* ps_e, float* ps_u,
                                   float* ps_v, swe::DevCtl* ctl, const double* dt_fixed, double* dt_hist,
                                   cudaStream_t st);

namespace {

struct NoallocScratch {
    swe::DevCtl ctl;          // CFL reduction slots and step bookkeeping; cleared by every call
    double dt_in;             // a caller's fixed step size, copied in
    double dt_used[2];        // the step size the call used
    float planes[3][SWE_NOALLOC_MAX_CELLS];  // predicted eta, u, v
};

// 12 MB + a few hundred bytes, resident on every device that loads the library.
static __device__ __align__(256) NoallocScratch g_swe_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoallocScratch* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (host code may not use
// the symbol itself: it names a host-side stand-in).
cudaError_t scratch_on(int device, NoallocScratch** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_swe_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (!ptr) return cudaErrorInvalidSymbol;
        g_dev_ptr[device] = static_cast<NoallocScratch*>(ptr);
    }
    *out = g_dev_ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" swe_status swe_step_plain_f32_noalloc(const swe_params* p, const float* z, const float* eta,
                                                 const float* u, const float* v, float* eta_out, float* u_out,
                                                 float* v_out, double dt_fixed, double* dt_out, void* stream) {
    if (!p || !z || !eta || !u || !v || !eta_out || !u_out || !v_out) return SWE_ERR_ARG;
    if (p->nx < 1 || p->ny < 1) return SWE_ERR_ARG;
    if ((long long)p->nx * (long long)p->ny > (long long)SWE_NOALLOC_MAX_CELLS) return SWE_ERR_ARG;
    if (!(p->dx > 0) || !(p->dy > 0) || !(p->g > 0) || !(p->cfl > 0) || !(p->h_dry > 0) || !(p->dt_max > 0))
        return SWE_ERR_ARG;
    if (!(p->kappa >= 0) || !(p->kappa <= 0.25) || !(p->manning_n >= 0)) return SWE_ERR_ARG;
    if (p->dir_cycle < 0 || p->dir_cycle > 7) return SWE_ERR_ARG;
    for (int s = 0; s < 4; ++s)
        if (p->bc[s] < SWE_BC_WALL || p->bc[s] > SWE_BC_OUTFLOW) return SWE_ERR_ARG;
    if (!(dt_fixed >= 0)) return SWE_ERR_ARG;
    // the corrector reads the input level while writing the output level
    const float* ins[3] = {eta, u, v};
    const float* outs[3] = {eta_out, u_out, v_out};
    for (const float* a : ins)
        for (const float* b : outs)
            if (a == b) return SWE_ERR_ARG;

    cudaStream_t st = (cudaStream_t)stream;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SWE_ERR_CUDA;
    NoallocScratch* s = nullptr;
    if (scratch_on(dev, &s) != cudaSuccess) return SWE_ERR_CUDA;

    // the scratch keeps the previous call's contents: clear the control block
    if (cudaMemsetAsync(&s->ctl, 0, sizeof(s->ctl), st) != cudaSuccess) return SWE_ERR_CUDA;
    const double* dtp = nullptr;
    if (dt_fixed > 0) {
        if (cudaMemcpyAsync(&s->dt_in, &dt_fixed, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return SWE_ERR_CUDA;
        dtp = &s->dt_in;
    }
    cudaError_t e = swe_plain_step_f32_raw(p, p->nx, z, eta, u, v, eta_out, u_out, v_out, s->planes[0],
                                           s->planes[1], s->planes[2], &s->ctl, dtp, s->dt_used, st);
    if (e != cudaSuccess) return SWE_ERR_CUDA;
    if (dt_out) {
        if (cudaMemcpyAsync(dt_out, &s->dt_used[0], sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SWE_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return SWE_ERR_CUDA;
    }
    return SWE_OK;
}
