// swe_noalloc.cu -- the no-allocation FP32 step (swe_step_plain_f32_noalloc).
//
// For callers that must not allocate device memory: engines whose device
// memory is all handed out by their own pool (a cudaMalloc behind the pool's
// back breaks its budget), plug-ins running inside a host application that
// owns the device memory, and loops with hard latency limits that cannot wait
// on the allocator (cudaMalloc and cudaFree may synchronise the device).
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
    double dt_in;             // a caller's fixed step size (k_noalloc_set_dt)
    double dt_used[2];        // the step size the call used
    float planes[3][SWE_NOALLOC_MAX_CELLS];  // predicted eta, u, v
};

// 12 MB + a few hundred bytes, resident on every device that loads the library.
static __device__ __align__(256) NoallocScratch g_swe_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoallocScratch* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (host code may not use
// the symbol itself: it names a host-side stand-in).  Looked up once per
// device and kept for the life of the process; after a cudaDeviceReset the
// module is loaded anew and the kept address is stale, so the entry point
// must not be called on a device that was reset.
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

// Stores a caller's fixed step size, passed by value, where the step kernels
// read it.
__global__ void k_noalloc_set_dt(double* dst, double dt) { *dst = dt; }

// Whether the byte ranges [a, a + n) and [b, b + n) share a byte.
bool overlap(const void* a, const void* b, size_t n) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + n && y < x + n;
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
    if (p->friction != 0 || p->dissipation != 0) return SWE_ERR_UNSUPPORTED;  // the ablation forms
    for (int s = 0; s < 4; ++s)
        if (p->bc[s] < SWE_BC_WALL || p->bc[s] > SWE_BC_OUTFLOW) return SWE_ERR_ARG;
    if (!(dt_fixed >= 0)) return SWE_ERR_ARG;
    // The corrector reads the input level (and the bed) while it writes the
    // output level: no output may share a byte with an input or another output.
    const size_t bytes = (size_t)p->nx * (size_t)p->ny * sizeof(float);
    const void* ins[4] = {z, eta, u, v};
    const void* outs[3] = {eta_out, u_out, v_out};
    for (int i = 0; i < 3; ++i) {
        for (const void* a : ins)
            if (overlap(a, outs[i], bytes)) return SWE_ERR_ARG;
        for (int j = i + 1; j < 3; ++j)
            if (overlap(outs[i], outs[j], bytes)) return SWE_ERR_ARG;
    }

    cudaStream_t st = (cudaStream_t)stream;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SWE_ERR_CUDA;
    NoallocScratch* s = nullptr;
    if (scratch_on(dev, &s) != cudaSuccess) return SWE_ERR_CUDA;

    // the scratch keeps the previous call's contents: clear the control block
    if (cudaMemsetAsync(&s->ctl, 0, sizeof(s->ctl), st) != cudaSuccess) return SWE_ERR_CUDA;
    const double* dtp = nullptr;
    if (dt_fixed > 0) {
        k_noalloc_set_dt<<<1, 1, 0, st>>>(&s->dt_in, dt_fixed);
        if (cudaGetLastError() != cudaSuccess) return SWE_ERR_CUDA;
        dtp = &s->dt_in;
    }
    cudaError_t e = swe_plain_step_f32_raw(p, p->nx, z, eta, u, v, eta_out, u_out, v_out, s->planes[0],
                                           s->planes[1], s->planes[2], &s->ctl, dtp, s->dt_used, st);
    if (e != cudaSuccess) return SWE_ERR_CUDA;
    if (dt_out) {
        unsigned flags = 0u;
        if (cudaMemcpyAsync(dt_out, &s->dt_used[0], sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SWE_ERR_CUDA;
        if (cudaMemcpyAsync(&flags, &s->ctl.flags, sizeof(flags), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SWE_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return SWE_ERR_CUDA;
        if (flags & SWE_FLAG_NONFINITE) return SWE_ERR_NONFINITE;
    }
    return SWE_OK;
}
