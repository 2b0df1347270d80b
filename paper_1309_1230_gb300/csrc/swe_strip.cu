// swe_strip.cu -- row-strip decomposition of one domain over several
// contexts (the paper's Sec. 6.1 proposal: horizontal strips of rows, each
// with halo rows copied from its neighbours, so that a step needs no
// synchronisation inside it).  A strip context steps its own rows and a halo
// of two rows per cut side (the step's dependency radius in rows); between
// steps the halos are refreshed from the neighbours' own rows and the CFL
// maxima of the strips are combined, so every strip takes the same step size
// and its own rows equal the undecomposed domain's bit for bit.  Here the
// strips are contexts on one GPU and the exchange is device-to-device
// copies; across GPUs the same calls would move the rows by peer copies.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "swe_internal.cuh"

using namespace swe;

namespace {

swe_status sfail(swe_ctx* c, swe_status s, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

constexpr int MAX_STRIPS = 64;

struct CtlList {
    DevCtl* ctl[MAX_STRIPS];
};

__global__ void k_cfl_combine(CtlList L, int n, int slot) {
    unsigned long long m = 0ull;
    for (int q = 0; q < n; ++q) {
        const unsigned long long b = L.ctl[q]->smax[slot];
        m = b > m ? b : m;  // non-negative FP64 bit patterns order like their values
    }
    for (int q = 0; q < n; ++q) L.ctl[q]->smax[slot] = m;
}

// Makes `waiter` wait for the work queued so far on `on`.
cudaError_t stream_after(cudaStream_t waiter, cudaStream_t on) {
    if (waiter == on) return cudaSuccess;
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev, on);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(waiter, ev, 0);
    cudaEventDestroy(ev);
    return e;
}

}  // namespace

extern "C" {

swe_status swe_set_own_rows(swe_ctx* c, int32_t lo, int32_t hi) {
    if (!c) return SWE_ERR_ARG;
    if (c->poisoned) return sfail(c, SWE_ERR_STATE, "context poisoned by an earlier CUDA error");
    if (lo < 0 || hi > c->p.ny || lo >= hi) return sfail(c, SWE_ERR_ARG, "own rows [%d, %d) outside [0, %d)", lo, hi, c->p.ny);
    if (cudaSetDevice(c->p.device) != cudaSuccess) return sfail(c, SWE_ERR_CUDA, "cudaSetDevice failed");
    c->own_lo = lo;
    c->own_hi = hi;
    if (c->state_set) {  // the current level's CFL maximum over the own rows only
        cudaError_t e = swe_launch_prologue(c);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { c->poisoned = true; return sfail(c, SWE_ERR_CUDA, "prologue: %s", cudaGetErrorString(e)); }
    }
    return SWE_OK;
}

swe_status swe_copy_rows(swe_ctx* dst, int32_t dst_row, const swe_ctx* src, int32_t src_row, int32_t nrows) {
    if (!dst || !src) return SWE_ERR_ARG;
    if (dst->poisoned) return sfail(dst, SWE_ERR_STATE, "context poisoned by an earlier CUDA error");
    if (!dst->state_set || !src->state_set) return sfail(dst, SWE_ERR_STATE, "both states must be set");
    if (dst->p.nx != src->p.nx || dst->real_size != src->real_size || dst->p.device != src->p.device)
        return sfail(dst, SWE_ERR_ARG, "strips differ in nx, precision or device");
    if (nrows < 0 || dst_row < 0 || src_row < 0 || dst_row + nrows > dst->p.ny || src_row + nrows > src->p.ny)
        return sfail(dst, SWE_ERR_ARG, "rows out of range");
    if (nrows == 0) return SWE_OK;
    if (cudaSetDevice(dst->p.device) != cudaSuccess) return sfail(dst, SWE_ERR_CUDA, "cudaSetDevice failed");
    const size_t es = (size_t)dst->real_size;
    cudaError_t e = stream_after(dst->stream, src->stream);
    void* d[3] = {dst->eta[dst->cur], dst->u[dst->cur], dst->v[dst->cur]};
    const void* s[3] = {src->eta[src->cur], src->u[src->cur], src->v[src->cur]};
    for (int f = 0; f < 3 && e == cudaSuccess; ++f)
        e = cudaMemcpy2DAsync((char*)d[f] + (size_t)dst_row * dst->pitch * es, dst->pitch * es,
                              (const char*)s[f] + (size_t)src_row * src->pitch * es, src->pitch * es, dst->p.nx * es,
                              nrows, cudaMemcpyDeviceToDevice, dst->stream);
    // rows changed outside the step: the dry-skip flags no longer hold
    if (e == cudaSuccess) e = swe_fused_reset_flags(dst);
    if (e == cudaSuccess) e = stream_after(src->stream, dst->stream);  // src may not overwrite them early
    if (e != cudaSuccess) { dst->poisoned = true; return sfail(dst, SWE_ERR_CUDA, "copy rows: %s", cudaGetErrorString(e)); }
    return SWE_OK;
}

swe_status swe_cfl_combine(swe_ctx* const* ctxs, int32_t n) {
    if (!ctxs || n < 1 || n > MAX_STRIPS) return SWE_ERR_ARG;
    swe_ctx* c0 = ctxs[0];
    if (!c0) return SWE_ERR_ARG;
    for (int q = 0; q < n; ++q) {
        if (!ctxs[q]) return SWE_ERR_ARG;
        if (ctxs[q]->poisoned) return sfail(ctxs[q], SWE_ERR_STATE, "context poisoned by an earlier CUDA error");
        if (ctxs[q]->step != c0->step || ctxs[q]->p.device != c0->p.device)
            return sfail(c0, SWE_ERR_ARG, "strip %d is at another step or device", q);
    }
    if (cudaSetDevice(c0->p.device) != cudaSuccess) return sfail(c0, SWE_ERR_CUDA, "cudaSetDevice failed");
    CtlList L;
    memset(&L, 0, sizeof(L));
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < n && e == cudaSuccess; ++q) {
        L.ctl[q] = ctxs[q]->ctl;
        e = stream_after(c0->stream, ctxs[q]->stream);
    }
    if (e == cudaSuccess) {
        k_cfl_combine<<<1, 1, 0, c0->stream>>>(L, n, (int)(c0->step % 3));
        e = cudaGetLastError();
    }
    for (int q = 1; q < n && e == cudaSuccess; ++q) e = stream_after(ctxs[q]->stream, c0->stream);
    if (e != cudaSuccess) { c0->poisoned = true; return sfail(c0, SWE_ERR_CUDA, "cfl combine: %s", cudaGetErrorString(e)); }
    return SWE_OK;
}

}  // extern "C"
