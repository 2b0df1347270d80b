// swe_api.cu -- the C ABI of include/swe.h: context life cycle, host and
// device transfers, and the step loop that queues the step kernels on the
// context's stream.  No step arithmetic lives here.
#include <cmath>
#include <cstdarg>
#include <vector>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "swe_internal.cuh"

using namespace swe;

namespace {

swe_status fail(swe_ctx* c, swe_status s, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

swe_status cuda_fail(swe_ctx* c, cudaError_t e, const char* what) {
    if (c) c->poisoned = true;
    return fail(c, SWE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(c, expr)                                             \
    do {                                                        \
        cudaError_t e__ = (expr);                               \
        if (e__ != cudaSuccess) return cuda_fail((c), e__, #expr); \
    } while (0)

bool params_ok(const swe_params* p, char* why, size_t n) {
    if (!p) { snprintf(why, n, "params is NULL"); return false; }
    if (p->nx < 1 || p->ny < 1) { snprintf(why, n, "nx, ny must be >= 1"); return false; }
    if ((double)p->nx * (double)p->ny > 4.0e9) { snprintf(why, n, "grid too large"); return false; }
    if (!(p->dx > 0) || !(p->dy > 0)) { snprintf(why, n, "dx, dy must be > 0"); return false; }
    if (!(p->g > 0) || !(p->cfl > 0) || !(p->h_dry > 0) || !(p->dt_max > 0)) {
        snprintf(why, n, "g, cfl, h_dry, dt_max must be > 0"); return false;
    }
    if (!(p->kappa >= 0) || !(p->kappa <= 0.25)) { snprintf(why, n, "kappa must lie in [0, 0.25]"); return false; }
    if (!(p->manning_n >= 0)) { snprintf(why, n, "manning_n must be >= 0"); return false; }
    for (int s = 0; s < 4; ++s) {
        if (p->bc[s] < SWE_BC_WALL || p->bc[s] > SWE_BC_OUTFLOW) { snprintf(why, n, "bad bc[%d]", s); return false; }
        if (!std::isfinite(p->q_in[s])) { snprintf(why, n, "bad q_in[%d]", s); return false; }
    }
    if (p->precision != SWE_FP64 && p->precision != SWE_FP32) { snprintf(why, n, "bad precision"); return false; }
    if (p->dir_cycle < 0 || p->dir_cycle > 7) { snprintf(why, n, "dir_cycle must lie in [0, 7]"); return false; }
    if (p->kernel < SWE_KERNEL_FUSED || p->kernel > SWE_KERNEL_PAPER_SHARED_DEVDT) { snprintf(why, n, "bad kernel"); return false; }
    if (p->seg_rows < 0 || p->seg_rows > 4096 || p->cta_warps < 0 || p->cta_warps > 16) {
        snprintf(why, n, "bad seg_rows / cta_warps"); return false;
    }
    if (p->friction < 0 || p->friction > 1 || p->dissipation < 0 || p->dissipation > 1) {
        snprintf(why, n, "friction and dissipation must be 0 or 1"); return false;
    }
    return true;
}

template <class F>
void free_all(swe_ctx* c, F&& f) {
    for (int b = 0; b < 2; ++b) { f(c->eta[b]); f(c->u[b]); f(c->v[b]); f(c->seg_wet[b]); }
    f(c->z); f(c->z64); f(c->n2);
    for (int q = 0; q < 3; ++q) f(c->ps[q]);
    f(c->ctl); f(c->diag); f(c->diag_part); f(c->diag_wet); f(c->diag_bad);
    f(c->dt_hist); f(c->dt_fixed); f(c->stage); f(c->seg_same); f(c->bad_flag);
}

swe_status ensure_stage(swe_ctx* c, size_t elems) {
    if (c->stage_elems >= elems) return SWE_OK;
    if (c->stage) cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_elems = 0;
    CK(c, cudaMalloc(&c->stage, elems * sizeof(double)));
    c->stage_elems = elems;
    return SWE_OK;
}

swe_status ensure_hist(swe_ctx* c, int n) {
    if (n <= c->dt_hist_cap) return SWE_OK;
    int cap = n < 1024 ? 1024 : n;
    if (c->dt_hist) cudaFree(c->dt_hist);
    c->dt_hist = nullptr;
    c->dt_hist_cap = 0;
    CK(c, cudaMalloc(&c->dt_hist, (size_t)cap * sizeof(double)));
    c->dt_hist_cap = cap;
    return SWE_OK;
}

swe_status ensure_fixed(swe_ctx* c, int n) {
    if (n <= c->dt_fixed_alloc) return SWE_OK;
    int cap = n < 1024 ? 1024 : n;
    if (c->dt_fixed) cudaFree(c->dt_fixed);
    c->dt_fixed = nullptr;
    c->dt_fixed_alloc = 0;
    CK(c, cudaMalloc(&c->dt_fixed, (size_t)cap * sizeof(double)));
    c->dt_fixed_alloc = cap;
    return SWE_OK;
}

swe_status check_ctx(swe_ctx* c) {
    if (!c) return SWE_ERR_ARG;
    if (c->poisoned) return fail(c, SWE_ERR_STATE, "context poisoned by an earlier CUDA error");
    cudaError_t e = cudaSetDevice(c->p.device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return SWE_OK;
}

// After set_state: the first step's CFL reduction and the dry-skip flags.
swe_status after_state(swe_ctx* c) {
    CK(c, swe_launch_prologue(c));
    if (c->p.kernel == SWE_KERNEL_FUSED) CK(c, swe_fused_prepare(c));
    c->state_set = true;
    return SWE_OK;
}

}  // namespace

extern "C" {

void swe_params_default(swe_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nx = 1; p->ny = 1;
    p->dx = 1.0; p->dy = 1.0;
    p->g = 9.81; p->cfl = 0.5; p->h_dry = 1e-3; p->dt_max = 10.0;
    p->kappa = 0.0; p->manning_n = 0.0;
    p->precision = SWE_FP64;
    p->dir_cycle = 1;
    p->device = 0;
    p->kernel = SWE_KERNEL_FUSED;
    p->use_graph = 1;
    p->dry_skip = 1;
}

const char* swe_status_string(swe_status s) {
    switch (s) {
    case SWE_OK: return "ok";
    case SWE_ERR_ARG: return "invalid argument";
    case SWE_ERR_CUDA: return "CUDA error";
    case SWE_ERR_NONFINITE: return "non-finite state";
    case SWE_ERR_NEGDEPTH: return "negative depth";
    case SWE_ERR_TIMEOUT: return "device wait timed out";
    case SWE_ERR_STATE: return "call out of order or context poisoned";
    case SWE_ERR_UNSUPPORTED: return "unsupported configuration";
    case SWE_ERR_CHECK: return "device-side check failed";
    }
    return "unknown status";
}

const char* swe_last_error(const swe_ctx* c) { return c ? c->err : "no context"; }

void* swe_stream(const swe_ctx* c) { return c ? (void*)c->stream : nullptr; }

swe_status swe_create(const swe_params* p, swe_ctx** out) {
    if (!out) return SWE_ERR_ARG;
    *out = nullptr;
    char why[256];
    if (!params_ok(p, why, sizeof(why))) return SWE_ERR_ARG;
    // the ablation forms run in the plain and paper-layout kernels only
    if ((p->friction != 0 || p->dissipation != 0) && p->kernel == SWE_KERNEL_FUSED) return SWE_ERR_UNSUPPORTED;
    swe_ctx* c = new (std::nothrow) swe_ctx();
    if (!c) return SWE_ERR_ARG;
    memset(c->err, 0, sizeof(c->err));
    c->p = *p;
    c->real_size = p->precision == SWE_FP64 ? 8 : 4;
    c->pitch = ((p->nx + 31) / 32) * 32;
    c->plane = (size_t)c->pitch * p->ny;
    auto bail = [&](cudaError_t e, const char* what) {
        fprintf(stderr, "swe_create: %s: %s\n", what, cudaGetErrorString(e));
        free_all(c, [](void* q) { if (q) cudaFree(q); });
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        if (c->h_ctl) cudaFreeHost(c->h_ctl);
        swe_fused_release(c);
        swe_paper_release(c);
        delete c;
        return SWE_ERR_CUDA;
    };
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return bail(e, "cudaSetDevice");
    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(e, "cudaStreamCreate");
        c->own_stream = true;
    }
    const size_t bytes = c->plane * c->real_size;
#ifdef SWE_CHECKED
    // every byte 0xff (a NaN in FP32 and FP64) until set: a read of a plane's
    // padding or of a cell never written shows as a non-finite state
    const int fill = 0xff;
#else
    const int fill = 0;
#endif
    for (int b = 0; b < 2; ++b) {
        void** bufs[3] = {&c->eta[b], &c->u[b], &c->v[b]};
        for (void** q : bufs) {
            if ((e = cudaMalloc(q, bytes)) != cudaSuccess) return bail(e, "cudaMalloc state");
            if ((e = cudaMemset(*q, fill, bytes)) != cudaSuccess) return bail(e, "cudaMemset");
        }
    }
    if ((e = cudaMalloc(&c->z, bytes)) != cudaSuccess) return bail(e, "cudaMalloc bed");
    if ((e = cudaMemset(c->z, fill, bytes)) != cudaSuccess) return bail(e, "cudaMemset");
    if ((e = cudaMalloc(&c->z64, (size_t)p->nx * p->ny * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc bed64");
    if ((e = cudaMemset(c->z64, 0, (size_t)p->nx * p->ny * sizeof(double))) != cudaSuccess) return bail(e, "cudaMemset");
    if (p->kernel == SWE_KERNEL_PLAIN) {
        for (int q = 0; q < 3; ++q)
            if ((e = cudaMalloc(&c->ps[q], bytes)) != cudaSuccess) return bail(e, "cudaMalloc scratch");
    }
    if ((e = cudaMalloc(&c->ctl, sizeof(DevCtl))) != cudaSuccess) return bail(e, "cudaMalloc ctl");
    if ((e = cudaMemset(c->ctl, 0, sizeof(DevCtl))) != cudaSuccess) return bail(e, "cudaMemset");
    if ((e = cudaMallocHost(&c->h_ctl, sizeof(DevCtl))) != cudaSuccess) return bail(e, "cudaMallocHost");
    c->diag_blocks = 1024;
    if ((e = cudaMalloc(&c->diag, sizeof(DevDiag))) != cudaSuccess) return bail(e, "cudaMalloc diag");
    if ((e = cudaMalloc(&c->diag_part, c->diag_blocks * sizeof(double))) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c->diag_wet, c->diag_blocks * sizeof(long long))) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c->diag_bad, sizeof(unsigned int))) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c->bad_flag, sizeof(unsigned int))) != cudaSuccess) return bail(e, "cudaMalloc");
    c->cur = 0;
    c->step = 0;
    c->own_lo = 0;
    c->own_hi = p->ny;
    // the set-up memsets ran on the legacy default stream, which the
    // context's non-blocking stream does not wait for
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(e, "cudaDeviceSynchronize");
    *out = c;
    if (ensure_hist(c, 1024) != SWE_OK) { swe_destroy(c); *out = nullptr; return SWE_ERR_CUDA; }
    return SWE_OK;
}

void swe_destroy(swe_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->p.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 6; ++b)
            if (c->graph[a][b]) cudaGraphExecDestroy(c->graph[a][b]);
    free_all(c, [](void* q) { if (q) cudaFree(q); });
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    swe_fused_release(c);  // work plan
    swe_paper_release(c);
    delete c;
}

swe_status swe_set_clock(swe_ctx* c, int64_t step, double t) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return s;
    if (step < 0 || !std::isfinite(t)) return fail(c, SWE_ERR_ARG, "bad clock");
    // the CFL slot of the current level moves with the step index
    if (c->state_set) {
        CK(c, cudaStreamSynchronize(c->stream));
        CK(c, cudaMemcpy(c->h_ctl, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost));
        unsigned long long m = c->h_ctl->smax[c->step % 3];
        c->h_ctl->smax[0] = c->h_ctl->smax[1] = c->h_ctl->smax[2] = 0ull;
        c->h_ctl->smax[step % 3] = m;
    } else {
        CK(c, cudaMemcpy(c->h_ctl, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost));
    }
    c->h_ctl->t = t;
    CK(c, cudaMemcpy(c->ctl, c->h_ctl, sizeof(DevCtl), cudaMemcpyHostToDevice));
    c->step = step;
    return SWE_OK;
}

swe_status swe_set_bed(swe_ctx* c, const double* z, const double* n_field) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return s;
    if (!z) return fail(c, SWE_ERR_ARG, "z is NULL");
    const size_t n = (size_t)c->p.nx * c->p.ny;
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(z[k])) return fail(c, SWE_ERR_ARG, "non-finite bed at %zu", k);
    if (n_field)
        for (size_t k = 0; k < n; ++k)
            if (!std::isfinite(n_field[k]) || n_field[k] < 0) return fail(c, SWE_ERR_ARG, "bad n_field at %zu", k);
    if ((s = ensure_stage(c, 3 * n)) != SWE_OK) return s;
    CK(c, cudaMemcpyAsync(c->z64, z, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c, swe_launch_to_real(c, c->z64, c->z, 1, false));
    if (n_field) {
        if (!c->n2) CK(c, cudaMalloc(&c->n2, c->plane * c->real_size));
        CK(c, cudaMemcpyAsync(c->stage, n_field, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(c, swe_launch_to_real(c, c->stage, c->n2, 1, true));
    } else if (c->n2) {
        CK(c, cudaFree(c->n2));
        c->n2 = nullptr;
    }
    CK(c, cudaStreamSynchronize(c->stream));
    swe_paper_bed_changed(c);
    c->state_set = false;  // the state must be set (and normalised) against the new bed
    return SWE_OK;
}

swe_status swe_set_bed_device(swe_ctx* c, const void* z, const void* n_field) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return s;
    if (!z) return fail(c, SWE_ERR_ARG, "z is NULL");
    CK(c, swe_launch_dense_copy(c, z, c->z, true));
    CK(c, swe_launch_to_double(c, c->z, c->z64));
    swe_paper_bed_changed(c);
    if (n_field) {
        if (!c->n2) CK(c, cudaMalloc(&c->n2, c->plane * c->real_size));
        // a device n field is given as g*n^2 is not assumed: convert n -> g n^2 through FP64
        const size_t n = (size_t)c->p.nx * c->p.ny;
        if ((s = ensure_stage(c, 3 * n)) != SWE_OK) return s;
        CK(c, swe_launch_dense_copy(c, n_field, c->n2, true));
        CK(c, swe_launch_to_double(c, c->n2, c->stage));
        CK(c, swe_launch_to_real(c, c->stage, c->n2, 1, true));
    } else if (c->n2) {
        CK(c, cudaStreamSynchronize(c->stream));
        CK(c, cudaFree(c->n2));
        c->n2 = nullptr;
    }
    c->state_set = false;
    return SWE_OK;
}

// Reads the set-state rejection bits, then prepares the first step.
static swe_status finish_state(swe_ctx* c) {
    CK(c, cudaMemcpyAsync(&c->h_ctl->pad, c->bad_flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    unsigned int bad = c->h_ctl->pad;
    if (bad & 1u) { c->state_set = false; return fail(c, SWE_ERR_ARG, "non-finite value in the state or bed"); }
    if (bad & 2u) { c->state_set = false; return fail(c, SWE_ERR_NEGDEPTH, "depth below -1e-12 m"); }
    return after_state(c);
}

swe_status swe_set_state(swe_ctx* c, const double* eta, const double* u, const double* v) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return s;
    if (!eta || !u || !v) return fail(c, SWE_ERR_ARG, "NULL state array");
    const size_t n = (size_t)c->p.nx * c->p.ny;
    if ((s = ensure_stage(c, 3 * n)) != SWE_OK) return s;
    CK(c, cudaMemcpyAsync(c->stage, eta, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->stage + n, u, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(c->stage + 2 * n, v, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    // checked and normalised in FP64 against the FP64 bed, then rounded
    CK(c, cudaMemsetAsync(c->bad_flag, 0, sizeof(unsigned int), c->stream));
    CK(c, swe_launch_normalise64(c, c->stage, c->bad_flag));
    CK(c, swe_launch_to_real(c, c->stage, c->eta[c->cur], 1, false));
    CK(c, swe_launch_to_real(c, c->stage + n, c->u[c->cur], 1, false));
    CK(c, swe_launch_to_real(c, c->stage + 2 * n, c->v[c->cur], 1, false));
    return finish_state(c);
}

swe_status swe_set_state_device(swe_ctx* c, const void* eta, const void* u, const void* v) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return s;
    if (!eta || !u || !v) return fail(c, SWE_ERR_ARG, "NULL state array");
    CK(c, swe_launch_dense_copy(c, eta, c->eta[c->cur], true));
    CK(c, swe_launch_dense_copy(c, u, c->u[c->cur], true));
    CK(c, swe_launch_dense_copy(c, v, c->v[c->cur], true));
    CK(c, cudaMemsetAsync(c->bad_flag, 0, sizeof(unsigned int), c->stream));
    CK(c, swe_launch_normalise(c, c->bad_flag));
    return finish_state(c);
}

swe_status swe_get_state(swe_ctx* c, double* eta, double* u, double* v) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return s;
    if (!eta || !u || !v) return fail(c, SWE_ERR_ARG, "NULL state array");
    const size_t n = (size_t)c->p.nx * c->p.ny;
    if ((s = ensure_stage(c, 3 * n)) != SWE_OK) return s;
    CK(c, swe_launch_to_double(c, c->eta[c->cur], c->stage));
    CK(c, swe_launch_to_double(c, c->u[c->cur], c->stage + n));
    CK(c, swe_launch_to_double(c, c->v[c->cur], c->stage + 2 * n));
    CK(c, cudaMemcpyAsync(eta, c->stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(u, c->stage + n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(v, c->stage + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return SWE_OK;
}

swe_status swe_get_state_device(swe_ctx* c, void* eta, void* u, void* v) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return s;
    if (!eta || !u || !v) return fail(c, SWE_ERR_ARG, "NULL state array");
    CK(c, swe_launch_dense_copy(c, c->eta[c->cur], eta, false));
    CK(c, swe_launch_dense_copy(c, c->u[c->cur], u, false));
    CK(c, swe_launch_dense_copy(c, c->v[c->cur], v, false));
    return SWE_OK;
}

static swe_status fill_info(swe_ctx* c, swe_step_info* info, bool run_diag) {
    if (run_diag) CK(c, swe_launch_diag(c));
    DevDiag d;
    CK(c, cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
    if (run_diag) CK(c, cudaMemcpyAsync(&d, c->diag, sizeof(DevDiag), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (!info) return SWE_OK;
    const DevCtl& h = *c->h_ctl;
    memset(info, 0, sizeof(*info));
    info->t = h.t;
    info->dt_last = h.dt_last;
    info->dt_min = h.dt_min > 1e299 ? 0.0 : h.dt_min;
    info->dt_max_seen = h.dt_maxs;
    info->clamp_volume = h.clamp;
    for (int s = 0; s < 4; ++s) info->bflux[s] = h.bflux[s];
    info->step = c->step;
    info->flags = (int32_t)h.flags;
    if (run_diag) {
        info->volume = d.volume;
        info->n_wet = d.n_wet;
        if (d.nonfinite) info->flags |= SWE_FLAG_NONFINITE;
    }
    return SWE_OK;
}

swe_status swe_get_info(swe_ctx* c, swe_step_info* info) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return s;
    if (!info) return fail(c, SWE_ERR_ARG, "info is NULL");
    return fill_info(c, info, true);
}

swe_status swe_step(swe_ctx* c, int32_t nsteps, const double* dt_fixed, double* dt_out, swe_step_info* info) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return s;
    if (!c->state_set) return fail(c, SWE_ERR_STATE, "swe_set_state must come first");
    if (nsteps < 0) return fail(c, SWE_ERR_ARG, "nsteps < 0");
    if (dt_fixed)
        for (int q = 0; q < nsteps; ++q)
            if (!(dt_fixed[q] > 0) || !std::isfinite(dt_fixed[q])) return fail(c, SWE_ERR_ARG, "dt_fixed[%d] invalid", q);
    if ((s = ensure_hist(c, nsteps)) != SWE_OK) return s;
    c->dt_fixed_cap = 0;
    if (dt_fixed && nsteps > 0) {
        if ((s = ensure_fixed(c, nsteps)) != SWE_OK) return s;
        CK(c, cudaMemcpyAsync(c->dt_fixed, dt_fixed, (size_t)nsteps * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        c->dt_fixed_cap = nsteps;
    }
    CK(c, swe_launch_call_begin(c));
    if (c->p.kernel == SWE_KERNEL_FUSED) {
        CK(c, swe_fused_run(c, nsteps));
    } else if (c->p.kernel == SWE_KERNEL_PLAIN) {
        for (int q = 0; q < nsteps; ++q) {
            CK(c, swe_launch_plain_step(c, q, c->step + q));
            c->cur = 1 - c->cur;
        }
    } else {
        for (int q = 0; q < nsteps; ++q) {
            CK(c, swe_launch_paper_step(c, q, c->step + q));
            c->cur = 1 - c->cur;
        }
    }
    c->step += nsteps;
    if (dt_out && nsteps > 0)
        CK(c, cudaMemcpyAsync(dt_out, c->dt_hist, (size_t)nsteps * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    swe_step_info local;
    if ((s = fill_info(c, info ? info : &local, info != nullptr)) != SWE_OK) return s;
    if (c->h_ctl->flags & SWE_FLAG_TIMEOUT) return fail(c, SWE_ERR_TIMEOUT, "a device-side wait gave up");
    if (c->h_ctl->flags & SWE_FLAG_CHECK)
        return fail(c, SWE_ERR_CHECK, "a device-side index or alignment check failed (checked build)");
    if ((c->h_ctl->flags & SWE_FLAG_NONFINITE) || (info && (info->flags & SWE_FLAG_NONFINITE)))
        return fail(c, SWE_ERR_NONFINITE, "non-finite value in the state");
    return SWE_OK;
}

int32_t swe_autotune_candidates(swe_ctx* c, int32_t* rows, int32_t cap) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return -(int32_t)s;
    if (c->p.kernel != SWE_KERNEL_FUSED)
        return -(int32_t)fail(c, SWE_ERR_UNSUPPORTED, "only the fused step has a work-item shape to tune");
    if (!rows || cap < 1) return -(int32_t)fail(c, SWE_ERR_ARG, "rows is NULL or cap < 1");
    return swe_fused_row_candidates(c, rows, cap);
}

swe_status swe_autotune(swe_ctx* c, int32_t probe_steps, const int32_t* rows, int32_t nrows, double* ms_per_step,
                        int32_t* chosen) {
    swe_status s = check_ctx(c);
    if (s != SWE_OK) return s;
    if (!c->state_set) return fail(c, SWE_ERR_STATE, "swe_set_state must come first");
    if (c->p.kernel != SWE_KERNEL_FUSED) return fail(c, SWE_ERR_UNSUPPORTED, "only the fused step has a work-item shape to tune");
    if (probe_steps < 1 || probe_steps > 10000) return fail(c, SWE_ERR_ARG, "probe_steps must lie in [1, 10000]");
    std::vector<int> cand;
    if (rows) {
        if (nrows < 1) return fail(c, SWE_ERR_ARG, "nrows < 1");
        for (int i = 0; i < nrows; ++i) {
            if (rows[i] < 1 || rows[i] > 4096) return fail(c, SWE_ERR_ARG, "rows[%d] must lie in [1, 4096]", i);
            cand.push_back(rows[i]);
        }
    } else {
        if (ms_per_step) return fail(c, SWE_ERR_ARG, "ms_per_step needs the candidate list");
        int tmp[16];
        const int n = swe_fused_row_candidates(c, tmp, 16);
        cand.assign(tmp, tmp + n);
    }
    if ((s = ensure_hist(c, probe_steps)) != SWE_OK) return s;
    c->dt_fixed_cap = 0;
    // the state, clock and tallies to come back to after every probe
    const int cur0 = c->cur;
    const long long step0 = c->step;
    const size_t bytes = c->plane * (size_t)c->real_size;
    DevCtl saved;
    CK(c, cudaMemcpyAsync(&saved, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    struct Scratch {
        void* p[3] = {nullptr, nullptr, nullptr};
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Scratch() {
            for (void* q : p)
                if (q) cudaFree(q);
            for (cudaEvent_t q : e)
                if (q) cudaEventDestroy(q);
        }
    } k;
    void* live[3] = {c->eta[cur0], c->u[cur0], c->v[cur0]};
    for (int f = 0; f < 3; ++f) {
        CK(c, cudaMalloc(&k.p[f], bytes));
        CK(c, cudaMemcpyAsync(k.p[f], live[f], bytes, cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(c, cudaEventCreate(&k.e[0]));
    CK(c, cudaEventCreate(&k.e[1]));
    auto restore = [&]() -> cudaError_t {
        c->cur = cur0;
        c->step = step0;
        cudaError_t e = cudaSuccess;
        for (int f = 0; f < 3 && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(live[f], k.p[f], bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->ctl, &saved, sizeof(DevCtl), cudaMemcpyHostToDevice, c->stream);
        return e;
    };
    int best = -1;
    float best_ms = 0.f;
    for (size_t i = 0; i < cand.size(); ++i) {
        c->p.seg_rows = cand[i];
        CK(c, swe_fused_prepare(c));
        CK(c, restore());
        CK(c, swe_launch_call_begin(c));
        CK(c, swe_fused_run(c, 1));  // warm-up
        c->step += 1;
        CK(c, cudaEventRecord(k.e[0], c->stream));
        CK(c, swe_fused_run(c, probe_steps));
        CK(c, cudaEventRecord(k.e[1], c->stream));
        CK(c, cudaEventSynchronize(k.e[1]));
        float ms = 0.f;
        CK(c, cudaEventElapsedTime(&ms, k.e[0], k.e[1]));
        ms /= (float)probe_steps;
        if (ms_per_step) ms_per_step[i] = ms;
        if (best < 0 || ms < best_ms) { best = (int)i; best_ms = ms; }
        unsigned flags = 0;
        CK(c, cudaMemcpy(&flags, &c->ctl->flags, sizeof(unsigned), cudaMemcpyDeviceToHost));
        if (flags & SWE_FLAG_TIMEOUT) {
            c->p.seg_rows = 0;
            return fail(c, SWE_ERR_TIMEOUT, "a device-side wait gave up while probing %d rows", cand[i]);
        }
    }
    c->p.seg_rows = cand[best];
    CK(c, swe_fused_prepare(c));
    CK(c, restore());
    CK(c, cudaStreamSynchronize(c->stream));
    if (chosen) *chosen = cand[best];
    return SWE_OK;
}

}  // extern "C"
