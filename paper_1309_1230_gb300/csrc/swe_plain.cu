// swe_plain.cu -- the plain GPU step: one thread per cell, the predictor
// (S1-S8) and the corrector with averaging, dissipation and fix (S9-S16) as
// two kernels per step, all data in global memory.  This mirrors the paper's
// non-shared-memory design (Sec. 3.1: kernel boundaries give the intra-step
// synchronisation, one thread per cell), except that the time-step
// reduction stays on the GPU.  It is the FP64/FP32 reference step that the
// fused sweep is compared with, and the utility kernels of the context.
#include "swe_plain.cuh"

namespace swe {

// ---------------------------------------------------------------- utilities
template <class T>
__global__ void k_to_real(const double* __restrict__ src, T* __restrict__ dst, int nx, int ny, int pitch,
                          double scale_sq) {
    size_t n = (size_t)pitch * ny;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(q / pitch), i = (int)(q % pitch);
        double x = (i < nx) ? src[(size_t)j * nx + i] : 0.0;
        if (scale_sq != 0.0) x = scale_sq * x * x;
        dst[q] = (T)x;
    }
}

template <class T>
__global__ void k_to_double(const T* __restrict__ src, double* __restrict__ dst, int nx, int ny, int pitch) {
    size_t n = (size_t)nx * ny;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(q / nx), i = (int)(q % nx);
        dst[q] = (double)src[(size_t)j * pitch + i];
    }
}

template <class T>
__global__ void k_dense_copy(const T* __restrict__ src, T* __restrict__ dst, int nx, int ny, int pitch,
                             int to_pitched) {
    size_t n = (size_t)nx * ny;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        int j = (int)(q / nx), i = (int)(q % nx);
        size_t pq = (size_t)j * pitch + i;
        if (to_pitched) dst[pq] = src[q]; else dst[q] = src[pq];
    }
}

// Set-state normalisation on the context's real type: reject non-finite
// values and depths below -1e-12 m (bad bits 1 and 2), clamp small negative
// depths to zero and zero the velocity of dry cells.
template <class T>
__global__ void k_normalise(T* e, T* u, T* v, const T* z, int nx, int ny, int pitch, T h_dry,
                            unsigned int* bad) {
    size_t n = (size_t)nx * ny;
    unsigned int b = 0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        size_t k = (q / nx) * (size_t)pitch + q % nx;
        T ee = e[k], uu = u[k], vv = v[k], zz = z[k];
        if (!isfinite(ee) || !isfinite(uu) || !isfinite(vv) || !isfinite(zz)) { b |= 1u; continue; }
        T h = ee - zz;
        if (h < T(-1e-12)) { b |= 2u; continue; }
        if (h < T(0)) { ee = zz; h = T(0); }
        if (h <= h_dry) { uu = T(0); vv = T(0); }
        e[k] = ee; u[k] = uu; v[k] = vv;
    }
    if (b) atomicOr(bad, b);
}

// The same normalisation in FP64 on dense staging planes (eta, u, v) against
// the FP64 bed, before the state is rounded to the context's real type.
__global__ void k_normalise64(double* st, const double* z64, size_t n, double h_dry, unsigned int* bad) {
    unsigned int b = 0;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        double ee = st[q], uu = st[n + q], vv = st[2 * n + q], zz = z64[q];
        if (!isfinite(ee) || !isfinite(uu) || !isfinite(vv) || !isfinite(zz)) { b |= 1u; continue; }
        double h = ee - zz;
        if (h < -1e-12) { b |= 2u; continue; }
        if (h < 0.0) { ee = zz; h = 0.0; }
        if (h <= h_dry) { uu = 0.0; vv = 0.0; }
        st[q] = ee; st[n + q] = uu; st[2 * n + q] = vv;
    }
    if (b) atomicOr(bad, b);
}

// CFL reduction of a freshly set state into slot `slot`; the other slots
// are cleared.
template <class T>
__global__ void k_prologue(GridK<T> G, const T* e, const T* u, const T* v, const T* z, DevCtl* ctl, int slot) {
    size_t n = (size_t)G.nx * G.ny;
    T m = T(0);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(q / G.nx);
        size_t k = (size_t)row * G.pitch + q % G.nx;
        T s = cfl_speed(e[k], u[k], v[k], z[k], G);
        if (row < G.own_lo || row >= G.own_hi) s = T(0);
        m = s > m ? s : m;
    }
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0 && m > T(0))
        atomicMax(&ctl->smax[slot], (unsigned long long)__double_as_longlong((double)m));
}

// Diagnostics: per-block FP64 partial volume (fixed row ranges, fixed order)
// and wet count, then one block sums the partials in order.
template <class T>
__global__ void k_diag_part(GridK<T> G, const T* e, const T* u, const T* v, const T* z, double* part,
                            long long* wet, unsigned int* bad, int rows_per_block) {
    __shared__ double sh[32];
    __shared__ long long shw[32];
    const int j0 = blockIdx.x * rows_per_block, j1 = min(G.ny, j0 + rows_per_block);
    double s = 0.0;
    long long w = 0;
    unsigned int b = 0;
    for (int j = j0; j < j1; ++j) {
        if (j < G.own_lo || j >= G.own_hi) continue;  // halo rows of a strip
        for (int i = threadIdx.x; i < G.nx; i += blockDim.x) {
            size_t k = (size_t)j * G.pitch + i;
            double h = (double)e[k] - (double)z[k];
            s += h;
            w += (T)(e[k] - z[k]) > G.h_dry;
            if (!isfinite(e[k]) || !isfinite(u[k]) || !isfinite(v[k])) b = 1;
        }
    }
    s = warp_sum(s);
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[wid] = s; shw[wid] = w; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        long long tw = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { t += sh[q]; tw += shw[q]; }
        part[blockIdx.x] = t;
        wet[blockIdx.x] = tw;
    }
    if (b) atomicOr(bad, 1u);
}

__global__ void k_diag_final(const double* part, const long long* wet, int nparts, DevDiag* out, double area,
                             const unsigned int* bad) {
    double t = 0.0;
    long long w = 0;
    for (int q = 0; q < nparts; ++q) { t += part[q]; w += wet[q]; }
    out->volume = t * area;
    out->n_wet = w;
    out->nonfinite = *bad;
}

__global__ void k_call_begin(DevCtl* ctl) {
    ctl->dt_min = 1e300;
    ctl->dt_maxs = 0.0;
    ctl->flags = 0u;
    ctl->qctr[0] = ctl->qctr[1] = ctl->qctr[2] = 0u;
    for (int q = 0; q < 3; ++q) ctl->wcnt[q][0] = ctl->wcnt[q][1] = 0u;
}

}  // namespace swe

using namespace swe;

static int util_blocks(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

cudaError_t swe_launch_plain_step(swe_ctx* c, int s, long long k) {
    if (c->real_size == 8) return plain_step_dir<double>(c, s, k);
    return plain_step_dir<float>(c, s, k);
}

cudaError_t swe_launch_to_real(swe_ctx* c, const double* src, void* dst, int n_planes, bool square_n) {
    size_t n = c->plane;
    double scale = square_n ? c->p.g : 0.0;
    for (int pl = 0; pl < n_planes; ++pl) {
        const double* s = src + (size_t)pl * c->p.nx * c->p.ny;
        if (c->real_size == 8)
            k_to_real<double><<<util_blocks(n), 256, 0, c->stream>>>(s, (double*)dst + pl * n, c->p.nx, c->p.ny, c->pitch, scale);
        else
            k_to_real<float><<<util_blocks(n), 256, 0, c->stream>>>(s, (float*)dst + pl * n, c->p.nx, c->p.ny, c->pitch, scale);
    }
    return cudaGetLastError();
}

cudaError_t swe_launch_to_double(swe_ctx* c, const void* src, double* dst) {
    size_t n = (size_t)c->p.nx * c->p.ny;
    if (c->real_size == 8)
        k_to_double<double><<<util_blocks(n), 256, 0, c->stream>>>((const double*)src, dst, c->p.nx, c->p.ny, c->pitch);
    else
        k_to_double<float><<<util_blocks(n), 256, 0, c->stream>>>((const float*)src, dst, c->p.nx, c->p.ny, c->pitch);
    return cudaGetLastError();
}

cudaError_t swe_launch_dense_copy(swe_ctx* c, const void* src, void* dst, bool to_pitched) {
    size_t n = (size_t)c->p.nx * c->p.ny;
    if (c->real_size == 8)
        k_dense_copy<double><<<util_blocks(n), 256, 0, c->stream>>>((const double*)src, (double*)dst, c->p.nx, c->p.ny, c->pitch, to_pitched);
    else
        k_dense_copy<float><<<util_blocks(n), 256, 0, c->stream>>>((const float*)src, (float*)dst, c->p.nx, c->p.ny, c->pitch, to_pitched);
    return cudaGetLastError();
}

cudaError_t swe_launch_normalise(swe_ctx* c, unsigned int* bad) {
    size_t n = (size_t)c->p.nx * c->p.ny;
    int a = c->cur;
    if (c->real_size == 8)
        k_normalise<double><<<util_blocks(n), 256, 0, c->stream>>>((double*)c->eta[a], (double*)c->u[a], (double*)c->v[a],
                                                                  (const double*)c->z, c->p.nx, c->p.ny, c->pitch, c->p.h_dry, bad);
    else
        k_normalise<float><<<util_blocks(n), 256, 0, c->stream>>>((float*)c->eta[a], (float*)c->u[a], (float*)c->v[a],
                                                                 (const float*)c->z, c->p.nx, c->p.ny, c->pitch, (float)c->p.h_dry, bad);
    return cudaGetLastError();
}

cudaError_t swe_launch_normalise64(swe_ctx* c, double* stage, unsigned int* bad) {
    size_t n = (size_t)c->p.nx * c->p.ny;
    k_normalise64<<<util_blocks(n), 256, 0, c->stream>>>(stage, c->z64, n, c->p.h_dry, bad);
    return cudaGetLastError();
}

cudaError_t swe_launch_prologue(swe_ctx* c) {
    size_t n = (size_t)c->p.nx * c->p.ny;
    int a = c->cur;
    int slot = (int)(c->step % 3);
    cudaError_t e = cudaMemsetAsync(c->ctl->smax, 0, sizeof(c->ctl->smax), c->stream);
    if (e != cudaSuccess) return e;
    if (c->real_size == 8)
        k_prologue<double><<<util_blocks(n), 256, 0, c->stream>>>(grid_of<double>(c), (const double*)c->eta[a], (const double*)c->u[a],
                                                                 (const double*)c->v[a], (const double*)c->z, c->ctl, slot);
    else
        k_prologue<float><<<util_blocks(n), 256, 0, c->stream>>>(grid_of<float>(c), (const float*)c->eta[a], (const float*)c->u[a],
                                                                (const float*)c->v[a], (const float*)c->z, c->ctl, slot);
    return cudaGetLastError();
}

cudaError_t swe_launch_diag(swe_ctx* c) {
    int a = c->cur;
    int rpb = (c->p.ny + c->diag_blocks - 1) / c->diag_blocks;
    int nb = (c->p.ny + rpb - 1) / rpb;
    cudaError_t e = cudaMemsetAsync(c->diag_bad, 0, sizeof(unsigned int), c->stream);
    if (e != cudaSuccess) return e;
    if (c->real_size == 8)
        k_diag_part<double><<<nb, 256, 0, c->stream>>>(grid_of<double>(c), (const double*)c->eta[a], (const double*)c->u[a],
                                                        (const double*)c->v[a], (const double*)c->z, c->diag_part, c->diag_wet,
                                                        c->diag_bad, rpb);
    else
        k_diag_part<float><<<nb, 256, 0, c->stream>>>(grid_of<float>(c), (const float*)c->eta[a], (const float*)c->u[a],
                                                       (const float*)c->v[a], (const float*)c->z, c->diag_part, c->diag_wet,
                                                       c->diag_bad, rpb);
    k_diag_final<<<1, 1, 0, c->stream>>>(c->diag_part, c->diag_wet, nb, c->diag, c->p.dx * c->p.dy, c->diag_bad);
    return cudaGetLastError();
}

cudaError_t swe_launch_call_begin(swe_ctx* c) {
    k_call_begin<<<1, 1, 0, c->stream>>>(c->ctl);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = swe_fused_reset_flags(c);
    return e;
}

// One plain FP32 step on caller-provided dense buffers (row pitch `pitch`)
// with caller-provided scratch: the predicted planes ps_*, a control block
// (already cleared) and a dt slot.  compute_cfl: run the CFL reduction of the
// input first; otherwise *dt_fixed (device) gives the step size.
cudaError_t swe_plain_step_f32_raw(const swe_params* p, int pitch, const float* z, const float* e, const float* u,
                                   const float* v, float* e1, float* u1, float* v1, float* ps_e, float* ps_u,
                                   float* ps_v, DevCtl* ctl, const double* dt_fixed, double* dt_hist,
                                   cudaStream_t st) {
    GridK<float> G;
    G.nx = p->nx; G.ny = p->ny; G.pitch = pitch;
    G.g = (float)p->g; G.h_dry = (float)p->h_dry; G.kappa = (float)p->kappa;
    G.gn2 = (float)(p->g * p->manning_n * p->manning_n);
    G.inv_dx = (float)(1.0 / p->dx); G.inv_dy = (float)(1.0 / p->dy);
    for (int s = 0; s < 4; ++s) { G.bc[s] = p->bc[s]; G.qin[s] = (float)p->q_in[s]; }
    const size_t n = (size_t)p->nx * p->ny;
    if (!dt_fixed) k_prologue<float><<<util_blocks(n), 256, 0, st>>>(G, e, u, v, z, ctl, 0);
    k_plain_dt<<<1, 1, 0, st>>>(ctl, 0, 1, dt_fixed, 0, dt_hist, p->cfl, p->dt_max, 1.0 / p->dx, 1.0 / p->dy, p->g);
    int sx, sy;
    step_dirs(p->dir_cycle, 0, &sx, &sy);
    dim3 blk(32, 8), grd((p->nx + 31) / 32, (p->ny + 7) / 8);
    const double area = p->dx * p->dy;
#define SWE_RAW_STEP(SX_, SY_)                                                                                   \
    do {                                                                                                         \
        k_plain_pred<float, SX_, SY_><<<grd, blk, 0, st>>>(G, &ctl->cur.dt, p->dx, p->dy, p->g, e, u, v, z,     \
                                                           nullptr, ps_e, ps_u, ps_v, ctl, area);                \
        k_plain_corr<float, SX_, SY_><<<grd, blk, 0, st>>>(G, ctl, &ctl->cur.dt, p->dx, p->dy, p->g, e, u, v, z, \
                                                           nullptr, ps_e, ps_u, ps_v, e1, u1, v1, 1, area);      \
    } while (0)
    if (sx > 0 && sy > 0) SWE_RAW_STEP(1, 1);
    else if (sx > 0) SWE_RAW_STEP(1, -1);
    else if (sy > 0) SWE_RAW_STEP(-1, 1);
    else SWE_RAW_STEP(-1, -1);
#undef SWE_RAW_STEP
    return cudaGetLastError();
}
