// swe_adjoint.cu -- discrete adjoint of the time step (reverse mode) for the
// gradient of a gauge-misfit loss with respect to the per-cell Manning n and
// the initial elevation.
//
// The step is differentiated with its step size frozen (the CFL minimum is
// not differentiable) and in the regime where it is smooth: no dissipation
// (kappa = 0) and every cell wet, so the wet/dry fixes are the identity.
// The bed elevation enters the step only through the depth h = eta - z (and
// the ghost cells' copy of the adjacent bed), so every cotangent record below
// keeps the part that reached a cell through its depth (h) apart from the
// part that reached its elevation directly (e): the cotangent of eta is
// e + h, that of the bed is -h.
// One reverse step, for the level-n state q^n and the cotangent lambda of
// level n+1:
//   1. recompute the predicted state q* (the plain predictor kernel);
//   2. per cell, the local vector-Jacobian product of its corrector stage
//      (which reads q* at the cell and its two upwind neighbours and q^n at
//      the cell): the parts for the cell and for each neighbour are stored;
//   3. per cell, gather the cotangent of q* from itself and the two cells
//      that read it, then the local product of its predictor stage;
//   4. per cell, gather the cotangent of q^n.
// Gathering instead of scattering keeps the result deterministic.  Ghost
// cells fold their cotangent back into the boundary cell they copy.
//
// The driver checkpoints the state every K steps (K = ceil(sqrt(T)) by
// default), runs the forward, then for each segment from the last one
// recomputes its levels with the plain step (bitwise equal to the fused one)
// and runs the reverse steps.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <vector>

#include "swe_plain.cuh"

namespace swe {
namespace adj {

template <class T>
struct Vjp3 {
    T e, u, v;
};

// Cotangent of a cell: elevation (direct), velocities, and depth.
template <class T>
struct Vjp4 {
    T e, u, v, h;
};

// Cotangent of ghost(in, side) folded into the cotangent of `in` (the ghost
// copies the cell's elevation and bed, hence its depth).
template <class T>
__device__ __forceinline__ void ghost_vjp(const Cell<T>& in, int side, const GridK<T>& G, const Vjp4<T>& lg,
                                          Vjp4<T>& li) {
    li.e += lg.e;
    li.h += lg.h;
    const int bc = G.bc[side];
    const bool xs = side < 2;
    if (bc == BC_WALL) {
        if (xs) { li.u -= lg.u; li.v += lg.v; } else { li.u += lg.u; li.v -= lg.v; }
    } else if (bc == BC_INFLOW) {
        const T h = in.e - in.z;
        if (h > G.h_dry) {  // the ghost velocity q_in / h
            const T sgn = (side == SIDE_W || side == SIDE_S) ? T(1) : T(-1);
            li.h += -sgn * G.qin[side] / (h * h) * (xs ? lg.u : lg.v);
        }
    } else {
        li.u += lg.u; li.v += lg.v;
    }
}

// Local vector-Jacobian product of stage<DX,DY> (swe_cell.cuh) at one cell:
// given the cotangents (le, lu, lv) of its outputs, the cotangents of the
// differenced cell c, its x and y neighbours, the four face fluxes, the
// level-n base values and g n^2.
template <int DX, int DY, class T>
__device__ __forceinline__ void stage_vjp(const Cell<T>& c, const Cell<T>& xn, const Cell<T>& yn, T e0, T u0, T v0,
                                          T gn2, const StepK<T>& S, T h_dry, T le, T lu, T lv, Vjp4<T>& lc,
                                          Vjp4<T>& lx, Vjp4<T>& ly, T (&lf)[4], Vjp3<T>& lb, T& lgn2) {
    // forward values
    const T h = c.e - c.z;
    const bool wet = h > h_dry;
    const T s2 = c.u * c.u + c.v * c.v;
    const T mag = s2 > T(0) ? rsq_sqrt(s2) : T(0);
    const T P = wet ? pow_m43(h) : T(0);
    const T cf = wet ? gn2 * mag * P : T(0);
    const bool xwall = !((xn.e - xn.z) > h_dry) && xn.z > c.e;
    const bool ywall = !((yn.e - yn.z) > h_dry) && yn.z > c.e;
    const T ex = xwall ? c.e : xn.e, ey = ywall ? c.e : yn.e;
    const T D = T(DX), E = T(DY);
    const T dux = D * (xn.u - c.u), dvx = D * (xn.v - c.v), dex = D * (ex - c.e);
    const T duy = E * (yn.u - c.u), dvy = E * (yn.v - c.v), dey = E * (ey - c.e);
    const T au = c.u * (S.dtdx * dux) + c.v * (S.dtdy * duy) + S.g_dtdx * dex;
    const T av = c.u * (S.dtdx * dvx) + c.v * (S.dtdy * dvy) + S.g_dtdy * dey;
    const T r = T(1) / (T(1) + S.dt * cf);
    // continuity: eo = e0 - (dtdx (fe - fw) + dtdy (fn - fs))
    lb.e += le;
    lf[0] += -S.dtdx * le;
    lf[1] += S.dtdx * le;
    lf[2] += -S.dtdy * le;
    lf[3] += S.dtdy * le;
    // momentum: uo = (u0 - au) r, vo = (v0 - av) r
    lb.u += r * lu;
    lb.v += r * lv;
    const T lau = -r * lu, lav = -r * lv;
    const T lr = (u0 - au) * lu + (v0 - av) * lv;
    const T lcf = -S.dt * r * r * lr;
    lc.u += S.dtdx * dux * lau + S.dtdx * dvx * lav;
    lc.v += S.dtdy * duy * lau + S.dtdy * dvy * lav;
    const T ldux = c.u * S.dtdx * lau, lduy = c.v * S.dtdy * lau, ldex = S.g_dtdx * lau;
    const T ldvx = c.u * S.dtdx * lav, ldvy = c.v * S.dtdy * lav, ldey = S.g_dtdy * lav;
    lx.u += D * ldux; lc.u -= D * ldux;
    lx.v += D * ldvx; lc.v -= D * ldvx;
    ly.u += E * lduy; lc.u -= E * lduy;
    ly.v += E * ldvy; lc.v -= E * ldvy;
    lc.e -= D * ldex + E * ldey;
    if (xwall) lc.e += D * ldex; else lx.e += D * ldex;
    if (ywall) lc.e += E * ldey; else ly.e += E * ldey;
    // friction C = g n^2 |U| h^(-4/3)
    if (wet) {
        lgn2 += mag * P * lcf;
        if (mag > T(0)) {
            lc.u += gn2 * (c.u / mag) * P * lcf;
            lc.v += gn2 * (c.v / mag) * P * lcf;
        }
        lc.h += T(-4) / T(3) * cf / h * lcf;
    }
}

// Face-flux cotangents (fe, fw, fn, fs) of a stage with directions DX, DY at
// cell (i, j) back to the fluxes of the cell and its neighbours, then to
// their eta and velocity (flux = (eta - z) * velocity).
template <int DX, int DY, class T>
__device__ __forceinline__ void faces_vjp(int i, int j, const GridK<T>& G, const Cell<T>& c, const Cell<T>& xn,
                                          const Cell<T>& yn, const T (&lf)[4], Vjp4<T>& lc, Vjp4<T>& lx,
                                          Vjp4<T>& ly) {
    T lqc_x = T(0), lqn_x = T(0), lqc_y = T(0), lqn_y = T(0);
    // east / north faces
    if (i == G.nx - 1) { if (G.bc[SIDE_E] == BC_OUTFLOW) lqc_x += lf[0]; }
    else if (DX > 0) lqn_x += lf[0]; else lqc_x += lf[0];
    if (i == 0) { if (G.bc[SIDE_W] == BC_OUTFLOW) lqc_x += lf[1]; }
    else if (DX > 0) lqc_x += lf[1]; else lqn_x += lf[1];
    if (j == G.ny - 1) { if (G.bc[SIDE_N] == BC_OUTFLOW) lqc_y += lf[2]; }
    else if (DY > 0) lqn_y += lf[2]; else lqc_y += lf[2];
    if (j == 0) { if (G.bc[SIDE_S] == BC_OUTFLOW) lqc_y += lf[3]; }
    else if (DY > 0) lqc_y += lf[3]; else lqn_y += lf[3];
    lc.h += c.u * lqc_x + c.v * lqc_y;
    lc.u += (c.e - c.z) * lqc_x;
    lc.v += (c.e - c.z) * lqc_y;
    lx.h += xn.u * lqn_x;
    lx.u += (xn.e - xn.z) * lqn_x;
    ly.h += yn.v * lqn_y;
    ly.v += (yn.e - yn.z) * lqn_y;
}

template <class T>
__device__ __forceinline__ Cell<T> cell_at(const T* e, const T* u, const T* v, const T* z, size_t k) {
    Cell<T> c;
    c.e = e[k]; c.u = u[k]; c.v = v[k]; c.z = z[k];
    return c;
}

template <class T>
struct Planes3 {
    T* e; T* u; T* v;
};

template <class T>
struct Planes4 {
    T* e; T* u; T* v; T* h;
};

template <class T>
__device__ __forceinline__ void put4(const Planes4<T>& P, size_t k, const Vjp4<T>& a) {
    P.e[k] = a.e; P.u[k] = a.u; P.v[k] = a.v; P.h[k] = a.h;
}

// Step 2: corrector stage VJP (directions -SX, -SY) at every cell.
template <class T, int SX, int SY>
__global__ void __launch_bounds__(256) k_adj_corr(GridK<T> G, StepK<T> S, const T* __restrict__ z,
                                                  const T* __restrict__ n2, Planes3<T> qn, Planes3<T> qs,
                                                  Planes3<T> lam, Planes4<T> Sc, Planes4<T> GX, Planes4<T> GY,
                                                  Planes3<T> Bc, T* __restrict__ ggn2, unsigned* dry) {
    constexpr int CX = -SX, CY = -SY;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const size_t k = (size_t)j * G.pitch + i;
    const Cell<T> cs = cell_at(qs.e, qs.u, qs.v, z, k);
    if (!(cs.e - cs.z > G.h_dry)) atomicOr(dry, 1u);  // outside the differentiated regime
    const bool gx = !(i + CX >= 0 && i + CX < G.nx), gy = !(j + CY >= 0 && j + CY < G.ny);
    const int sidex = CX > 0 ? SIDE_E : SIDE_W, sidey = CY > 0 ? SIDE_N : SIDE_S;
    const Cell<T> xs = gx ? ghost(cs, sidex, G) : cell_at(qs.e, qs.u, qs.v, z, (size_t)((ptrdiff_t)k + CX));
    const Cell<T> ys = gy ? ghost(cs, sidey, G)
                          : cell_at(qs.e, qs.u, qs.v, z, (size_t)((ptrdiff_t)k + (ptrdiff_t)CY * G.pitch));
    const T gn2 = n2 ? n2[k] : G.gn2;
    const T le = T(0.5) * lam.e[k], lu = T(0.5) * lam.u[k], lv = T(0.5) * lam.v[k];
    Vjp4<T> lc{le, lu, lv, 0}, lx{0, 0, 0, 0}, ly{0, 0, 0, 0};  // averaging passes half to q* directly
    Vjp3<T> lb{0, 0, 0};
    T lf[4] = {0, 0, 0, 0}, lg = T(0);
    stage_vjp<CX, CY>(cs, xs, ys, qn.e[k], qn.u[k], qn.v[k], gn2, S, G.h_dry, le, lu, lv, lc, lx, ly, lf, lb, lg);
    faces_vjp<CX, CY>(i, j, G, cs, xs, ys, lf, lc, lx, ly);
    if (gx) { ghost_vjp(cs, sidex, G, lx, lc); lx = Vjp4<T>{0, 0, 0, 0}; }
    if (gy) { ghost_vjp(cs, sidey, G, ly, lc); ly = Vjp4<T>{0, 0, 0, 0}; }
    put4(Sc, k, lc);
    put4(GX, k, lx);
    put4(GY, k, ly);
    Bc.e[k] = lb.e; Bc.u[k] = lb.u; Bc.v[k] = lb.v;
    ggn2[k] += lg;
}

// Step 3: gather the cotangent of q*, then the predictor stage VJP.
template <class T, int SX, int SY>
__global__ void __launch_bounds__(256) k_adj_pred(GridK<T> G, StepK<T> S, const T* __restrict__ z,
                                                  const T* __restrict__ n2, Planes3<T> qn, Planes4<T> Sc,
                                                  Planes4<T> GX, Planes4<T> GY, Planes3<T> Bc, Planes4<T> Pc,
                                                  Planes4<T> PX, Planes4<T> PY, T* __restrict__ ggn2,
                                                  T* __restrict__ ggz, unsigned* dry) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const size_t k = (size_t)j * G.pitch + i;
    // the corrector of cell m reads q* of m - SX and m - SY (its upwind side)
    T ls_e = Sc.e[k], ls_u = Sc.u[k], ls_v = Sc.v[k], ls_h = Sc.h[k];
    if (i + SX >= 0 && i + SX < G.nx) {
        const size_t m = (size_t)((ptrdiff_t)k + SX);
        ls_e += GX.e[m]; ls_u += GX.u[m]; ls_v += GX.v[m]; ls_h += GX.h[m];
    }
    if (j + SY >= 0 && j + SY < G.ny) {
        const size_t m = (size_t)((ptrdiff_t)k + (ptrdiff_t)SY * G.pitch);
        ls_e += GY.e[m]; ls_u += GY.u[m]; ls_v += GY.v[m]; ls_h += GY.h[m];
    }
    // the predicted depth h* = eta* - z (the fix is the identity when wet)
    ls_e += ls_h;
    ggz[k] -= ls_h;
    const Cell<T> c = cell_at(qn.e, qn.u, qn.v, z, k);
    if (!(c.e - c.z > G.h_dry)) atomicOr(dry, 1u);
    const bool gx = !(i + SX >= 0 && i + SX < G.nx), gy = !(j + SY >= 0 && j + SY < G.ny);
    const int sidex = SX > 0 ? SIDE_E : SIDE_W, sidey = SY > 0 ? SIDE_N : SIDE_S;
    const Cell<T> xn = gx ? ghost(c, sidex, G) : cell_at(qn.e, qn.u, qn.v, z, (size_t)((ptrdiff_t)k + SX));
    const Cell<T> yn = gy ? ghost(c, sidey, G)
                          : cell_at(qn.e, qn.u, qn.v, z, (size_t)((ptrdiff_t)k + (ptrdiff_t)SY * G.pitch));
    const T gn2 = n2 ? n2[k] : G.gn2;
    Vjp4<T> lc{0, 0, 0, 0}, lx{0, 0, 0, 0}, ly{0, 0, 0, 0};
    Vjp3<T> lb{Bc.e[k], Bc.u[k], Bc.v[k]};
    T lf[4] = {0, 0, 0, 0}, lg = T(0);
    stage_vjp<SX, SY>(c, xn, yn, c.e, c.u, c.v, gn2, S, G.h_dry, ls_e, ls_u, ls_v, lc, lx, ly, lf, lb, lg);
    faces_vjp<SX, SY>(i, j, G, c, xn, yn, lf, lc, lx, ly);
    if (gx) { ghost_vjp(c, sidex, G, lx, lc); lx = Vjp4<T>{0, 0, 0, 0}; }
    if (gy) { ghost_vjp(c, sidey, G, ly, lc); ly = Vjp4<T>{0, 0, 0, 0}; }
    lc.e += lb.e; lc.u += lb.u; lc.v += lb.v;
    put4(Pc, k, lc);
    put4(PX, k, lx);
    put4(PY, k, ly);
    ggn2[k] += lg;
}

// Step 4: the cotangent of q^n: the cell's own part and the parts its
// downwind predictor neighbours computed for it.
template <class T, int SX, int SY>
__global__ void __launch_bounds__(256) k_adj_gather(GridK<T> G, Planes4<T> Pc, Planes4<T> PX, Planes4<T> PY,
                                                    Planes3<T> lam, T* __restrict__ ggz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const size_t k = (size_t)j * G.pitch + i;
    T e = Pc.e[k], u = Pc.u[k], v = Pc.v[k], h = Pc.h[k];
    if (i - SX >= 0 && i - SX < G.nx) {
        const size_t m = (size_t)((ptrdiff_t)k - SX);
        e += PX.e[m]; u += PX.u[m]; v += PX.v[m]; h += PX.h[m];
    }
    if (j - SY >= 0 && j - SY < G.ny) {
        const size_t m = (size_t)((ptrdiff_t)k - (ptrdiff_t)SY * G.pitch);
        e += PY.e[m]; u += PY.u[m]; v += PY.v[m]; h += PY.h[m];
    }
    // level n's depth h = eta - z
    lam.e[k] = e + h; lam.u[k] = u; lam.v[k] = v;
    ggz[k] -= h;
}

// Gauge values of a level into out[g]; residuals into lambda_eta at gauges.
template <class T>
__global__ void k_gauge_read(const T* e, const long long* gidx, int ng, int nx, int pitch, double* out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const long long q = gidx[g];
    out[g] = (double)e[(size_t)(q / nx) * pitch + (size_t)(q % nx)];
}
template <class T>
__global__ void k_gauge_add(T* le, const long long* gidx, int ng, int nx, int pitch, const double* res) {
    // gauges may repeat: one thread adds them all in order
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int g = 0; g < ng; ++g) {
        const long long q = gidx[g];
        le[(size_t)(q / nx) * pitch + (size_t)(q % nx)] += (T)res[g];
    }
}

// Flags a level that has a cell at or below the wet threshold.
template <class T>
__global__ void k_wet_check(const T* e, const T* z, int nx, int ny, int pitch, T h_dry, unsigned* dry) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const size_t k = (size_t)j * pitch + i;
    if (!(e[k] - z[k] > h_dry)) atomicOr(dry, 1u);
}

template <class T>
__global__ void k_zero(T* p, size_t n) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) p[q] = T(0);
}

}  // namespace adj
}  // namespace swe

using namespace swe;
using namespace swe::adj;

namespace {

swe_status afail(swe_ctx* c, swe_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
    return s;
}

struct DevBuf {  // freed at scope exit; cleared on the context's stream
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit DevBuf(cudaStream_t s) : st(s) {}
    ~DevBuf() {
        cudaStreamSynchronize(st);
        for (void* p : ptrs) cudaFree(p);
    }
    template <class U>
    cudaError_t get(U** p, size_t bytes) {
        cudaError_t e = cudaMalloc((void**)p, bytes);
        if (e == cudaSuccess) { ptrs.push_back((void*)*p); e = cudaMemsetAsync((void*)*p, 0, bytes, st); }
        return e;
    }
};

#define ACK(expr)                                                                              \
    do {                                                                                       \
        cudaError_t e__ = (expr);                                                              \
        if (e__ != cudaSuccess) {                                                              \
            c->poisoned = true;                                                                \
            return afail(c, SWE_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e__));           \
        }                                                                                      \
    } while (0)

template <class T>
GridK<T> grid_k(const swe_ctx* c) {
    GridK<T> G;
    const swe_params& p = c->p;
    G.nx = p.nx; G.ny = p.ny; G.pitch = c->pitch;
    G.g = (T)p.g; G.h_dry = (T)p.h_dry; G.kappa = (T)p.kappa;
    G.gn2 = (T)(p.g * p.manning_n * p.manning_n);
    G.inv_dx = (T)(1.0 / p.dx); G.inv_dy = (T)(1.0 / p.dy);
    for (int s = 0; s < 4; ++s) { G.bc[s] = p.bc[s]; G.qin[s] = (T)p.q_in[s]; }
    return G;
}

// One plain step on given buffers with a frozen step size (device pointer).
template <class T, int SX, int SY>
void plain_step_raw(const swe_ctx* c, const GridK<T>& G, DevCtl* ctl, const double* dtp, Planes3<T> in,
                    Planes3<T> ps, Planes3<T> out) {
    const swe_params& p = c->p;
    dim3 blk(32, 8), grd((p.nx + 31) / 32, (p.ny + 7) / 8);
    const double area = p.dx * p.dy;
    k_plain_pred<T, SX, SY><<<grd, blk, 0, c->stream>>>(G, dtp, p.dx, p.dy, p.g, in.e, in.u, in.v, (const T*)c->z,
                                                        (const T*)c->n2, ps.e, ps.u, ps.v, ctl, area);
    k_plain_corr<T, SX, SY><<<grd, blk, 0, c->stream>>>(G, ctl, dtp, p.dx, p.dy, p.g, in.e, in.u, in.v,
                                                        (const T*)c->z, (const T*)c->n2, ps.e, ps.u, ps.v, out.e,
                                                        out.u, out.v, 1, area);
}

template <class T, int SX, int SY>
void adj_step_raw(const swe_ctx* c, const GridK<T>& G, double dt, DevCtl* ctl, const double* dtp, Planes3<T> qn,
                  Planes3<T> qs, Planes3<T> lam, Planes4<T> Sc, Planes4<T> GX, Planes4<T> GY, Planes3<T> Bc,
                  Planes4<T> Pc, Planes4<T> PX, Planes4<T> PY, T* ggn2, T* ggz, unsigned* dry) {
    const swe_params& p = c->p;
    dim3 blk(32, 8), grd((p.nx + 31) / 32, (p.ny + 7) / 8);
    const StepK<T> S = make_stepk<T>(dt, 1.0 / p.dx, 1.0 / p.dy, p.g);
    // 1. the predicted state of this level
    k_plain_pred<T, SX, SY><<<grd, blk, 0, c->stream>>>(G, dtp, p.dx, p.dy, p.g, qn.e, qn.u, qn.v, (const T*)c->z,
                                                        (const T*)c->n2, qs.e, qs.u, qs.v, ctl, p.dx * p.dy);
    // 2-4. corrector VJP, gather + predictor VJP, gather
    k_adj_corr<T, SX, SY><<<grd, blk, 0, c->stream>>>(G, S, (const T*)c->z, (const T*)c->n2, qn, qs, lam, Sc, GX,
                                                      GY, Bc, ggn2, dry);
    k_adj_pred<T, SX, SY><<<grd, blk, 0, c->stream>>>(G, S, (const T*)c->z, (const T*)c->n2, qn, Sc, GX, GY, Bc, Pc,
                                                      PX, PY, ggn2, ggz, dry);
    k_adj_gather<T, SX, SY><<<grd, blk, 0, c->stream>>>(G, Pc, PX, PY, lam, ggz);
}

template <class T>
void dispatch_plain(const swe_ctx* c, const GridK<T>& G, long long k, DevCtl* ctl, const double* dtp,
                    Planes3<T> in, Planes3<T> ps, Planes3<T> out) {
    int sx, sy;
    step_dirs(c->p.dir_cycle, k, &sx, &sy);
    if (sx > 0 && sy > 0) plain_step_raw<T, 1, 1>(c, G, ctl, dtp, in, ps, out);
    else if (sx > 0) plain_step_raw<T, 1, -1>(c, G, ctl, dtp, in, ps, out);
    else if (sy > 0) plain_step_raw<T, -1, 1>(c, G, ctl, dtp, in, ps, out);
    else plain_step_raw<T, -1, -1>(c, G, ctl, dtp, in, ps, out);
}

template <class T>
void dispatch_adj(const swe_ctx* c, const GridK<T>& G, long long k, double dt, DevCtl* ctl, const double* dtp,
                  Planes3<T> qn, Planes3<T> qs, Planes3<T> lam, Planes4<T> Sc, Planes4<T> GX,
                  Planes4<T> GY, Planes3<T> Bc, Planes4<T> Pc, Planes4<T> PX, Planes4<T> PY, T* ggn2, T* ggz,
                  unsigned* dry) {
    int sx, sy;
    step_dirs(c->p.dir_cycle, k, &sx, &sy);
#define SWE_ADJ(A_, B_) \
    adj_step_raw<T, A_, B_>(c, G, dt, ctl, dtp, qn, qs, lam, Sc, GX, GY, Bc, Pc, PX, PY, ggn2, ggz, dry)
    if (sx > 0 && sy > 0) SWE_ADJ(1, 1);
    else if (sx > 0) SWE_ADJ(1, -1);
    else if (sy > 0) SWE_ADJ(-1, 1);
    else SWE_ADJ(-1, -1);
#undef SWE_ADJ
}

// Runs the work `enqueue` puts on the context's stream, captured as a CUDA
// graph: segments of the same shape re-use one executable graph (updated in
// place), so a segment costs one launch instead of one per kernel.  When the
// stream cannot be captured the work is enqueued directly and graphs stay off
// for the rest of the call.  `enqueue` must be repeatable: it is called again
// when a capture fails.
struct SegGraph {
    cudaStream_t st;
    bool on;
    cudaGraphExec_t exec = nullptr;
    SegGraph(cudaStream_t s, bool use) : st(s), on(use) {}
    ~SegGraph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
    template <class F>
    cudaError_t run(F&& enqueue) {
        if (on) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                enqueue();
                const cudaError_t le = cudaGetLastError();
                e = cudaStreamEndCapture(st, &g);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess && exec) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(exec, g, &info) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(exec);
                    exec = nullptr;
                }
            }
            if (e == cudaSuccess && !exec) e = cudaGraphInstantiate(&exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e == cudaSuccess) return cudaGraphLaunch(exec, st);
            cudaGetLastError();  // capture unavailable: direct launches from here on
            on = false;
        }
        enqueue();
        return cudaGetLastError();
    }
};

template <class T>
swe_status adjoint_t(swe_ctx* c, int T_, const int64_t* gauges, int ng, const double* obs, int kcp, double* loss,
                     double* grad_n, double* grad_eta0, double* grad_z) {
    const swe_params& p = c->p;
    const size_t plane = c->plane, n = (size_t)p.nx * p.ny;
    const GridK<T> G = grid_k<T>(c);
    const int K = kcp > 0 ? kcp : (int)std::ceil(std::sqrt((double)(T_ > 0 ? T_ : 1)));
    const int nseg = (T_ + K - 1) / K;
    DevBuf buf(c->stream);
    auto planes = [&](Planes3<T>& P) -> cudaError_t {
        cudaError_t e;
        if ((e = buf.get(&P.e, plane * sizeof(T))) != cudaSuccess) return e;
        if ((e = buf.get(&P.u, plane * sizeof(T))) != cudaSuccess) return e;
        return buf.get(&P.v, plane * sizeof(T));
    };
    std::vector<Planes3<T>> cp(nseg > 0 ? nseg : 1), seg(K + 1);
    for (auto& q : cp) ACK(planes(q));
    for (auto& q : seg) ACK(planes(q));
    Planes3<T> qs, lam, Bc;
    Planes3<T>* all3[3] = {&qs, &lam, &Bc};
    for (int q = 0; q < 3; ++q) ACK(planes(*all3[q]));
    Planes4<T> Sc, GX, GY, Pc, PX, PY;
    Planes4<T>* all4[6] = {&Sc, &GX, &GY, &Pc, &PX, &PY};
    for (int q = 0; q < 6; ++q) {
        Planes3<T> t3;
        ACK(planes(t3));
        all4[q]->e = t3.e; all4[q]->u = t3.u; all4[q]->v = t3.v;
        ACK(buf.get(&all4[q]->h, plane * sizeof(T)));
    }
    T *ggn2 = nullptr, *ggz = nullptr;
    ACK(buf.get(&ggn2, plane * sizeof(T)));
    ACK(buf.get(&ggz, plane * sizeof(T)));
    long long* gd = nullptr;
    double *gv = nullptr, *res = nullptr;
    StepSlot* ssd = nullptr;  // per step: the frozen step size and its constants (the recompute kernels read them)
    DevCtl* ctl = nullptr;
    unsigned* dry = nullptr;
    ACK(buf.get(&dry, sizeof(unsigned)));
    ACK(buf.get(&gd, (ng > 0 ? ng : 1) * sizeof(long long)));
    ACK(buf.get(&gv, (size_t)(T_ > 0 ? T_ : 1) * (ng > 0 ? ng : 1) * sizeof(double)));
    ACK(buf.get(&res, (size_t)(T_ > 0 ? T_ : 1) * (ng > 0 ? ng : 1) * sizeof(double)));
    ACK(buf.get(&ssd, (size_t)(T_ > 0 ? T_ : 1) * sizeof(StepSlot)));
    ACK(buf.get(&ctl, sizeof(DevCtl)));
    if (ng > 0) ACK(cudaMemcpyAsync(gd, gauges, ng * sizeof(long long), cudaMemcpyHostToDevice, c->stream));

    // ---- forward: the library's own step, checkpoints every K steps, gauge series
    std::vector<double> dts(T_ > 0 ? T_ : 1);
    const long long step0 = c->step;
    SegGraph fgraph(c->stream, c->p.use_graph != 0), rgraph(c->stream, c->p.use_graph != 0);
    if (T_ > 0) {
        if (c->dt_hist_cap < T_) {
            if (c->dt_hist) cudaFree(c->dt_hist);
            c->dt_hist = nullptr;
            ACK(cudaMalloc(&c->dt_hist, (size_t)T_ * sizeof(double)));
            c->dt_hist_cap = T_;
        }
        c->dt_fixed_cap = 0;
        ACK(swe_launch_call_begin(c));
        // segment by segment: its checkpoint, then its steps with the gauge reads
        const int cur0 = c->cur;
        for (int sg = 0; sg < nseg; ++sg) {
            const int s0 = sg * K, s1 = (s0 + K < T_) ? s0 + K : T_;
            cudaError_t le = cudaSuccess;
            auto enqueue = [&]() {
                le = cudaSuccess;
                c->cur = (cur0 + s0) & 1;
                const Planes3<T>& d = cp[sg];
                cudaMemcpyAsync(d.e, c->eta[c->cur], plane * sizeof(T), cudaMemcpyDeviceToDevice, c->stream);
                cudaMemcpyAsync(d.u, c->u[c->cur], plane * sizeof(T), cudaMemcpyDeviceToDevice, c->stream);
                cudaMemcpyAsync(d.v, c->v[c->cur], plane * sizeof(T), cudaMemcpyDeviceToDevice, c->stream);
                for (int s = s0; s < s1 && le == cudaSuccess; ++s) {
                    le = c->p.kernel == SWE_KERNEL_FUSED ? swe_launch_fused_step(c, s, step0 + s)
                                                         : swe_launch_plain_step(c, s, step0 + s);
                    c->cur = 1 - c->cur;
                    if (ng > 0)
                        k_gauge_read<T><<<(ng + 127) / 128, 128, 0, c->stream>>>((const T*)c->eta[c->cur], gd, ng,
                                                                                  p.nx, c->pitch, gv + (size_t)s * ng);
                }
            };
            // the first segment runs uncaptured: it makes the kernels' first launches
            if (sg == 0) {
                enqueue();
                ACK(le);
            } else {
                ACK(fgraph.run(enqueue));
                ACK(le);
            }
        }
        {  // the final level must be wet too
            dim3 blk(32, 8), grd((p.nx + 31) / 32, (p.ny + 7) / 8);
            k_wet_check<T><<<grd, blk, 0, c->stream>>>((const T*)c->eta[c->cur], (const T*)c->z, p.nx, p.ny, c->pitch,
                                                        (T)p.h_dry, dry);
        }
        ACK(cudaGetLastError());
        c->step += T_;
        ACK(cudaMemcpyAsync(dts.data(), c->dt_hist, (size_t)T_ * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    std::vector<double> g((size_t)(T_ > 0 ? T_ : 1) * (ng > 0 ? ng : 1));
    if (T_ > 0 && ng > 0)
        ACK(cudaMemcpyAsync(g.data(), gv, (size_t)T_ * ng * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    ACK(cudaStreamSynchronize(c->stream));
    double L = 0.0;
    for (int s = 0; s < T_; ++s)
        for (int q = 0; q < ng; ++q) {
            const double r = g[(size_t)s * ng + q] - obs[(size_t)s * ng + q];
            g[(size_t)s * ng + q] = r;
            L += 0.5 * r * r;
        }
    if (!std::isfinite(L)) return afail(c, SWE_ERR_NONFINITE, "non-finite loss");
    *loss = L;
    std::vector<StepSlot> slots(T_ > 0 ? T_ : 1);
    for (int s = 0; s < T_; ++s) slots[s] = make_slot(dts[s], 1.0 / p.dx, 1.0 / p.dy, p.g);
    if (T_ > 0)
        ACK(cudaMemcpyAsync(ssd, slots.data(), (size_t)T_ * sizeof(StepSlot), cudaMemcpyHostToDevice, c->stream));
    if (T_ > 0 && ng > 0)
        ACK(cudaMemcpyAsync(res, g.data(), (size_t)T_ * ng * sizeof(double), cudaMemcpyHostToDevice, c->stream));

    // ---- reverse
    const int zb = 1024;
    T* zq[5] = {lam.e, lam.u, lam.v, ggn2, ggz};
    for (int q = 0; q < 5; ++q) k_zero<T><<<zb, 256, 0, c->stream>>>(zq[q], plane);
    if (T_ > 0 && ng > 0) k_gauge_add<T><<<1, 1, 0, c->stream>>>(lam.e, gd, ng, p.nx, c->pitch, res + (size_t)(T_ - 1) * ng);
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int s0 = sg * K, s1 = (s0 + K < T_) ? s0 + K : T_;
        auto enqueue = [&]() {
            // levels s0 .. s1-1 of this segment, recomputed from its checkpoint
            cudaMemcpyAsync(seg[0].e, cp[sg].e, plane * sizeof(T), cudaMemcpyDeviceToDevice, c->stream);
            cudaMemcpyAsync(seg[0].u, cp[sg].u, plane * sizeof(T), cudaMemcpyDeviceToDevice, c->stream);
            cudaMemcpyAsync(seg[0].v, cp[sg].v, plane * sizeof(T), cudaMemcpyDeviceToDevice, c->stream);
            for (int s = s0; s + 1 < s1; ++s)
                dispatch_plain<T>(c, G, step0 + s, ctl, &ssd[s].dt, seg[s - s0], qs, seg[s - s0 + 1]);
            for (int s = s1 - 1; s >= s0; --s) {
                dispatch_adj<T>(c, G, step0 + s, dts[s], ctl, &ssd[s].dt, seg[s - s0], qs, lam, Sc, GX, GY, Bc, Pc, PX,
                                PY, ggn2, ggz, dry);
                if (s >= 1 && ng > 0)
                    k_gauge_add<T><<<1, 1, 0, c->stream>>>(lam.e, gd, ng, p.nx, c->pitch, res + (size_t)(s - 1) * ng);
            }
        };
        // the first segment handled (the last in time) runs uncaptured: first launches
        if (sg == nseg - 1) {
            enqueue();
            ACK(cudaGetLastError());
        } else {
            ACK(rgraph.run(enqueue));
        }
    }
    // ---- outputs: d/d eta0, d/dz, and d/dn = d/d(g n^2) * 2 g n
    unsigned hdry = 0;
    ACK(cudaMemcpyAsync(&hdry, dry, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    ACK(cudaStreamSynchronize(c->stream));
    if (hdry)
        return afail(c, SWE_ERR_UNSUPPORTED,
                     "a cell was at or below the wet threshold during the run: the adjoint covers the fully wet regime");
    std::vector<T> hb(plane), hg(plane), hn(plane), hz(grad_z ? plane : 1);
    ACK(cudaMemcpyAsync(hb.data(), lam.e, plane * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    ACK(cudaMemcpyAsync(hg.data(), ggn2, plane * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    if (grad_z) ACK(cudaMemcpyAsync(hz.data(), ggz, plane * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    if (c->n2) ACK(cudaMemcpyAsync(hn.data(), c->n2, plane * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    ACK(cudaStreamSynchronize(c->stream));
    for (int j = 0; j < p.ny; ++j)
        for (int i = 0; i < p.nx; ++i) {
            const size_t k = (size_t)j * c->pitch + i, o = (size_t)j * p.nx + i;
            if (grad_eta0) grad_eta0[o] = (double)hb[k];
            if (grad_z) grad_z[o] = (double)hz[k];
            if (grad_n) {
                const double gn2 = c->n2 ? (double)hn[k] : p.g * p.manning_n * p.manning_n;
                grad_n[o] = (double)hg[k] * 2.0 * std::sqrt(p.g * gn2);
            }
        }
    (void)n;
    return SWE_OK;
}

}  // namespace

extern "C" swe_status swe_adjoint(swe_ctx* c, int32_t nsteps, const int64_t* gauges, int32_t ngauges,
                                  const double* obs, int32_t checkpoint_every, double* loss, double* grad_n,
                                  double* grad_eta0, double* grad_z) {
    if (!c) return SWE_ERR_ARG;
    if (c->poisoned) return afail(c, SWE_ERR_STATE, "context poisoned by an earlier CUDA error");
    if (cudaSetDevice(c->p.device) != cudaSuccess) return afail(c, SWE_ERR_CUDA, "cudaSetDevice failed");
    if (!c->state_set) return afail(c, SWE_ERR_STATE, "swe_set_state must come first");
    if (nsteps < 0 || ngauges < 0 || (ngauges > 0 && (!gauges || !obs)) || !loss || checkpoint_every < 0)
        return afail(c, SWE_ERR_ARG, "bad adjoint arguments");
    if (c->p.kappa != 0.0) return afail(c, SWE_ERR_UNSUPPORTED, "the adjoint needs kappa = 0");
    if (c->p.friction != 0 || c->p.dissipation != 0)
        return afail(c, SWE_ERR_UNSUPPORTED, "the adjoint differentiates the default friction and dissipation forms");
    if (c->p.kernel != SWE_KERNEL_FUSED && c->p.kernel != SWE_KERNEL_PLAIN)
        return afail(c, SWE_ERR_UNSUPPORTED, "the adjoint runs with the fused or the plain step");
    const long long ncell = (long long)c->p.nx * c->p.ny;
    for (int g = 0; g < ngauges; ++g)
        if (gauges[g] < 0 || gauges[g] >= ncell) return afail(c, SWE_ERR_ARG, "gauge %d out of range", g);
    if (c->real_size == 8)
        return adjoint_t<double>(c, nsteps, gauges, ngauges, obs, checkpoint_every, loss, grad_n, grad_eta0, grad_z);
    return adjoint_t<float>(c, nsteps, gauges, ngauges, obs, checkpoint_every, loss, grad_n, grad_eta0, grad_z);
}
