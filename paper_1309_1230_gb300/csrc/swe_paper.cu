// swe_paper.cu -- the step in the paper's own GPU layout (Seitz et al. 2013,
// Sec. 3.1): one kernel per sub-step, every intermediate through global
// memory, one thread per cell in one-dimensional blocks along a row, and
// (SWE_KERNEL_PAPER) the step size computed on the host from a
// device-to-host copy of the state before every step, as the paper does to
// avoid a serial reduction on the GPU.  SWE_KERNEL_PAPER_DEVDT keeps the same
// kernels but reduces the CFL speed on the GPU in the last sub-step, as the
// fused and plain steps do.
//
// SWE_KERNEL_PAPER_SHARED (and its _DEVDT form) is the paper's second design
// (Sec. 3.2): the sub-steps that read neighbours run in 16 x 16 blocks with
// the cells and their halo staged in shared memory.
//
// It exists to measure the paper's design next to the fused sweep on the
// same GPU.  The per-cell arithmetic is swe_cell.cuh's, split at the
// sub-step boundaries, so with the same step sizes its results equal the
// plain and fused steps bit for bit.
//
// Sub-steps (one kernel each; S2 is the step size):
//   S1 depth and wet mask       S9  ghost cells of the predicted level
//   S3 ghost cells of level n   S10 fluxes of the predicted level
//   S4 fluxes h u, h v          S11 corrector continuity
//   S5 predictor continuity     S12 friction coefficient, predicted level
//   S6 friction coefficient     S13 corrector momentum
//   S7 predictor momentum       S14 average of predictor and corrector
//   S8 predictor wet/dry fix    S15 dissipation of level n
//                               S16 final wet/dry fix, tallies (and the CFL
//                                   reduction on the GPU in the DEVDT form)
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "swe_plain.cuh"

namespace swe {
namespace pp {

constexpr int BX = 256;  // threads per block, along a row

template <int V>
struct IntC {
    static constexpr int value = V;
};
template <int X, int Y>
struct Dirs {
    static constexpr int x = X, y = Y;
};

template <class T>
struct Ghosts {  // ghost cells of one level, per side (W/E: ny entries, S/N: nx)
    Cell<T>* side[4];
};

template <class T>
struct Scratch {
    T *h, *qx, *qy, *C, *es, *us, *vs, *qxs, *qys, *Cs, *ec, *uc, *vc;
    unsigned char* wet;
    Ghosts<T> gn, gs;
    double* d_dt;          // the step size the host computed
    T *hst_e, *hst_u, *hst_v, *hst_z;  // pinned host copies for the host step size
    bool z_on_host;
};

__device__ __forceinline__ bool cell_of(const int nx, const int ny, int& i, int& j) {
    i = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y;
    return i < nx && j < ny;
}

template <class T>
__device__ __forceinline__ Cell<T> at(const T* e, const T* u, const T* v, const T* z, size_t k) {
    Cell<T> c;
    c.e = e[k]; c.u = u[k]; c.v = v[k]; c.z = z[k];
    return c;
}

// Neighbour of (i, j) in direction (DX, DY) of a level, or its ghost cell.
template <int DX, int DY, class T>
__device__ __forceinline__ Cell<T> nbr(const GridK<T>& G, const T* e, const T* u, const T* v, const T* z,
                                       const Ghosts<T>& g, int i, int j, size_t k) {
    const int ii = i + DX, jj = j + DY;
    if (ii < 0) return g.side[SIDE_W][j];
    if (ii >= G.nx) return g.side[SIDE_E][j];
    if (jj < 0) return g.side[SIDE_S][i];
    if (jj >= G.ny) return g.side[SIDE_N][i];
    return at(e, u, v, z, (size_t)((ptrdiff_t)k + DX + (ptrdiff_t)DY * G.pitch));
}

// Step size and clock bookkeeping of step s (S2's result on the device).
__global__ void k_paper_dt(DevCtl* ctl, const double* dtv, int from_smax, int slot, int slot_next, int s,
                           double* dt_hist, double cfl, double dt_max, double rdx, double rdy, double g) {
    const double dt = from_smax ? dt_from_speed(__longlong_as_double((long long)ctl->smax[slot]), cfl, dt_max) : *dtv;
    ctl->cur = make_slot(dt, rdx, rdy, g);
    ctl->dt_last = dt;
    ctl->t += dt;
    ctl->dt_min = fmin(ctl->dt_min, dt);
    ctl->dt_maxs = fmax(ctl->dt_maxs, dt);
    dt_hist[s] = dt;
    ctl->smax[slot_next] = 0ull;
}

// S1
template <class T>
__global__ void __launch_bounds__(BX) k_s1(GridK<T> G, const T* __restrict__ e, const T* __restrict__ z,
                                           T* __restrict__ h, unsigned char* __restrict__ wet) {
    int i, j;
    if (!cell_of(G.nx, G.ny, i, j)) return;
    const size_t k = (size_t)j * G.pitch + i;
    const T d = e[k] - z[k];
    h[k] = d;
    wet[k] = d > G.h_dry ? 1 : 0;
}

// S3 / S9: the ghost cells of the four sides of one level.
template <class T>
__global__ void k_ghosts(GridK<T> G, const T* __restrict__ e, const T* __restrict__ u, const T* __restrict__ v,
                         const T* __restrict__ z, Ghosts<T> g) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < G.ny) {
        const size_t kw = (size_t)q * G.pitch, ke = kw + (G.nx - 1);
        g.side[SIDE_W][q] = ghost(at(e, u, v, z, kw), SIDE_W, G);
        g.side[SIDE_E][q] = ghost(at(e, u, v, z, ke), SIDE_E, G);
    }
    if (q < G.nx) {
        const size_t ks = (size_t)q, kn = (size_t)(G.ny - 1) * G.pitch + q;
        g.side[SIDE_S][q] = ghost(at(e, u, v, z, ks), SIDE_S, G);
        g.side[SIDE_N][q] = ghost(at(e, u, v, z, kn), SIDE_N, G);
    }
}

// S4 / S10: the cell fluxes h u and h v of a level.
template <class T>
__global__ void __launch_bounds__(BX) k_fluxes(GridK<T> G, const T* __restrict__ e, const T* __restrict__ u,
                                               const T* __restrict__ v, const T* __restrict__ z, T* __restrict__ qx,
                                               T* __restrict__ qy) {
    int i, j;
    if (!cell_of(G.nx, G.ny, i, j)) return;
    const size_t k = (size_t)j * G.pitch + i;
    const T d = e[k] - z[k];
    qx[k] = d * u[k];
    qy[k] = d * v[k];
}

// S5 / S11: continuity with the one-sided face fluxes in directions (DX, DY);
// e0 is level n, the fluxes those of the differenced level.
template <class T, int DX, int DY>
__global__ void __launch_bounds__(BX) k_continuity(GridK<T> G, const double* __restrict__ dtp, double dx, double dy,
                                                   double g, const T* __restrict__ e0, const T* __restrict__ qx,
                                                   const T* __restrict__ qy, Ghosts<T> gh, T* __restrict__ eo) {
    int i, j;
    if (!cell_of(G.nx, G.ny, i, j)) return;
    const StepK<T> S = step_consts<T>(dtp);
    const size_t k = (size_t)j * G.pitch + i;
    T qxn, qyn;
    if (i + DX >= 0 && i + DX < G.nx) qxn = qx[(size_t)((ptrdiff_t)k + DX)];
    else { const Cell<T> q = gh.side[DX > 0 ? SIDE_E : SIDE_W][j]; qxn = (q.e - q.z) * q.u; }
    if (j + DY >= 0 && j + DY < G.ny) qyn = qy[(size_t)((ptrdiff_t)k + (ptrdiff_t)DY * G.pitch)];
    else { const Cell<T> q = gh.side[DY > 0 ? SIDE_N : SIDE_S][i]; qyn = (q.e - q.z) * q.v; }
    T fe, fw, fn, fs;
    faces<DX>(qx[k], qxn, i == 0, i == G.nx - 1, SIDE_W, SIDE_E, G, fe, fw);
    faces<DY>(qy[k], qyn, j == 0, j == G.ny - 1, SIDE_S, SIDE_N, G, fn, fs);
    eo[k] = continuity(e0[k], fe, fw, fn, fs, S);
}

// S6 / S12: the Manning coefficient of a level.
template <class T>
__global__ void __launch_bounds__(BX) k_friction(GridK<T> G, const T* __restrict__ e, const T* __restrict__ u,
                                                 const T* __restrict__ v, const T* __restrict__ z,
                                                 const T* __restrict__ n2, T* __restrict__ C) {
    int i, j;
    if (!cell_of(G.nx, G.ny, i, j)) return;
    const size_t k = (size_t)j * G.pitch + i;
    C[k] = friction(at(e, u, v, z, k), n2 ? n2[k] : G.gn2, G.h_dry);
}

// S7 / S13: momentum differenced on level (e, u, v) in directions (DX, DY),
// updating the level-n velocities u0, v0.
template <class T, int DX, int DY, int FR>
__global__ void __launch_bounds__(BX) k_momentum(GridK<T> G, const double* __restrict__ dtp, double dx, double dy,
                                                 double g, const T* __restrict__ e, const T* __restrict__ u,
                                                 const T* __restrict__ v, const T* __restrict__ z, Ghosts<T> gh,
                                                 const T* __restrict__ C, const T* __restrict__ u0,
                                                 const T* __restrict__ v0, T* __restrict__ uo, T* __restrict__ vo) {
    int i, j;
    if (!cell_of(G.nx, G.ny, i, j)) return;
    const StepK<T> S = step_consts<T>(dtp);
    const size_t k = (size_t)j * G.pitch + i;
    const Cell<T> c = at(e, u, v, z, k);
    const Cell<T> xn = nbr<DX, 0>(G, e, u, v, z, gh, i, j, k);
    const Cell<T> yn = nbr<0, DY>(G, e, u, v, z, gh, i, j, k);
    T a, b;
    momentum<DX, DY, FR>(c, xn, yn, C[k], u0[k], v0[k], S, G.h_dry, a, b);
    uo[k] = a;
    vo[k] = b;
}

// S8: the predictor's wet/dry fix in place; a predicted clamp counts half.
template <class T>
__global__ void __launch_bounds__(BX) k_fix_pred(GridK<T> G, T* __restrict__ e, T* __restrict__ u,
                                                 T* __restrict__ v, const T* __restrict__ z, DevCtl* ctl,
                                                 double area) {
    int i, j;
    T added = T(0);
    if (cell_of(G.nx, G.ny, i, j)) {
        const size_t k = (size_t)j * G.pitch + i;
        T a = e[k], b = u[k], d = v[k];
        added = wetdry_fix(a, b, d, z[k], G.h_dry);
        e[k] = a; u[k] = b; v[k] = d;
    }
    if (__any_sync(0xffffffffu, added != T(0))) {
        const double s = warp_sum((double)added);
        if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(&ctl->clamp, 0.5 * s * area);
    }
}

// S14: average of the predicted and corrected levels.
template <class T>
__global__ void __launch_bounds__(BX) k_average(GridK<T> G, const T* __restrict__ es, const T* __restrict__ us,
                                                const T* __restrict__ vs, const T* __restrict__ ec,
                                                const T* __restrict__ uc, const T* __restrict__ vc, T* __restrict__ e1,
                                                T* __restrict__ u1, T* __restrict__ v1) {
    int i, j;
    if (!cell_of(G.nx, G.ny, i, j)) return;
    const size_t k = (size_t)j * G.pitch + i;
    e1[k] = T(0.5) * (es[k] + ec[k]);
    u1[k] = T(0.5) * (us[k] + uc[k]);
    v1[k] = T(0.5) * (vs[k] + vc[k]);
}

// S15: dissipation of level n added to the new level (or the TVD term of
// the ablation).
template <class T>
__global__ void __launch_bounds__(BX) k_dissipation(GridK<T> G, const double* __restrict__ dtp, double dx, double dy,
                                                    double g, const T* __restrict__ e, const T* __restrict__ u,
                                                    const T* __restrict__ v, const T* __restrict__ z,
                                                    T* __restrict__ e1, T* __restrict__ u1, T* __restrict__ v1) {
    int i, j;
    if (!cell_of(G.nx, G.ny, i, j)) return;
    const size_t k = (size_t)j * G.pitch + i;
    T a = e1[k], b = u1[k], d = v1[k];
    if (G.dissipation == 1) tvd_at(G, step_consts<T>(dtp), i, j, e, u, v, z, a, b, d);
    else dissipation_at(G, i, j, e, u, v, z, e[k], u[k], v[k], z[k], a, b, d);
    e1[k] = a; u1[k] = b; v1[k] = d;
}

// S16: final wet/dry fix, clamp and boundary-flux tallies, non-finite flag;
// with `reduce`, the next step's CFL speed maximum into slot_next.
template <class T>
__global__ void __launch_bounds__(BX) k_final(GridK<T> G, const double* __restrict__ dtp, double dx, double dy,
                                              const T* __restrict__ e, const T* __restrict__ u,
                                              const T* __restrict__ v, const T* __restrict__ z,
                                              const T* __restrict__ qxs, const T* __restrict__ qys,
                                              T* __restrict__ e1, T* __restrict__ u1, T* __restrict__ v1, DevCtl* ctl,
                                              int reduce, int slot_next, double area) {
    int i, j;
    T added = T(0), speed = T(0);
    double bw = 0.0, be = 0.0, bs = 0.0, bn = 0.0;
    bool bad = false;
    const double dtd = *dtp;
    if (cell_of(G.nx, G.ny, i, j)) {
        const size_t k = (size_t)j * G.pitch + i;
        const T zc = z[k];
        T en = e1[k], un = u1[k], vn = v1[k];
        added = wetdry_fix(en, un, vn, zc, G.h_dry);
        e1[k] = en; u1[k] = un; v1[k] = vn;
        speed = cfl_speed(en, un, vn, zc, G);
        bad = !isfinite(en + un + vn);
        const T e0 = e[k], u0 = u[k], v0 = v[k];
        const T qxn = (e0 - zc) * u0, qyn = (e0 - zc) * v0;
        if (i == 0) bw = 0.5 * ((double)face_bnd(SIDE_W, qxn, G) + (double)face_bnd(SIDE_W, qxs[k], G));
        if (i == G.nx - 1) be = -0.5 * ((double)face_bnd(SIDE_E, qxn, G) + (double)face_bnd(SIDE_E, qxs[k], G));
        if (j == 0) bs = 0.5 * ((double)face_bnd(SIDE_S, qyn, G) + (double)face_bnd(SIDE_S, qys[k], G));
        if (j == G.ny - 1) bn = -0.5 * ((double)face_bnd(SIDE_N, qyn, G) + (double)face_bnd(SIDE_N, qys[k], G));
    }
    const int lane = threadIdx.x & 31;
    if (reduce) {
        const T m = warp_max(speed);
        if (lane == 0 && m > T(0)) atomicMax(&ctl->smax[slot_next], (unsigned long long)__double_as_longlong((double)m));
    }
    if (__any_sync(0xffffffffu, added != T(0))) {
        const double s = warp_sum((double)added);
        if (lane == 0 && s != 0.0) atomicAdd(&ctl->clamp, s * area);
    }
    if (__any_sync(0xffffffffu, bw != 0.0 || be != 0.0 || bs != 0.0 || bn != 0.0)) {
        const double a = warp_sum(bw), b = warp_sum(be), c2 = warp_sum(bs), d = warp_sum(bn);
        if (lane == 0) {
            if (a != 0.0) atomicAdd(&ctl->bflux[0], a * dtd * dy);
            if (b != 0.0) atomicAdd(&ctl->bflux[1], b * dtd * dy);
            if (c2 != 0.0) atomicAdd(&ctl->bflux[2], c2 * dtd * dx);
            if (d != 0.0) atomicAdd(&ctl->bflux[3], d * dtd * dx);
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&ctl->flags, (unsigned)SWE_FLAG_NONFINITE);
}

// ---------------------------------------------------------------- 16x16 shared-memory form
// The paper's second design (Sec. 3.2): two-dimensional blocks of 16 by 16
// threads; each thread copies its cell into shared memory, the threads at the
// block's edges also copy the halo cells, and the sub-steps that read
// neighbours (S5/S11 continuity, S7/S13 momentum, S15 dissipation) take them
// from shared memory.  The per-cell sub-steps read no neighbour and keep their
// row blocks.  The arithmetic is the same per-cell functions, so the results
// equal the other layouts' bit for bit.
constexpr int SB = 16;

// Level value at (x, y) or, just outside the grid, the ghost cell there (the
// one the neighbour reads of nbr() return); zeros farther out (never read).
template <class T>
__device__ __forceinline__ Cell<T> cell_or_ghost(const GridK<T>& G, const T* e, const T* u, const T* v, const T* z,
                                                 const Ghosts<T>& g, int x, int y) {
    if (x >= 0 && x < G.nx && y >= 0 && y < G.ny) return at(e, u, v, z, (size_t)y * G.pitch + x);
    if (y >= 0 && y < G.ny) {
        if (x == -1) return g.side[SIDE_W][y];
        if (x == G.nx) return g.side[SIDE_E][y];
    }
    if (x >= 0 && x < G.nx) {
        if (y == -1) return g.side[SIDE_S][x];
        if (y == G.ny) return g.side[SIDE_N][x];
    }
    Cell<T> c;
    c.e = c.u = c.v = c.z = T(0);
    return c;
}

// S5 / S11 with the block's cell fluxes and one halo column/row (on the DX /
// DY side) in shared memory.
template <class T, int DX, int DY>
__global__ void __launch_bounds__(SB * SB) k_continuity_sh(GridK<T> G, const double* __restrict__ dtp, double dx,
                                                           double dy, double g, const T* __restrict__ e0,
                                                           const T* __restrict__ qx, const T* __restrict__ qy,
                                                           Ghosts<T> gh, T* __restrict__ eo) {
    __shared__ T sx[SB][SB + 1];  // column c is grid column i0 + c + XL
    __shared__ T sy[SB + 1][SB];  // row r is grid row j0 + r + YL
    constexpr int XL = DX > 0 ? 0 : -1, YL = DY > 0 ? 0 : -1;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * SB, j0 = blockIdx.y * SB;
    const int i = i0 + tx, j = j0 + ty;
    auto qxat = [&](int x, int y) -> T {  // the flux a face of column x sees (ghost flux just outside)
        if (y < 0 || y >= G.ny) return T(0);
        if (x >= 0 && x < G.nx) return qx[(size_t)y * G.pitch + x];
        if (x == -1 || x == G.nx) { const Cell<T> q = gh.side[x < 0 ? SIDE_W : SIDE_E][y]; return (q.e - q.z) * q.u; }
        return T(0);
    };
    auto qyat = [&](int x, int y) -> T {
        if (x < 0 || x >= G.nx) return T(0);
        if (y >= 0 && y < G.ny) return qy[(size_t)y * G.pitch + x];
        if (y == -1 || y == G.ny) { const Cell<T> q = gh.side[y < 0 ? SIDE_S : SIDE_N][x]; return (q.e - q.z) * q.v; }
        return T(0);
    };
    sx[ty][tx - XL] = qxat(i, j);
    sy[ty - YL][tx] = qyat(i, j);
    if (tx == 0) sx[ty][DX > 0 ? SB : 0] = qxat(i0 + (DX > 0 ? SB : -1), j);
    if (ty == 0) sy[DY > 0 ? SB : 0][tx] = qyat(i, j0 + (DY > 0 ? SB : -1));
    __syncthreads();
    if (i >= G.nx || j >= G.ny) return;
    const StepK<T> S = step_consts<T>(dtp);
    const size_t k = (size_t)j * G.pitch + i;
    const T qxc = sx[ty][tx - XL], qxn = sx[ty][tx - XL + DX];
    const T qyc = sy[ty - YL][tx], qyn = sy[ty - YL + DY][tx];
    T fe, fw, fn, fs;
    faces<DX>(qxc, qxn, i == 0, i == G.nx - 1, SIDE_W, SIDE_E, G, fe, fw);
    faces<DY>(qyc, qyn, j == 0, j == G.ny - 1, SIDE_S, SIDE_N, G, fn, fs);
    eo[k] = continuity(e0[k], fe, fw, fn, fs, S);
}

// S7 / S13 with the block's cells and one halo column/row in shared memory.
template <class T, int DX, int DY, int FR>
__global__ void __launch_bounds__(SB * SB) k_momentum_sh(GridK<T> G, const double* __restrict__ dtp, double dx,
                                                         double dy, double g, const T* __restrict__ e,
                                                         const T* __restrict__ u, const T* __restrict__ v,
                                                         const T* __restrict__ z, Ghosts<T> gh,
                                                         const T* __restrict__ C, const T* __restrict__ u0,
                                                         const T* __restrict__ v0, T* __restrict__ uo,
                                                         T* __restrict__ vo) {
    __shared__ Cell<T> sc[SB][SB];
    __shared__ Cell<T> hx[SB];  // the column past the block on the DX side
    __shared__ Cell<T> hy[SB];  // the row past the block on the DY side
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * SB, j0 = blockIdx.y * SB;
    const int i = i0 + tx, j = j0 + ty;
    sc[ty][tx] = cell_or_ghost(G, e, u, v, z, gh, i, j);
    if (tx == 0) hx[ty] = cell_or_ghost(G, e, u, v, z, gh, i0 + (DX > 0 ? SB : -1), j);
    if (ty == 0) hy[tx] = cell_or_ghost(G, e, u, v, z, gh, i, j0 + (DY > 0 ? SB : -1));
    __syncthreads();
    if (i >= G.nx || j >= G.ny) return;
    const StepK<T> S = step_consts<T>(dtp);
    const size_t k = (size_t)j * G.pitch + i;
    const int txn = tx + DX, tyn = ty + DY;
    const Cell<T> xn = (txn >= 0 && txn < SB) ? sc[ty][txn] : hx[ty];
    const Cell<T> yn = (tyn >= 0 && tyn < SB) ? sc[tyn][tx] : hy[tx];
    T a, b;
    momentum<DX, DY, FR>(sc[ty][tx], xn, yn, C[k], u0[k], v0[k], S, G.h_dry, a, b);
    uo[k] = a;
    vo[k] = b;
}

// S15 (or the TVD term) with the block's depths and e, u, v (halo 2) in
// shared memory, each at the clamped grid position the global form reads.
template <class T>
__global__ void __launch_bounds__(SB * SB) k_dissipation_sh(GridK<T> G, const double* __restrict__ dtp, double dx,
                                                            double dy, double g, const T* __restrict__ e,
                                                            const T* __restrict__ u, const T* __restrict__ v,
                                                            const T* __restrict__ z, T* __restrict__ e1,
                                                            T* __restrict__ u1, T* __restrict__ v1) {
    __shared__ T sh[SB + 4][SB + 4];
    __shared__ T sf[3][SB + 4][SB + 4];
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * SB + tx;
    const int i0 = blockIdx.x * SB, j0 = blockIdx.y * SB;
    auto clampx = [&](int x) { return x < 0 ? 0 : (x >= G.nx ? G.nx - 1 : x); };
    auto clampy = [&](int y) { return y < 0 ? 0 : (y >= G.ny ? G.ny - 1 : y); };
    for (int q = t; q < (SB + 4) * (SB + 4); q += SB * SB) {
        const int r = q / (SB + 4), c = q % (SB + 4);
        const size_t k = (size_t)clampy(j0 + r - 2) * G.pitch + clampx(i0 + c - 2);
        sh[r][c] = e[k] - z[k];
    }
    for (int q = t; q < (SB + 4) * (SB + 4); q += SB * SB) {
        const int r = q / (SB + 4), c = q % (SB + 4);
        const size_t k = (size_t)clampy(j0 + r - 2) * G.pitch + clampx(i0 + c - 2);
        sf[0][r][c] = e[k];
        sf[1][r][c] = u[k];
        sf[2][r][c] = v[k];
    }
    __syncthreads();
    const int i = i0 + tx, j = j0 + ty;
    if (i >= G.nx || j >= G.ny) return;
    const size_t k = (size_t)j * G.pitch + i;
    auto hat = [&](int ii, int jj) -> T { return sh[jj - j0 + 2][ii - i0 + 2]; };
    auto atf = [&](int f, int ii, int jj) -> T { return sf[f][jj - j0 + 2][ii - i0 + 2]; };
    T a = e1[k], b = u1[k], d = v1[k];
    if (G.dissipation == 1)
        tvd_core(G, step_consts<T>(dtp), i, j, hat, atf, a, b, d);
    else
        dissipation_core(G, i, j, hat, atf, sf[0][ty + 2][tx + 2], sf[1][ty + 2][tx + 2], sf[2][ty + 2][tx + 2], z[k], a,
                         b, d);
    e1[k] = a; u1[k] = b; v1[k] = d;
}

template <class T>
void free_scratch(Scratch<T>* q) {
    T* dev[] = {q->h, q->qx, q->qy, q->C, q->es, q->us, q->vs, q->qxs, q->qys, q->Cs, q->ec, q->uc, q->vc};
    for (T* p : dev)
        if (p) cudaFree(p);
    if (q->wet) cudaFree(q->wet);
    for (int s = 0; s < 4; ++s) {
        if (q->gn.side[s]) cudaFree(q->gn.side[s]);
        if (q->gs.side[s]) cudaFree(q->gs.side[s]);
    }
    if (q->d_dt) cudaFree(q->d_dt);
    T* host[] = {q->hst_e, q->hst_u, q->hst_v, q->hst_z};
    for (T* p : host)
        if (p) cudaFreeHost(p);
    free(q);
}

template <class T>
cudaError_t get_scratch(swe_ctx* c, Scratch<T>** out) {
    if (c->paper) { *out = (Scratch<T>*)c->paper; return cudaSuccess; }
    Scratch<T>* q = (Scratch<T>*)calloc(1, sizeof(Scratch<T>));
    if (!q) return cudaErrorMemoryAllocation;
    const size_t bytes = c->plane * sizeof(T);
    cudaError_t e = cudaSuccess;
    T** dev[] = {&q->h, &q->qx, &q->qy, &q->C, &q->es, &q->us, &q->vs, &q->qxs, &q->qys, &q->Cs, &q->ec, &q->uc, &q->vc};
    for (T** p : dev)
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&q->wet, c->plane);
    const size_t side = (size_t)(c->p.nx > c->p.ny ? c->p.nx : c->p.ny) * sizeof(Cell<T>);
    for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
        e = cudaMalloc(&q->gn.side[s], side);
        if (e == cudaSuccess) e = cudaMalloc(&q->gs.side[s], side);
    }
    if (e == cudaSuccess) e = cudaMalloc(&q->d_dt, sizeof(double));
    T** host[] = {&q->hst_e, &q->hst_u, &q->hst_v, &q->hst_z};
    for (T** p : host)
        if (e == cudaSuccess) e = cudaMallocHost(p, bytes);
    if (e != cudaSuccess) {
        free_scratch(q);
        return e;
    }
    c->paper = q;
    *out = q;
    return cudaSuccess;
}

// S2 on the host: copy the level to pinned host memory, wait, and take the
// CFL maximum over the wet cells in FP64 (one thread, as the paper's CPU code).
template <class T>
cudaError_t host_dt(swe_ctx* c, Scratch<T>* q, double* dt) {
    const size_t bytes = c->plane * sizeof(T);
    cudaError_t e;
    if (!q->z_on_host) {
        if ((e = cudaMemcpyAsync(q->hst_z, c->z, bytes, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return e;
        q->z_on_host = true;
    }
    if ((e = cudaMemcpyAsync(q->hst_e, c->eta[c->cur], bytes, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(q->hst_u, c->u[c->cur], bytes, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(q->hst_v, c->v[c->cur], bytes, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    const swe_params& p = c->p;
    double smax = 0.0;
    for (int j = 0; j < p.ny; ++j)
        for (int i = 0; i < p.nx; ++i) {
            const size_t k = (size_t)j * c->pitch + i;
            const double h = (double)q->hst_e[k] - (double)q->hst_z[k];
            if (!(h > p.h_dry)) continue;
            const double cw = std::sqrt(p.g * h);
            const double s = (std::fabs((double)q->hst_u[k]) + cw) / p.dx + (std::fabs((double)q->hst_v[k]) + cw) / p.dy;
            smax = s > smax ? s : smax;
        }
    *dt = dt_from_speed(smax, p.cfl, p.dt_max);
    return cudaSuccess;
}

template <class T, int SX, int SY>
cudaError_t step_t(swe_ctx* c, Scratch<T>* q, int s, long long k) {
    constexpr int CX = -SX, CY = -SY;
    const swe_params& p = c->p;
    const GridK<T> G = grid_of<T>(c);
    const int a = c->cur, b = 1 - c->cur;
    const T* e = (const T*)c->eta[a];
    const T* u = (const T*)c->u[a];
    const T* v = (const T*)c->v[a];
    const T* z = (const T*)c->z;
    const T* n2 = (const T*)c->n2;
    T* e1 = (T*)c->eta[b];
    T* u1 = (T*)c->u[b];
    T* v1 = (T*)c->v[b];
    const double area = p.dx * p.dy;
    const int slot = (int)(k % 3), slot_next = (int)((k + 1) % 3);
    cudaError_t err;
    // S2: the step size
    const bool fixed = c->dt_fixed_cap > 0 && c->dt_fixed;
    const bool devdt = p.kernel == SWE_KERNEL_PAPER_DEVDT || p.kernel == SWE_KERNEL_PAPER_SHARED_DEVDT;
    const bool shared = p.kernel == SWE_KERNEL_PAPER_SHARED || p.kernel == SWE_KERNEL_PAPER_SHARED_DEVDT;
    const dim3 sblk(SB, SB), sgrd((p.nx + SB - 1) / SB, (p.ny + SB - 1) / SB);
    const double* dtv = fixed ? c->dt_fixed + s : q->d_dt;
    if (!fixed && !devdt) {
        double dt = 0.0;
        if ((err = host_dt<T>(c, q, &dt)) != cudaSuccess) return err;
        if ((err = cudaMemcpyAsync(q->d_dt, &dt, sizeof(double), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
            return err;
    }
    k_paper_dt<<<1, 1, 0, c->stream>>>(c->ctl, dtv, (!fixed && devdt) ? 1 : 0, slot, slot_next, s, c->dt_hist, p.cfl,
                                       p.dt_max, 1.0 / p.dx, 1.0 / p.dy, p.g);
    const double* dtp = &c->ctl->cur.dt;
    const dim3 blk(BX), grd((p.nx + BX - 1) / BX, p.ny);
    const int nside = p.nx > p.ny ? p.nx : p.ny;
    const int gb = (nside + 255) / 256;
    k_s1<T><<<grd, blk, 0, c->stream>>>(G, e, z, q->h, q->wet);                                           // S1
    k_ghosts<T><<<gb, 256, 0, c->stream>>>(G, e, u, v, z, q->gn);                                          // S3
    k_fluxes<T><<<grd, blk, 0, c->stream>>>(G, e, u, v, z, q->qx, q->qy);                                  // S4
    if (shared)
        k_continuity_sh<T, SX, SY><<<sgrd, sblk, 0, c->stream>>>(G, dtp, p.dx, p.dy, p.g, e, q->qx, q->qy, q->gn, q->es);
    else
        k_continuity<T, SX, SY><<<grd, blk, 0, c->stream>>>(G, dtp, p.dx, p.dy, p.g, e, q->qx, q->qy, q->gn, q->es);  // S5
    k_friction<T><<<grd, blk, 0, c->stream>>>(G, e, u, v, z, n2, q->C);                                    // S6
    // S7 (FR: the friction form)
    auto mom = [&](auto fr, const T* me, const T* mu, const T* mv, const Ghosts<T>& mg, const T* mC, T* ou, T* ov,
                   auto dirs) {
        constexpr int F = decltype(fr)::value, MX = decltype(dirs)::x, MY = decltype(dirs)::y;
        if (shared)
            k_momentum_sh<T, MX, MY, F><<<sgrd, sblk, 0, c->stream>>>(G, dtp, p.dx, p.dy, p.g, me, mu, mv, z, mg, mC, u,
                                                                      v, ou, ov);
        else
            k_momentum<T, MX, MY, F><<<grd, blk, 0, c->stream>>>(G, dtp, p.dx, p.dy, p.g, me, mu, mv, z, mg, mC, u, v,
                                                                 ou, ov);
    };
    if (p.friction == 1) mom(IntC<1>(), e, u, v, q->gn, q->C, q->us, q->vs, Dirs<SX, SY>());
    else mom(IntC<0>(), e, u, v, q->gn, q->C, q->us, q->vs, Dirs<SX, SY>());
    k_fix_pred<T><<<grd, blk, 0, c->stream>>>(G, q->es, q->us, q->vs, z, c->ctl, area);                    // S8
    k_ghosts<T><<<gb, 256, 0, c->stream>>>(G, q->es, q->us, q->vs, z, q->gs);                              // S9
    k_fluxes<T><<<grd, blk, 0, c->stream>>>(G, q->es, q->us, q->vs, z, q->qxs, q->qys);                    // S10
    if (shared)
        k_continuity_sh<T, CX, CY><<<sgrd, sblk, 0, c->stream>>>(G, dtp, p.dx, p.dy, p.g, e, q->qxs, q->qys, q->gs,
                                                                 q->ec);
    else
        k_continuity<T, CX, CY><<<grd, blk, 0, c->stream>>>(G, dtp, p.dx, p.dy, p.g, e, q->qxs, q->qys, q->gs,
                                                            q->ec);                                        // S11
    k_friction<T><<<grd, blk, 0, c->stream>>>(G, q->es, q->us, q->vs, z, n2, q->Cs);                       // S12
    if (p.friction == 1) mom(IntC<1>(), q->es, q->us, q->vs, q->gs, q->Cs, q->uc, q->vc, Dirs<CX, CY>());  // S13
    else mom(IntC<0>(), q->es, q->us, q->vs, q->gs, q->Cs, q->uc, q->vc, Dirs<CX, CY>());
    k_average<T><<<grd, blk, 0, c->stream>>>(G, q->es, q->us, q->vs, q->ec, q->uc, q->vc, e1, u1, v1);     // S14
    if (p.kappa != 0.0 || p.dissipation == 1) {                                                            // S15
        if (shared) k_dissipation_sh<T><<<sgrd, sblk, 0, c->stream>>>(G, dtp, p.dx, p.dy, p.g, e, u, v, z, e1, u1, v1);
        else k_dissipation<T><<<grd, blk, 0, c->stream>>>(G, dtp, p.dx, p.dy, p.g, e, u, v, z, e1, u1, v1);
    }
    k_final<T><<<grd, blk, 0, c->stream>>>(G, dtp, p.dx, p.dy, e, u, v, z, q->qxs, q->qys, e1, u1, v1, c->ctl,
                                           devdt ? 1 : 0, slot_next, area);                                // S16
    return cudaGetLastError();
}

template <class T>
cudaError_t step_dir(swe_ctx* c, int s, long long k) {
    Scratch<T>* q = nullptr;
    cudaError_t e = get_scratch<T>(c, &q);
    if (e != cudaSuccess) return e;
    int sx, sy;
    step_dirs(c->p.dir_cycle, k, &sx, &sy);
    if (sx > 0 && sy > 0) return step_t<T, 1, 1>(c, q, s, k);
    if (sx > 0 && sy < 0) return step_t<T, 1, -1>(c, q, s, k);
    if (sx < 0 && sy > 0) return step_t<T, -1, 1>(c, q, s, k);
    return step_t<T, -1, -1>(c, q, s, k);
}

}  // namespace pp
}  // namespace swe

using namespace swe;

cudaError_t swe_launch_paper_step(swe_ctx* c, int s, long long k) {
    if (c->real_size == 8) return pp::step_dir<double>(c, s, k);
    return pp::step_dir<float>(c, s, k);
}

void swe_paper_release(swe_ctx* c) {
    if (!c->paper) return;
    if (c->real_size == 8) pp::free_scratch((pp::Scratch<double>*)c->paper);
    else pp::free_scratch((pp::Scratch<float>*)c->paper);
    c->paper = nullptr;
}

// The bed on the host copy is stale after swe_set_bed*.
void swe_paper_bed_changed(swe_ctx* c) {
    if (!c->paper) return;
    if (c->real_size == 8) ((pp::Scratch<double>*)c->paper)->z_on_host = false;
    else ((pp::Scratch<float>*)c->paper)->z_on_host = false;
}
