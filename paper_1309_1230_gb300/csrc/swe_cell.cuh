// swe_cell.cuh -- per-cell arithmetic of one MacCormack stage of the 2D
// shallow-water step (Seitz et al. 2013, Sec. 1: explicit predictor/corrector
// MacCormack on elevation and two velocities, split into 16 per-cell
// sub-steps).  Every GPU kernel form (plain, fused, batched, adjoint
// recompute) evaluates a cell through these functions, so a cell's result
// does not depend on which kernel, tile shape or batch computed it.
//
// Real type T is float (FP32 form) or double (FP64 form).  In FP32 the
// translation unit is compiled with approximate division/square root and
// flush-to-zero; FP64 is IEEE throughout.  The library is compiled without
// implicit multiply-add contraction: every fused multiply-add below is
// written out (fma_), so the rounding of a cell is fixed by this file alone.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace swe {

enum { BC_WALL = 0, BC_INFLOW = 1, BC_OUTFLOW = 2 };
enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };

// Guard of the dissipation switch denominator (m).
#define SWE_NU_TINY 1e-12

template <class T>
struct Cell {
    T e, u, v, z;  // elevation, velocities, bed
};

// Grid-wide constants of one scenario.
template <class T>
struct GridK {
    int nx, ny, pitch;       // cells; row pitch in elements
    T g, h_dry, kappa;
    T gn2;                   // g * n^2 of the uniform Manning n
    T inv_dx, inv_dy;        // for the CFL speed
    T qin[4];                // inflow discharge into the domain per side
    int bc[4];
};

// Step constants, rounded from the FP64 step size.
template <class T>
struct StepK {
    T dt, dtdx, dtdy, g_dtdx, g_dtdy;
};

template <class T>
__host__ __device__ inline StepK<T> make_stepk(double dt, double dx, double dy, double g) {
    StepK<T> s;
    s.dt = (T)dt;
    s.dtdx = (T)(dt / dx);
    s.dtdy = (T)(dt / dy);
    s.g_dtdx = (T)(g * dt / dx);
    s.g_dtdy = (T)(g * dt / dy);
    return s;
}

template <class T>
__device__ __forceinline__ T fma_(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ float pow_m43(float h) { return __powf(h, -1.33333333f); }
__device__ __forceinline__ double pow_m43(double h) {
    double r = rcbrt(h);
    double r2 = r * r;
    return r2 * r2;
}

template <class T>
__device__ __forceinline__ T rsq_sqrt(T x) { return sqrt(x); }
template <>
__device__ __forceinline__ float rsq_sqrt<float>(float x) { return sqrtf(x); }

template <class T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// Elevation of neighbour nb seen by the pressure term of a cell at elevation
// eta_self: a dry neighbour whose bed is above eta_self acts as a wall.
template <class T>
__device__ __forceinline__ T eta_seen(const Cell<T>& nb, T eta_self, T h_dry) {
    bool dry = !((nb.e - nb.z) > h_dry);
    return (dry && nb.z > eta_self) ? eta_self : nb.e;
}

// Ghost cell of side `side` from the adjacent interior cell `in` (S3/S9).
template <class T>
__device__ __forceinline__ Cell<T> ghost(const Cell<T>& in, int side, const GridK<T>& G) {
    Cell<T> g = in;
    int bc = G.bc[side];
    bool xside = side < 2;
    if (bc == BC_WALL) {
        if (xside) g.u = -in.u; else g.v = -in.v;
    } else if (bc == BC_INFLOW) {
        T h = in.e - in.z;
        T sgn = (side == SIDE_W || side == SIDE_S) ? T(1) : T(-1);
        T vn = sgn * G.qin[side] / tmax(h, G.h_dry);
        if (xside) { g.u = vn; g.v = T(0); } else { g.v = vn; g.u = T(0); }
    }
    return g;
}

// Flux through a boundary face of side `side`, given the adjacent cell's flux.
template <class T>
__device__ __forceinline__ T face_bnd(int side, T qc, const GridK<T>& G) {
    int bc = G.bc[side];
    if (bc == BC_WALL) return T(0);
    if (bc == BC_INFLOW) return (side == SIDE_W || side == SIDE_S) ? G.qin[side] : -G.qin[side];
    return qc;
}

// Face fluxes (east/west or north/south) of a cell for a one-sided
// difference in direction D (+1 forward: a face carries the flux of the cell
// above it; -1 backward: of the cell below it).  qc: the cell's flux,
// qn: the flux of the neighbour in direction D.  lo/hi: the cell touches the
// low/high boundary of this axis.
template <int D, class T>
__device__ __forceinline__ void faces(T qc, T qn, bool lo, bool hi, int side_lo, int side_hi,
                                      const GridK<T>& G, T& f_hi, T& f_lo) {
    if (D > 0) { f_hi = qn; f_lo = qc; } else { f_hi = qc; f_lo = qn; }
    if (hi) f_hi = face_bnd(side_hi, qc, G);
    if (lo) f_lo = face_bnd(side_lo, qc, G);
}

// Manning coefficient of a cell (S6/S12): g n^2 |U| / h^(4/3) when wet.
template <class T>
__device__ __forceinline__ T friction(const Cell<T>& c, T gn2, T h_dry) {
    T h = c.e - c.z;
    T s2 = fma_(c.u, c.u, c.v * c.v);
    T mag = s2 > T(0) ? rsq_sqrt(s2) : T(0);
    return (h > h_dry) ? gn2 * mag * pow_m43(h) : T(0);
}

// One MacCormack stage of a cell (S5-S8 for the predictor, S11-S13 for the
// corrector before averaging).  c: the differenced state at the cell (level n
// for the predictor, predicted for the corrector); xn/yn: its neighbours in
// the stage's one-sided directions DX/DY (ghost cells at the boundary);
// f*: face fluxes; e0,u0,v0: the level-n values the stage updates from.
template <int DX, int DY, class T>
__device__ __forceinline__ void stage(const Cell<T>& c, const Cell<T>& xn, const Cell<T>& yn,
                                      T fe, T fw, T fn, T fs, T e0, T u0, T v0, T gn2,
                                      const StepK<T>& S, T h_dry, T& eo, T& uo, T& vo) {
    eo = e0 - fma_(S.dtdx, fe - fw, S.dtdy * (fn - fs));
    T cf = friction(c, gn2, h_dry);
    T ex = eta_seen(xn, c.e, h_dry);
    T ey = eta_seen(yn, c.e, h_dry);
    T dux, dvx, dex, duy, dvy, dey;
    if (DX > 0) { dux = xn.u - c.u; dvx = xn.v - c.v; dex = ex - c.e; }
    else        { dux = c.u - xn.u; dvx = c.v - xn.v; dex = c.e - ex; }
    if (DY > 0) { duy = yn.u - c.u; dvy = yn.v - c.v; dey = ey - c.e; }
    else        { duy = c.u - yn.u; dvy = c.v - yn.v; dey = c.e - ey; }
    T au = fma_(c.u, S.dtdx * dux, fma_(c.v, S.dtdy * duy, S.g_dtdx * dex));
    T av = fma_(c.u, S.dtdx * dvx, fma_(c.v, S.dtdy * dvy, S.g_dtdy * dey));
    T r = T(1) / fma_(S.dt, cf, T(1));
    uo = (u0 - au) * r;
    vo = (v0 - av) * r;
}

// Wet/dry fix (S8/S16): negative depth -> eta = z (returns the added depth),
// dry -> zero velocity.
template <class T>
__device__ __forceinline__ T wetdry_fix(T& e, T& u, T& v, T z, T h_dry) {
    T h = e - z;
    T added = T(0);
    if (h < T(0)) { added = -h; e = z; h = T(0); }
    if (h <= h_dry) { u = T(0); v = T(0); }
    return added;
}

// Dissipation switch of a cell along one axis (S15).
template <class T>
__device__ __forceinline__ T nu_switch(T hl, T hc, T hr) {
    T num = fabs(fma_(T(-2), hc, hl + hr));
    T den = fma_(T(2), fabs(hc), fabs(hl) + fabs(hr)) + T(SWE_NU_TINY);
    return num / den;
}

// Face coefficient of the dissipation: interior face between two wet cells.
template <class T>
__device__ __forceinline__ T face_eps(bool wet_a, bool wet_b, T nu_a, T nu_b) {
    return (wet_a && wet_b) ? tmax(nu_a, nu_b) : T(0);
}

// S15 dissipation flux through one face: eps * (phi_above - phi_below).
template <class T>
__device__ __forceinline__ T dflux(T eps, T hi, T lo) { return eps * (hi - lo); }

// S15 for one field of a cell from its four face fluxes (east, west, north,
// south): out + kappa * ((fe - fw) + (fn - fs)).  Every kernel form builds the
// same face fluxes with dflux, so a face is rounded the same from both sides.
template <class T>
__device__ __forceinline__ T dissip_faces(T out, T fe, T fw, T fn, T fs, T kappa) {
    return fma_(kappa, (fe - fw) + (fn - fs), out);
}

// CFL speed of a cell (S2); 0 for dry cells.
template <class T>
__device__ __forceinline__ T cfl_speed(T e, T u, T v, T z, const GridK<T>& G) {
    T h = e - z;
    if (!(h > G.h_dry)) return T(0);
    T c = rsq_sqrt(G.g * h);
    return fma_(fabs(u) + c, G.inv_dx, (fabs(v) + c) * G.inv_dy);
}

// Step size from the reduced CFL speed (S2), FP64.
__host__ __device__ inline double dt_from_speed(double smax, double cfl, double dt_max) {
    if (!(smax > 0.0)) return dt_max;
    double dt = cfl / smax;
    return dt < dt_max ? dt : dt_max;
}

// Predictor direction of step k (+1 forward, -1 backward) per axis.
__host__ __device__ inline void step_dirs(int dir_cycle, long long k, int* sx, int* sy) {
    int ax = (dir_cycle & 2) ? -1 : 1;
    int ay = (dir_cycle & 4) ? -1 : 1;
    if ((dir_cycle & 1) && (k & 1)) { ax = -ax; ay = -ay; }
    *sx = ax; *sy = ay;
}

}  // namespace swe
