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
//
// The stage functions are generic in the value type R: a scalar T, or a
// lane vector vecn<T, N> holding the N cells one lane of the fused kernel
// owns in a row.  vecn<float, 2> adds, multiplies and multiply-adds both
// cells with one packed instruction (mul/fma.rn.ftz.f32x2, sm_100 and later;
// sums as a multiply-add with a unit factor); everything else acts per cell.  Per component a packed
// operation rounds exactly like its scalar one (IEEE round to nearest, FP32
// subnormals flushed), so a cell's result does not depend on the value type
// it was computed in.
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
    // Rows [own_lo, own_hi) are the grid's own; the others are halo rows
    // copied from a neighbouring strip of a decomposed domain: they are
    // stepped like any row but enter no tally and no CFL maximum.
    int own_lo = 0, own_hi = 1 << 30;
    // Ablation forms (plain and paper-layout kernels): explicit friction, and
    // the TVD-MacCormack term in place of S15's switch form.
    int friction = 0, dissipation = 0;
};

// Step constants, rounded from the FP64 step size.
template <class T>
struct StepK {
    T dt, dtdx, dtdy, g_dtdx, g_dtdy;
};

// rdx, rdy: 1/dx and 1/dy in FP64, divided once on the host, so that a
// device thread computing the constants does no FP64 division beyond the
// step size's own (GB300's FP64 pipe takes tens of cycles per warp
// instruction).
template <class T>
__host__ __device__ inline StepK<T> make_stepk(double dt, double rdx, double rdy, double g) {
    StepK<T> s;
    s.dt = (T)dt;
    s.dtdx = (T)(dt * rdx);
    s.dtdy = (T)(dt * rdy);
    s.g_dtdx = (T)(g * dt * rdx);
    s.g_dtdy = (T)(g * dt * rdy);
    return s;
}

// The step size with its constants in both real types, computed once per
// step by one thread (or on the host) from the same FP64 step size: kernels
// that run one thread per cell read them here instead of dividing in FP64 in
// every thread (GB300's FP64 rate is a small fraction of its FP32 rate).  A
// pointer to `dt` is a pointer to the slot.
struct StepSlot {
    double dt;
    StepK<float> f;
    StepK<double> d;
};

__host__ __device__ inline StepSlot make_slot(double dt, double rdx, double rdy, double g) {
    StepSlot s;
    s.dt = dt;
    s.f = make_stepk<float>(dt, rdx, rdy, g);
    s.d = make_stepk<double>(dt, rdx, rdy, g);
    return s;
}

// The constants of the slot whose step size dtp points at.
template <class T>
__device__ __forceinline__ StepK<T> step_consts(const double* dtp);
template <>
__device__ __forceinline__ StepK<float> step_consts<float>(const double* dtp) {
    return reinterpret_cast<const StepSlot*>(dtp)->f;
}
template <>
__device__ __forceinline__ StepK<double> step_consts<double>(const double* dtp) {
    return reinterpret_cast<const StepSlot*>(dtp)->d;
}

// Scalar fused multiply-add, round to nearest (FP32: subnormals flushed,
// stated explicitly so that the packed form below rounds the same).
__device__ __forceinline__ float fma_(float a, float b, float c) {
    float d;
    asm("fma.rn.ftz.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ float pow_m43(float h) { return __powf(h, -1.33333333f); }
__device__ __forceinline__ double pow_m43(double h) {
    double r = rcbrt(h);
    double r2 = r * r;
    return r2 * r2;
}

__device__ __forceinline__ float rsq_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double rsq_sqrt(double x) { return sqrt(x); }

// Reciprocal and quotient.  FP32: the hardware reciprocal (PTX rcp.approx,
// about 1 ulp) times the numerator, with no range scaling: the denominators
// here (a friction factor >= 1, a switch denominator of depths plus
// SWE_NU_TINY) stay far inside the normal FP32 range.  FP64: IEEE division.
__device__ __forceinline__ float rcp_(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float div_(float a, float b) { return a * rcp_(b); }
__device__ __forceinline__ double div_(double a, double b) { return a / b; }

template <class T>
__device__ __forceinline__ T sel(bool c, T a, T b) { return c ? a : b; }

// Per-cell (never packed) multiply: the friction update below keeps it so
// that the fused kernel's cells stay bitwise equal to the one-thread-per-cell
// kernel's (with the packed multiply there, a few cells differed by one ulp,
// although the packed and scalar products of the same operands agreed when
// compared in the kernel).
__device__ __forceinline__ float smul(float a, float b) { return a * b; }
__device__ __forceinline__ double smul(double a, double b) { return a * b; }

// ---------------------------------------------------------------- lane vectors
template <int N>
struct maskn {
    bool c[N];
    friend __device__ __forceinline__ maskn operator&&(maskn a, maskn b) {
        maskn r;
#pragma unroll
        for (int i = 0; i < N; ++i) r.c[i] = a.c[i] && b.c[i];
        return r;
    }
    friend __device__ __forceinline__ maskn operator||(maskn a, maskn b) {
        maskn r;
#pragma unroll
        for (int i = 0; i < N; ++i) r.c[i] = a.c[i] || b.c[i];
        return r;
    }
    friend __device__ __forceinline__ maskn operator!(maskn a) {
        maskn r;
#pragma unroll
        for (int i = 0; i < N; ++i) r.c[i] = !a.c[i];
        return r;
    }
};

// N cells of a lane, arithmetic per component (the generic form).
template <class T, int N>
struct vecn {
    T c[N];
    vecn() = default;
    __device__ __forceinline__ vecn(T s) {
#pragma unroll
        for (int i = 0; i < N; ++i) c[i] = s;
    }
    __device__ __forceinline__ T& operator[](int i) { return c[i]; }
    __device__ __forceinline__ const T& operator[](int i) const { return c[i]; }
#define SWE_VEC_OP(OP)                                                         \
    friend __device__ __forceinline__ vecn operator OP(vecn a, vecn b) {       \
        vecn r;                                                                \
        _Pragma("unroll") for (int i = 0; i < N; ++i) r.c[i] = a.c[i] OP b.c[i]; \
        return r;                                                              \
    }
    SWE_VEC_OP(+)
    SWE_VEC_OP(-)
    SWE_VEC_OP(*)
    SWE_VEC_OP(/)
#undef SWE_VEC_OP
#define SWE_VEC_CMP(OP)                                                        \
    friend __device__ __forceinline__ maskn<N> operator OP(vecn a, vecn b) {   \
        maskn<N> r;                                                            \
        _Pragma("unroll") for (int i = 0; i < N; ++i) r.c[i] = a.c[i] OP b.c[i]; \
        return r;                                                              \
    }
    SWE_VEC_CMP(>)
    SWE_VEC_CMP(<)
    SWE_VEC_CMP(<=)
    SWE_VEC_CMP(>=)
    SWE_VEC_CMP(==)
#undef SWE_VEC_CMP
    friend __device__ __forceinline__ vecn operator-(vecn a) {
        vecn r;
#pragma unroll
        for (int i = 0; i < N; ++i) r.c[i] = -a.c[i];
        return r;
    }
    friend __device__ __forceinline__ vecn fma_(vecn a, vecn b, vecn d) {
        vecn r;
#pragma unroll
        for (int i = 0; i < N; ++i) r.c[i] = fma_(a.c[i], b.c[i], d.c[i]);
        return r;
    }
    friend __device__ __forceinline__ vecn smul(vecn a, vecn b) { return a * b; }
    friend __device__ __forceinline__ vecn sel(maskn<N> m, vecn a, vecn b) {
        vecn r;
#pragma unroll
        for (int i = 0; i < N; ++i) r.c[i] = m.c[i] ? a.c[i] : b.c[i];
        return r;
    }
    friend __device__ __forceinline__ vecn rcp_(vecn a) {
        vecn r;
#pragma unroll
        for (int i = 0; i < N; ++i) r.c[i] = rcp_(a.c[i]);
        return r;
    }
    friend __device__ __forceinline__ vecn div_(vecn a, vecn b) {
        vecn r;
#pragma unroll
        for (int i = 0; i < N; ++i) r.c[i] = div_(a.c[i], b.c[i]);
        return r;
    }
    friend __device__ __forceinline__ vecn rsq_sqrt(vecn a) {
        vecn r;
#pragma unroll
        for (int i = 0; i < N; ++i) r.c[i] = rsq_sqrt(a.c[i]);
        return r;
    }
    friend __device__ __forceinline__ vecn pow_m43(vecn a) {
        vecn r;
#pragma unroll
        for (int i = 0; i < N; ++i) r.c[i] = pow_m43(a.c[i]);
        return r;
    }
};

// Two FP32 cells: add, subtract, multiply and multiply-add as one packed
// instruction each; the rest per component.
template <>
struct vecn<float, 2> {
    float2 v;
    vecn() = default;
    __device__ __forceinline__ vecn(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ vecn(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ float& operator[](int i) { return i == 0 ? v.x : v.y; }
    __device__ __forceinline__ const float& operator[](int i) const { return i == 0 ? v.x : v.y; }
#define SWE_PACKED(NAME, INSN)                                                                            \
    friend __device__ __forceinline__ vecn NAME(vecn a, vecn b) {                                         \
        vecn r;                                                                                           \
        asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n " INSN           \
            " rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"                                                     \
            : "=f"(r.v.x), "=f"(r.v.y) : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));                 \
        return r;                                                                                         \
    }
    SWE_PACKED(operator*, "mul.rn.ftz.f32x2")
#undef SWE_PACKED
    // Sums and differences as a multiply-add with a unit factor: a + b =
    // fma(a, 1, b) and a - b = fma(b, -1, a) round exactly as the add (the
    // product is exact, signed zeros included).  With a packed add.rn, ptxas
    // was seen to contract a packed product feeding it into one FFMA2 in some
    // builds (1-ulp differences from the scalar kernels), although add.rn
    // forbids that; a sum that already is a multiply-add leaves nothing to
    // contract into.
    friend __device__ __forceinline__ vecn operator+(vecn a, vecn b) {
        vecn r;
        asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
            " mov.b64 rc, 0x3F8000003F800000;\n fma.rn.ftz.f32x2 rd, ra, rc, rb;\n mov.b64 {%0, %1}, rd;\n}"
            : "=f"(r.v.x), "=f"(r.v.y) : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));
        return r;
    }
    friend __device__ __forceinline__ vecn operator-(vecn a, vecn b) {
        vecn r;
        asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
            " mov.b64 rc, 0xBF800000BF800000;\n fma.rn.ftz.f32x2 rd, rb, rc, ra;\n mov.b64 {%0, %1}, rd;\n}"
            : "=f"(r.v.x), "=f"(r.v.y) : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));
        return r;
    }
    friend __device__ __forceinline__ vecn operator/(vecn a, vecn b) { return vecn(a.v.x / b.v.x, a.v.y / b.v.y); }
    friend __device__ __forceinline__ vecn smul(vecn a, vecn b) { return vecn(a.v.x * b.v.x, a.v.y * b.v.y); }
    friend __device__ __forceinline__ vecn fma_(vecn a, vecn b, vecn d) {
        vecn r;
        asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
            " mov.b64 rc, {%6, %7};\n fma.rn.ftz.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
            : "=f"(r.v.x), "=f"(r.v.y)
            : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y), "f"(d.v.x), "f"(d.v.y));
        return r;
    }
    friend __device__ __forceinline__ vecn operator-(vecn a) { return vecn(-a.v.x, -a.v.y); }
#define SWE_PCMP(OP)                                                        \
    friend __device__ __forceinline__ maskn<2> operator OP(vecn a, vecn b) { \
        maskn<2> r;                                                         \
        r.c[0] = a.v.x OP b.v.x;                                            \
        r.c[1] = a.v.y OP b.v.y;                                            \
        return r;                                                           \
    }
    SWE_PCMP(>)
    SWE_PCMP(<)
    SWE_PCMP(<=)
    SWE_PCMP(>=)
    SWE_PCMP(==)
#undef SWE_PCMP
    friend __device__ __forceinline__ vecn sel(maskn<2> m, vecn a, vecn b) {
        return vecn(m.c[0] ? a.v.x : b.v.x, m.c[1] ? a.v.y : b.v.y);
    }
    friend __device__ __forceinline__ vecn rsq_sqrt(vecn a) { return vecn(sqrtf(a.v.x), sqrtf(a.v.y)); }
    friend __device__ __forceinline__ vecn rcp_(vecn a) { return vecn(rcp_(a.v.x), rcp_(a.v.y)); }
    friend __device__ __forceinline__ vecn div_(vecn a, vecn b) { return a * vecn(rcp_(b.v.x), rcp_(b.v.y)); }
    friend __device__ __forceinline__ vecn pow_m43(vecn a) { return vecn(pow_m43(a.v.x), pow_m43(a.v.y)); }
};

// Maximum of two switch values or speeds (never NaN in a finite state; a
// non-finite state is flagged separately).
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
template <class T, int N>
__device__ __forceinline__ vecn<T, N> tmax(vecn<T, N> a, vecn<T, N> b) {
    vecn<T, N> r;
#pragma unroll
    for (int i = 0; i < N; ++i) r[i] = tmax(a[i], b[i]);
    return r;
}

// The WET forms below serve stencils whose every cell is known to be wet (h
// > h_dry) in the state they read and, where they clamp, in the state they
// produce: each wet/dry select then picks the value the arithmetic computes,
// so they return that value and round exactly like the general form.  The
// caller checks the wetness and recomputes with the general form where it
// fails.

// Elevation of neighbour nb seen by the pressure term of a cell at elevation
// eta_self: a dry neighbour whose bed is above eta_self acts as a wall.
template <bool WET = false, class R, class T>
__device__ __forceinline__ R eta_seen(const Cell<R>& nb, R eta_self, T h_dry) {
    if constexpr (WET) return nb.e;
    const auto dry = !((nb.e - nb.z) > R(h_dry));
    return sel(dry && (nb.z > eta_self), eta_self, nb.e);
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
template <bool WET = false, class R, class T>
__device__ __forceinline__ R friction(const Cell<R>& c, R gn2, T h_dry) {
    const R h = c.e - c.z;
    const R s2 = fma_(c.u, c.u, c.v * c.v);  // >= +0, and sqrt(+0) = +0
    const R mag = rsq_sqrt(s2);
    if constexpr (WET) return gn2 * mag * pow_m43(h);
    return sel(h > R(h_dry), gn2 * mag * pow_m43(h), R(0));
}

// One MacCormack stage of a cell (S5-S8 for the predictor, S11-S13 for the
// corrector before averaging).  c: the differenced state at the cell (level n
// for the predictor, predicted for the corrector); xn/yn: its neighbours in
// the stage's one-sided directions DX/DY (ghost cells at the boundary);
// f*: face fluxes; e0,u0,v0: the level-n values the stage updates from.
// Continuity of one stage (S5/S11): the elevation update from the face
// fluxes.
template <class R, class T>
__device__ __forceinline__ R continuity(R e0, R fe, R fw, R fn, R fs, const StepK<T>& S) {
    return e0 - fma_(R(S.dtdx), fe - fw, R(S.dtdy) * (fn - fs));
}

// Momentum of one stage (S7/S13): advection and the wet/dry-aware pressure
// gradient from the one-sided differences in directions DX/DY, with the
// point-implicit friction of coefficient cf (FR = 1: explicit friction,
// vel0 - dt A - dt cf vel, the ablation form).
template <int DX, int DY, int FR = 0, bool WET = false, class R, class T>
__device__ __forceinline__ void momentum(const Cell<R>& c, const Cell<R>& xn, const Cell<R>& yn, R cf, R u0, R v0,
                                         const StepK<T>& S, T h_dry, R& uo, R& vo) {
    const R ex = eta_seen<WET>(xn, c.e, h_dry);
    const R ey = eta_seen<WET>(yn, c.e, h_dry);
    R dux, dvx, dex, duy, dvy, dey;
    if (DX > 0) { dux = xn.u - c.u; dvx = xn.v - c.v; dex = ex - c.e; }
    else        { dux = c.u - xn.u; dvx = c.v - xn.v; dex = c.e - ex; }
    if (DY > 0) { duy = yn.u - c.u; dvy = yn.v - c.v; dey = ey - c.e; }
    else        { duy = c.u - yn.u; dvy = c.v - yn.v; dey = c.e - ey; }
    const R au = fma_(c.u, R(S.dtdx) * dux, fma_(c.v, R(S.dtdy) * duy, R(S.g_dtdx) * dex));
    const R av = fma_(c.u, R(S.dtdx) * dvx, fma_(c.v, R(S.dtdy) * dvy, R(S.g_dtdy) * dey));
    if (FR == 1) {
        const R dc = R(S.dt) * cf;
        uo = fma_(-dc, c.u, u0 - au);
        vo = fma_(-dc, c.v, v0 - av);
        return;
    }
    const R r = rcp_(fma_(R(S.dt), cf, R(T(1))));
    uo = smul(u0 - au, r);
    vo = smul(v0 - av, r);
}

template <int DX, int DY, int FR = 0, bool WET = false, class R, class T>
__device__ __forceinline__ void stage(const Cell<R>& c, const Cell<R>& xn, const Cell<R>& yn,
                                      R fe, R fw, R fn, R fs, R e0, R u0, R v0, R gn2,
                                      const StepK<T>& S, T h_dry, R& eo, R& uo, R& vo) {
    eo = continuity(e0, fe, fw, fn, fs, S);
    const R cf = friction<WET>(c, gn2, h_dry);
    momentum<DX, DY, FR, WET>(c, xn, yn, cf, u0, v0, S, h_dry, uo, vo);
}

// Wet/dry fix (S8/S16): negative depth -> eta = z (returns the added depth),
// dry -> zero velocity.
template <class R, class T>
__device__ __forceinline__ R wetdry_fix(R& e, R& u, R& v, R z, T h_dry) {
    const R h = e - z;
    const auto neg = h < R(T(0));
    const R added = tmax(-h, R(T(0)));  // z - e (= -h exactly) when h < 0, else +0
    e = sel(neg, z, e);
    const auto dry = h <= R(h_dry);            // includes h < 0 (h_dry > 0)
    u = sel(dry, R(T(0)), u);
    v = sel(dry, R(T(0)), v);
    return added;
}

// Dissipation switch of a cell along one axis (S15).
// The depths are never negative (the wet/dry fix keeps eta >= z, ghost
// cells copy an interior depth), so |h| = h in the denominator.
__device__ __forceinline__ float absv(float x) { return fabsf(x); }
__device__ __forceinline__ double absv(double x) { return fabs(x); }
template <class T, int N>
__device__ __forceinline__ vecn<T, N> absv(vecn<T, N> x) {
    vecn<T, N> r;
#pragma unroll
    for (int i = 0; i < N; ++i) r[i] = absv(x[i]);
    return r;
}
template <class R>
__device__ __forceinline__ R nu_switch(R hl, R hc, R hr) {
    const R s = hl + hr;
    const R num = absv(fma_(R(-2.0f), hc, s));
    const R den = fma_(R(2.0f), hc, s) + R(SWE_NU_TINY);
    return div_(num, den);
}

// Face coefficient of the dissipation: interior face between two wet cells.
template <class M, class R>
__device__ __forceinline__ R face_eps(M wet_a, M wet_b, R nu_a, R nu_b) {
    return sel(wet_a && wet_b, tmax(nu_a, nu_b), R(0.0f));
}
// The same between two cells known to be wet.
template <class R>
__device__ __forceinline__ R face_eps_wet(R nu_a, R nu_b) {
    return tmax(nu_a, nu_b);
}

// S15 dissipation flux through one face: eps * (phi_above - phi_below).
template <class T>
__device__ __forceinline__ T dflux(T eps, T hi, T lo) { return eps * (hi - lo); }

// S15 for one field of a cell from its four face fluxes (east, west, north,
// south): out + kappa * (((fe - fw) - fs) + fn).  Every kernel form builds the
// same face fluxes with dflux, so a face is rounded the same from both sides,
// and sums them in this order (the fused sweep carries east - west - south
// from one row to the next and adds the north face when it arrives).
template <class R, class T>
__device__ __forceinline__ R dissip_faces(R out, R fe, R fw, R fn, R fs, T kappa) {
    return fma_(R(kappa), ((fe - fw) - fs) + fn, out);
}

// CFL speed of a cell (S2); 0 for dry cells.
template <bool WET = false, class T>
__device__ __forceinline__ T cfl_speed(T e, T u, T v, T z, const GridK<T>& G) {
    T h = e - z;
    if (!WET && !(h > G.h_dry)) return T(0);
    T c = rsq_sqrt(G.g * h);
    return fma_(fabs(u) + c, G.inv_dx, (fabs(v) + c) * G.inv_dy);
}

template <bool WET = false, class T, int N>
__device__ __forceinline__ vecn<T, N> cfl_speed(vecn<T, N> e, vecn<T, N> u, vecn<T, N> v, vecn<T, N> z,
                                                const GridK<T>& G) {
    vecn<T, N> r;
#pragma unroll
    for (int i = 0; i < N; ++i) r[i] = cfl_speed<WET>(e[i], u[i], v[i], z[i], G);
    return r;
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
