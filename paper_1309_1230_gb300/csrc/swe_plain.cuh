// swe_plain.cuh -- the plain GPU step's kernels (one thread per cell,
// predictor and corrector as two kernels), shared by the context path, the
// no-allocation step and the adjoint's forward recompute.
#pragma once
#include <cfloat>

#include "swe_internal.cuh"

namespace swe {

template <class T>
__device__ __forceinline__ Cell<T> ld(const T* e, const T* u, const T* v, const T* z, size_t k) {
    Cell<T> c;
    c.e = e[k]; c.u = u[k]; c.v = v[k]; c.z = z[k];
    return c;
}

__device__ __forceinline__ double warp_sum(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
template <class T>
__device__ __forceinline__ T warp_max(T x) {
    for (int o = 16; o > 0; o >>= 1) {
        T y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y > x ? y : x;
    }
    return x;
}

// Step size of step s of a call: replayed or from the level's CFL reduction.
static __global__ void k_plain_dt(DevCtl* ctl, int slot, int slot_next, const double* dt_fixed, int s,
                           double* dt_hist, double cfl, double dt_max, double rdx, double rdy, double g) {
    double dt;
    if (dt_fixed) dt = dt_fixed[s];
    else dt = dt_from_speed(__longlong_as_double((long long)ctl->smax[slot]), cfl, dt_max);
    ctl->cur = make_slot(dt, rdx, rdy, g);
    ctl->dt_last = dt;
    ctl->t += dt;
    ctl->dt_min = fmin(ctl->dt_min, dt);
    ctl->dt_maxs = fmax(ctl->dt_maxs, dt);
    dt_hist[s] = dt;
    ctl->smax[slot_next] = 0ull;
}

// S15 at cell (i, j): the face-form dissipation of level n (e, u, v, bed z;
// the cell's own values e0, u0, v0, zc) added to the averaged en, un, vn.
// Neighbour depths outside the grid repeat the edge cell; faces on the
// boundary carry none.
// The arithmetic, given accessors of the neighbours' depth hat(ii, jj) and of
// field f (0: e, 1: u, 2: v) at(f, ii, jj), both at the clamped position.
template <class T, class HAT, class AT>
__device__ __forceinline__ void dissipation_core(const GridK<T>& G, int i, int j, HAT&& hat, AT&& at, T e0, T u0,
                                                 T v0, T zc, T& en, T& un, T& vn) {
    const T hc = e0 - zc;
    const T hxm2 = hat(i - 2, j), hxm1 = hat(i - 1, j), hxp1 = hat(i + 1, j), hxp2 = hat(i + 2, j);
    const T hym2 = hat(i, j - 2), hym1 = hat(i, j - 1), hyp1 = hat(i, j + 1), hyp2 = hat(i, j + 2);
    const T hd = G.h_dry;
    const bool wc = hc > hd;
    const T nxc = nu_switch(hxm1, hc, hxp1), nyc = nu_switch(hym1, hc, hyp1);
    T ee = (i + 1 < G.nx) ? face_eps(wc, hxp1 > hd, nxc, nu_switch(hc, hxp1, hxp2)) : T(0);
    T ew = (i - 1 >= 0) ? face_eps(hxm1 > hd, wc, nu_switch(hxm2, hxm1, hc), nxc) : T(0);
    T en2 = (j + 1 < G.ny) ? face_eps(wc, hyp1 > hd, nyc, nu_switch(hc, hyp1, hyp2)) : T(0);
    T es2 = (j - 1 >= 0) ? face_eps(hym1 > hd, wc, nu_switch(hym2, hym1, hc), nyc) : T(0);
    en = dissip_faces(en, dflux(ee, at(0, i + 1, j), e0), dflux(ew, e0, at(0, i - 1, j)),
                      dflux(en2, at(0, i, j + 1), e0), dflux(es2, e0, at(0, i, j - 1)), G.kappa);
    un = dissip_faces(un, dflux(ee, at(1, i + 1, j), u0), dflux(ew, u0, at(1, i - 1, j)),
                      dflux(en2, at(1, i, j + 1), u0), dflux(es2, u0, at(1, i, j - 1)), G.kappa);
    vn = dissip_faces(vn, dflux(ee, at(2, i + 1, j), v0), dflux(ew, v0, at(2, i - 1, j)),
                      dflux(en2, at(2, i, j + 1), v0), dflux(es2, v0, at(2, i, j - 1)), G.kappa);
}

template <class T>
__device__ __forceinline__ void dissipation_at(const GridK<T>& G, int i, int j, const T* __restrict__ e,
                                               const T* __restrict__ u, const T* __restrict__ v,
                                               const T* __restrict__ z, T e0, T u0, T v0, T zc, T& en, T& un,
                                               T& vn) {
    auto hat = [&](int ii, int jj) -> T {
        ii = ii < 0 ? 0 : (ii >= G.nx ? G.nx - 1 : ii);
        jj = jj < 0 ? 0 : (jj >= G.ny ? G.ny - 1 : jj);
        size_t q = (size_t)jj * G.pitch + ii;
        return e[q] - z[q];
    };
    auto at = [&](int f, int ii, int jj) -> T {
        ii = ii < 0 ? 0 : (ii >= G.nx ? G.nx - 1 : ii);
        jj = jj < 0 ? 0 : (jj >= G.ny ? G.ny - 1 : jj);
        const T* p = f == 0 ? e : (f == 1 ? u : v);
        return p[(size_t)jj * G.pitch + ii];
    };
    dissipation_core(G, i, j, hat, at, e0, u0, v0, zc, en, un, vn);
}

// The TVD-MacCormack term (the ablation form of S15; Davis 1984, for shallow
// water Garcia-Navarro, Alcrudo and Saviron 1992) at cell (i, j), per axis
// and field phi of level n, with D the face differences (0 beyond the grid,
// which clamped accessors give):
//   r+_i = D_{i-1/2} D_{i+1/2} / D_{i+1/2}^2, r-_i = D_{i-1/2} D_{i+1/2} / D_{i-1/2}^2 (0 on a zero denominator),
//   psi(r) = max(0, min(2 r, 1)), C(nu) = nu (1 - nu) up to nu = 1/2, then 1/4,
//   nu = (|vel| + sqrt(g h)) dt / dx on a wet cell (0 on a dry one), G = C (1 - psi) / 2,
//   T_{i+1/2} = (G(nu_i, r+_i) + G(nu_{i+1}, r-_{i+1})) D_{i+1/2} between two wet
// interior cells; phi += (T_e - T_w) + (T_n - T_s).
template <class T>
__device__ __forceinline__ T tvd_psi(T r) {
    T m = r + r;
    m = m < T(1) ? m : T(1);
    return m > T(0) ? m : T(0);
}
template <class T>
__device__ __forceinline__ T tvd_cnu(T nu) { return nu <= T(0.5) ? nu * (T(1) - nu) : T(0.25); }
template <class T>
__device__ __forceinline__ T tvd_ratio(T num, T den) { return den != T(0) ? div_(num, den) : T(0); }
template <class T>
__device__ __forceinline__ T tvd_face(T dm, T d, T dp, T nua, T nub) {
    const T rpa = tvd_ratio(dm * d, d * d);
    const T rmb = tvd_ratio(d * dp, d * d);
    const T ga = T(0.5) * tvd_cnu(nua) * (T(1) - tvd_psi(rpa));
    const T gb = T(0.5) * tvd_cnu(nub) * (T(1) - tvd_psi(rmb));
    return (ga + gb) * d;
}

template <class T, class HAT, class AT>
__device__ __forceinline__ void tvd_core(const GridK<T>& G, const StepK<T>& S, int i, int j, HAT&& hat, AT&& at,
                                         T& en, T& un, T& vn) {
    const T hd = G.h_dry;
    auto nux = [&](int ii) -> T {
        const T h = hat(ii, j);
        return h > hd ? (fabs(at(1, ii, j)) + rsq_sqrt(G.g * h)) * S.dtdx : T(0);
    };
    auto nuy = [&](int jj) -> T {
        const T h = hat(i, jj);
        return h > hd ? (fabs(at(2, i, jj)) + rsq_sqrt(G.g * h)) * S.dtdy : T(0);
    };
    const bool wc = hat(i, j) > hd;
    const bool we = i + 1 < G.nx && wc && hat(i + 1, j) > hd, ww = i - 1 >= 0 && wc && hat(i - 1, j) > hd;
    const bool wn = j + 1 < G.ny && wc && hat(i, j + 1) > hd, ws = j - 1 >= 0 && wc && hat(i, j - 1) > hd;
    const T nxc = nux(i), nxe = nux(i + 1), nxw = nux(i - 1);
    const T nyc = nuy(j), nyn = nuy(j + 1), nys = nuy(j - 1);
    T* out[3] = {&en, &un, &vn};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        auto Dx = [&](int ii) -> T { return at(f, ii + 1, j) - at(f, ii, j); };
        auto Dy = [&](int jj) -> T { return at(f, i, jj + 1) - at(f, i, jj); };
        const T te = we ? tvd_face(Dx(i - 1), Dx(i), Dx(i + 1), nxc, nxe) : T(0);
        const T tw = ww ? tvd_face(Dx(i - 2), Dx(i - 1), Dx(i), nxw, nxc) : T(0);
        const T tn = wn ? tvd_face(Dy(j - 1), Dy(j), Dy(j + 1), nyc, nyn) : T(0);
        const T ts = ws ? tvd_face(Dy(j - 2), Dy(j - 1), Dy(j), nys, nyc) : T(0);
        *out[f] = *out[f] + ((te - tw) + (tn - ts));
    }
}

template <class T>
__device__ __forceinline__ void tvd_at(const GridK<T>& G, const StepK<T>& S, int i, int j, const T* __restrict__ e,
                                       const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ z,
                                       T& en, T& un, T& vn) {
    auto hat = [&](int ii, int jj) -> T {
        ii = ii < 0 ? 0 : (ii >= G.nx ? G.nx - 1 : ii);
        jj = jj < 0 ? 0 : (jj >= G.ny ? G.ny - 1 : jj);
        size_t q = (size_t)jj * G.pitch + ii;
        return e[q] - z[q];
    };
    auto at = [&](int f, int ii, int jj) -> T {
        ii = ii < 0 ? 0 : (ii >= G.nx ? G.nx - 1 : ii);
        jj = jj < 0 ? 0 : (jj >= G.ny ? G.ny - 1 : jj);
        const T* p = f == 0 ? e : (f == 1 ? u : v);
        return p[(size_t)jj * G.pitch + ii];
    };
    tvd_core(G, S, i, j, hat, at, en, un, vn);
}

template <class T, int SX, int SY, int FR = 0>
__global__ void __launch_bounds__(256) k_plain_pred(GridK<T> G, const double* __restrict__ dtp, double dx,
                                                    double dy, double g, const T* __restrict__ e,
                                                    const T* __restrict__ u, const T* __restrict__ v,
                                                    const T* __restrict__ z, const T* __restrict__ n2,
                                                    T* __restrict__ es, T* __restrict__ us,
                                                    T* __restrict__ vs, DevCtl* ctl_w, double area) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const StepK<T> S = step_consts<T>(dtp);
    T added = T(0);
    if (i < G.nx && j < G.ny) {
        const size_t k = (size_t)j * G.pitch + i;
        Cell<T> c = ld(e, u, v, z, k);
        Cell<T> xn = (i + SX >= 0 && i + SX < G.nx) ? ld(e, u, v, z, (size_t)((ptrdiff_t)k + SX))
                                                   : ghost(c, SX > 0 ? SIDE_E : SIDE_W, G);
        Cell<T> yn = (j + SY >= 0 && j + SY < G.ny) ? ld(e, u, v, z, (size_t)((ptrdiff_t)k + (ptrdiff_t)SY * G.pitch))
                                                   : ghost(c, SY > 0 ? SIDE_N : SIDE_S, G);
        T gn2 = n2 ? n2[k] : G.gn2;
        T fe, fw, fn, fs;
        faces<SX>((c.e - c.z) * c.u, (xn.e - xn.z) * xn.u, i == 0, i == G.nx - 1, SIDE_W, SIDE_E, G, fe, fw);
        faces<SY>((c.e - c.z) * c.v, (yn.e - yn.z) * yn.v, j == 0, j == G.ny - 1, SIDE_S, SIDE_N, G, fn, fs);
        T eo, uo, vo;
        stage<SX, SY, FR>(c, xn, yn, fe, fw, fn, fs, c.e, c.u, c.v, gn2, S, G.h_dry, eo, uo, vo);
        added = wetdry_fix(eo, uo, vo, c.z, G.h_dry);
        es[k] = eo; us[k] = uo; vs[k] = vo;
        if (j < G.own_lo || j >= G.own_hi) added = T(0);
    }
    // predictor clamps count half (the average keeps half of the predicted level)
    if (__any_sync(0xffffffffu, added != T(0))) {
        double s = warp_sum((double)added);
        if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(&ctl_w->clamp, 0.5 * s * area);
    }
}

template <class T, int SX, int SY, int FR = 0>
__global__ void __launch_bounds__(256) k_plain_corr(GridK<T> G, DevCtl* ctl, const double* __restrict__ dtp,
                                                    double dx, double dy, double g,
                                                    const T* __restrict__ e, const T* __restrict__ u,
                                                    const T* __restrict__ v, const T* __restrict__ z,
                                                    const T* __restrict__ n2, const T* __restrict__ es,
                                                    const T* __restrict__ us, const T* __restrict__ vs,
                                                    T* __restrict__ e1, T* __restrict__ u1,
                                                    T* __restrict__ v1, int slot_next, double area) {
    constexpr int CX = -SX, CY = -SY;  // corrector directions
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const double dtd = *dtp;
    const StepK<T> S = step_consts<T>(dtp);
    T added = T(0), speed = T(0);
    double bw = 0.0, be = 0.0, bs = 0.0, bn = 0.0;
    bool bad = false;
    if (i < G.nx && j < G.ny) {
        const size_t k = (size_t)j * G.pitch + i;
        const T zc = z[k];
        Cell<T> cs = ld(es, us, vs, z, k);
        Cell<T> xs = (i + CX >= 0 && i + CX < G.nx) ? ld(es, us, vs, z, (size_t)((ptrdiff_t)k + CX))
                                                   : ghost(cs, CX > 0 ? SIDE_E : SIDE_W, G);
        Cell<T> ys = (j + CY >= 0 && j + CY < G.ny) ? ld(es, us, vs, z, (size_t)((ptrdiff_t)k + (ptrdiff_t)CY * G.pitch))
                                                   : ghost(cs, CY > 0 ? SIDE_N : SIDE_S, G);
        const T e0 = e[k], u0 = u[k], v0 = v[k];
        T gn2 = n2 ? n2[k] : G.gn2;
        T fe, fw, fn, fs;
        const T qxs = (cs.e - cs.z) * cs.u, qys = (cs.e - cs.z) * cs.v;
        faces<CX>(qxs, (xs.e - xs.z) * xs.u, i == 0, i == G.nx - 1, SIDE_W, SIDE_E, G, fe, fw);
        faces<CY>(qys, (ys.e - ys.z) * ys.v, j == 0, j == G.ny - 1, SIDE_S, SIDE_N, G, fn, fs);
        T eo, uo, vo;
        stage<CX, CY, FR>(cs, xs, ys, fe, fw, fn, fs, e0, u0, v0, gn2, S, G.h_dry, eo, uo, vo);
        // S14: average
        T en = T(0.5) * (cs.e + eo), un = T(0.5) * (cs.u + uo), vn = T(0.5) * (cs.v + vo);
        // S15: dissipation of level n (or the TVD term of the ablation)
        if (G.dissipation == 1) tvd_at(G, S, i, j, e, u, v, z, en, un, vn);
        else if (G.kappa != T(0)) dissipation_at(G, i, j, e, u, v, z, e0, u0, v0, zc, en, un, vn);
        // S16: fix, tallies
        added = wetdry_fix(en, un, vn, zc, G.h_dry);
        e1[k] = en; u1[k] = un; v1[k] = vn;
        speed = cfl_speed(en, un, vn, zc, G);
        bad = !isfinite(en + un + vn);
        const T qxn = (e0 - zc) * u0, qyn = (e0 - zc) * v0;
        if (i == 0) bw = 0.5 * ((double)face_bnd(SIDE_W, qxn, G) + (double)face_bnd(SIDE_W, qxs, G));
        if (i == G.nx - 1) be = -0.5 * ((double)face_bnd(SIDE_E, qxn, G) + (double)face_bnd(SIDE_E, qxs, G));
        if (j == 0) bs = 0.5 * ((double)face_bnd(SIDE_S, qyn, G) + (double)face_bnd(SIDE_S, qys, G));
        if (j == G.ny - 1) bn = -0.5 * ((double)face_bnd(SIDE_N, qyn, G) + (double)face_bnd(SIDE_N, qys, G));
        if (j < G.own_lo || j >= G.own_hi) { added = T(0); speed = T(0); bad = false; bw = be = bs = bn = 0.0; }
    }
    const int lane = threadIdx.x & 31;
    T m = warp_max(speed);
    if (lane == 0 && m > T(0))
        atomicMax(&ctl->smax[slot_next], (unsigned long long)__double_as_longlong((double)m));
    if (__any_sync(0xffffffffu, added != T(0))) {
        double s = warp_sum((double)added);
        if (lane == 0 && s != 0.0) atomicAdd(&ctl->clamp, s * area);
    }
    if (__any_sync(0xffffffffu, bw != 0.0 || be != 0.0 || bs != 0.0 || bn != 0.0)) {
        double a = warp_sum(bw), b = warp_sum(be), c2 = warp_sum(bs), d = warp_sum(bn);
        if (lane == 0) {
            if (a != 0.0) atomicAdd(&ctl->bflux[0], a * dtd * dy);
            if (b != 0.0) atomicAdd(&ctl->bflux[1], b * dtd * dy);
            if (c2 != 0.0) atomicAdd(&ctl->bflux[2], c2 * dtd * dx);
            if (d != 0.0) atomicAdd(&ctl->bflux[3], d * dtd * dx);
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&ctl->flags, (unsigned)SWE_FLAG_NONFINITE);
}

template <class T>
static GridK<T> grid_of(const swe_ctx* c) {
    GridK<T> G;
    const swe_params& p = c->p;
    G.nx = p.nx; G.ny = p.ny; G.pitch = c->pitch;
    G.g = (T)p.g; G.h_dry = (T)p.h_dry; G.kappa = (T)p.kappa;
    G.gn2 = (T)(p.g * p.manning_n * p.manning_n);
    G.inv_dx = (T)(1.0 / p.dx); G.inv_dy = (T)(1.0 / p.dy);
    for (int s = 0; s < 4; ++s) { G.bc[s] = p.bc[s]; G.qin[s] = (T)p.q_in[s]; }
    G.own_lo = c->own_lo; G.own_hi = c->own_hi;
    G.friction = p.friction; G.dissipation = p.dissipation;
    return G;
}

template <class T, int SX, int SY, int FR>
static cudaError_t plain_step_t(swe_ctx* c, int s, long long k) {
    const swe_params& p = c->p;
    GridK<T> G = grid_of<T>(c);
    int slot = (int)(k % 3), slot_next = (int)((k + 1) % 3);
    k_plain_dt<<<1, 1, 0, c->stream>>>(c->ctl, slot, slot_next, c->dt_fixed_cap > 0 && c->dt_fixed ? c->dt_fixed : nullptr,
                                       s, c->dt_hist, p.cfl, p.dt_max, 1.0 / p.dx, 1.0 / p.dy, p.g);
    dim3 blk(32, 8), grd((p.nx + 31) / 32, (p.ny + 7) / 8);
    const int a = c->cur, b = 1 - c->cur;
    const double area = p.dx * p.dy;
    k_plain_pred<T, SX, SY, FR><<<grd, blk, 0, c->stream>>>(
        G, &c->ctl->cur.dt, p.dx, p.dy, p.g, (const T*)c->eta[a], (const T*)c->u[a], (const T*)c->v[a], (const T*)c->z,
        (const T*)c->n2, (T*)c->ps[0], (T*)c->ps[1], (T*)c->ps[2], c->ctl, area);
    k_plain_corr<T, SX, SY, FR><<<grd, blk, 0, c->stream>>>(
        G, c->ctl, &c->ctl->cur.dt, p.dx, p.dy, p.g, (const T*)c->eta[a], (const T*)c->u[a], (const T*)c->v[a], (const T*)c->z,
        (const T*)c->n2, (const T*)c->ps[0], (const T*)c->ps[1], (const T*)c->ps[2], (T*)c->eta[b], (T*)c->u[b],
        (T*)c->v[b], slot_next, area);
    return cudaGetLastError();
}

template <class T>
static cudaError_t plain_step_dir(swe_ctx* c, int s, long long k) {
    int sx, sy;
    step_dirs(c->p.dir_cycle, k, &sx, &sy);
    if (c->p.friction == 1) {  // the explicit-friction ablation
        if (sx > 0 && sy > 0) return plain_step_t<T, 1, 1, 1>(c, s, k);
        if (sx > 0 && sy < 0) return plain_step_t<T, 1, -1, 1>(c, s, k);
        if (sx < 0 && sy > 0) return plain_step_t<T, -1, 1, 1>(c, s, k);
        return plain_step_t<T, -1, -1, 1>(c, s, k);
    }
    if (sx > 0 && sy > 0) return plain_step_t<T, 1, 1, 0>(c, s, k);
    if (sx > 0 && sy < 0) return plain_step_t<T, 1, -1, 0>(c, s, k);
    if (sx < 0 && sy > 0) return plain_step_t<T, -1, 1, 0>(c, s, k);
    return plain_step_t<T, -1, -1, 0>(c, s, k);
}

}  // namespace swe
