// swe_fused.cuh -- the fused MacCormack step: all 16 sub-steps of one time
// step (Seitz et al. 2013, Sec. 1) in one sweep over the grid, one kernel
// launch per step.  Device code and launch templates; the explicit
// instantiations are spread over swe_fused_*.cu so they compile in parallel,
// the host set-up (tensor maps, work plan) is in swe_fused.cu.
#pragma once
//
// Decomposition.  A work item is a column strip of 32*CPT cells (one warp, CPT
// cells per lane) by a segment of L rows.  Along x the warp outputs 31 of its
// 32 lanes: the remaining lane (lane 0 when the predictor differences
// forward, lane 31 when backward) only computes the predicted values its
// neighbour's corrector needs.  Along y the warp marches row by row; the
// dependency radius of one step is one row for predictor and corrector and
// two rows for the dissipation switch, so the warp loads the segment plus two
// rows above and below.
//
// Data movement.  Level-n rows (eta, u, v, z) stream into a per-warp ring in
// shared memory with TMA (cp.async.bulk.tensor.2d, completion on an
// mbarrier), NPRE rows ahead of use; a row stays in the ring while any of the
// four rows of the step's stencil window still needs it.  The two predicted
// rows and the y dissipation switches the corrector needs are carried in
// registers from one row to the next.  x neighbours come from adjacent lanes
// by shuffles; the strip's output-side edge lane reads the ring's halo
// columns (the other edge lane never outputs).  Boundary handling runs under
// warp-uniform branches: per row for the y sides, per item for the x sides.  The new level is stored with
// 16-byte vector stores.  Out-of-grid rows and columns read as zeros (TMA
// fill) and are replaced by the ghost cells of the boundary conditions.
//
// Reductions.  The CFL speed of the new level (the next step's S2) is reduced
// per warp, per CTA, then with one atomicMax per CTA on the FP64 bit
// pattern (exact, order-free).  Each CTA derives this step's dt from the
// previous step's reduction, in FP64.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>

#include "swe_internal.cuh"

namespace swe {
namespace fz {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NWARP = 4;           // warps per CTA
constexpr int NSLOT = 8;           // ring slots per warp (a power of two)
constexpr int NPRE = NSLOT - 4;    // rows loaded ahead of the current row
constexpr unsigned long long WAIT_LIMIT = 4000000000ull;  // cycles (~2 s) before a wait gives up

template <class T, int CPT>
struct Geo {
    static constexpr int W = 32 * CPT;                    // window columns
    static constexpr int OUT = W - CPT;                   // output columns per item
    static constexpr int BW = W + 8;                      // TMA box width (elements)
    static constexpr int ALIGN = 16 / (int)sizeof(T);     // TMA x alignment (elements)
    static constexpr int FSTRIDE = ((BW * (int)sizeof(T) + 127) / 128) * 128;  // bytes per field row
    static constexpr int SLOT = 4 * FSTRIDE;              // bytes per ring slot (eta, u, v, z)
    static constexpr int WARP_SMEM = NSLOT * SLOT;
};

template <class T>
struct Args {
    GridK<T> G;
    T* e1; T* u1; T* v1;           // new level (pitched)
    const T* n2;                   // per-cell g n^2 or null
    DevCtl* ctl;
    const double* dt_fixed;        // null: CFL step
    double* dt_hist;
    double dx, dy, g, cfl, dt_max, area;
    int s;                         // step within the call
    int slot_cur, slot_next, slot_zero;
    int nxs, nys, L, nitems;
};

__device__ __forceinline__ unsigned saddr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(saddr(b)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait; false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
    if (mbar_try(b, parity)) return true;
    unsigned long long t0 = clock64();
    while (!mbar_try(b, parity))
        if (clock64() - t0 > WAIT_LIMIT) return false;
    return true;
}
__device__ __forceinline__ void tma_row(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(saddr(dst)), "l"(map), "r"(x), "r"(y), "r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <class T, int CPT>
__device__ __forceinline__ void ld_vec(const T* p, T (&o)[CPT]) {
    if constexpr (sizeof(T) * CPT == 16) {
        if constexpr (sizeof(T) == 4) {
            float4 q = *reinterpret_cast<const float4*>(p);
            o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
        } else {
            double2 q = *reinterpret_cast<const double2*>(p);
            o[0] = q.x; o[1] = q.y;
        }
    } else if constexpr (sizeof(T) * CPT == 8) {
        float2 q = *reinterpret_cast<const float2*>(p);
        o[0] = q.x; o[1] = q.y;
    } else {
#pragma unroll
        for (int c = 0; c < CPT; ++c) o[c] = p[c];
    }
}
template <class T, int CPT>
__device__ __forceinline__ void st_vec(T* p, const T (&o)[CPT]) {
    if constexpr (sizeof(T) * CPT == 16) {
        if constexpr (sizeof(T) == 4) *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
        else *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    } else if constexpr (sizeof(T) * CPT == 8) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    } else {
#pragma unroll
        for (int c = 0; c < CPT; ++c) p[c] = o[c];
    }
}

template <class T, int CPT>
struct Row {  // eta, u, v, z of the lane's CPT cells in one row
    T e[CPT], u[CPT], v[CPT], z[CPT];
};
template <class T, int CPT>
struct PRow {  // predicted eta, u, v
    T e[CPT], u[CPT], v[CPT];
};

template <class T, int CPT>
__device__ __forceinline__ void ld_row(const unsigned char* slot, int col, Row<T, CPT>& r) {
    ld_vec<T, CPT>(reinterpret_cast<const T*>(slot + 0 * Geo<T, CPT>::FSTRIDE) + col, r.e);
    ld_vec<T, CPT>(reinterpret_cast<const T*>(slot + 1 * Geo<T, CPT>::FSTRIDE) + col, r.u);
    ld_vec<T, CPT>(reinterpret_cast<const T*>(slot + 2 * Geo<T, CPT>::FSTRIDE) + col, r.v);
    ld_vec<T, CPT>(reinterpret_cast<const T*>(slot + 3 * Geo<T, CPT>::FSTRIDE) + col, r.z);
}
template <class T, int CPT>
__device__ __forceinline__ T ld1(const unsigned char* slot, int f, int col) {
    return reinterpret_cast<const T*>(slot + f * Geo<T, CPT>::FSTRIDE)[col];
}

template <class T, int CPT>
__device__ __forceinline__ void ghost_row(Row<T, CPT>& r, int side, const GridK<T>& G) {
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        Cell<T> q; q.e = r.e[c]; q.u = r.u[c]; q.v = r.v[c]; q.z = r.z[c];
        q = ghost(q, side, G);
        r.e[c] = q.e; r.u[c] = q.u; r.v[c] = q.v; r.z[c] = q.z;
    }
}

template <class T>
__device__ __forceinline__ T shdn(T x) { return __shfl_down_sync(FULL, x, 1); }
template <class T>
__device__ __forceinline__ T shup(T x) { return __shfl_up_sync(FULL, x, 1); }

// Neighbours of the lane's cells one column to the right (D > 0) or left
// (D < 0): the next cell of the lane, else the adjacent lane's end cell;
// the strip-edge lane takes the ring's halo column value h.
template <int D, class T, int CPT>
__device__ __forceinline__ void shift(const T (&a)[CPT], T halo, bool edge_lane, T (&o)[CPT]) {
    if (D > 0) {
#pragma unroll
        for (int c = 0; c + 1 < CPT; ++c) o[c] = a[c + 1];
        T t = shdn(a[0]);
        o[CPT - 1] = edge_lane ? halo : t;
    } else {
#pragma unroll
        for (int c = 1; c < CPT; ++c) o[c] = a[c - 1];
        T t = shup(a[CPT - 1]);
        o[0] = edge_lane ? halo : t;
    }
}

// x neighbours of a level-n row on side D; the halo is read on that side only.
template <int D, class T, int CPT>
__device__ __forceinline__ void row_shift(const Row<T, CPT>& r, const unsigned char* slot, int col, int lane,
                                          Row<T, CPT>& o) {
    const int hc = D > 0 ? col + CPT : col - 1;
    const bool el = D > 0 ? lane == 31 : lane == 0;
    shift<D, T, CPT>(r.e, ld1<T, CPT>(slot, 0, hc), el, o.e);
    shift<D, T, CPT>(r.u, ld1<T, CPT>(slot, 1, hc), el, o.u);
    shift<D, T, CPT>(r.v, ld1<T, CPT>(slot, 2, hc), el, o.v);
    shift<D, T, CPT>(r.z, ld1<T, CPT>(slot, 3, hc), el, o.z);
}
// x neighbours without a halo (the lane that would need it never outputs).
template <int D, class T, int CPT>
__device__ __forceinline__ void row_shift_nohalo(const Row<T, CPT>& r, Row<T, CPT>& o) {
    shift<D, T, CPT>(r.e, T(0), false, o.e);
    shift<D, T, CPT>(r.u, T(0), false, o.u);
    shift<D, T, CPT>(r.v, T(0), false, o.v);
    shift<D, T, CPT>(r.z, T(0), false, o.z);
}

struct Acc {
    double clamp, bw, be, bs, bn;
    double smax;
    bool bad;
};

// Process one work item: rows [y0, y1) of the strip whose window starts at xw.
// One loop iteration per ring row r: y switch and predictor of row r-1,
// corrector/average/dissipation/fix of row r-2.
template <class T, int CPT, int SX, int SY, bool KAPPA>
__device__ __forceinline__ void run_item(const Args<T>& A, const StepK<T>& S, Acc& acc, unsigned char* ring,
                                         uint64_t* bars, int lane, int xw, int y0, int y1, unsigned& g0,
                                         const CUtensorMap* tme, const CUtensorMap* tmu, const CUtensorMap* tmv,
                                         const CUtensorMap* tmz, bool& timed_out) {
    using Gm = Geo<T, CPT>;
    constexpr int CX = -SX, CY = -SY;
    const GridK<T>& G = A.G;
    const int ny = G.ny, nx = G.nx;
    const T hd = G.h_dry;
    const int xb = (xw - 2) & ~(Gm::ALIGN - 1);  // TMA box start, 16-byte aligned
    const int col = (xw - xb) + CPT * lane;      // ring column of the lane's first cell
    const int x0c = xw + CPT * lane;             // grid column of the lane's first cell
    const int nr = y1 - y0 + 4;
    const bool out_lane = SX > 0 ? lane != 0 : lane != 31;
    const bool edge = (xw - 2 < 0) || (xw + Gm::W + 1 > nx - 1);  // strip touches the x boundary
    constexpr unsigned BYTES = 4u * Gm::BW * sizeof(T);

    auto issue = [&](int k) {
        if (lane == 0 && k < nr) {
            const unsigned g = g0 + (unsigned)k;
            uint64_t* bar = bars + (g & (NSLOT - 1));
            unsigned char* dst = ring + (g & (NSLOT - 1)) * Gm::SLOT;
            const int y = y0 - 2 + k;
            mbar_expect(bar, BYTES);
            tma_row(dst + 0 * Gm::FSTRIDE, tme, bar, xb, y);
            tma_row(dst + 1 * Gm::FSTRIDE, tmu, bar, xb, y);
            tma_row(dst + 2 * Gm::FSTRIDE, tmv, bar, xb, y);
            tma_row(dst + 3 * Gm::FSTRIDE, tmz, bar, xb, y);
        }
    };
    fence_async_smem();  // the previous item's rows were read through the generic proxy
#pragma unroll
    for (int k = 0; k < NPRE; ++k) issue(k);

    auto slot_of = [&](int row) -> const unsigned char* {  // clamped to the grid
        const int src = row < 0 ? 0 : (row >= ny ? ny - 1 : row);
        return ring + ((g0 + (unsigned)(src - (y0 - 2))) & (NSLOT - 1)) * Gm::SLOT;
    };

    PRow<T, CPT> PA, PB;   // predicted rows C-1 and C
    T NA[CPT], NB[CPT];    // y switches of rows C-1 and C
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
        NA[j] = NB[j] = T(0);
        PA.e[j] = PA.u[j] = PA.v[j] = PB.e[j] = PB.u[j] = PB.v[j] = T(0);
    }
    T clamp_i = T(0), bw_i = T(0), be_i = T(0), bs_i = T(0), bn_i = T(0), smax_i = T(0);
    bool bad_i = false;
    int waited = 0;

#pragma unroll 1
    for (int k = 0; k < nr; ++k) {
        const int r = y0 - 2 + k;
        fence_async_smem();
        issue(k + NPRE);  // into the slot of ring row k-4, consumed last iteration
        {
            const unsigned g = g0 + (unsigned)k;
            const bool ok = mbar_wait(bars + (g & (NSLOT - 1)), (g / NSLOT) & 1u);
            if (__any_sync(FULL, !ok)) { timed_out = true; break; }
            waited = k + 1;
        }
        if (k < 2) { __syncwarp(); continue; }
        // rows r (0), r-1 (1), r-2 (2), r-3 (3); ghosted outside [0, ny)
        const bool brow = (r - 3 < 0) || (r >= ny);
        const unsigned char* s0 = slot_of(r);
        const unsigned char* s1 = slot_of(r - 1);
        const unsigned char* s2 = slot_of(r - 2);
        const unsigned char* s3 = slot_of(r - 3);
        Row<T, CPT> R0, R1, R2, R3;
        ld_row<T, CPT>(s0, col, R0);
        ld_row<T, CPT>(s1, col, R1);
        ld_row<T, CPT>(s2, col, R2);
        if (KAPPA || k >= 4) ld_row<T, CPT>(s3, col, R3);
        if (brow) {
            if (r < 0) ghost_row(R0, SIDE_S, G); else if (r >= ny) ghost_row(R0, SIDE_N, G);
            if (r - 1 < 0) ghost_row(R1, SIDE_S, G); else if (r - 1 >= ny) ghost_row(R1, SIDE_N, G);
            if (r - 2 < 0) ghost_row(R2, SIDE_S, G); else if (r - 2 >= ny) ghost_row(R2, SIDE_N, G);
            if (r - 3 < 0) ghost_row(R3, SIDE_S, G); else if (r - 3 >= ny) ghost_row(R3, SIDE_N, G);
        }
        // ---------------- y switch of row r-1 (S15 input)
        T NN[CPT];
        if (KAPPA) {
#pragma unroll
            for (int j = 0; j < CPT; ++j) NN[j] = nu_switch(R2.e[j] - R2.z[j], R1.e[j] - R1.z[j], R0.e[j] - R0.z[j]);
        }
        // ---------------- predictor of row p = r-1 (S1-S8)
        PRow<T, CPT> PN;
        const int p = r - 1;
        {
            const Row<T, CPT>& c = R1;
            const Row<T, CPT>& yn = SY > 0 ? R0 : R2;
            Row<T, CPT> xn;
            row_shift<SX, T, CPT>(c, s1, col, lane, xn);
            T hc[CPT], qxc[CPT], qyc[CPT], fe[CPT], fw[CPT], fn[CPT], fs[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                hc[j] = c.e[j] - c.z[j];
                qxc[j] = hc[j] * c.u[j];
                qyc[j] = hc[j] * c.v[j];
                const T qxn = (xn.e[j] - xn.z[j]) * xn.u[j];
                const T qyn = (yn.e[j] - yn.z[j]) * yn.v[j];
                if (SX > 0) { fe[j] = qxn; fw[j] = qxc[j]; } else { fe[j] = qxc[j]; fw[j] = qxn; }
                if (SY > 0) { fn[j] = qyn; fs[j] = qyc[j]; } else { fn[j] = qyc[j]; fs[j] = qyn; }
            }
            if (edge) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    const int x = x0c + j;
                    if (x == 0) fw[j] = face_bnd(SIDE_W, qxc[j], G);
                    if (x == nx - 1) fe[j] = face_bnd(SIDE_E, qxc[j], G);
                    if (SX > 0 ? x == nx - 1 : x == 0) {
                        Cell<T> q; q.e = c.e[j]; q.u = c.u[j]; q.v = c.v[j]; q.z = c.z[j];
                        q = ghost(q, SX > 0 ? SIDE_E : SIDE_W, G);
                        xn.e[j] = q.e; xn.u[j] = q.u; xn.v[j] = q.v; xn.z[j] = q.z;
                    }
                }
            }
            if (p == 0) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) fs[j] = face_bnd(SIDE_S, qyc[j], G);
            }
            if (p == ny - 1) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) fn[j] = face_bnd(SIDE_N, qyc[j], G);
            }
            T gn2v[CPT];
            if (A.n2 != nullptr) {
                int xc = x0c < 0 ? 0 : (x0c > G.pitch - CPT ? G.pitch - CPT : x0c);
                const int pr = p < 0 ? 0 : (p >= ny ? ny - 1 : p);
                ld_vec<T, CPT>(A.n2 + (size_t)pr * G.pitch + xc, gn2v);
            } else {
#pragma unroll
                for (int j = 0; j < CPT; ++j) gn2v[j] = G.gn2;
            }
            T added = T(0);
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                Cell<T> cc, cx, cy;
                cc.e = c.e[j]; cc.u = c.u[j]; cc.v = c.v[j]; cc.z = c.z[j];
                cx.e = xn.e[j]; cx.u = xn.u[j]; cx.v = xn.v[j]; cx.z = xn.z[j];
                cy.e = yn.e[j]; cy.u = yn.u[j]; cy.v = yn.v[j]; cy.z = yn.z[j];
                T eo, uo, vo;
                stage<SX, SY>(cc, cx, cy, fe[j], fw[j], fn[j], fs[j], cc.e, cc.u, cc.v, gn2v[j], S, hd, eo, uo, vo);
                T ad = wetdry_fix(eo, uo, vo, cc.z, hd);
                if (edge && x0c + j >= nx) ad = T(0);
                added += ad;
                PN.e[j] = eo; PN.u[j] = uo; PN.v[j] = vo;
            }
            // a predicted clamp counts once per cell: in the item and lane that output it
            // (a lane's CPT cells never straddle column 0)
            const bool own = out_lane && p >= y0 && p < y1 && x0c >= 0;
            if (own) clamp_i = fma_(T(0.5), added, clamp_i);
        }
        // ---------------- corrector/average/dissipation/fix of row C = r-2 (S9-S16)
        const int C = r - 2;
        if (k >= 4) {
            const Row<T, CPT>& n0 = R2;
            Row<T, CPT> cs, ys, xs;
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                cs.e[j] = PB.e[j]; cs.u[j] = PB.u[j]; cs.v[j] = PB.v[j]; cs.z[j] = n0.z[j];
                if (CY < 0) { ys.e[j] = PA.e[j]; ys.u[j] = PA.u[j]; ys.v[j] = PA.v[j]; ys.z[j] = R3.z[j]; }
                else        { ys.e[j] = PN.e[j]; ys.u[j] = PN.u[j]; ys.v[j] = PN.v[j]; ys.z[j] = R1.z[j]; }
            }
            if (CY < 0 ? C == 0 : C == ny - 1) { ys = cs; ghost_row(ys, CY < 0 ? SIDE_S : SIDE_N, G); }
            row_shift_nohalo<CX, T, CPT>(cs, xs);  // the lane that would need a halo never outputs
            T qxs[CPT], qys[CPT], fe[CPT], fw[CPT], fn[CPT], fs[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const T h = cs.e[j] - cs.z[j];
                qxs[j] = h * cs.u[j];
                qys[j] = h * cs.v[j];
                const T qxn = (xs.e[j] - xs.z[j]) * xs.u[j];
                const T qyn = (ys.e[j] - ys.z[j]) * ys.v[j];
                if (CX > 0) { fe[j] = qxn; fw[j] = qxs[j]; } else { fe[j] = qxs[j]; fw[j] = qxn; }
                if (CY > 0) { fn[j] = qyn; fs[j] = qys[j]; } else { fn[j] = qys[j]; fs[j] = qyn; }
            }
            if (edge) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    const int x = x0c + j;
                    if (x == 0) fw[j] = face_bnd(SIDE_W, qxs[j], G);
                    if (x == nx - 1) fe[j] = face_bnd(SIDE_E, qxs[j], G);
                    if (CX > 0 ? x == nx - 1 : x == 0) {
                        Cell<T> q; q.e = cs.e[j]; q.u = cs.u[j]; q.v = cs.v[j]; q.z = cs.z[j];
                        q = ghost(q, CX > 0 ? SIDE_E : SIDE_W, G);
                        xs.e[j] = q.e; xs.u[j] = q.u; xs.v[j] = q.v; xs.z[j] = q.z;
                    }
                }
            }
            if (C == 0) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) fs[j] = face_bnd(SIDE_S, qys[j], G);
            }
            if (C == ny - 1) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) fn[j] = face_bnd(SIDE_N, qys[j], G);
            }
            T gn2v[CPT];
            if (A.n2 != nullptr) {
                int xc = x0c < 0 ? 0 : (x0c > G.pitch - CPT ? G.pitch - CPT : x0c);
                ld_vec<T, CPT>(A.n2 + (size_t)C * G.pitch + xc, gn2v);
            } else {
#pragma unroll
                for (int j = 0; j < CPT; ++j) gn2v[j] = G.gn2;
            }
            T oe[CPT], ou[CPT], ov[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                Cell<T> cc, cx, cy;
                cc.e = cs.e[j]; cc.u = cs.u[j]; cc.v = cs.v[j]; cc.z = cs.z[j];
                cx.e = xs.e[j]; cx.u = xs.u[j]; cx.v = xs.v[j]; cx.z = xs.z[j];
                cy.e = ys.e[j]; cy.u = ys.u[j]; cy.v = ys.v[j]; cy.z = ys.z[j];
                T eo, uo, vo;
                stage<CX, CY>(cc, cx, cy, fe[j], fw[j], fn[j], fs[j], n0.e[j], n0.u[j], n0.v[j], gn2v[j], S, hd, eo,
                              uo, vo);
                oe[j] = T(0.5) * (cc.e + eo);
                ou[j] = T(0.5) * (cc.u + uo);
                ov[j] = T(0.5) * (cc.v + vo);
            }
            if (KAPPA) {
                // level-n neighbours of row C; the halo is needed on the output side only
                Row<T, CPT> nl, nr;
                if (SX > 0) {
                    row_shift_nohalo<-1, T, CPT>(n0, nl);
                    row_shift<+1, T, CPT>(n0, s2, col, lane, nr);
                } else {
                    row_shift<-1, T, CPT>(n0, s2, col, lane, nl);
                    row_shift_nohalo<+1, T, CPT>(n0, nr);
                }
                T h0[CPT], hl[CPT], hr[CPT];
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    h0[j] = n0.e[j] - n0.z[j];
                    hl[j] = nl.e[j] - nl.z[j];
                    hr[j] = nr.e[j] - nr.z[j];
                }
                if (edge) {  // ghost depth at columns -1 and nx is the adjacent interior depth
#pragma unroll
                    for (int j = 0; j < CPT; ++j) {
                        if (x0c + j == 0) hl[j] = h0[j];
                        if (x0c + j == nx - 1) hr[j] = h0[j];
                    }
                }
                T nuc[CPT], nul[CPT], nur[CPT];
#pragma unroll
                for (int j = 0; j < CPT; ++j) nuc[j] = nu_switch(hl[j], h0[j], hr[j]);
                {
                    // switch one column outside the lane: from the adjacent lane, or
                    // computed from the ring on the output side of the strip edge
                    T lo = shup(nuc[CPT - 1]), hi = shdn(nuc[0]);
                    if (SX > 0) {
                        const T h2 = ld1<T, CPT>(s2, 0, col + CPT + 1) - ld1<T, CPT>(s2, 3, col + CPT + 1);
                        const T ext = nu_switch(h0[CPT - 1], hr[CPT - 1], h2);
                        hi = lane == 31 ? ext : hi;
                    } else {
                        const T h2 = ld1<T, CPT>(s2, 0, col - 2) - ld1<T, CPT>(s2, 3, col - 2);
                        const T ext = nu_switch(h2, hl[0], h0[0]);
                        lo = lane == 0 ? ext : lo;
                    }
#pragma unroll
                    for (int j = 1; j < CPT; ++j) nul[j] = nuc[j - 1];
#pragma unroll
                    for (int j = 0; j + 1 < CPT; ++j) nur[j] = nuc[j + 1];
                    nul[0] = lo;
                    nur[CPT - 1] = hi;
                }
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    const bool wc = h0[j] > hd;
                    T ee = face_eps(wc, hr[j] > hd, nuc[j], nur[j]);
                    T ew = face_eps(hl[j] > hd, wc, nul[j], nuc[j]);
                    T en = face_eps(wc, (R1.e[j] - R1.z[j]) > hd, NB[j], NN[j]);
                    T es = face_eps((R3.e[j] - R3.z[j]) > hd, wc, NA[j], NB[j]);
                    if (edge) {
                        if (x0c + j + 1 >= nx) ee = T(0);
                        if (x0c + j - 1 < 0) ew = T(0);
                    }
                    if (C + 1 >= ny) en = T(0);
                    if (C - 1 < 0) es = T(0);
                    oe[j] = dissip(oe[j], n0.e[j], nl.e[j], nr.e[j], R3.e[j], R1.e[j], ee, ew, en, es, G.kappa);
                    ou[j] = dissip(ou[j], n0.u[j], nl.u[j], nr.u[j], R3.u[j], R1.u[j], ee, ew, en, es, G.kappa);
                    ov[j] = dissip(ov[j], n0.v[j], nl.v[j], nr.v[j], R3.v[j], R1.v[j], ee, ew, en, es, G.kappa);
                }
            }
            // S16: fix, the next step's CFL speed, tallies, store
            T added = T(0), sp = T(0);
            bool badc = false;
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                T ad = wetdry_fix(oe[j], ou[j], ov[j], n0.z[j], hd);
                T spj = cfl_speed(oe[j], ou[j], ov[j], n0.z[j], G);
                const T sum = oe[j] + ou[j] + ov[j];
                const bool bj = !((sum - sum) == T(0));
                if (edge && x0c + j >= nx) { ad = T(0); spj = T(0); }
                added += ad;
                sp = spj > sp ? spj : sp;
                badc = badc || bj;
            }
            if (out_lane && x0c >= 0 && x0c < nx) {
                clamp_i += added;
                smax_i = sp > smax_i ? sp : smax_i;
                bad_i = bad_i || badc;
                const size_t o = (size_t)C * G.pitch + x0c;
                st_vec<T, CPT>(A.e1 + o, oe);
                st_vec<T, CPT>(A.u1 + o, ou);
                st_vec<T, CPT>(A.v1 + o, ov);
                if (edge) {
#pragma unroll
                    for (int j = 0; j < CPT; ++j) {
                        const T qxn = (n0.e[j] - n0.z[j]) * n0.u[j];
                        if (x0c + j == 0) bw_i += T(0.5) * (face_bnd(SIDE_W, qxn, G) + face_bnd(SIDE_W, qxs[j], G));
                        if (x0c + j == nx - 1) be_i -= T(0.5) * (face_bnd(SIDE_E, qxn, G) + face_bnd(SIDE_E, qxs[j], G));
                    }
                }
                if (C == 0 || C == ny - 1) {
#pragma unroll
                    for (int j = 0; j < CPT; ++j) {
                        if (edge && x0c + j >= nx) continue;
                        const T qyn = (n0.e[j] - n0.z[j]) * n0.v[j];
                        if (C == 0) bs_i += T(0.5) * (face_bnd(SIDE_S, qyn, G) + face_bnd(SIDE_S, qys[j], G));
                        if (C == ny - 1) bn_i -= T(0.5) * (face_bnd(SIDE_N, qyn, G) + face_bnd(SIDE_N, qys[j], G));
                    }
                }
            }
        }
        // rotate the register window
        if (SY > 0) {
#pragma unroll
            for (int j = 0; j < CPT; ++j) { PA.e[j] = PB.e[j]; PA.u[j] = PB.u[j]; PA.v[j] = PB.v[j]; }
        }
#pragma unroll
        for (int j = 0; j < CPT; ++j) { PB.e[j] = PN.e[j]; PB.u[j] = PN.u[j]; PB.v[j] = PN.v[j]; }
        if (KAPPA) {
#pragma unroll
            for (int j = 0; j < CPT; ++j) { NA[j] = NB[j]; NB[j] = NN[j]; }
        }
        __syncwarp();
    }
    if (timed_out) {
        // drain this item's loads still in flight (bounded) before the ring is reused or left
        const int issued = nr < waited + NPRE ? nr : waited + NPRE;
        for (int k = waited; k < issued; ++k) {
            const unsigned g = g0 + (unsigned)k;
            unsigned long long t0 = clock64();
            while (!mbar_try(bars + (g & (NSLOT - 1)), (g / NSLOT) & 1u))
                if (clock64() - t0 > WAIT_LIMIT / 8) break;
        }
    }
    g0 += (unsigned)nr;
    acc.clamp += (double)clamp_i;
    acc.bw += (double)bw_i; acc.be += (double)be_i; acc.bs += (double)bs_i; acc.bn += (double)bn_i;
    acc.smax = fmax(acc.smax, (double)smax_i);
    acc.bad = acc.bad || bad_i;
}

template <class T, int CPT, int SX, int SY, bool KAPPA>
__global__ void __launch_bounds__(NWARP * 32, (sizeof(T) == 4 ? 4 : 2))
k_fused(const __grid_constant__ CUtensorMap tme, const __grid_constant__ CUtensorMap tmu,
        const __grid_constant__ CUtensorMap tmv, const __grid_constant__ CUtensorMap tmz, const Args<T> A) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[NWARP][NSLOT];
    __shared__ double sh_dt;
    __shared__ double red[NWARP][6];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        double dt = A.dt_fixed ? A.dt_fixed[A.s]
                               : dt_from_speed(__longlong_as_double((long long)A.ctl->smax[A.slot_cur]), A.cfl, A.dt_max);
        sh_dt = dt;
        if (blockIdx.x == 0) {
            DevCtl* c = A.ctl;
            c->dt_last = dt;
            c->t += dt;
            c->dt_min = fmin(c->dt_min, dt);
            c->dt_maxs = fmax(c->dt_maxs, dt);
            A.dt_hist[A.s] = dt;
            c->smax[A.slot_zero] = 0ull;
        }
    }
    if (lane == 0)
        for (int s = 0; s < NSLOT; ++s) mbar_init(&bars[warp][s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    const double dt = sh_dt;
    const StepK<T> S = make_stepk<T>(dt, A.dx, A.dy, A.g);

    Acc acc;
    acc.clamp = acc.bw = acc.be = acc.bs = acc.bn = 0.0;
    acc.smax = 0.0;
    acc.bad = false;
    bool timed_out = false;
    unsigned g0 = 0;
    unsigned char* ring = smem + warp * Geo<T, CPT>::WARP_SMEM;
    const int gw = blockIdx.x * NWARP + warp, nw = gridDim.x * NWARP;
    for (int item = gw; item < A.nitems && !timed_out; item += nw) {
        const int kx = item % A.nxs, ky = item / A.nxs;
        const int x0 = kx * Geo<T, CPT>::OUT;
        const int xw = SX > 0 ? x0 - CPT : x0;
        const int y0 = ky * A.L;
        const int y1 = min(A.G.ny, y0 + A.L);
        run_item<T, CPT, SX, SY, KAPPA>(A, S, acc, ring, bars[warp], lane, xw, y0, y1, g0, &tme, &tmu, &tmv, &tmz,
                                        timed_out);
    }

    // ---- reductions: warp, CTA, then one atomic per CTA
    double v[6] = {acc.smax, acc.clamp, acc.bw, acc.be, acc.bs, acc.bn};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = fmax(v[0], __shfl_xor_sync(FULL, v[0], o));
#pragma unroll
        for (int m = 1; m < 6; ++m) v[m] += __shfl_xor_sync(FULL, v[m], o);
    }
    const bool bad = __any_sync(FULL, acc.bad);
    const bool tmo = __any_sync(FULL, timed_out);
    if (lane == 0) {
#pragma unroll
        for (int m = 0; m < 6; ++m) red[warp][m] = v[m];
        if (bad) atomicOr(&A.ctl->flags, (unsigned)SWE_FLAG_NONFINITE);
        if (tmo) atomicOr(&A.ctl->flags, (unsigned)SWE_FLAG_TIMEOUT);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[6] = {0, 0, 0, 0, 0, 0};
        for (int w = 0; w < NWARP; ++w) {
            t[0] = fmax(t[0], red[w][0]);
            for (int m = 1; m < 6; ++m) t[m] += red[w][m];
        }
        if (t[0] > 0.0) {
            unsigned long long bits = (unsigned long long)__double_as_longlong(t[0]);
            unsigned long long* slot = &A.ctl->smax[A.slot_next];
            if (bits > *(volatile unsigned long long*)slot) atomicMax(slot, bits);
        }
        if (t[1] != 0.0) atomicAdd(&A.ctl->clamp, t[1] * A.area);
        if (t[2] != 0.0) atomicAdd(&A.ctl->bflux[0], t[2] * dt * A.dy);
        if (t[3] != 0.0) atomicAdd(&A.ctl->bflux[1], t[3] * dt * A.dy);
        if (t[4] != 0.0) atomicAdd(&A.ctl->bflux[2], t[4] * dt * A.dx);
        if (t[5] != 0.0) atomicAdd(&A.ctl->bflux[3], t[5] * dt * A.dx);
    }
}

}  // namespace fz
}  // namespace swe

namespace swe {
namespace fz {

struct Plan {
    CUtensorMap e[2], u[2], v[2], z;
    int nxs, nys, L, nitems, grid;
    bool ready;
};

template <class T, int CPT>
constexpr int cpt_smem() { return NWARP * Geo<T, CPT>::WARP_SMEM; }

template <class T, int CPT, int SX, int SY, bool KAPPA>
cudaError_t launch_t(swe_ctx* c, const Plan& pl, int s, long long k) {
    Args<T> A;
    const swe_params& p = c->p;
    A.G.nx = p.nx; A.G.ny = p.ny; A.G.pitch = c->pitch;
    A.G.g = (T)p.g; A.G.h_dry = (T)p.h_dry; A.G.kappa = (T)p.kappa;
    A.G.gn2 = (T)(p.g * p.manning_n * p.manning_n);
    A.G.inv_dx = (T)(1.0 / p.dx); A.G.inv_dy = (T)(1.0 / p.dy);
    for (int q = 0; q < 4; ++q) { A.G.bc[q] = p.bc[q]; A.G.qin[q] = (T)p.q_in[q]; }
    const int a = c->cur, b = 1 - c->cur;
    A.e1 = (T*)c->eta[b]; A.u1 = (T*)c->u[b]; A.v1 = (T*)c->v[b];
    A.n2 = (const T*)c->n2;
    A.ctl = c->ctl;
    A.dt_fixed = c->dt_fixed_cap > 0 ? c->dt_fixed : nullptr;
    A.dt_hist = c->dt_hist;
    A.dx = p.dx; A.dy = p.dy; A.g = p.g; A.cfl = p.cfl; A.dt_max = p.dt_max; A.area = p.dx * p.dy;
    A.s = s;
    A.slot_cur = (int)(k % 3); A.slot_next = (int)((k + 1) % 3); A.slot_zero = (int)((k + 2) % 3);
    A.nxs = pl.nxs; A.nys = pl.nys; A.L = pl.L; A.nitems = pl.nitems;
    auto kern = k_fused<T, CPT, SX, SY, KAPPA>;
    constexpr int SM = cpt_smem<T, CPT>();
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    kern<<<pl.grid, NWARP * 32, SM, c->stream>>>(pl.e[a], pl.u[a], pl.v[a], pl.z, A);
    return cudaGetLastError();
}

template <class T, int CPT, bool KAPPA>
cudaError_t launch_dir(swe_ctx* c, const Plan& pl, int s, long long k) {
    int sx, sy;
    step_dirs(c->p.dir_cycle, k, &sx, &sy);
    if (sx > 0 && sy > 0) return launch_t<T, CPT, 1, 1, KAPPA>(c, pl, s, k);
    if (sx > 0 && sy < 0) return launch_t<T, CPT, 1, -1, KAPPA>(c, pl, s, k);
    if (sx < 0 && sy > 0) return launch_t<T, CPT, -1, 1, KAPPA>(c, pl, s, k);
    return launch_t<T, CPT, -1, -1, KAPPA>(c, pl, s, k);
}

// Explicit instantiations live in swe_fused_<type><kappa>.cu (one per
// translation unit so that they compile in parallel).
cudaError_t launch_f32_k(swe_ctx* c, const Plan& pl, int s, long long k);
cudaError_t launch_f32_0(swe_ctx* c, const Plan& pl, int s, long long k);
cudaError_t launch_f64_k(swe_ctx* c, const Plan& pl, int s, long long k);
cudaError_t launch_f64_0(swe_ctx* c, const Plan& pl, int s, long long k);
int occupancy_f32(swe_ctx* c);
int occupancy_f64(swe_ctx* c);


}  // namespace fz
}  // namespace swe
