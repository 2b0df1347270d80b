// swe_fused.cuh -- the fused MacCormack step: all 16 sub-steps of one time
// step (Seitz et al. 2013, Sec. 1) in one sweep over the grid, one kernel
// launch per step.  Device code and launch templates; the explicit
// instantiations are spread over swe_fused_*.cu so they compile in parallel,
// the host set-up (tensor maps, work plan) is in swe_fused.cu.
#pragma once
//
// Decomposition.  A work item is a column strip of 32*CPT cells (one warp,
// CPT cells per lane) by a segment of L rows; the resident warps take items
// from a per-step atomic queue, costliest first, so that they finish
// together.  Along x the warp outputs 31 of its 32 lanes: the remaining lane
// (lane 0 when the predictor differences forward, lane 31 when backward) only
// computes the predicted values its neighbour's corrector needs.  Along y the
// warp marches row by row; the dependency radius of one step is one row for
// predictor and corrector and two rows for the dissipation switch, so the
// warp loads the segment plus two rows above and below.
//
// Data movement.  Level-n rows (eta, u, v, z) stream into a per-warp ring in
// shared memory with TMA (cp.async.bulk.tensor.2d, boxes two rows high, one
// mbarrier per pair of rows), two pairs ahead of use; a row stays in the ring
// while any of the four rows of the step's stencil window still needs it.  The two predicted rows, the y dissipation
// switch and the partial dissipation sum the corrector needs are carried in
// registers from one row to the next.  The level-n x neighbours outside a
// lane's cells are read from the ring (its columns extend two cells beyond
// the strip on both sides); the predicted ones come from adjacent lanes by
// shuffles (the lane that would need a halo there never outputs).  Boundary
// handling runs under warp-uniform branches: per row for the y sides, per
// item for the x sides.  The new level is stored with one vector store per
// field and lane (both cells).  Out-of-grid rows and columns read as zeros
// (TMA fill) and are replaced by the ghost cells of the boundary conditions.
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
constexpr int NWARP = 1;           // warps per CTA (one: item and row branches are then CTA-uniform)
constexpr int NSLOT = 8;           // ring rows per warp (a power of two): the pair in use, the
                                   // pair before it (the stencil's rows r-1, r-2) and two pairs in flight
constexpr int NPAIR = NSLOT / 2;   // ring slots: rows are loaded and waited for in pairs
constexpr unsigned long long WAIT_LIMIT = 4000000000ull;  // cycles (~2 s) before a wait gives up
constexpr int CPT_F32 = 2;         // cells per lane of the FP32 form (FP64: 2)
constexpr unsigned WET_SHARE = 50; // see sh_wet in k_fused

template <class T, int CPT>
struct Geo {
    static constexpr int W = 32 * CPT;                    // window columns
    static constexpr int OUT = W - CPT;                   // output columns per item
    static constexpr int BW = W + 8;                      // TMA box width (elements)
    static constexpr int ALIGN = 16 / (int)sizeof(T);     // TMA x alignment (elements)
    static constexpr int RSTRIDE = BW * (int)sizeof(T);   // bytes of one field row (one TMA box row)
    static constexpr int FSTRIDE = ((2 * RSTRIDE + 127) / 128) * 128;  // bytes per field of a slot (two rows)
    static constexpr int SLOT = 4 * FSTRIDE;              // bytes per ring slot (eta, u, v, z of two rows)
    static constexpr int WARP_SMEM = NPAIR * SLOT;
    // CTAs per SM the register budget must allow (FP32: 15 leaves the compiler
    // 136 registers; it uses at most 128, so 16 CTAs still fit)
    static constexpr int MINB = (sizeof(T) == 4 && CPT <= 2) ? 15 : 8;
};

// What one work item reads and writes: its scenario's constants and the
// new-level planes, with pointers at the scenario's row 0.
template <class T>
struct ItemIO {
    GridK<T> G;
    T* e1; T* u1; T* v1;
    const T* n2;
};

template <class T>
struct Args : ItemIO<T> {
    DevCtl* ctl;
    const double* dt_fixed;        // null: CFL step
    double* dt_hist;
    double dx, dy, g, cfl, dt_max, area;
    double rdx, rdy;               // 1/dx, 1/dy (divided on the host)
    int s;                         // step within the call
    int slot_cur, slot_next, slot_zero;
    int nxs, nys, L, nitems;
    int nfull;                     // row bands of the full L rows
    // per-item flags, written for level k+1 in step k: bit 0 = no wet output
    // cell, bit 1 = both ping-pong copies of the item agree (both for the
    // dry-item skip), bit 2 = some output cell not known to be wet (the
    // all-wet pass is not tried next to it); null: none
    const unsigned* fl_in;
    unsigned* fl_out;
    bool skip;                     // dry-item skip
    int inflow_mask;               // bit s: side s has an inflow boundary
};

// Work item of queue position q.  Items are handed out through an atomic
// counter in order of decreasing cost: the strips at the x boundary (their
// rows run the boundary code), then the interior strips, then the short last
// row band.
__device__ __forceinline__ void item_of(int q, int nxs, int nfull, int& kx, int& ky) {
    const int ne = nxs >= 2 ? 2 : 1;
    const int n_edge = ne * nfull, n_full = nxs * nfull;
    if (q < n_edge) {
        ky = q / ne;
        kx = (q - ky * ne) == 0 ? 0 : nxs - 1;
    } else if (q < n_full) {
        const int r = q - n_edge, ni = nxs - ne;
        ky = r / ni;
        kx = 1 + (r - ky * ni);
    } else {
        ky = nfull;
        kx = q - n_full;
    }
}

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

// The CPT cells of a lane in one row (swe_cell.cuh: packed for two FP32 cells).
template <class T, int CPT>
using Vec = vecn<T, CPT>;

template <class T, int CPT>
__device__ __forceinline__ void ld_vec(const T* p, Vec<T, CPT>& o) {
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
__device__ __forceinline__ void st_vec(T* p, const Vec<T, CPT>& o) {
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
    Vec<T, CPT> e, u, v, z;
};

template <class T, int CPT>
struct PR {  // a predicted row as the corrector needs it: eta*, u*, v*, bed, h* v*
    Vec<T, CPT> e, u, v, z, qy;
};

// State carried from one row to the next, double-buffered by row parity so
// that unrolling the row loop by two needs no register copies: the values of
// the row just produced go to index PAR, the previous row's are at 1 - PAR.
template <class T, int CPT>
struct Carry {
    PR<T, CPT> P[2];         // predicted rows
    Vec<T, CPT> NY[2];       // y dissipation switch of a level-n row
    // S15 dissipation of a row (eta, u, v) without its north face flux: east
    // minus west, minus south (the south face is the previous row's north face)
    Vec<T, CPT> DX[2][3];
};

// Totals that change once per item (a lane's totals over the warp's items)
// or only in boundary rows (an item's side tallies) sit in shared memory,
// one slot per lane at stride 32, so that they hold no registers through the
// row loop.  They are kept in the state's real type and reduced over the
// warp in FP64 once, at the end of the launch: GB300's FP64 pipe takes tens
// of cycles per warp instruction, and a reduction per item kept it busy a
// fifth of the time.
template <class T>
struct Acc {  // p[m * 32], m = 0 smax, 1 clamp, 2..5 sides W, E, S, N
    T* p;
    bool bad;
};

template <class T>
struct ItemAcc {  // per-item totals in the state's real type
    T clamp, smax;
    bool bad;
    T* side;      // side[q * 32]: boundary inflow through side q = W, E, S, N
};

template <class T, int CPT>
struct ItemCtx {
    unsigned char* ring;
    uint64_t* bars;
    int lane, xw, xb, col, x0c, y0, y1, nr;
    int yoff;                    // tensor row of the scenario's row 0
    bool out_lane, edge;
    bool st_lane;                // the lane outputs and its first cell is in the grid
    int plo, phi;                // rows of the item whose predicted clamps this item tallies
    unsigned g0;
    unsigned* chk;               // checked builds: set when a check fails (shared memory)
};

// Checked builds (SWE_CHECKED): a failed index or alignment check of the row
// step sets *I.chk and the access is made safe instead (a clamped column, the
// ring's first row, a store left out, an aligned TMA coordinate); the kernel
// reports SWE_FLAG_CHECK.  Nothing traps.  Other builds compile the checks out.
#ifdef SWE_CHECKED
#define SWE_CHK(I, cond) ((cond) ? true : (*(I).chk = 1u, false))
#else
#define SWE_CHK(I, cond) true
#endif

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

// Values one column to the right (D > 0) or left (D < 0) of the lane's
// cells: the lane's next cell; for the outer one, `halo` when `use_halo`
// (the caller read it from the ring), else the adjacent lane's end cell by
// a shuffle.
template <int D, class T, int CPT>
__device__ __forceinline__ Vec<T, CPT> shift(const Vec<T, CPT>& a, T halo, bool use_halo) {
    Vec<T, CPT> o;
    if (D > 0) {
#pragma unroll
        for (int c = 0; c + 1 < CPT; ++c) o[c] = a[c + 1];
        const T t = shdn(a[0]);
        o[CPT - 1] = use_halo ? halo : t;
    } else {
#pragma unroll
        for (int c = 1; c < CPT; ++c) o[c] = a[c - 1];
        const T t = shup(a[CPT - 1]);
        o[0] = use_halo ? halo : t;
    }
    return o;
}

template <class T, int CPT>
__device__ __forceinline__ Cell<Vec<T, CPT>> cells(const Row<T, CPT>& r) {
    Cell<Vec<T, CPT>> c;
    c.e = r.e; c.u = r.u; c.v = r.v; c.z = r.z;
    return c;
}

// The ring.  Ring row g (counted over the warp's items, even at an item's
// start) sits in slot (g / 2) % NPAIR, at row g % 2 of each field's two; a
// slot's two rows are one TMA box per field and complete one barrier.

// Row base of ring row g (field f at + f * FSTRIDE); ODD = g % 2.
template <class T, int CPT, int ODD>
__device__ __forceinline__ const unsigned char* ring_row(const ItemCtx<T, CPT>& I, unsigned g) {
    return I.ring + ((g >> 1) & (NPAIR - 1)) * Geo<T, CPT>::SLOT + ODD * Geo<T, CPT>::RSTRIDE;
}
template <class T, int CPT>
__device__ __forceinline__ const unsigned char* ring_row(const ItemCtx<T, CPT>& I, unsigned g) {
    return I.ring + ((g >> 1) & (NPAIR - 1)) * Geo<T, CPT>::SLOT + (g & 1u) * Geo<T, CPT>::RSTRIDE;
}

// Predicated issue of the item's ring rows 2q and 2q + 1: lane 0 arms the
// slot's barrier and starts the four two-row tile loads, if `want` (no branch).
template <class T, int CPT>
__device__ __forceinline__ void issue_pair(const ItemCtx<T, CPT>& I, int q, const CUtensorMap* tme,
                                           const CUtensorMap* tmu, const CUtensorMap* tmv, const CUtensorMap* tmz,
                                           bool want = true) {
    using Gm = Geo<T, CPT>;
    const unsigned sl = ((I.g0 >> 1) + (unsigned)q) & (NPAIR - 1);
    const unsigned bar = saddr(I.bars + sl);
    const unsigned dst = saddr(I.ring + sl * Gm::SLOT);
    const unsigned pred = (I.lane == 0 && want) ? 1u : 0u;
    const int y = I.yoff + I.y0 - 2 + 2 * q;
    int xb = I.xb;
    if (!SWE_CHK(I, (xb * (int)sizeof(T)) % 16 == 0)) xb &= ~(Gm::ALIGN - 1);  // TMA x: 16-byte multiple
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %0, 0;\n @p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%1], %2;\n}"
                 ::"r"(pred), "r"(bar), "r"(4u * 2u * (unsigned)Gm::RSTRIDE) : "memory");
    const CUtensorMap* maps[4] = {tme, tmu, tmv, tmz};
#pragma unroll
    for (int f = 0; f < 4; ++f)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %0, 0;\n"
            " @p cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%1], [%2, {%3, %4}], [%5];\n}"
            ::"r"(pred), "r"(dst + f * Gm::FSTRIDE), "l"(maps[f]), "r"(xb), "r"(y), "r"(bar) : "memory");
}

// Barrier and phase parity of the item's ring rows 2q and 2q + 1.
template <class T, int CPT>
__device__ __forceinline__ uint64_t* pair_bar(const ItemCtx<T, CPT>& I, int q, unsigned& par) {
    const unsigned p = (I.g0 >> 1) + (unsigned)q;
    par = (p / NPAIR) & 1u;
    return I.bars + (p & (NPAIR - 1));
}

// Waits for the item's ring rows 2q and 2q + 1; false (for the whole warp)
// when the wait gave up.
template <class T, int CPT>
__device__ __forceinline__ bool wait_pair(const ItemCtx<T, CPT>& I, int q) {
    unsigned par;
    uint64_t* bar = pair_bar(I, q, par);
    if (__all_sync(FULL, mbar_try(bar, par))) return true;
    const unsigned long long t0 = clock64();
    while (!__all_sync(FULL, mbar_try(bar, par)))
        if (clock64() - t0 > WAIT_LIMIT) return false;
    return true;
}

template <class T, int CPT>
__device__ __forceinline__ const unsigned char* slot_clamped(const ItemCtx<T, CPT>& I, int row, int ny) {
    const int src = row < 0 ? 0 : (row >= ny ? ny - 1 : row);
    return ring_row(I, I.g0 + (unsigned)(src - (I.y0 - 2)));
}

// One ring row r (ring index k) of an item: y switch of row r-1, the
// predictor and x dissipation of row r-1, and the corrector, average,
// dissipation and fix of row C = r-2 (S1-S16).  PAR is k's parity.  The
// arithmetic works on the lane's CPT cells at once (Vec); boundary cases
// patch single cells.  NF (lean rows): 1 when a per-cell Manning field is
// set, so that a lean row has no branch on it.  WET (lean rows; `wet` in the
// general ones): the item runs on the assumption that every cell it reads or
// produces is wet; a lean row then leaves out every wet/dry select (the WET
// forms of swe_cell.cuh), and every row checks the assumption into `ok` (the
// level-n row entering the window, the ring's halo cells a lean row reads,
// the predicted and the new cells), so that the caller recomputes the item
// without it where it fails.  Without it, `ok` collects whether every new
// cell the item outputs is wet (the hint for the next step).
// The checks of the all-wet assumption keep the running minimum of the
// depths they cover; NaN propagates (min.NaN), so "every depth > h_dry" is
// the minimum > h_dry, NaN included, in one instruction per depth.
__device__ __forceinline__ float nanmin(float a, float b) {
    float d;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ double nanmin(double a, double b) { return (a != a) ? a : ((b != b) ? b : fmin(a, b)); }
template <class R, class T>
__device__ __forceinline__ void chk_min(T& mn, const R& v) {
#pragma unroll
    for (int i = 0; i < (int)(sizeof(R) / sizeof(T)); ++i) mn = nanmin(mn, v[i]);
}

template <class M>
__device__ __forceinline__ bool all_of(const M& m) {
    bool r = true;
#pragma unroll
    for (int i = 0; i < (int)(sizeof(m.c) / sizeof(m.c[0])); ++i) r = r && m.c[i];
    return r;
}

template <class T, int CPT, int SX, int SY, bool KAPPA, int PAR, bool GEN, int NF, bool WET, bool PRED_ONLY = false>
__device__ __forceinline__ void row_step(const ItemIO<T>& A, const StepK<T>& S, const ItemCtx<T, CPT>& I, int k,
                                         Carry<T, CPT>& Cy, ItemAcc<T>& ia, const CUtensorMap* tme,
                                         const CUtensorMap* tmu, const CUtensorMap* tmv, const CUtensorMap* tmz,
                                         bool& timed_out, T& mn, bool wet) {
    constexpr bool WA = WET && !GEN;  // wet arithmetic: the lean row without selects
    const bool ck = GEN ? wet : WET;  // check the all-wet assumption
    using V = Vec<T, CPT>;
    constexpr int CX = -SX, CY = -SY;
    constexpr int Q = PAR, O = 1 - PAR;  // this row's buffers, the previous row's
    const GridK<T>& G = A.G;
    const int ny = G.ny, nx = G.nx;
    const T hd = G.h_dry;
    const V hdv(hd);
    const int lane = I.lane;
    const int r = I.y0 - 2 + k;

    if (GEN && k < 2) return;  // the item's first pair of ring rows only loads

    // -------- level-n rows r, r-1, r-2 (ghost cells outside [0, ny)).  The
    // lean instantiation (GEN false) serves interior rows of items away from
    // the x boundary, where every boundary test below is false.
    const bool brow = GEN && ((r - 2 <= 0) || (r >= ny));
    const bool edge = GEN && I.edge;
    const bool nfield = GEN ? A.n2 != nullptr : NF != 0;
    const unsigned g = I.g0 + (unsigned)k;  // g % 2 = PAR
    const unsigned char* s0 = ring_row<T, CPT, PAR>(I, g);
    const unsigned char* s1 = ring_row<T, CPT, 1 - PAR>(I, g - 1u);
    const unsigned char* s2 = ring_row<T, CPT, PAR>(I, g - 2u);
    if (brow) {
        s0 = slot_clamped(I, r, ny);
        s1 = slot_clamped(I, r - 1, ny);
        s2 = slot_clamped(I, r - 2, ny);
    }
    int col = I.col;
#ifdef SWE_CHECKED
    {   // the rows in the ring, their columns col - 2 .. col + CPT + 1 in the row, vector-aligned
        using Gm = Geo<T, CPT>;
        const unsigned char* sp[3] = {s0, s1, s2};
        bool in = true;
        for (int q = 0; q < 3; ++q) {  // a slot's first or second row
            const long off = (long)(sp[q] - I.ring), r = off % Gm::SLOT;
            in = in && off >= 0 && off + 3 * Gm::FSTRIDE + Gm::RSTRIDE <= Gm::WARP_SMEM &&
                 (r == 0 || r == Gm::RSTRIDE);
        }
        if (!SWE_CHK(I, in)) s0 = s1 = s2 = I.ring;
        if (!SWE_CHK(I, col >= 2 && col + CPT + 2 <= Gm::BW && col % CPT == 0)) col = 2 * CPT;
    }
#endif
    Row<T, CPT> R0, R1, R2;
    ld_row<T, CPT>(s0, col, R0);
    ld_row<T, CPT>(s1, col, R1);
    ld_row<T, CPT>(s2, col, R2);
    if (brow) {
        if (r < 0) ghost_row(R0, SIDE_S, G); else if (r >= ny) ghost_row(R0, SIDE_N, G);
        if (r - 1 < 0) ghost_row(R1, SIDE_S, G); else if (r - 1 >= ny) ghost_row(R1, SIDE_N, G);
        if (r - 2 < 0) ghost_row(R2, SIDE_S, G); else if (r - 2 >= ny) ghost_row(R2, SIDE_N, G);
    }
    const V h0 = R0.e - R0.z, h1 = R1.e - R1.z, h2 = R2.e - R2.z;
    if (ck) chk_min(mn, h0);  // each level-n row of the window enters once as row r

    // -------- y switch of row r-1, y dissipation flux through the face between
    // rows r-2 and r-1 (north face of the corrector's row, south face of the predictor's)
    V FYQ[3];
    if (KAPPA) {
        const bool face_in = !brow || (r - 2 >= 0 && r - 1 < ny);
        const V nyn = nu_switch(h2, h1, h0);
        V eps;
        if (WA) eps = face_eps_wet(Cy.NY[O], nyn);
        else eps = face_eps(h2 > hdv, h1 > hdv, Cy.NY[O], nyn);
        if (!face_in) eps = V(T(0));
        FYQ[0] = dflux(eps, R1.e, R2.e);
        FYQ[1] = dflux(eps, R1.u, R2.u);
        FYQ[2] = dflux(eps, R1.v, R2.v);
        Cy.NY[Q] = nyn;
    }

    // -------- predictor and x dissipation of row p = r-1
    auto predictor = [&]() {
        const int p = r - 1;
        const Row<T, CPT>& c = R1;
        const Row<T, CPT>& yn = SY > 0 ? R0 : R2;
        const V hyn = SY > 0 ? h0 : h2;
        // x neighbours on the predictor's side: the lane's next cells, the outer one from the ring
        const int hcol = SX > 0 ? col + CPT : col - 1;
        Row<T, CPT> xn;
        xn.e = shift<SX, T, CPT>(c.e, ld1<T, CPT>(s1, 0, hcol), true);
        xn.u = shift<SX, T, CPT>(c.u, ld1<T, CPT>(s1, 1, hcol), true);
        xn.v = shift<SX, T, CPT>(c.v, ld1<T, CPT>(s1, 2, hcol), true);
        xn.z = shift<SX, T, CPT>(c.z, ld1<T, CPT>(s1, 3, hcol), true);
        if (brow && (r - 1 < 0 || r - 1 >= ny)) {  // the cell read from the ring in a ghost row
            constexpr int j = SX > 0 ? CPT - 1 : 0;
            Cell<T> q; q.e = xn.e[j]; q.u = xn.u[j]; q.v = xn.v[j]; q.z = xn.z[j];
            q = ghost(q, r - 1 < 0 ? SIDE_S : SIDE_N, G);
            xn.e[j] = q.e; xn.u[j] = q.u; xn.v[j] = q.v; xn.z[j] = q.z;
        }
        const V qx = h1 * c.u, qy = h1 * c.v;
        const V hxn = xn.e - xn.z;
        const V qxn = hxn * xn.u;
        const V qyn = hyn * yn.v;
        if (WA) mn = nanmin(mn, hxn[SX > 0 ? CPT - 1 : 0]);  // the ring's halo cell
        V fe, fw, fn, fs;
        if (SX > 0) { fe = qxn; fw = qx; } else { fe = qx; fw = qxn; }
        if (SY > 0) { fn = qyn; fs = qy; } else { fn = qy; fs = qyn; }
        if (edge) {
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const int x = I.x0c + j;
                if (x == 0) fw[j] = face_bnd(SIDE_W, qx[j], G);
                if (x == nx - 1) fe[j] = face_bnd(SIDE_E, qx[j], G);
                if (SX > 0 ? x == nx - 1 : x == 0) {
                    Cell<T> q; q.e = c.e[j]; q.u = c.u[j]; q.v = c.v[j]; q.z = c.z[j];
                    q = ghost(q, SX > 0 ? SIDE_E : SIDE_W, G);
                    xn.e[j] = q.e; xn.u[j] = q.u; xn.v[j] = q.v; xn.z[j] = q.z;
                }
            }
        }
        if (brow) {
            if (p == 0) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) fs[j] = face_bnd(SIDE_S, qy[j], G);
            }
            if (p == ny - 1) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) fn[j] = face_bnd(SIDE_N, qy[j], G);
            }
        }
        V gn2v;
        if (nfield) {
            const int xc = I.x0c < 0 ? 0 : (I.x0c > G.pitch - CPT ? G.pitch - CPT : I.x0c);
            const int pr = p < 0 ? 0 : (p >= ny ? ny - 1 : p);
            ld_vec<T, CPT>(A.n2 + (size_t)pr * G.pitch + xc, gn2v);
        } else {
            gn2v = V(G.gn2);
        }
        PR<T, CPT>& P = Cy.P[Q];
        V eo, uo, vo;
        stage<SX, SY, 0, WA>(cells(c), cells(xn), cells(yn), fe, fw, fn, fs, c.e, c.u, c.v, gn2v, S, hd, eo, uo, vo);
        if (!WA) {
            V ad = wetdry_fix(eo, uo, vo, c.z, hd);
            if (edge) {
#pragma unroll
                for (int j = 0; j < CPT; ++j)
                    if (I.x0c + j >= nx) ad[j] = T(0);
            }
            T added = T(0);
#pragma unroll
            for (int j = 0; j < CPT; ++j) added += ad[j];
            // a predicted clamp counts once per cell: in the item and lane that output it
            if (I.st_lane && p >= I.plo && p < I.phi)
                ia.clamp = fma_(T(0.5), added, ia.clamp);
        }
        P.e = eo; P.u = uo; P.v = vo; P.z = c.z;
        const V hp = eo - c.z;
        P.qy = hp * vo;
        if (ck && (!GEN || (p >= 0 && p < ny))) chk_min(mn, hp);  // every lane's predicted cells feed a corrector
        if (KAPPA) {
            // x dissipation of row r-1; the outer neighbour on the other side
            // from the ring as well
            Row<T, CPT> xo;
            const int ocol = SX > 0 ? col - 1 : col + CPT;
            xo.e = shift<-SX, T, CPT>(c.e, ld1<T, CPT>(s1, 0, ocol), true);
            xo.u = shift<-SX, T, CPT>(c.u, ld1<T, CPT>(s1, 1, ocol), true);
            xo.v = shift<-SX, T, CPT>(c.v, ld1<T, CPT>(s1, 2, ocol), true);
            xo.z = shift<-SX, T, CPT>(c.z, ld1<T, CPT>(s1, 3, ocol), true);
            const Row<T, CPT>& L = SX > 0 ? xo : xn;  // left neighbours
            const Row<T, CPT>& Rr = SX > 0 ? xn : xo; // right neighbours
            V hl = L.e - L.z, hr = Rr.e - Rr.z;
            if (WA) mn = nanmin(mn, SX > 0 ? hl[0] : hr[CPT - 1]);  // the ring's other halo cell
            if (edge) {  // ghost depth at columns -1 and nx is the adjacent interior depth
#pragma unroll
                for (int j = 0; j < CPT; ++j) {
                    if (I.x0c + j == 0) hl[j] = h1[j];
                    if (I.x0c + j == nx - 1) hr[j] = h1[j];
                }
            }
            const V nuc = nu_switch(hl, h1, hr);
            // switch one column outside the lane: on the predictor's side every lane
            // computes it from the ring (at the grid edge with the ghost depth
            // beyond it, as the adjacent lane would); on the other side the
            // adjacent lane's (the edge lane there never outputs)
            T nu_lo, nu_hi;
            if (SX > 0) {
                T h2x = ld1<T, CPT>(s1, 0, col + CPT + 1) - ld1<T, CPT>(s1, 3, col + CPT + 1);
                if (edge && I.x0c + CPT == nx - 1) h2x = hr[CPT - 1];
                nu_hi = nu_switch(h1[CPT - 1], hr[CPT - 1], h2x);
                nu_lo = shup(nuc[CPT - 1]);
            } else {
                T h2x = ld1<T, CPT>(s1, 0, col - 2) - ld1<T, CPT>(s1, 3, col - 2);
                if (edge && I.x0c - 1 == 0) h2x = hl[0];
                nu_lo = nu_switch(h2x, hl[0], h1[0]);
                nu_hi = shdn(nuc[0]);
            }
            // east face of every cell
            V nur;
#pragma unroll
            for (int j = 0; j + 1 < CPT; ++j) nur[j] = nuc[j + 1];
            nur[CPT - 1] = nu_hi;
            V eps;
            if (WA) eps = face_eps_wet(nuc, nur);
            else eps = face_eps(h1 > hdv, hr > hdv, nuc, nur);
            if (edge) {
#pragma unroll
                for (int j = 0; j < CPT; ++j)
                    if (I.x0c + j + 1 >= nx) eps[j] = T(0);
            }
            V fr[3] = {dflux(eps, Rr.e, c.e), dflux(eps, Rr.u, c.u), dflux(eps, Rr.v, c.v)};
            // west face of the first cell; the others' west faces are their left neighbours' east faces
            T e0;
            if (WA) e0 = face_eps_wet(nu_lo, nuc[0]);
            else e0 = face_eps(hl[0] > hd, h1[0] > hd, nu_lo, nuc[0]);
            if (edge && I.x0c - 1 < 0) e0 = T(0);
            T fl0[3] = {dflux(e0, c.e[0], L.e[0]), dflux(e0, c.u[0], L.u[0]), dflux(e0, c.v[0], L.v[0])};
            if (edge) {
                // a face on the x boundary carries +0, whatever lies beyond the grid
                // (the one-thread-per-cell kernel's difference of a cell with its
                // clamped self)
#pragma unroll
                for (int f = 0; f < 3; ++f) {
#pragma unroll
                    for (int j = 0; j < CPT; ++j)
                        if (I.x0c + j + 1 >= nx) fr[f][j] = T(0);
                    if (I.x0c - 1 < 0) fl0[f] = T(0);
                }
            }
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                V west;
                west[0] = fl0[f];
#pragma unroll
                for (int j = 1; j < CPT; ++j) west[j] = fr[f][j - 1];
                Cy.DX[Q][f] = (fr[f] - west) - FYQ[f];
            }
        }
    };

    // -------- corrector, average, dissipation and fix of row C = r-2
    auto corrector = [&]() {
        const int C = r - 2;
        const PR<T, CPT>& pc = Cy.P[O];       // predicted row C
        PR<T, CPT> ys = Cy.P[Q];              // row C-1 (forward predictor) or C+1 (backward)
        Row<T, CPT> cs;
        cs.e = pc.e; cs.u = pc.u; cs.v = pc.v; cs.z = pc.z;
        if (brow && (CY < 0 ? C == 0 : C == ny - 1)) {
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                Cell<T> q; q.e = cs.e[j]; q.u = cs.u[j]; q.v = cs.v[j]; q.z = cs.z[j];
                q = ghost(q, CY < 0 ? SIDE_S : SIDE_N, G);
                ys.e[j] = q.e; ys.u[j] = q.u; ys.v[j] = q.v; ys.z[j] = q.z;
                ys.qy[j] = (q.e - q.z) * q.v;
            }
        }
        Row<T, CPT> xs;  // the lane that would need a halo on this side never outputs
        xs.e = shift<CX, T, CPT>(cs.e, T(0), false);
        xs.u = shift<CX, T, CPT>(cs.u, T(0), false);
        xs.v = shift<CX, T, CPT>(cs.v, T(0), false);
        xs.z = shift<CX, T, CPT>(cs.z, T(0), false);
        const V qx = (cs.e - cs.z) * cs.u;
        const V qxn = (xs.e - xs.z) * xs.u;
        V fe, fw, fn, fs;
        if (CX > 0) { fe = qxn; fw = qx; } else { fe = qx; fw = qxn; }
        if (CY > 0) { fn = ys.qy; fs = pc.qy; } else { fn = pc.qy; fs = ys.qy; }
        if (edge) {
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const int x = I.x0c + j;
                if (x == 0) fw[j] = face_bnd(SIDE_W, qx[j], G);
                if (x == nx - 1) fe[j] = face_bnd(SIDE_E, qx[j], G);
                if (CX > 0 ? x == nx - 1 : x == 0) {
                    Cell<T> q; q.e = cs.e[j]; q.u = cs.u[j]; q.v = cs.v[j]; q.z = cs.z[j];
                    q = ghost(q, CX > 0 ? SIDE_E : SIDE_W, G);
                    xs.e[j] = q.e; xs.u[j] = q.u; xs.v[j] = q.v; xs.z[j] = q.z;
                }
            }
        }
        if (brow) {
            if (C == 0) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) fs[j] = face_bnd(SIDE_S, pc.qy[j], G);
            }
            if (C == ny - 1) {
#pragma unroll
                for (int j = 0; j < CPT; ++j) fn[j] = face_bnd(SIDE_N, pc.qy[j], G);
            }
        }
        V gn2v;
        if (nfield) {
            const int xc = I.x0c < 0 ? 0 : (I.x0c > G.pitch - CPT ? G.pitch - CPT : I.x0c);
            const int cr = SWE_CHK(I, C >= 0 && C < ny) ? C : 0;
            ld_vec<T, CPT>(A.n2 + (size_t)cr * G.pitch + xc, gn2v);
        } else {
            gn2v = V(G.gn2);
        }
        Cell<V> cy;
        cy.e = ys.e; cy.u = ys.u; cy.v = ys.v; cy.z = ys.z;
        V eo, uo, vo;
        stage<CX, CY, 0, WA>(cells(cs), cells(xs), cy, fe, fw, fn, fs, R2.e, R2.u, R2.v, gn2v, S, hd, eo, uo, vo);
        const V half(T(0.5));
        V oe = half * (cs.e + eo);
        V ou = half * (cs.u + uo);
        V ov = half * (cs.v + vo);
        if (KAPPA) {
            // east minus west minus south face flux, plus the north one
            const V kap(G.kappa);
            oe = fma_(kap, Cy.DX[O][0] + FYQ[0], oe);
            ou = fma_(kap, Cy.DX[O][1] + FYQ[1], ou);
            ov = fma_(kap, Cy.DX[O][2] + FYQ[2], ov);
        }
        // a lean row of an item's first pair (k < 4) runs the corrector on rows
        // of the item above: nothing of it is stored or tallied
        bool st = I.st_lane && (GEN || k >= 4);
#ifdef SWE_CHECKED
        if (st && !SWE_CHK(I, C >= 0 && C < ny && I.x0c >= 0 && I.x0c + CPT <= G.pitch && I.x0c % CPT == 0)) st = false;
#endif
        // the new cells the item outputs are wet (the fix below keeps a cell
        // whose depth is above h_dry as it is)
        const V hn = oe - cs.z;
        T wn = T(INFINITY);
#pragma unroll
        for (int j = 0; j < CPT; ++j) wn = nanmin(wn, (edge && I.x0c + j >= nx) ? T(INFINITY) : hn[j]);
        mn = st ? nanmin(mn, wn) : mn;
        V ad;
        if (WA) ad = V(T(0));
        else ad = wetdry_fix(oe, ou, ov, cs.z, hd);
        V spj = cfl_speed<WA>(oe, ou, ov, cs.z, G);
        const V sum = oe + ou + ov;
        V dsum = sum - sum;  // NaN for a non-finite cell
        if (edge) {  // a lane's cells beyond the grid are computed, not output
#pragma unroll
            for (int j = 0; j < CPT; ++j)
                if (I.x0c + j >= nx) { ad[j] = T(0); spj[j] = T(0); dsum[j] = T(0); }
        }
        // the row's speed maximum (speeds are >= 0 and never NaN in a finite
        // state; a NaN speed is left out, as the max of fmax does) and the sum of
        // the cells' NaN probes (0 unless one is NaN)
        T sp = T(0), dprobe = T(0);
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            sp = tmax(sp, spj[j]);
            dprobe += dsum[j];
        }
        // halo rows of a strip are stored, not tallied (the all-wet pass runs
        // only on items of own rows)
        const bool own = WA ? st : (st && C >= G.own_lo && C < G.own_hi);
        if (!WA) {
            T added = T(0);
#pragma unroll
            for (int j = 0; j < CPT; ++j) added += ad[j];
            ia.clamp += own ? added : T(0);
        }
        ia.smax = tmax(ia.smax, own ? sp : T(0));
        ia.bad = ia.bad || (own && !(dprobe == T(0)));
        if constexpr (sizeof(T) == 4 && CPT == 2) {  // predicated stores: no branch in the row
            const size_t o = (size_t)C * G.pitch + I.x0c;
            asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %0, 0;\n"
                         " @p st.global.v2.f32 [%1], {%2, %3};\n @p st.global.v2.f32 [%4], {%5, %6};\n"
                         " @p st.global.v2.f32 [%7], {%8, %9};\n}"
                         ::"r"((unsigned)st), "l"(A.e1 + o), "f"(oe[0]), "f"(oe[1]), "l"(A.u1 + o), "f"(ou[0]), "f"(ou[1]),
                           "l"(A.v1 + o), "f"(ov[0]), "f"(ov[1]) : "memory");
        } else if (st) {
            const size_t o = (size_t)C * G.pitch + I.x0c;
            st_vec<T, CPT>(A.e1 + o, oe);
            st_vec<T, CPT>(A.u1 + o, ou);
            st_vec<T, CPT>(A.v1 + o, ov);
        }
        if (edge) {
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const T qxn0 = h2[j] * R2.u[j];
                const T w = T(0.5) * (face_bnd(SIDE_W, qxn0, G) + face_bnd(SIDE_W, qx[j], G));
                const T e = T(0.5) * (face_bnd(SIDE_E, qxn0, G) + face_bnd(SIDE_E, qx[j], G));
                ia.side[0] += (own && I.x0c + j == 0) ? w : T(0);
                ia.side[32] -= (own && I.x0c + j == nx - 1) ? e : T(0);
            }
        }
        if (brow && (C == 0 || C == ny - 1)) {
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const bool in = own && !(edge && I.x0c + j >= nx);
                const T qyn = h2[j] * R2.v[j];
                const T sv = T(0.5) * (face_bnd(SIDE_S, qyn, G) + face_bnd(SIDE_S, pc.qy[j], G));
                const T nv = T(0.5) * (face_bnd(SIDE_N, qyn, G) + face_bnd(SIDE_N, pc.qy[j], G));
                ia.side[64] += (in && C == 0) ? sv : T(0);
                ia.side[96] -= (in && C == ny - 1) ? nv : T(0);
            }
        }
    };

    if (SY > 0) {  // the corrector reads P(C-1) from the buffer the predictor overwrites
        if (!PRED_ONLY && (!GEN || k >= 4)) corrector();
        predictor();
    } else {       // the corrector reads P(C+1), which the predictor produces
        predictor();
        if (!PRED_ONLY && (!GEN || k >= 4)) corrector();
    }
    // the ring slot refilled next was read two rows ago: lean rows come in pairs
    // and sync after the second
    if (GEN || PAR == 1) __syncwarp();
}

// The rows of one item.  wet (only with TRY_WET): on the assumption that
// every cell is wet (row_step).  Returns 2 (for the whole warp) when that
// assumption failed, as soon as a pair of rows or the item shows it, with the
// pass's loads drained; else 0 when every new cell the item outputs is wet,
// 1 when not.  I.g0 has moved past the pass's loads either way.
template <class T, int CPT, int SX, int SY, bool KAPPA, bool TRY_WET>
__device__ __forceinline__ int run_rows(const ItemIO<T>& A, const StepK<T>& S, ItemCtx<T, CPT>& I,
                                        Carry<T, CPT>& Cy, ItemAcc<T>& ia, const CUtensorMap* tme,
                                        const CUtensorMap* tmu, const CUtensorMap* tmv, const CUtensorMap* tmz,
                                        bool& timed_out, bool wet) {
    wet = TRY_WET && wet;
    fence_async_smem();  // the previous pass's rows were read through the generic proxy
    const int nr = I.nr;
    const int np = (nr + 1) / 2;  // pairs of ring rows (an odd count loads one row more)
    issue_pair<T, CPT>(I, 0, tme, tmu, tmv, tmz);
    issue_pair<T, CPT>(I, 1, tme, tmu, tmv, tmz, np > 1);
    Cy.NY[0] = Cy.NY[1] = Vec<T, CPT>(T(0));
#pragma unroll
    for (int f = 0; f < 3; ++f) Cy.DX[0][f] = Cy.DX[1][f] = Vec<T, CPT>(T(0));
    ia.clamp = ia.smax = T(0);
    ia.bad = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) ia.side[q * 32] = T(0);
    T mn = T(INFINITY);  // the minimum of the depths checked (ok: mn > h_dry)
    bool held = true;
    const T hdc = A.G.h_dry;
    int drain_from = 0, issued = 0;  // after a failed wait or check: the pairs to drain, [drain_from, issued)
    int k = 0;
    const int ny = A.G.ny;
    // Lean rows: pairs from the item's second on (the first, k = 0 and 1, only
    // loads) whose rows r = y0 - 2 + k and r + 1 keep two rows from the y
    // sides (r - 2 > 0, r + 1 < ny), in items away from the x sides; with the
    // all-wet pass compiled in, only for an item that takes it (the others, a
    // few per launch, run the general rows, so that a launch keeps one lean
    // loop hot).
    const int klo = max(2, 5 - I.y0);
    const int khi = (I.edge || (TRY_WET && !wet)) ? 0 : min(nr - 1, ny - I.y0 + 1);
#pragma unroll 1
    for (; k < nr; k += 2) {
        const int q = k >> 1;
        // the slot refilled held the pair before last, read up to the previous pair
        fence_async_smem();
        issue_pair<T, CPT>(I, q + 2, tme, tmu, tmv, tmz, q + 2 < np);
        if (!wait_pair<T, CPT>(I, q)) { timed_out = true; drain_from = q; issued = min(np, q + 3); break; }
        if (k >= klo && k < khi) {
#define SWE_PAIR(NF, W, PO)                                                                                       \
    row_step<T, CPT, SX, SY, KAPPA, 0, false, NF, W, PO>(A, S, I, k, Cy, ia, tme, tmu, tmv, tmz, timed_out, mn, wet); \
    row_step<T, CPT, SX, SY, KAPPA, 1, false, NF, W, PO>(A, S, I, k + 1, Cy, ia, tme, tmu, tmv, tmz, timed_out, mn, wet)
            // the item's first lean pair (k = 2, 3) has no corrector rows yet
            if (A.n2 != nullptr) {
                if (k < 4) { SWE_PAIR(1, TRY_WET, true); } else { SWE_PAIR(1, TRY_WET, false); }
            } else {
                if (k < 4) { SWE_PAIR(0, TRY_WET, true); } else { SWE_PAIR(0, TRY_WET, false); }
            }
#undef SWE_PAIR
        } else {
            row_step<T, CPT, SX, SY, KAPPA, 0, true, 0, false>(A, S, I, k, Cy, ia, tme, tmu, tmv, tmz, timed_out, mn, wet);
            if (k + 1 < nr)  // the last row of an odd count runs alone
                row_step<T, CPT, SX, SY, KAPPA, 1, true, 0, false>(A, S, I, k + 1, Cy, ia, tme, tmu, tmv, tmz, timed_out,
                                                                   mn, wet);
        }
        if (TRY_WET && wet && !__all_sync(FULL, mn > hdc)) {
            held = false; drain_from = q + 1; issued = min(np, q + 3); break;
        }
    }
    const bool all_ok = held && __all_sync(FULL, mn > hdc);
    if (TRY_WET && wet && held && !timed_out && !all_ok) { held = false; drain_from = np; issued = np; }
    if (timed_out || !held) {
        // drain this pass's loads still in flight (bounded) before the ring is reused or left
        for (int q = drain_from; q < issued; ++q) {
            unsigned par;
            uint64_t* bar = pair_bar(I, q, par);
            unsigned long long t0 = clock64();
            while (!mbar_try(bar, par))
                if (clock64() - t0 > WAIT_LIMIT / 8) break;
        }
        I.g0 += 2u * (unsigned)issued;
        __syncwarp();
        return held ? 1 : 2;
    }
    I.g0 += 2u * (unsigned)np;
    return all_ok ? 0 : 1;
}

// Returns (for the whole warp) whether any output cell of the item is wet;
// all_wet: whether every output cell is.  try_wet: run the item on the
// all-wet assumption first, and again in the general form where it fails
// (only when TRY_WET: the FP32 form, where the wet/dry selects are a large
// share of the row's instructions).  The item's tallies are added to the
// lane's totals acc.p[m * 32].
template <class T, int CPT, int SX, int SY, bool KAPPA, bool TRY_WET>
__device__ __forceinline__ bool run_item(const ItemIO<T>& A, const StepK<T>& S, Acc<T>& acc, ItemCtx<T, CPT>& I,
                                         Carry<T, CPT>& Cy, const CUtensorMap* tme, const CUtensorMap* tmu,
                                         const CUtensorMap* tmv, const CUtensorMap* tmz, bool& timed_out,
                                         bool try_wet, bool& all_wet, T* side) {
    I.st_lane = I.out_lane && I.x0c >= 0 && I.x0c < A.G.nx;
    I.plo = max(I.y0, A.G.own_lo);
    I.phi = min(I.y1, A.G.own_hi);
    ItemAcc<T> ia;
    ia.side = side;
    const bool wet = TRY_WET && try_wet && !I.edge && I.y0 >= A.G.own_lo && I.y1 <= A.G.own_hi;
    int st = 0;
    bool w = wet;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {  // one call site: the rows' code is not inlined twice
        st = run_rows<T, CPT, SX, SY, KAPPA, TRY_WET>(A, S, I, Cy, ia, tme, tmu, tmv, tmz, timed_out, w);
        if (st != 2 || timed_out) break;
        w = false;
    }
    all_wet = st == 0;
    acc.p[0] = tmax(acc.p[0], ia.smax);
    acc.p[32] += ia.clamp;
#pragma unroll
    for (int q = 0; q < 4; ++q) acc.p[(2 + q) * 32] += ia.side[q * 32];
    acc.bad = acc.bad || ia.bad;
    return __any_sync(FULL, ia.smax > T(0));
}

// The work-item loop of one launch.  TRY_WET: items whose neighbourhood was
// all wet take the all-wet pass (run_item); the loop is compiled once with
// and once without it, and a launch runs one of the two.  wc: the counts of
// interior items with and without an all-wet neighbourhood (shared memory).
template <class T, int CPT, int SX, int SY, bool KAPPA, bool TRY_WET>
__device__ __forceinline__ void item_loop(const Args<T>& A, const StepK<T>& S, const CUtensorMap* tme,
                                          const CUtensorMap* tmu, const CUtensorMap* tmv, const CUtensorMap* tmz,
                                          unsigned char* ring, uint64_t* bars, int lane, Acc<T>& acc, bool& timed_out,
                                          unsigned* wc, T* side, unsigned* chk) {
    ItemCtx<T, CPT> I;
    I.ring = ring;
    I.bars = bars;
    I.chk = chk;
    I.lane = lane;
    I.out_lane = SX > 0 ? lane != 0 : lane != 31;
    I.g0 = 0;
    Carry<T, CPT> Cy;
#pragma unroll
    for (int b = 0; b < 2; ++b) Cy.P[b].e = Cy.P[b].u = Cy.P[b].v = Cy.P[b].z = Cy.P[b].qy = Vec<T, CPT>(T(0));
    I.yoff = 0;
    // items from the step's queue; the next index is fetched while an item runs
    unsigned* qc = &A.ctl->qctr[A.slot_cur];
    int item = 0;
    if (lane == 0) item = (int)atomicAdd(qc, 1u);
    item = __shfl_sync(FULL, item, 0);
    while (item < A.nitems && !timed_out) {
        int nxt = 0;
        if (lane == 0) nxt = (int)atomicAdd(qc, 1u);
        int kx, ky;
        item_of(item, A.nxs, A.nfull, kx, ky);
        const int fi = ky * A.nxs + kx;
        bool dry = false, try_wet = true;
        if (A.fl_in) {
            // lane q < 9 reads the flags of item (kx + q % 3 - 1, ky + q / 3 - 1),
            // the 3x3 neighbourhood (a radius of at least 2 cells); an item
            // outside the grid counts as dry and as all wet
            const int qx = kx + lane % 3 - 1, qy = ky + lane / 3 - 1;
            const bool in = lane < 9 && qx >= 0 && qy >= 0 && qx < A.nxs && qy < A.nys;
            const unsigned f = in ? A.fl_in[qy * A.nxs + qx] : 1u;
            const unsigned fc = __shfl_sync(FULL, f, 4);
            // an item whose neighbourhood held no wet cell keeps its values; if its
            // other copy already holds them too, it is skipped
            dry = A.skip && __all_sync(FULL, f & 1u) &&
                  !(((A.inflow_mask >> SIDE_W) & 1) && kx == 0) && !(((A.inflow_mask >> SIDE_E) & 1) && kx == A.nxs - 1) &&
                  !(((A.inflow_mask >> SIDE_S) & 1) && ky == 0) && !(((A.inflow_mask >> SIDE_N) & 1) && ky == A.nys - 1);
            // a neighbourhood whose every cell was wet is tried on the all-wet assumption
            try_wet = !__any_sync(FULL, f & 4u);
            if (dry && (fc & 2u)) {
                if (lane == 0) A.fl_out[fi] = 7u;
                item = __shfl_sync(FULL, nxt, 0);
                continue;
            }
        }
        const int x0 = kx * Geo<T, CPT>::OUT;
        I.xw = SX > 0 ? x0 - CPT : x0;
        I.xb = (I.xw - 2) & ~(Geo<T, CPT>::ALIGN - 1);
        I.col = (I.xw - I.xb) + CPT * lane;
        I.x0c = I.xw + CPT * lane;
        I.y0 = ky * A.L;
        I.y1 = min(A.G.ny, I.y0 + A.L);
        I.nr = I.y1 - I.y0 + 4;
        I.edge = (I.xw - 2 < 0) || (I.xw + Geo<T, CPT>::W + 1 > A.G.nx - 1);
        if (lane == 0 && !I.edge) atomicAdd(&wc[try_wet ? 0 : 1], 1u);
        bool all_wet;
        const bool wet = run_item<T, CPT, SX, SY, KAPPA, TRY_WET>(A, S, acc, I, Cy, tme, tmu, tmv, tmz, timed_out,
                                                                  try_wet, all_wet, side);
        if (A.fl_in && lane == 0) A.fl_out[fi] = (wet ? 0u : 1u) | (dry ? 2u : 0u) | (all_wet ? 0u : 4u);
        item = __shfl_sync(FULL, nxt, 0);
    }

}

template <class T, int CPT, int SX, int SY, bool KAPPA>
__global__ void __launch_bounds__(NWARP * 32, Geo<T, CPT>::MINB)
k_fused(const __grid_constant__ CUtensorMap tme, const __grid_constant__ CUtensorMap tmu,
        const __grid_constant__ CUtensorMap tmv, const __grid_constant__ CUtensorMap tmz, const Args<T> A) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[NWARP][NPAIR];
    __shared__ double sh_dt;
    __shared__ StepK<T> sh_S;  // the step's constants, divided once per CTA in FP64
    __shared__ bool sh_wet;    // this step runs the all-wet pass where an item's neighbourhood allows it
    __shared__ unsigned sh_wc[2];  // the CTA's interior items with and without an all-wet neighbourhood
    __shared__ unsigned sh_chk;    // checked builds: a check of the row step failed
    __shared__ double red[NWARP][6];
    __shared__ T sh_tot[NWARP][6][32];    // Acc
    __shared__ T sh_side[NWARP][4][32];   // ItemAcc::side
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        double dt = A.dt_fixed ? A.dt_fixed[A.s]
                               : dt_from_speed(__longlong_as_double((long long)A.ctl->smax[A.slot_cur]), A.cfl, A.dt_max);
        sh_dt = dt;
        sh_S = make_stepk<T>(dt, A.rdx, A.rdy, A.g);
        // The all-wet pass and the general lean rows are two large blocks of
        // code; where both run in one step they contend for the instruction
        // cache, which costs more than the pass saves.  So the pass runs only
        // when, in the previous step, the computed interior items that could
        // not take it were at most 1/WET_SHARE of those that could (every item
        // can after a reset of the counts).
        const unsigned* wc = A.ctl->wcnt[A.slot_cur];
        sh_wet = (unsigned long long)wc[1] * WET_SHARE <= (unsigned long long)wc[0];
        sh_wc[0] = sh_wc[1] = 0u;
        sh_chk = 0u;
        if (blockIdx.x == 0) {
            DevCtl* c = A.ctl;
            c->dt_last = dt;
            c->t += dt;
            c->dt_min = fmin(c->dt_min, dt);
            c->dt_maxs = fmax(c->dt_maxs, dt);
            A.dt_hist[A.s] = dt;
            c->smax[A.slot_zero] = 0ull;
            c->qctr[A.slot_zero] = 0u;  // the previous step's queue (all its CTAs have finished)
            c->wcnt[A.slot_zero][0] = c->wcnt[A.slot_zero][1] = 0u;
        }
    }
    if (lane == 0)
        for (int s = 0; s < NPAIR; ++s) mbar_init(&bars[warp][s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();
    const double dt = sh_dt;
    const StepK<T> S = sh_S;
    const bool use_wet = sh_wet;

    Acc<T> acc;
    acc.p = &sh_tot[warp][0][lane];
#pragma unroll
    for (int m = 0; m < 6; ++m) acc.p[m * 32] = T(0);
    __syncwarp();
    acc.bad = false;
    bool timed_out = false;
    if constexpr (sizeof(T) == 4) {
        if (use_wet)
            item_loop<T, CPT, SX, SY, KAPPA, true>(A, S, &tme, &tmu, &tmv, &tmz, smem + warp * Geo<T, CPT>::WARP_SMEM,
                                                   bars[warp], lane, acc, timed_out, sh_wc, &sh_side[warp][0][lane],
                                                   &sh_chk);
        else
            item_loop<T, CPT, SX, SY, KAPPA, false>(A, S, &tme, &tmu, &tmv, &tmz, smem + warp * Geo<T, CPT>::WARP_SMEM,
                                                    bars[warp], lane, acc, timed_out, sh_wc, &sh_side[warp][0][lane],
                                                   &sh_chk);
    } else {
        item_loop<T, CPT, SX, SY, KAPPA, false>(A, S, &tme, &tmu, &tmv, &tmz, smem + warp * Geo<T, CPT>::WARP_SMEM,
                                                bars[warp], lane, acc, timed_out, sh_wc, &sh_side[warp][0][lane],
                                                   &sh_chk);
    }

    // ---- reductions: warp, CTA, then one atomic per CTA
    __syncwarp();
    // the lanes' totals reduced over the warp in the real type, in FP64 from
    // there on (lane 0)
    T w[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) w[m] = acc.p[m * 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        w[0] = tmax(w[0], __shfl_xor_sync(FULL, w[0], o));
#pragma unroll
        for (int m = 1; m < 6; ++m) w[m] += __shfl_xor_sync(FULL, w[m], o);
    }
    double v[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) v[m] = (double)w[m];
    const bool bad = __any_sync(FULL, acc.bad);
    const bool tmo = __any_sync(FULL, timed_out);
    if (lane == 0) {
#pragma unroll
        for (int m = 0; m < 6; ++m) red[warp][m] = v[m];
        if (bad) atomicOr(&A.ctl->flags, (unsigned)SWE_FLAG_NONFINITE);
        if (tmo) atomicOr(&A.ctl->flags, (unsigned)SWE_FLAG_TIMEOUT);
        if (sh_chk) atomicOr(&A.ctl->flags, (unsigned)SWE_FLAG_CHECK);
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
        if (sh_wc[0]) atomicAdd(&A.ctl->wcnt[A.slot_next][0], sh_wc[0]);
        if (sh_wc[1]) atomicAdd(&A.ctl->wcnt[A.slot_next][1], sh_wc[1]);
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
    unsigned* flags;  // [2][nitems] dry-skip flags by step parity (device)
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
    A.G.own_lo = c->own_lo; A.G.own_hi = c->own_hi;
    const int a = c->cur, b = 1 - c->cur;
    A.e1 = (T*)c->eta[b]; A.u1 = (T*)c->u[b]; A.v1 = (T*)c->v[b];
    A.n2 = (const T*)c->n2;
    A.ctl = c->ctl;
    A.dt_fixed = c->dt_fixed_cap > 0 ? c->dt_fixed : nullptr;
    A.dt_hist = c->dt_hist;
    A.dx = p.dx; A.dy = p.dy; A.g = p.g; A.cfl = p.cfl; A.dt_max = p.dt_max; A.area = p.dx * p.dy;
    A.rdx = 1.0 / p.dx; A.rdy = 1.0 / p.dy;
    A.s = s;
    A.slot_cur = (int)(k % 3); A.slot_next = (int)((k + 1) % 3); A.slot_zero = (int)((k + 2) % 3);
    A.nxs = pl.nxs; A.nys = pl.nys; A.L = pl.L; A.nitems = pl.nitems; A.nfull = p.ny / pl.L;
    A.fl_in = nullptr; A.fl_out = nullptr; A.inflow_mask = 0;
    A.skip = p.dry_skip != 0;
    if (pl.flags) {
        A.fl_in = pl.flags + (size_t)(k & 1) * pl.nitems;
        A.fl_out = pl.flags + (size_t)((k + 1) & 1) * pl.nitems;
        for (int q = 0; q < 4; ++q)
            if (p.bc[q] == SWE_BC_INFLOW) A.inflow_mask |= 1 << q;
    }
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
