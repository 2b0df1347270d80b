// swe_batch.cu -- the batched form: many independent scenarios of uneven
// grid size advanced together, FP32, in one persistent cooperative launch
// per call (captured in a CUDA graph), each scenario with its own CFL step.
//
// Layout.  All scenarios share one arena per field: scenario s occupies rows
// [row0_s, row0_s + ny_s) and columns [0, nx_s) of a plane whose width is the
// largest nx; one TMA tensor map per field covers the whole arena, and the
// fused row step of swe_fused.cuh runs on it with the scenario's row offset.
// Cells outside a scenario (other scenarios' rows, padding columns) are read
// but always replaced by the scenario's ghost cells.
//
// Schedule.  The work items of every scenario (column strip x row segment)
// form one queue, largest scenarios first; in each step the CTAs claim items
// with an atomic counter, then meet at a bounded grid barrier before the next
// step.  An item whose 3x3 neighbourhood of items held no wet cell, and whose
// two ping-pong copies already agree, is skipped: an all-dry neighbourhood
// (radius 2 in cells) leaves the cells unchanged.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "swe_fused.cuh"

namespace swe {
namespace bt {

using fz::Acc;
using fz::Carry;
using fz::Geo;
using fz::ItemCtx;
using fz::ItemIO;

constexpr int CPT = 2;
using T = float;
using Gm = Geo<T, CPT>;

struct Scen {  // per-scenario constants on the device
    int nx, ny, row0, nxs, nys, item0;
    float gn2;
};

struct BItem {  // one work item: scenario, strip, segment, index of its flags (scenario-major)
    int s, kx, ky, fi;
};

struct BatchArgs {
    GridK<T> G;            // shared constants (nx, ny, gn2 are per scenario)
    const Scen* scen;
    const BItem* items;
    DevCtl* ctl;           // one control block per scenario
    unsigned* flags;       // [2][nitems]: bit 0 wet, bit 1 both copies equal
    unsigned* counters;    // [3] item claim counters by step % 3
    unsigned* bar;         // [2] grid barrier: arrivals, generation
    T* planes[2][3];       // eta, u, v of the two ping-pong copies
    const T* zp;           // bed
    double dx, dy, g, cfl, dt_max, area;
    double rdx, rdy;  // 1/dx, 1/dy (divided on the host)
    long long step0;
    int nsteps, nitems, nscen, L, cur0, dir_cycle, dry_skip;
    int inflow_side[4];
    unsigned long long bar_limit;  // grid-barrier wait limit, cycles
    int withhold;          // test hook: CTA withhold - 1 skips its first barrier arrival (0: none)
};

constexpr unsigned long long BARRIER_LIMIT = 4000000000ull;  // cycles (~2 s)

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_acquire32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded grid barrier (one warp per CTA); false when the wait gave up.  A
// CTA told to withhold its arrival (a test hook) returns false at once, and
// the other CTAs' waits run out after `limit` cycles.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned long long limit, bool withhold) {
    __syncwarp();
    if (withhold) return false;
    unsigned ok = 1;
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire32(bar + 1);
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = clock64();
            while (ld_acquire32(bar + 1) == gen) {
                if (clock64() - t0 > limit) { ok = 0; break; }
                __nanosleep(100);
            }
        }
        __threadfence();
        // the next step's TMA loads (async proxy) read rows other CTAs stored
        // with ordinary stores (generic proxy)
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    return ok != 0;
}

__device__ __forceinline__ double scen_dt(const BatchArgs& B, int s, long long k) {
    const unsigned long long bits = ld_acquire(&B.ctl[s].smax[k % 3]);
    return dt_from_speed(__longlong_as_double((long long)bits), B.cfl, B.dt_max);
}

// The persistent kernel holds both sweep directions of the row step, so it
// needs more registers than the single-grid kernel: 12 CTAs per SM (163
// registers) run it without spills, which measured faster than 16 with spills.
constexpr int BATCH_MINB = 12;

template <bool KAPPA>
__global__ void __launch_bounds__(32, BATCH_MINB)
k_batch(const __grid_constant__ CUtensorMap eA, const __grid_constant__ CUtensorMap uA,
        const __grid_constant__ CUtensorMap vA, const __grid_constant__ CUtensorMap eB,
        const __grid_constant__ CUtensorMap uB, const __grid_constant__ CUtensorMap vB,
        const __grid_constant__ CUtensorMap zz, const BatchArgs B) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[fz::NPAIR];
    __shared__ T sh_tot[6][32];       // fz::Acc of the current item
    __shared__ T sh_side[4][32];      // fz::ItemAcc::side
    const int lane = threadIdx.x & 31;
    if (lane == 0)
        for (int q = 0; q < fz::NPAIR; ++q) fz::mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();

    __shared__ unsigned sh_chk;       // checked builds: a check of the row step failed (fz::SWE_CHK)
    if (lane == 0) sh_chk = 0u;
    __syncwarp();
    ItemCtx<T, CPT> I;
    I.ring = smem;
    I.bars = bars;
    I.lane = lane;
    I.g0 = 0;
    I.chk = &sh_chk;
    Carry<T, CPT> Cy;
#pragma unroll
    for (int b = 0; b < 2; ++b)
        Cy.P[b].e = Cy.P[b].u = Cy.P[b].v = Cy.P[b].z = Cy.P[b].qy = fz::Vec<T, CPT>(0.f);
    bool timed_out = false;

    for (int st = 0; st < B.nsteps && !timed_out; ++st) {
        const long long k = B.step0 + st;
        const int cur = (B.cur0 + st) & 1;
        const unsigned* fl_in = B.flags + (size_t)(st & 1) * B.nitems;
        unsigned* fl_out = B.flags + (size_t)((st + 1) & 1) * B.nitems;
        if (blockIdx.x == 0) {
            // bookkeeping of every scenario for this step; the claim counter of the next step
            for (int s = lane; s < B.nscen; s += 32) {
                const double dt = scen_dt(B, s, k);
                DevCtl* c = &B.ctl[s];
                c->dt_last = dt;
                c->t += dt;
                c->dt_min = fmin(c->dt_min, dt);
                c->dt_maxs = fmax(c->dt_maxs, dt);
                c->smax[(k + 2) % 3] = 0ull;
            }
            if (lane == 0) B.counters[(k + 1) % 3] = 0u;
        }
        int sx, sy;
        step_dirs(B.dir_cycle, k, &sx, &sy);
        const CUtensorMap* me = cur ? &eB : &eA;
        const CUtensorMap* mu = cur ? &uB : &uA;
        const CUtensorMap* mv = cur ? &vB : &vA;
        for (;;) {
            unsigned it = 0;
            if (lane == 0) it = atomicAdd(&B.counters[k % 3], 1u);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= (unsigned)B.nitems) break;
            const BItem bi = B.items[it];
            const Scen sc = B.scen[bi.s];
            // dry skip: no wet cell in the 3x3 items around, both copies already equal
            bool dry = true;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int qx = bi.kx + dx, qy = bi.ky + dy;
                    if (qx < 0 || qy < 0 || qx >= sc.nxs || qy >= sc.nys) continue;
                    dry = dry && !(__ldcg(fl_in + sc.item0 + qy * sc.nxs + qx) & 1u);  // written by other SMs
                }
            const bool touches_inflow = (B.inflow_side[SIDE_W] && bi.kx == 0) ||
                                        (B.inflow_side[SIDE_E] && bi.kx == sc.nxs - 1) ||
                                        (B.inflow_side[SIDE_S] && bi.ky == 0) ||
                                        (B.inflow_side[SIDE_N] && bi.ky == sc.nys - 1);
            dry = dry && !touches_inflow;
            if (B.dry_skip && dry && (__ldcg(fl_in + bi.fi) & 2u)) {
                if (lane == 0) fl_out[bi.fi] = 2u;
                continue;
            }
            ItemIO<T> io;
            io.G = B.G;
            io.G.nx = sc.nx;
            io.G.ny = sc.ny;
            io.G.gn2 = sc.gn2;
            const size_t off = (size_t)sc.row0 * B.G.pitch;
            io.e1 = B.planes[1 - cur][0] + off;
            io.u1 = B.planes[1 - cur][1] + off;
            io.v1 = B.planes[1 - cur][2] + off;
            io.n2 = nullptr;
            // the scenario's step size and constants: FP64 divisions in one lane, then broadcast
            double dt = 0.0;
            StepK<T> S;
            if (lane == 0) {
                dt = scen_dt(B, bi.s, k);
                S = make_stepk<T>(dt, B.rdx, B.rdy, B.g);
            }
            dt = __shfl_sync(0xffffffffu, dt, 0);
            S.dt = __shfl_sync(0xffffffffu, S.dt, 0);
            S.dtdx = __shfl_sync(0xffffffffu, S.dtdx, 0);
            S.dtdy = __shfl_sync(0xffffffffu, S.dtdy, 0);
            S.g_dtdx = __shfl_sync(0xffffffffu, S.g_dtdx, 0);
            S.g_dtdy = __shfl_sync(0xffffffffu, S.g_dtdy, 0);
            const int x0 = bi.kx * Gm::OUT;
            I.xw = sx > 0 ? x0 - CPT : x0;
            I.xb = (I.xw - 2) & ~(Gm::ALIGN - 1);
            I.col = (I.xw - I.xb) + CPT * lane;
            I.x0c = I.xw + CPT * lane;
            I.y0 = bi.ky * B.L;
            I.y1 = min(sc.ny, I.y0 + B.L);
            I.nr = I.y1 - I.y0 + 4;
            I.yoff = sc.row0;
            I.out_lane = sx > 0 ? lane != 0 : lane != 31;
            I.edge = (I.xw - 2 < 0) || (I.xw + Gm::W + 1 > sc.nx - 1);
            Acc<T> acc;
            acc.p = &sh_tot[0][lane];
#pragma unroll
            for (int m = 0; m < 6; ++m) acc.p[m * 32] = T(0);
            acc.bad = false;
            bool all_wet;
            if (sx > 0) fz::run_item<T, CPT, 1, 1, KAPPA, false>(io, S, acc, I, Cy, me, mu, mv, &zz, timed_out, false, all_wet, &sh_side[0][lane]);
            else fz::run_item<T, CPT, -1, -1, KAPPA, false>(io, S, acc, I, Cy, me, mu, mv, &zz, timed_out, false, all_wet, &sh_side[0][lane]);
            // per-scenario reductions of this item
            // the item's totals, reduced over the warp in FP32, in FP64 from there
            T w[6];
#pragma unroll
            for (int m = 0; m < 6; ++m) w[m] = acc.p[m * 32];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                w[0] = fmaxf(w[0], __shfl_xor_sync(0xffffffffu, w[0], o));
#pragma unroll
                for (int m = 1; m < 6; ++m) w[m] += __shfl_xor_sync(0xffffffffu, w[m], o);
            }
            double v[6];
#pragma unroll
            for (int m = 0; m < 6; ++m) v[m] = (double)w[m];
            const bool bad = __any_sync(0xffffffffu, acc.bad);
            if (lane == 0) {
                DevCtl* c = &B.ctl[bi.s];
                if (v[0] > 0.0) atomicMax(&c->smax[(k + 1) % 3], (unsigned long long)__double_as_longlong(v[0]));
                if (v[1] != 0.0) atomicAdd(&c->clamp, v[1] * B.area);
                if (v[2] != 0.0) atomicAdd(&c->bflux[0], v[2] * dt * B.dy);
                if (v[3] != 0.0) atomicAdd(&c->bflux[1], v[3] * dt * B.dy);
                if (v[4] != 0.0) atomicAdd(&c->bflux[2], v[4] * dt * B.dx);
                if (v[5] != 0.0) atomicAdd(&c->bflux[3], v[5] * dt * B.dx);
                if (bad) atomicOr(&c->flags, (unsigned)SWE_FLAG_NONFINITE);
                if (sh_chk) { atomicOr(&c->flags, (unsigned)SWE_FLAG_CHECK); sh_chk = 0u; }
                fl_out[bi.fi] = (v[0] > 0.0 ? 1u : 0u) | (dry ? 2u : 0u);
            }
            if (timed_out) break;
        }
        const bool hold = B.withhold > 0 && blockIdx.x == (unsigned)(B.withhold - 1) && st == 0;
        if (timed_out || !grid_barrier(B.bar, gridDim.x, B.bar_limit, hold)) {
            timed_out = true;
            if (lane == 0) atomicOr(&B.ctl[0].flags, (unsigned)SWE_FLAG_TIMEOUT);
        }
    }
}

// CFL reduction of every scenario's freshly set state (one CTA per scenario)
// and the wet flags of its items; the flags start "copies differ".
__global__ void k_batch_prologue(const BatchArgs B, long long k) {
    __shared__ float red[32];
    const int s = blockIdx.x;
    const Scen sc = B.scen[s];
    const T* e = B.planes[B.cur0][0];
    const T* u = B.planes[B.cur0][1];
    const T* v = B.planes[B.cur0][2];
    GridK<T> G = B.G;
    G.nx = sc.nx; G.ny = sc.ny;
    float m = 0.f;
    for (int q = threadIdx.x; q < sc.nx * sc.ny; q += blockDim.x) {
        const int j = q / sc.nx, i = q % sc.nx;
        const size_t o = (size_t)(sc.row0 + j) * B.G.pitch + i;
        const float sp = cfl_speed(e[o], u[o], v[o], B.zp[o], G);
        if (sp > 0.f) {
            const int item = sc.item0 + (j / B.L) * sc.nxs + (i / Gm::OUT);
            if (!(B.flags[item] & 1u)) atomicOr(&B.flags[item], 1u);
        }
        m = fmaxf(m, sp);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
        DevCtl* c = &B.ctl[s];
        c->smax[0] = c->smax[1] = c->smax[2] = 0ull;
        c->smax[k % 3] = (unsigned long long)__double_as_longlong((double)t);
    }
}

// Scenario plane in, dense FP64 out (and the reverse).
__global__ void k_pack(const double* src, T* dst, int nx, int ny, int pitch, int row0) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nx * ny; q += gridDim.x * blockDim.x) {
        const int j = q / nx, i = q % nx;
        dst[(size_t)(row0 + j) * pitch + i] = (T)src[q];
    }
}
__global__ void k_unpack(const T* src, double* dst, int nx, int ny, int pitch, int row0) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nx * ny; q += gridDim.x * blockDim.x) {
        const int j = q / nx, i = q % nx;
        dst[q] = (double)src[(size_t)(row0 + j) * pitch + i];
    }
}

// FP64 volume of one scenario (one CTA, fixed order) and its wet-cell count.
__global__ void k_batch_volume(const BatchArgs B, int cur, double* vol, long long* wet) {
    __shared__ double sv[8];
    __shared__ long long sw[8];
    const int s = blockIdx.x;
    const Scen sc = B.scen[s];
    const T* e = B.planes[cur][0];
    double acc = 0.0;
    long long w = 0;
    for (int q = threadIdx.x; q < sc.nx * sc.ny; q += blockDim.x) {
        const int j = q / sc.nx, i = q % sc.nx;
        const size_t o = (size_t)(sc.row0 + j) * B.G.pitch + i;
        acc += (double)e[o] - (double)B.zp[o];
        w += (e[o] - B.zp[o]) > B.G.h_dry;
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = acc; sw[threadIdx.x >> 5] = w; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        long long tw = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { t += sv[q]; tw += sw[q]; }
        vol[s] = t * B.area;
        wet[s] = tw;
    }
}

__global__ void k_batch_begin(DevCtl* ctl, int n) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        ctl[s].dt_min = 1e300;
        ctl[s].dt_maxs = 0.0;
        ctl[s].flags = 0u;
    }
}

}  // namespace bt
}  // namespace swe

using namespace swe;
using namespace swe::bt;

struct swe_batch {
    swe_params p;
    int count = 0;
    std::vector<int> nx, ny, row0, order;
    std::vector<double> n;
    std::vector<std::vector<double>> zhost;
    std::vector<char> bed_set, state_set;
    int width = 0, pitch = 0;
    long long rows = 0;
    size_t plane = 0;
    T* pl[2][3] = {};
    T* z = nullptr;
    DevCtl* ctl = nullptr;
    DevCtl* h_ctl = nullptr;
    Scen* scen = nullptr;
    BItem* items = nullptr;
    unsigned* flags = nullptr;
    unsigned* counters = nullptr;
    unsigned* bar = nullptr;
    double* stage = nullptr;
    size_t stage_elems = 0;
    double* vol = nullptr;
    long long* wet = nullptr;
    int nitems = 0, grid = 0, L = 64;
    unsigned long long bar_limit = BARRIER_LIMIT;  // cycles; params reserved[0] (test hook)
    int withhold = 0;      // params reserved[1] (test hook), cleared after the next launch
    CUtensorMap tm[2][3];
    CUtensorMap tmz;
    cudaStream_t stream = nullptr;
    bool own_stream = false, poisoned = false;
    long long step = 0;
    int cur = 0;
    bool need_prologue = true;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = -1, graph_cur = -1;
    long long graph_k = -1;
    char err[512] = {};
};

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;

swe_status bfail(swe_batch* b, swe_status s, const char* fmt, ...) {
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define BCK(b, expr)                                                                         \
    do {                                                                                     \
        cudaError_t e__ = (expr);                                                            \
        if (e__ != cudaSuccess) {                                                            \
            (b)->poisoned = true;                                                            \
            return bfail((b), SWE_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e__));       \
        }                                                                                    \
    } while (0)

cudaError_t encode_plane(CUtensorMap* m, void* base, const swe_batch* b) {
    if (!g_enc) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
        g_enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    cuuint64_t dims[2] = {(cuuint64_t)b->width, (cuuint64_t)b->rows};
    cuuint64_t strides[1] = {(cuuint64_t)b->pitch * sizeof(T)};
    cuuint32_t box[2] = {(cuuint32_t)Gm::BW, 2u};  // two rows: one ring slot of the fused row step
    cuuint32_t es[2] = {1u, 1u};
    CUresult r = g_enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

BatchArgs make_args(const swe_batch* b, int nsteps) {
    BatchArgs B;
    memset(&B, 0, sizeof(B));
    const swe_params& p = b->p;
    B.G.nx = 0; B.G.ny = 0; B.G.pitch = b->pitch;
    B.G.own_lo = 0; B.G.own_hi = 1 << 30;  // every row of a scenario is its own
    B.G.g = (T)p.g; B.G.h_dry = (T)p.h_dry; B.G.kappa = (T)p.kappa; B.G.gn2 = 0.f;
    B.G.inv_dx = (T)(1.0 / p.dx); B.G.inv_dy = (T)(1.0 / p.dy);
    for (int s = 0; s < 4; ++s) {
        B.G.bc[s] = p.bc[s];
        B.G.qin[s] = (T)p.q_in[s];
        B.inflow_side[s] = p.bc[s] == SWE_BC_INFLOW;
    }
    B.scen = b->scen; B.items = b->items; B.ctl = b->ctl; B.flags = b->flags;
    B.counters = b->counters; B.bar = b->bar;
    for (int q = 0; q < 2; ++q)
        for (int f = 0; f < 3; ++f) B.planes[q][f] = b->pl[q][f];
    B.zp = b->z;
    B.dx = p.dx; B.dy = p.dy; B.g = p.g; B.cfl = p.cfl; B.dt_max = p.dt_max; B.area = p.dx * p.dy;
    B.rdx = 1.0 / p.dx; B.rdy = 1.0 / p.dy;
    B.step0 = b->step;
    B.nsteps = nsteps; B.nitems = b->nitems; B.nscen = b->count; B.L = b->L; B.cur0 = b->cur;
    B.dir_cycle = p.dir_cycle; B.dry_skip = p.dry_skip;
    B.bar_limit = b->bar_limit;
    B.withhold = b->withhold;
    return B;
}

swe_status ensure_stage(swe_batch* b, size_t elems) {
    if (b->stage_elems >= elems) return SWE_OK;
    if (b->stage) cudaFree(b->stage);
    b->stage = nullptr;
    b->stage_elems = 0;
    BCK(b, cudaMalloc(&b->stage, elems * sizeof(double)));
    b->stage_elems = elems;
    return SWE_OK;
}

void free_batch(swe_batch* b) {
    for (int q = 0; q < 2; ++q)
        for (int f = 0; f < 3; ++f)
            if (b->pl[q][f]) cudaFree(b->pl[q][f]);
    void* ptrs[] = {b->z, b->ctl, b->scen, b->items, b->flags, b->counters, b->bar, b->stage, b->vol, b->wet};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

swe_status check_batch(swe_batch* b) {
    if (!b) return SWE_ERR_ARG;
    if (b->poisoned) return bfail(b, SWE_ERR_STATE, "batch poisoned by an earlier CUDA error");
    if (cudaSetDevice(b->p.device) != cudaSuccess) return bfail(b, SWE_ERR_CUDA, "cudaSetDevice failed");
    return SWE_OK;
}

// (Re)builds the work items for L rows per item: the per-scenario table, the
// claim order (scenarios by decreasing size, so the largest are claimed
// first; the flags stay indexed scenario-major) and cleared dry-skip flags.
cudaError_t build_items(swe_batch* b, int L) {
    const int count = b->count;
    std::vector<Scen> sc(count);
    std::vector<BItem> items;
    for (int s = 0; s < count; ++s) {
        sc[s].nx = b->nx[s]; sc[s].ny = b->ny[s]; sc[s].row0 = b->row0[s];
        sc[s].nxs = (b->nx[s] + Gm::OUT - 1) / Gm::OUT;
        sc[s].nys = (b->ny[s] + L - 1) / L;
        sc[s].gn2 = (T)(b->p.g * b->n[s] * b->n[s]);
    }
    std::vector<int> item0(count);
    for (int s = 0; s < count; ++s) {  // item index = item0 + ky * nxs + kx, scenario-major
        item0[s] = (int)items.size();
        for (int ky = 0; ky < sc[s].nys; ++ky)
            for (int kx = 0; kx < sc[s].nxs; ++kx) items.push_back({s, kx, ky, (int)items.size()});
    }
    for (int s = 0; s < count; ++s) sc[s].item0 = item0[s];
    std::vector<BItem> claim;
    claim.reserve(items.size());
    for (int s : b->order)
        for (int q = 0; q < sc[s].nxs * sc[s].nys; ++q) claim.push_back(items[item0[s] + q]);
    cudaError_t e;
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return e;
    void* old[3] = {b->scen, b->items, b->flags};
    for (void* q : old)
        if (q && (e = cudaFree(q)) != cudaSuccess) return e;
    b->scen = nullptr; b->items = nullptr; b->flags = nullptr;
    b->nitems = (int)items.size();
    b->L = L;
    if ((e = cudaMalloc(&b->scen, count * sizeof(Scen))) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(b->scen, sc.data(), count * sizeof(Scen), cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(&b->items, b->nitems * sizeof(BItem))) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(b->items, claim.data(), b->nitems * sizeof(BItem), cudaMemcpyHostToDevice, b->stream)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMalloc(&b->flags, 2 * (size_t)b->nitems * sizeof(unsigned))) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->flags, 0, 2 * (size_t)b->nitems * sizeof(unsigned), b->stream)) != cudaSuccess) return e;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }  // captured the old item count
    b->graph_steps = -1;
    return cudaStreamSynchronize(b->stream);
}

int occupancy_batch(bool kappa) {
    int nb = 0;
    const int smem = Gm::WARP_SMEM;
    if (kappa) {
        cudaFuncSetAttribute(k_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<true>, 32, smem);
    } else {
        cudaFuncSetAttribute(k_batch<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<false>, 32, smem);
    }
    return nb;
}

}  // namespace

extern "C" {

swe_status swe_batch_create(const swe_params* p, int32_t count, const int32_t* nx, const int32_t* ny,
                            const double* manning_n, swe_batch** out) {
    if (!out) return SWE_ERR_ARG;
    *out = nullptr;
    if (!p || count < 1 || !nx || !ny || !manning_n) return SWE_ERR_ARG;
    if (p->precision != SWE_FP32) return SWE_ERR_UNSUPPORTED;
    if (p->dir_cycle != 0 && p->dir_cycle != 1) return SWE_ERR_UNSUPPORTED;
    if (p->friction != 0 || p->dissipation != 0) return SWE_ERR_UNSUPPORTED;  // ablation forms: plain/paper only
    if (!(p->dx > 0) || !(p->dy > 0) || !(p->g > 0) || !(p->cfl > 0) || !(p->h_dry > 0) || !(p->dt_max > 0))
        return SWE_ERR_ARG;
    if (!(p->kappa >= 0) || !(p->kappa <= 0.25)) return SWE_ERR_ARG;
    for (int s = 0; s < 4; ++s)
        if (p->bc[s] < SWE_BC_WALL || p->bc[s] > SWE_BC_OUTFLOW || !std::isfinite(p->q_in[s])) return SWE_ERR_ARG;
    for (int s = 0; s < count; ++s)
        if (nx[s] < 1 || ny[s] < 1 || !(manning_n[s] >= 0)) return SWE_ERR_ARG;
    // test hooks: the barrier wait limit (microseconds, at most 10 s) and a CTA withholding its arrival
    if (p->reserved[0] < 0 || p->reserved[0] > 10000000 || p->reserved[1] < 0) return SWE_ERR_ARG;
    swe_batch* b = new (std::nothrow) swe_batch();
    if (!b) return SWE_ERR_ARG;
    b->p = *p;
    // clock64 counts SM cycles: 2000 per microsecond at the GB300's 2.07 GHz maximum clock
    if (p->reserved[0] > 0) b->bar_limit = (unsigned long long)p->reserved[0] * 2000ull;
    b->withhold = p->reserved[1];
    b->count = count;
    b->nx.assign(nx, nx + count);
    b->ny.assign(ny, ny + count);
    b->n.assign(manning_n, manning_n + count);
    b->zhost.resize(count);
    b->bed_set.assign(count, 0);
    b->state_set.assign(count, 0);
    b->width = *std::max_element(nx, nx + count);
    b->pitch = ((b->width + 31) / 32) * 32;
    b->row0.resize(count);
    long long r = 0;
    for (int s = 0; s < count; ++s) { b->row0[s] = (int)r; r += ny[s]; }
    b->rows = r;
    b->plane = (size_t)b->pitch * (size_t)b->rows;
    b->L = p->seg_rows > 0 ? p->seg_rows : 192;
    auto bail = [&](const char* what, cudaError_t e) {
        fprintf(stderr, "swe_batch_create: %s: %s\n", what, cudaGetErrorString(e));
        free_batch(b);
        delete b;
        return SWE_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaSetDevice(p->device)) != cudaSuccess) return bail("cudaSetDevice", e);
    if (p->stream) b->stream = (cudaStream_t)p->stream;
    else {
        if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail("stream", e);
        b->own_stream = true;
    }
#ifdef SWE_CHECKED
    // every byte 0xff (a NaN) until set: a read beyond a scenario's cells shows
    const int fill = 0xff;
#else
    const int fill = 0;
#endif
    for (int q = 0; q < 2; ++q)
        for (int f = 0; f < 3; ++f) {
            if ((e = cudaMalloc(&b->pl[q][f], b->plane * sizeof(T))) != cudaSuccess) return bail("planes", e);
            if ((e = cudaMemset(b->pl[q][f], fill, b->plane * sizeof(T))) != cudaSuccess) return bail("memset", e);
        }
    if ((e = cudaMalloc(&b->z, b->plane * sizeof(T))) != cudaSuccess) return bail("bed", e);
    if ((e = cudaMemset(b->z, fill, b->plane * sizeof(T))) != cudaSuccess) return bail("memset", e);
    b->order.resize(count);
    for (int q = 0; q < count; ++q) b->order[q] = q;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int a, int c) { return (long long)nx[a] * ny[a] > (long long)nx[c] * ny[c]; });
    if ((e = build_items(b, b->L)) != cudaSuccess) return bail("work items", e);
    if ((e = cudaMalloc(&b->counters, 3 * sizeof(unsigned))) != cudaSuccess) return bail("counters", e);
    if ((e = cudaMemset(b->counters, 0, 3 * sizeof(unsigned))) != cudaSuccess) return bail("counters", e);
    if ((e = cudaMalloc(&b->bar, 2 * sizeof(unsigned))) != cudaSuccess) return bail("bar", e);
    if ((e = cudaMemset(b->bar, 0, 2 * sizeof(unsigned))) != cudaSuccess) return bail("bar", e);
    if ((e = cudaMalloc(&b->ctl, count * sizeof(DevCtl))) != cudaSuccess) return bail("ctl", e);
    if ((e = cudaMemset(b->ctl, 0, count * sizeof(DevCtl))) != cudaSuccess) return bail("ctl", e);
    if ((e = cudaMallocHost(&b->h_ctl, count * sizeof(DevCtl))) != cudaSuccess) return bail("ctl host", e);
    if ((e = cudaMalloc(&b->vol, count * sizeof(double))) != cudaSuccess) return bail("vol", e);
    if ((e = cudaMalloc(&b->wet, count * sizeof(long long))) != cudaSuccess) return bail("wet", e);
    for (int q = 0; q < 2; ++q)
        for (int f = 0; f < 3; ++f)
            if ((e = encode_plane(&b->tm[q][f], b->pl[q][f], b)) != cudaSuccess) return bail("tensor map", e);
    if ((e = encode_plane(&b->tmz, b->z, b)) != cudaSuccess) return bail("tensor map", e);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    const int per_sm = occupancy_batch(p->kappa != 0.0);
    if (per_sm < 1) return bail("occupancy", cudaErrorInvalidConfiguration);
    b->grid = sms * per_sm;
    // the set-up memsets and copies ran on the legacy default stream
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail("cudaDeviceSynchronize", e);
    *out = b;
    return SWE_OK;
}

void swe_batch_destroy(swe_batch* b) {
    if (!b) return;
    cudaSetDevice(b->p.device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
}

const char* swe_batch_last_error(const swe_batch* b) { return b ? b->err : "no batch"; }

swe_status swe_batch_set_bed(swe_batch* b, int32_t idx, const double* z) {
    swe_status s = check_batch(b);
    if (s != SWE_OK) return s;
    if (idx < 0 || idx >= b->count || !z) return bfail(b, SWE_ERR_ARG, "bad index or NULL bed");
    const size_t n = (size_t)b->nx[idx] * b->ny[idx];
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(z[k])) return bfail(b, SWE_ERR_ARG, "non-finite bed");
    b->zhost[idx].assign(z, z + n);
    if ((s = ensure_stage(b, 3 * n)) != SWE_OK) return s;
    BCK(b, cudaMemcpyAsync(b->stage, z, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    k_pack<<<256, 256, 0, b->stream>>>(b->stage, b->z, b->nx[idx], b->ny[idx], b->pitch, b->row0[idx]);
    BCK(b, cudaGetLastError());
    BCK(b, cudaStreamSynchronize(b->stream));
    b->bed_set[idx] = 1;
    b->state_set[idx] = 0;
    return SWE_OK;
}

// Set-state normalisation in FP64 against the scenario's FP64 bed, as in
// swe_set_state: reject h < -1e-12 m, clamp smaller negatives, zero the
// velocity of dry cells.
swe_status swe_batch_set_state(swe_batch* b, int32_t idx, const double* eta, const double* u, const double* v) {
    swe_status s = check_batch(b);
    if (s != SWE_OK) return s;
    if (idx < 0 || idx >= b->count || !eta || !u || !v) return bfail(b, SWE_ERR_ARG, "bad index or NULL state");
    if (!b->bed_set[idx]) return bfail(b, SWE_ERR_STATE, "set the bed of scenario %d first", idx);
    const size_t n = (size_t)b->nx[idx] * b->ny[idx];
    std::vector<double> e(eta, eta + n), uu(u, u + n), vv(v, v + n);
    const std::vector<double>& z = b->zhost[idx];
    for (size_t k = 0; k < n; ++k) {
        if (!std::isfinite(e[k]) || !std::isfinite(uu[k]) || !std::isfinite(vv[k]))
            return bfail(b, SWE_ERR_ARG, "non-finite state");
        double h = e[k] - z[k];
        if (h < -1e-12) return bfail(b, SWE_ERR_NEGDEPTH, "depth below -1e-12 m in scenario %d", idx);
        if (h < 0.0) { e[k] = z[k]; h = 0.0; }
        if (h <= b->p.h_dry) { uu[k] = 0.0; vv[k] = 0.0; }
    }
    if ((s = ensure_stage(b, 3 * n)) != SWE_OK) return s;
    const double* src[3] = {e.data(), uu.data(), vv.data()};
    for (int f = 0; f < 3; ++f) {
        BCK(b, cudaMemcpyAsync(b->stage + f * n, src[f], n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
        k_pack<<<256, 256, 0, b->stream>>>(b->stage + f * n, b->pl[b->cur][f], b->nx[idx], b->ny[idx], b->pitch,
                                           b->row0[idx]);
        BCK(b, cudaGetLastError());
    }
    BCK(b, cudaStreamSynchronize(b->stream));
    b->state_set[idx] = 1;
    b->need_prologue = true;
    return SWE_OK;
}

// Queues nsteps steps: one persistent cooperative launch, captured in a graph
// when `graph` is set (re-captured when the step count, starting step or
// buffer parity changes).
static cudaError_t launch_steps(swe_batch* b, int nsteps, bool graph) {
    BatchArgs B = make_args(b, nsteps);
    const bool kap = b->p.kappa != 0.0;
    void* kern = kap ? (void*)k_batch<true> : (void*)k_batch<false>;
    const CUtensorMap* A = b->tm[0];
    const CUtensorMap* Bm = b->tm[1];
    void* args[] = {(void*)&A[0], (void*)&A[1], (void*)&A[2], (void*)&Bm[0], (void*)&Bm[1], (void*)&Bm[2],
                    (void*)&b->tmz, (void*)&B};
    cudaError_t e;
    if ((e = cudaMemsetAsync(b->counters, 0, 3 * sizeof(unsigned), b->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned), b->stream)) != cudaSuccess) return e;
    if (!graph || b->withhold) return cudaLaunchCooperativeKernel(kern, dim3(b->grid), dim3(32), args, Gm::WARP_SMEM, b->stream);
    if (!b->graph || b->graph_steps != nsteps || b->graph_k != b->step || b->graph_cur != b->cur) {
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
        const cudaError_t le = cudaLaunchCooperativeKernel(kern, dim3(b->grid), dim3(32), args, Gm::WARP_SMEM, b->stream);
        const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return le != cudaSuccess ? le : ce;
        }
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        b->graph_steps = nsteps;
        b->graph_k = b->step;
        b->graph_cur = b->cur;
    }
    return cudaGraphLaunch(b->graph, b->stream);
}

static swe_status prologue(swe_batch* b) {
    BatchArgs B = make_args(b, 0);
    BCK(b, cudaMemsetAsync(b->flags, 0, 2 * (size_t)b->nitems * sizeof(unsigned), b->stream));
    k_batch_prologue<<<b->count, 256, 0, b->stream>>>(B, b->step);
    BCK(b, cudaGetLastError());
    return SWE_OK;
}

swe_status swe_batch_step(swe_batch* b, int32_t nsteps, swe_step_info* infos) {
    swe_status s = check_batch(b);
    if (s != SWE_OK) return s;
    if (nsteps < 0) return bfail(b, SWE_ERR_ARG, "nsteps < 0");
    for (int q = 0; q < b->count; ++q)
        if (!b->state_set[q]) return bfail(b, SWE_ERR_STATE, "scenario %d has no state", q);
    if (b->need_prologue) {
        // first call after a state was set: the initial CFL reductions and flags
        if ((s = prologue(b)) != SWE_OK) return s;
        b->need_prologue = false;
    }
    k_batch_begin<<<(b->count + 255) / 256, 256, 0, b->stream>>>(b->ctl, b->count);
    BCK(b, cudaGetLastError());
    if (nsteps > 0) {
        BCK(b, launch_steps(b, nsteps, b->p.use_graph != 0));
        b->withhold = 0;  // the test hook acts on one call
    }
    b->step += nsteps;
    b->cur = (b->cur + nsteps) & 1;
    BCK(b, cudaMemcpyAsync(b->h_ctl, b->ctl, b->count * sizeof(DevCtl), cudaMemcpyDeviceToHost, b->stream));
    std::vector<double> vol(b->count);
    std::vector<long long> wet(b->count);
    if (infos) {
        BatchArgs B = make_args(b, 0);
        k_batch_volume<<<b->count, 256, 0, b->stream>>>(B, b->cur, b->vol, b->wet);
        BCK(b, cudaGetLastError());
        BCK(b, cudaMemcpyAsync(vol.data(), b->vol, b->count * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        BCK(b, cudaMemcpyAsync(wet.data(), b->wet, b->count * sizeof(long long), cudaMemcpyDeviceToHost, b->stream));
    }
    BCK(b, cudaStreamSynchronize(b->stream));
    unsigned any = 0;
    for (int q = 0; q < b->count; ++q) {
        const DevCtl& h = b->h_ctl[q];
        any |= h.flags;
        if (infos) {
            swe_step_info& o = infos[q];
            memset(&o, 0, sizeof(o));
            o.t = h.t; o.dt_last = h.dt_last; o.dt_min = h.dt_min > 1e299 ? 0.0 : h.dt_min;
            o.dt_max_seen = h.dt_maxs; o.volume = vol[q]; o.clamp_volume = h.clamp;
            for (int k = 0; k < 4; ++k) o.bflux[k] = h.bflux[k];
            o.step = b->step; o.n_wet = wet[q]; o.flags = (int32_t)h.flags;
        }
    }
    if (any & SWE_FLAG_TIMEOUT) return bfail(b, SWE_ERR_TIMEOUT, "grid barrier or load wait gave up");
    if (any & SWE_FLAG_NONFINITE) return bfail(b, SWE_ERR_NONFINITE, "non-finite value in a scenario");
    if (any & SWE_FLAG_CHECK) return bfail(b, SWE_ERR_CHECK, "a device-side index or alignment check failed (checked build)");
    return SWE_OK;
}

swe_status swe_batch_get_state(swe_batch* b, int32_t idx, double* eta, double* u, double* v) {
    swe_status s = check_batch(b);
    if (s != SWE_OK) return s;
    if (idx < 0 || idx >= b->count || !eta || !u || !v) return bfail(b, SWE_ERR_ARG, "bad index or NULL state");
    const size_t n = (size_t)b->nx[idx] * b->ny[idx];
    if ((s = ensure_stage(b, 3 * n)) != SWE_OK) return s;
    double* dst[3] = {eta, u, v};
    for (int f = 0; f < 3; ++f) {
        k_unpack<<<256, 256, 0, b->stream>>>(b->pl[b->cur][f], b->stage + f * n, b->nx[idx], b->ny[idx], b->pitch,
                                             b->row0[idx]);
        BCK(b, cudaGetLastError());
        BCK(b, cudaMemcpyAsync(dst[f], b->stage + f * n, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    }
    BCK(b, cudaStreamSynchronize(b->stream));
    return SWE_OK;
}

// Built-in candidate rows per item of the batched step.
static const int kBatchRows[] = {32, 64, 96, 128, 192, 256, 384, 512};

int32_t swe_batch_autotune_candidates(swe_batch* b, int32_t* rows, int32_t cap) {
    swe_status s = check_batch(b);
    if (s != SWE_OK) return -(int32_t)s;
    if (!rows || cap < 1) return -(int32_t)bfail(b, SWE_ERR_ARG, "rows is NULL or cap < 1");
    const int n = (int)(sizeof(kBatchRows) / sizeof(kBatchRows[0]));
    for (int i = 0; i < n && i < cap; ++i) rows[i] = kBatchRows[i];
    return n < cap ? n : cap;
}

swe_status swe_batch_autotune(swe_batch* b, int32_t probe_steps, const int32_t* rows, int32_t nrows,
                              double* ms_per_step, int32_t* chosen) {
    swe_status s = check_batch(b);
    if (s != SWE_OK) return s;
    if (probe_steps < 1 || probe_steps > 10000) return bfail(b, SWE_ERR_ARG, "probe_steps must lie in [1, 10000]");
    for (int q = 0; q < b->count; ++q)
        if (!b->state_set[q]) return bfail(b, SWE_ERR_STATE, "scenario %d has no state", q);
    std::vector<int> cand;
    if (rows) {
        if (nrows < 1) return bfail(b, SWE_ERR_ARG, "nrows < 1");
        for (int i = 0; i < nrows; ++i) {
            if (rows[i] < 1 || rows[i] > 4096) return bfail(b, SWE_ERR_ARG, "rows[%d] must lie in [1, 4096]", i);
            cand.push_back(rows[i]);
        }
    } else {
        if (ms_per_step) return bfail(b, SWE_ERR_ARG, "ms_per_step needs the candidate list");
        cand.assign(std::begin(kBatchRows), std::end(kBatchRows));
    }
    if (b->need_prologue) {
        if ((s = prologue(b)) != SWE_OK) return s;
        b->need_prologue = false;
    }
    // the state, clocks and tallies to come back to after every probe
    const int cur0 = b->cur;
    const long long step0 = b->step;
    std::vector<DevCtl> saved(b->count);
    BCK(b, cudaMemcpyAsync(saved.data(), b->ctl, b->count * sizeof(DevCtl), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    struct Scratch {
        T* p[3] = {nullptr, nullptr, nullptr};
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Scratch() {
            for (T* q : p)
                if (q) cudaFree(q);
            for (cudaEvent_t q : e)
                if (q) cudaEventDestroy(q);
        }
    } k;
    const size_t bytes = b->plane * sizeof(T);
    for (int f = 0; f < 3; ++f) {
        BCK(b, cudaMalloc(&k.p[f], bytes));
        BCK(b, cudaMemcpyAsync(k.p[f], b->pl[cur0][f], bytes, cudaMemcpyDeviceToDevice, b->stream));
    }
    BCK(b, cudaEventCreate(&k.e[0]));
    BCK(b, cudaEventCreate(&k.e[1]));
    auto restore = [&]() -> swe_status {
        b->cur = cur0;
        b->step = step0;
        for (int f = 0; f < 3; ++f)
            BCK(b, cudaMemcpyAsync(b->pl[cur0][f], k.p[f], bytes, cudaMemcpyDeviceToDevice, b->stream));
        BCK(b, cudaMemcpyAsync(b->ctl, saved.data(), b->count * sizeof(DevCtl), cudaMemcpyHostToDevice, b->stream));
        // cleared flags: the first steps after this compute every item
        BCK(b, cudaMemsetAsync(b->flags, 0, 2 * (size_t)b->nitems * sizeof(unsigned), b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
        return SWE_OK;
    };
    int best = -1;
    float best_ms = 0.f;
    for (size_t i = 0; i < cand.size(); ++i) {
        BCK(b, build_items(b, cand[i]));
        if ((s = restore()) != SWE_OK) return s;
        k_batch_begin<<<(b->count + 255) / 256, 256, 0, b->stream>>>(b->ctl, b->count);
        BCK(b, cudaGetLastError());
        BCK(b, launch_steps(b, 1, false));  // warm-up
        b->step += 1;
        b->cur ^= 1;
        BCK(b, cudaEventRecord(k.e[0], b->stream));
        BCK(b, launch_steps(b, probe_steps, false));
        BCK(b, cudaEventRecord(k.e[1], b->stream));
        BCK(b, cudaEventSynchronize(k.e[1]));
        float ms = 0.f;
        BCK(b, cudaEventElapsedTime(&ms, k.e[0], k.e[1]));
        ms /= (float)probe_steps;
        if (ms_per_step) ms_per_step[i] = ms;
        if (best < 0 || ms < best_ms) { best = (int)i; best_ms = ms; }
        BCK(b, cudaMemcpy(b->h_ctl, b->ctl, b->count * sizeof(DevCtl), cudaMemcpyDeviceToHost));
        for (int q = 0; q < b->count; ++q)
            if (b->h_ctl[q].flags & SWE_FLAG_TIMEOUT)
                return bfail(b, SWE_ERR_TIMEOUT, "a device-side wait gave up while probing %d rows", cand[i]);
    }
    BCK(b, build_items(b, cand[best]));
    if ((s = restore()) != SWE_OK) return s;
    b->p.seg_rows = cand[best];
    if (chosen) *chosen = cand[best];
    return SWE_OK;
}

}  // extern "C"
