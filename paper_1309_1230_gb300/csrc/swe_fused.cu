// swe_fused.cu -- host side of the fused step: TMA tensor maps of the
// state planes and the work plan (rows per item, items per step, grid).  The
// kernel is in swe_fused.cuh.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "swe_fused.cuh"

using namespace swe;
using namespace swe::fz;

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encode() {
    if (g_encode) return cudaSuccess;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return cudaSuccess;
}

// Row boxes of W + 8 columns, two rows high (one ring slot).  No L2 fill
// promotion: a box row of 288 bytes at a 16-byte offset promoted to 256-byte
// fills fetched 8 % more from DRAM on the 8192^2 river than plain sector fills.
template <class T, int CPT>
cudaError_t encode(CUtensorMap* m, const void* base, const swe_ctx* c) {
    cuuint64_t dims[2] = {(cuuint64_t)c->p.nx, (cuuint64_t)c->p.ny};
    cuuint64_t strides[1] = {(cuuint64_t)c->pitch * sizeof(T)};
    cuuint32_t box[2] = {(cuuint32_t)Geo<T, CPT>::BW, 2u};  // two rows: one ring slot
    cuuint32_t es[2] = {1u, 1u};
    CUresult r = g_encode(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                          const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Rows per item: the warps take items from a queue, so the items only need
// to be small enough that the warps finish together (about ITEMS_PER_WARP
// each) while long enough that the four warm-up rows of an item stay a small
// share of its work.
constexpr int ITEMS_PER_WARP = 8;

int choose_rows(int ny, int nxs, int warps, int forced) {
    if (forced > 0) return forced;
    const double want = (double)ny * nxs / ((double)ITEMS_PER_WARP * warps);
    int L = ((int)want + 3) / 4 * 4;
    if (L < 32) L = 32;
    if (L > 512) L = 512;
    return L;
}

template <class T, int CPT>
cudaError_t prepare_t(swe_ctx* c, Plan& pl) {
    cudaError_t e = get_encode();
    if (e != cudaSuccess) return e;
    for (int b = 0; b < 2; ++b) {
        if ((e = encode<T, CPT>(&pl.e[b], c->eta[b], c)) != cudaSuccess) return e;
        if ((e = encode<T, CPT>(&pl.u[b], c->u[b], c)) != cudaSuccess) return e;
        if ((e = encode<T, CPT>(&pl.v[b], c->v[b], c)) != cudaSuccess) return e;
    }
    if ((e = encode<T, CPT>(&pl.z, c->z, c)) != cudaSuccess) return e;
    int dev = c->p.device, sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = sizeof(T) == 4 ? occupancy_f32(c) : occupancy_f64(c);
    pl.grid = sms * per_sm;
    const int warps = pl.grid * NWARP;
    pl.nxs = (c->p.nx + Geo<T, CPT>::OUT - 1) / Geo<T, CPT>::OUT;
    pl.L = choose_rows(c->p.ny, pl.nxs, warps, c->p.seg_rows);
    pl.nys = (c->p.ny + pl.L - 1) / pl.L;
    pl.nitems = pl.nxs * pl.nys;
    if (pl.grid * NWARP > pl.nitems) pl.grid = (pl.nitems + NWARP - 1) / NWARP;
    if (pl.flags) cudaFree(pl.flags);
    pl.flags = nullptr;
    if ((e = cudaMalloc(&pl.flags, 2 * (size_t)pl.nitems * sizeof(unsigned))) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(pl.flags, 0, 2 * (size_t)pl.nitems * sizeof(unsigned), c->stream)) != cudaSuccess) return e;
    pl.ready = true;
    return cudaSuccess;
}

}  // namespace

cudaError_t swe_fused_prepare(swe_ctx* c) {
    if (!c->tmaps) {
        c->tmaps = malloc(sizeof(Plan));
        if (!c->tmaps) return cudaErrorMemoryAllocation;
        memset(c->tmaps, 0, sizeof(Plan));
    }
    Plan& pl = *(Plan*)c->tmaps;
    if (c->real_size == 4) return prepare_t<float, CPT_F32>(c, pl);
    return prepare_t<double, 2>(c, pl);
}

// Candidate rows per item for the autotuner: the heights that give about q
// items per resident warp for q in {1, 2, 3, 4, 5, 6, 8}, and 16, 32, 64, 96
// and 128 rows; multiples of 4 in [16, 512], ascending, no repeats.
int swe_fused_row_candidates(swe_ctx* c, int* out, int cap) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->p.device);
    const int per_sm = c->real_size == 4 ? occupancy_f32(c) : occupancy_f64(c);
    const double warps = (double)sms * per_sm * NWARP;
    const int nxs = (c->p.nx + Geo<float, CPT_F32>::OUT - 1) / Geo<float, CPT_F32>::OUT;
    int v[12], n = 0;
    const int q[7] = {1, 2, 3, 4, 5, 6, 8};
    for (int i = 0; i < 7; ++i) {
        int L = ((int)std::ceil((double)c->p.ny * nxs / (q[i] * warps)) + 3) / 4 * 4;
        v[n++] = L < 16 ? 16 : (L > 512 ? 512 : L);
    }
    v[n++] = 16;
    v[n++] = 32;
    v[n++] = 64;
    v[n++] = 96;
    v[n++] = 128;
    std::sort(v, v + n);
    const int m = (int)(std::unique(v, v + n) - v);
    for (int i = 0; i < m && i < cap; ++i) out[i] = v[i];
    return m < cap ? m : cap;
}

void swe_fused_release(swe_ctx* c) {
    if (c->tmaps) {
        Plan& pl = *(Plan*)c->tmaps;
        if (pl.flags) cudaFree(pl.flags);
        free(c->tmaps);
        c->tmaps = nullptr;
    }
}

// Forgets what the dry-skip flags know (the state may have been replaced):
// the first two steps after this compute every item.
cudaError_t swe_fused_reset_flags(swe_ctx* c) {
    if (!c->tmaps) return cudaSuccess;
    Plan& pl = *(Plan*)c->tmaps;
    if (!pl.flags) return cudaSuccess;
    return cudaMemsetAsync(pl.flags, 0, 2 * (size_t)pl.nitems * sizeof(unsigned), c->stream);
}

cudaError_t swe_launch_fused_step(swe_ctx* c, int s, long long k) {
    Plan& pl = *(Plan*)c->tmaps;
    const bool kap = c->p.kappa != 0.0;
    if (c->real_size == 4) return kap ? launch_f32_k(c, pl, s, k) : launch_f32_0(c, pl, s, k);
    return kap ? launch_f64_k(c, pl, s, k) : launch_f64_0(c, pl, s, k);
}

cudaError_t swe_fused_run(swe_ctx* c, int nsteps) {
    if (!c->tmaps || !((Plan*)c->tmaps)->ready) {
        cudaError_t e = swe_fused_prepare(c);
        if (e != cudaSuccess) return e;
    }
    for (int q = 0; q < nsteps; ++q) {
        cudaError_t e = swe_launch_fused_step(c, q, c->step + q);
        if (e != cudaSuccess) return e;
        c->cur = 1 - c->cur;
    }
    return cudaSuccess;
}

int swe_fused_plan_info(swe_ctx* c, int* grid, int* L, int* nitems) {
    if (!c->tmaps) return 0;
    Plan& pl = *(Plan*)c->tmaps;
    *grid = pl.grid; *L = pl.L; *nitems = pl.nitems;
    return 1;
}
