// swe_fused.cu -- host side of the fused step: TMA tensor maps of the
// state planes and the work plan (rows per item chosen so that the items
// fill whole waves of the resident warps).  The kernel is in swe_fused.cuh.
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

template <class T, int CPT>
cudaError_t encode(CUtensorMap* m, const void* base, const swe_ctx* c) {
    cuuint64_t dims[2] = {(cuuint64_t)c->p.nx, (cuuint64_t)c->p.ny};
    cuuint64_t strides[1] = {(cuuint64_t)c->pitch * sizeof(T)};
    cuuint32_t box[2] = {(cuuint32_t)Geo<T, CPT>::BW, 1u};
    cuuint32_t es[2] = {1u, 1u};
    CUresult r = g_encode(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                          const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Rows per item chosen so that the items fill whole waves of the resident
// warps: minimise ceil(items / warps) * (L + 4) over L.
int choose_rows(int ny, int nxs, int warps, int forced) {
    if (forced > 0) return forced;
    int best = 64;
    double best_cost = 1e300;
    for (int L = 16; L <= 512; L += 4) {
        int nys = (ny + L - 1) / L;
        long long items = (long long)nxs * nys;
        long long rounds = (items + warps - 1) / warps;
        double cost = (double)rounds * (double)(L + 4);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = L; }
        if (L >= ny) break;
    }
    return best;
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
    if (c->real_size == 4) return prepare_t<float, 2>(c, pl);
    return prepare_t<double, 2>(c, pl);
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
