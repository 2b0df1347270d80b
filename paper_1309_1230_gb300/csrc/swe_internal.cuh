// swe_internal.cuh -- context layout and kernel entry points shared by the
// library's translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/swe.h"
#include "swe_cell.cuh"

namespace swe {

// Device-side control block of one grid: the CFL reductions (triple
// buffered by step index), the clock and the tallies.
struct DevCtl {
    unsigned long long smax[3];  // bits of the non-negative FP64 CFL speed max, slot k%3 = level k
    double t, dt_last, dt_min, dt_maxs;
    double clamp, bflux[4];
    unsigned int flags;
    unsigned int pad;
    StepSlot cur;                // plain and paper paths: step size and constants of the current step
    unsigned int qctr[3];        // fused path: work-queue counter, slot k%3 = step k
    unsigned int pad2;
    // fused FP32 path, slot (k+1)%3 = step k's computed interior items whose
    // neighbourhood was all wet, and those whose neighbourhood was not (step
    // k+1 runs the all-wet pass only when the second count is small)
    unsigned int wcnt[3][2];
};

// Per-call diagnostics reduction result.
struct DevDiag {
    double volume;
    long long n_wet;
    unsigned int nonfinite;
    unsigned int pad;
};

}  // namespace swe

struct swe_ctx {
    swe_params p;
    int real_size;          // 4 or 8
    int pitch;              // row pitch in elements
    size_t plane;           // pitch * ny elements
    cudaStream_t stream;
    bool own_stream;
    bool poisoned;
    bool state_set;
    int cur;                // buffer holding the current level
    long long step;
    void* eta[2];
    void* u[2];
    void* v[2];
    void* z;
    double* z64;            // dense FP64 copy of the bed (set-state checks)
    void* n2;               // per-cell g*n^2 (real type) or NULL
    unsigned int* bad_flag; // set-state rejection bits
    void* ps[3];            // plain path: predicted eta, u, v
    swe::DevCtl* ctl;
    swe::DevCtl* h_ctl;     // pinned mirror
    swe::DevDiag* diag;     // diag partials + result
    double* diag_part;      // per-block partial volumes
    long long* diag_wet;
    unsigned int* diag_bad;
    int diag_blocks;
    double* dt_hist;
    int dt_hist_cap;
    double* dt_fixed;
    int dt_fixed_cap;       // values valid for the current call (0: none)
    int dt_fixed_alloc;
    double* stage;          // FP64 staging for host <-> device conversion (3 planes)
    size_t stage_elems;
    // fused path
    uint8_t* seg_wet[2];    // per work item: any wet cell in the level held by buffer b
    uint8_t* seg_same;      // per work item: both buffers hold the same values
    int seg_rows, seg_cols, segs_x, segs_y;
    void* tmaps;            // device copy of the tensor maps (4 per buffer pair)
    void* paper;            // scratch of the paper-layout step (swe_paper.cu), or NULL
    int own_lo, own_hi;     // own rows of a strip of a decomposed domain (default all rows)
    cudaGraphExec_t graph[2][6];   // cached multi-step graphs by (has dt_fixed, step % 6)
    int graph_steps[2][6];
    char err[512];
};

// Launchers implemented in the kernel translation units; each returns the
// launch error (cudaSuccess when queued).
cudaError_t swe_launch_plain_step(swe_ctx* c, int s, long long k);
cudaError_t swe_launch_paper_step(swe_ctx* c, int s, long long k);  // waits for the GPU in host-dt mode
void swe_paper_release(swe_ctx* c);
void swe_paper_bed_changed(swe_ctx* c);
cudaError_t swe_launch_fused_step(swe_ctx* c, int s, long long k);
cudaError_t swe_fused_prepare(swe_ctx* c);
cudaError_t swe_fused_reset_flags(swe_ctx* c);
void swe_fused_release(swe_ctx* c);  // frees the work plan and its device flags
int swe_fused_row_candidates(swe_ctx* c, int* out, int cap);
cudaError_t swe_launch_prologue(swe_ctx* c);
cudaError_t swe_launch_diag(swe_ctx* c);
cudaError_t swe_launch_to_real(swe_ctx* c, const double* src, void* dst, int n_planes, bool square_n);
cudaError_t swe_launch_to_double(swe_ctx* c, const void* src, double* dst);
cudaError_t swe_launch_dense_copy(swe_ctx* c, const void* src, void* dst, bool to_pitched);
cudaError_t swe_launch_normalise(swe_ctx* c, unsigned int* bad);
cudaError_t swe_launch_normalise64(swe_ctx* c, double* stage, unsigned int* bad);
cudaError_t swe_launch_call_begin(swe_ctx* c);
cudaError_t swe_fused_run(swe_ctx* c, int nsteps);
