// launchers.h -- host-side launch entry points of the kernels (one
// translation unit per precision family so they compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include "hydro_internal.h"

namespace hydro {

// 2D step tile.
constexpr int STEP2D_TX = 32;
constexpr int STEP2D_TY = 8;

// Tile shapes of the 3D step (TX x TY threads, one column of cells each),
// chosen per solve or per batch by the autotuner.  The 512-thread 32 x 16
// tile is FP32 only: an FP64 thread needs about twice the 128 registers a
// 512-thread CTA can have.
struct TileShape { int tx, ty; };
// Variants 4..7 are the shapes of 0..3 staging the next plane with
// asynchronous copies one plane ahead (the staging depth the autotuner also
// chooses); 0..3 load each plane synchronously.
constexpr int TILE3D_VARIANTS = 8;
constexpr TileShape TILE3D_SHAPES[TILE3D_VARIANTS] = {{32, 8}, {32, 4}, {16, 16}, {32, 16},
                                                      {32, 8}, {32, 4}, {16, 16}, {32, 16}};
inline bool tile3d_available(int v, bool fp32) { return v >= 0 && v < TILE3D_VARIANTS && (v % 4 != 3 || fp32); }
// Paired-cell tiles (FP32 MUSCL-Hancock single solves only): variants
// PAIR_VARIANT0 + pv, each thread owning two x-adjacent cells of a tile of
// PAIR_SHAPES[pv] cells.
constexpr int PAIR_VARIANT0 = 8, PAIR_VARIANTS = 3;
constexpr TileShape PAIR_SHAPES[PAIR_VARIANTS] = {{32, 16}, {32, 8}, {16, 16}};
inline bool pair_variant(int v) { return v >= PAIR_VARIANT0 && v < PAIR_VARIANT0 + PAIR_VARIANTS; }
// cell tile of any 3D single-solve variant
inline TileShape tile_shape(int v) { return pair_variant(v) ? PAIR_SHAPES[v - PAIR_VARIANT0] : TILE3D_SHAPES[v]; }
inline bool tile3d_async(int v) { return v >= 4; }
constexpr int BATCH2D_TX = 32, BATCH2D_TY = 8;

// Persistent batched steps over the device-resident queue's work lists;
// `grid` CTAs claim the items.  *_max_grid: resident CTAs on the current
// device (SMs x occupancy).
cudaError_t launch_batch3d_f32(int variant, bool hse, const BatchInst *insts, BatchQueue *q, int parity, int grid,
                               cudaStream_t s);
cudaError_t launch_batch3d_f64(int variant, bool hse, const BatchInst *insts, BatchQueue *q, int parity, int grid,
                               cudaStream_t s);
int batch3d_max_grid_f32(int variant, bool hse);
int batch3d_max_grid_f64(int variant, bool hse);
inline cudaError_t launch_batch3d(int variant, bool fp32, bool hse, const BatchInst *insts, BatchQueue *q,
                                  int parity, int grid, cudaStream_t s)
{
    return fp32 ? launch_batch3d_f32(variant, hse, insts, q, parity, grid, s)
                : launch_batch3d_f64(variant, hse, insts, q, parity, grid, s);
}
cudaError_t launch_batch2d(bool fp32, const BatchInst *insts, BatchQueue *q, int parity, int grid, cudaStream_t s);
inline int batch3d_max_grid(int variant, bool fp32, bool hse)
{
    return fp32 ? batch3d_max_grid_f32(variant, hse) : batch3d_max_grid_f64(variant, hse);
}
int batch2d_max_grid(bool fp32);

// paired-cell FP32 MUSCL-Hancock step, pair variant pv (grid = tiles x z-chunks)
cudaError_t launch_pair3d(int pv, const StepArgs &a, dim3 grid, cudaStream_t s, bool hse);
// single-solve 3D step with tile variant v (grid = tiles x z-chunks)
cudaError_t launch_step3d_f64(int v, const StepArgs &a, dim3 grid, cudaStream_t s, bool hse);
cudaError_t launch_step3d_f32(int v, const StepArgs &a, dim3 grid, cudaStream_t s, bool hse);
// stage = STAGE_RK1 or STAGE_RK2 of the SSP-RK2 method of lines; recon =
// RECON_PLM or RECON_PPM (PPM without background subtraction)
cudaError_t launch_stage3d_f64(int stage, int v, const StepArgs &a, dim3 grid, cudaStream_t s, bool hse,
                               int recon);
cudaError_t launch_stage3d_f32(int stage, int v, const StepArgs &a, dim3 grid, cudaStream_t s, bool hse,
                               int recon);
// stage: STAGE_HANCOCK, STAGE_RK1 or STAGE_RK2; recon as above (stages only)
cudaError_t launch_step2d(const StepArgs &a, dim3 grid, cudaStream_t s, bool fp32, int stage = STAGE_HANCOCK,
                          int recon = RECON_PLM);

// corner transport upwind step (2D: same tile as the 2D step; 3D: blocks of
// cells, ctu3d_blocks of them)
cudaError_t launch_ctu2d(const StepArgs &a, dim3 grid, cudaStream_t s, bool fp32);
cudaError_t launch_ctu3d(const StepArgs &a, cudaStream_t s, bool fp32, bool hse);
long long ctu3d_blocks(const int n[3], bool fp32);

// Auxiliary kernels (aux.cu).  fp32 selects the stored precision.
struct AuxArgs {
    void *U;              // stored state (interior plane 0 of variable 0)
    int ndim, n[3];
    long long N, plane;   // cells, cells per plane
    long long vstride;    // distance between variable planes (N, or more with stored halos)
    double gamma, cfl, inv_dx[3], cell_volume;
    Ctrl *ctrl;
    double *partial;      // per-CTA partials (max_ctas * 5 doubles)
    const PlaneBG *bg;    // hse tables or nullptr
    int hse, fp32;
    int conserved_in;     // init conversion: staging holds conserved (1) or primitive (0) variables
};

// staging (FP64 total primitive, or with a.conserved_in total conserved,
// variables of cells [c0, c0 + m), planes of length m) -> stored state
cudaError_t launch_init_convert(const AuxArgs &a, const double *staging, long long c0,
                                long long m, cudaStream_t s);
// max signal speed of the state -> ctrl->dt_next (time unchanged)
cudaError_t launch_signal(const AuxArgs &a, cudaStream_t s);
// FP64 conserved totals (fixed-order two-stage sum) -> ctrl->totals
cudaError_t launch_totals(const AuxArgs &a, cudaStream_t s);
// state cells [c0, c0 + m) -> FP64 total conserved (what = 0) or primitive
// (what = 1) variables in staging (planes of length m)
cudaError_t launch_fields(const AuxArgs &a, double *staging, long long c0, long long m,
                          int what, cudaStream_t s);
// device arithmetic helpers over n values (0: 1/x, 1: y/x, 2: 1/sqrt(x), 3: MC slope of (x, y))
cudaError_t launch_math(int which, const double *x, const double *y, double *out, long long n,
                        cudaStream_t s);
// one stored value
cudaError_t launch_poke(const AuxArgs &a, int var, long long cell, double v, cudaStream_t s);

// grid of the reduction kernels (a fixed function of N, so sums are
// bitwise reproducible)
int aux_reduce_blocks(long long N);
constexpr int AUX_THREADS = 256;

}  // namespace hydro
