// hydro_internal.h -- structures shared by the host API and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>

namespace hydro {

enum { BC_OUTFLOW = 0, BC_PERIODIC = 1, BC_REFLECT = 2,
       BC_HALO = 3 };   // z only, internal: planes -2, -1 and nz, nz+1 are stored (slab decomposition)

// Device-resident time control; one per handle, at the start of the
// workspace.  Written only by the last CTA of a step (or of the dt kernel),
// read by every CTA of the next launch on the same stream.
struct __align__(16) Ctrl {
    double t;           // current time
    double dt_next;     // cfl / max signal speed of the current state
    double dt_last;     // dt taken by the last step
    double max_speed;   // max signal speed of the current state
    long long step;     // steps since init / set_state
    unsigned int counter;   // last-CTA arrival counter (returns to 0)
    int err;            // committed error bits (changed only at finalisation)
    int err_new;        // error bits raised by CTAs of the running step
    int pad0;
    double totals[5];   // last conserved-total reduction
    double pad[2];
};

// Per z-plane background constants of the hydrostatic-background mode for
// planes k = -2 .. nz+2 (entry k + 2).  Computed in FP64 on the host; the
// FP32 step reads a float copy so that no per-cell conversion is needed.
template <typename T>
struct PlaneBGT {
    T rho_c, p_c;   // background at the plane centre (0 for k = nz+2)
    T rho_f, p_f;   // background at the plane's low face z_lo + k dz
    T drho, dp;     // face(k+1) - face(k) (0 for k = nz+2)
    T B;            // (p_f(k+1) - p_f(k))/dz - rho_c g_z: discrete imbalance
    T pad;
};
using PlaneBG = PlaneBGT<double>;

// Arguments of one step launch (passed by value).
struct StepArgs {
    const void *U;      // state at t^n
    void *Unew;         // state at t^{n+1}
    int n[3];
    long long plane;    // nx*ny
    long long vstride;  // nx*ny*nz: distance between variable planes
    int bc_lo[3], bc_hi[3];
    double inv_dx[3];
    double gamma, cfl;
    double grav[3];
    double t_end;       // clamp target (+inf for a free step)
    long long step_end; // no further steps once ctrl->step reaches it
    Ctrl *ctrl;
    double *partial;    // per-CTA max signal speed
    const void *bgT;    // hse tables in the step's precision (nullptr in plain mode)
    const void *U0;     // second Runge-Kutta stage: U^n, read at the cell's own position
    int zchunk;         // planes per CTA (3D)
    int tiles_x;        // tiles along x
    // FP32 copies of gamma, 1/(gamma-1), 1/dx and g, each rounded once on
    // the host (fill_fp32_constants): an FP32 kernel uses them as operands
    // instead of converting the doubles, which the compiler would otherwise
    // redo on the FP64 pipe wherever it rematerialises them
    float gamma_f, igm1_f;
    float inv_dx_f[3], grav_f[3];
};

// Rounds the FP32 copies of a StepArgs' constants (the same values as a
// device-side conversion: IEEE round to nearest of the same doubles).
inline void fill_fp32_constants(StepArgs &a)
{
    a.gamma_f = static_cast<float>(a.gamma);
    a.igm1_f = static_cast<float>(1.0 / (a.gamma - 1.0));
    for (int d = 0; d < 3; ++d) {
        a.inv_dx_f[d] = static_cast<float>(a.inv_dx[d]);
        a.grav_f[d] = static_cast<float>(a.grav[d]);
    }
}

// One item of a batched step's work list: a tile and z-chunk of one instance.
struct BatchItem {
    int inst;    // instance index
    int tile;    // tile within the instance's x-y tiling
    int chunk;   // z-chunk (0 in 2D)
    int local;   // index of this item among the instance's items (its partial slot)
};

// Per-instance launch arguments for both ping-pong parities.
struct BatchInst {
    StepArgs a[2];
    int nitems;  // items of this instance in the work list
    int pad[3];
};

// Device-resident queue of a batch: the current work lists and their
// lengths, and per list and launch parity the counter of the next unclaimed
// item.  The persistent batched kernels read it at run time, so the host
// changes the batch's membership by rewriting it (stream-ordered copies
// between launches): the launch arguments, and a captured graph of launches,
// stay the same.  A launch's CTAs claim items one at a time from the counter
// (the host orders each list by decreasing item size); the last CTA to run
// out of items resets the counter and the exit count for the next launch.
struct BatchQueue {
    const BatchItem *items[2];   // [0]: 3D items, [1]: 2D items
    int nitems[2];
    unsigned next[2][2];         // [list][parity]: next unclaimed item
    unsigned exited[2][2];       // [list][parity]: CTAs that found no item left
};

// Workspace layout (offsets in bytes from the workspace base).
struct WorkLayout {
    size_t ctrl, partial, bg, bgf, stage, red, total;   // stage: first Runge-Kutta stage state
    int max_ctas;
};

// Kernel stage of a step: the MUSCL-Hancock step, or the first / second
// stage of the SSP-RK2 method of lines.
enum { STAGE_HANCOCK = 0, STAGE_RK1 = 1, STAGE_RK2 = 2 };

// Reconstruction of the face states: MC-limited linear, or the piecewise
// parabolic method (method-of-lines stages, no background subtraction).
enum { RECON_PLM = 0, RECON_PPM = 1 };

}  // namespace hydro
