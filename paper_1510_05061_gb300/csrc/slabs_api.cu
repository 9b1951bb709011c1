// slabs_api.cu -- domain decomposition of one 3D solve into z slabs.
//
// The paper's codes divide the star across nodes by domain decomposition and
// exchange nearest-neighbour data every step, plus a global reduction
// (introduction, "Capabilities needed").  Here a 3D grid is cut into R slabs
// along z, each stored with two halo planes below and above its interior.
// One step is: (1) halo exchange -- each internal slab face receives the two
// edge planes of its neighbour (periodic ends wrap); physical ends keep their
// boundary condition; (2) the step kernel on every slab (a halo side reads
// the stored planes instead of mapping a boundary); (3) a max-reduction of
// the slabs' CFL signal speeds that gives every slab the same next dt.
// With one GPU per box the slabs run as virtual ranks on one device (the
// exchange is device-to-device copies, the reduction a one-block kernel); on
// several GPUs the same plan maps to point-to-point sends and an allreduce.
// Given the same data and dt, every slab computes exactly the cells the
// undivided solve computes.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/hydro.h"
#include "hydro_internal.h"
#include "launchers.h"

using namespace hydro;

namespace {

constexpr size_t ALIGN = 256;
size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }
bool aligned(const void *p) { return (reinterpret_cast<uintptr_t>(p) % ALIGN) == 0; }
int tiles_along(int n, int t) { return (n + t - 1) / t; }

bool extent(const hydro_problem *g, int R, int r, int *z0, int *nz)
{
    if (!g || g->ndim != 3 || R <= 0 || r < 0 || r >= R) return false;
    const int base = g->n[2] / R, extra = g->n[2] % R;
    *nz = base + (r < extra ? 1 : 0);
    *z0 = r * base + std::min(r, extra);
    return *nz >= 2;
}

bool valid_global(const hydro_problem *g, int R)
{
    if (!g || g->ndim != 3 || R <= 0 || hydro_state_bytes(g) == 0) return false;
    if (g->scheme != HYDRO_SCHEME_HANCOCK) return false;   // slabs step MUSCL-Hancock
    return g->n[2] / R >= 2;   // every slab supplies two halo planes
}

struct SlabLayout {
    size_t ctrl, partial, bg, bgf, total;
};

SlabLayout slab_layout(const hydro_problem *g, int nz)
{
    SlabLayout L{};
    const long long N = (long long)g->n[0] * g->n[1] * nz;
    int m = 0;
    for (int v = 0; v < TILE3D_VARIANTS; ++v)
        m = std::max(m, tiles_along(g->n[0], TILE3D_SHAPES[v].tx) * tiles_along(g->n[1], TILE3D_SHAPES[v].ty) * nz);
    const size_t nparts = std::max((size_t)m, (size_t)5 * aux_reduce_blocks(N));
    size_t off = 0;
    L.ctrl = off;
    off = align_up(off + sizeof(Ctrl));
    L.partial = off;
    off = align_up(off + sizeof(double) * nparts);
    L.bg = L.bgf = 0;
    if (g->hse_subtract) {
        L.bg = off;
        off = align_up(off + sizeof(PlaneBG) * (size_t)(nz + 5));
        L.bgf = off;
        off = align_up(off + sizeof(PlaneBGT<float>) * (size_t)(nz + 5));
    }
    L.total = off;
    return L;
}

struct Slab {
    int z0, nz;
    long long N, vstride;          // interior cells, variable stride (nz + 4 planes)
    void *buf[2];                  // base of each ping-pong buffer (halo plane -2 of var 0)
    Ctrl *ctrl;
    double *partial;
    PlaneBG *bg;
    PlaneBGT<float> *bgf;
    int bc_lo, bc_hi;              // z boundaries of this slab
    int tiles_x, tiles_y;
};

// One halo copy: two planes of every variable from slab src (interior
// planes sp, sp+1) to slab dst (stored planes dp, dp+1; -2 or nz).
struct HaloCopy {
    int src, sp, dst, dp;
};

std::vector<HaloCopy> plan(const hydro_problem *g, int R)
{
    std::vector<HaloCopy> out;
    const bool per = g->bc_lo[2] == HYDRO_BC_PERIODIC;
    for (int r = 0; r < R; ++r) {
        int z0, nz, z0s, nzs;
        extent(g, R, r, &z0, &nz);
        if (r > 0 || per) {                       // low halo from the slab below
            const int s = (r - 1 + R) % R;
            extent(g, R, s, &z0s, &nzs);
            out.push_back(HaloCopy{s, nzs - 2, r, -2});
        }
        if (r < R - 1 || per) {                   // high halo from the slab above
            const int s = (r + 1) % R;
            out.push_back(HaloCopy{s, 0, r, nz});
        }
    }
    return out;
}

__global__ void dt_allreduce_kernel(Ctrl **ctrls, int R, double cfl)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double m = 0.0;
    int err = 0;
    for (int r = 0; r < R; ++r) {
        m = fmax(m, ctrls[r]->max_speed);
        err |= ctrls[r]->err;
    }
    const double dt = m > 0.0 ? cfl / m : 0.0;
    for (int r = 0; r < R; ++r) {
        ctrls[r]->max_speed = m;
        ctrls[r]->dt_next = dt;
        ctrls[r]->err |= err | (m > 0.0 && isfinite(m) ? 0 : 1);
    }
}

}  // namespace

struct hydro_slabs {
    hydro_problem g;
    int R, nvar, cur, variant, zchunk;
    int balanced;    // 0, or the balanced grid's z-chunk setting (-1: whole columns, -Z)
    size_t bytes_per;              // value size
    long long plane;
    std::vector<Slab> slab;
    std::vector<HaloCopy> copies;
    Ctrl **d_ctrls;                // device array of the slabs' control blocks
    cudaStream_t stream;
    // the slabs' step kernels run concurrently, one stream per slab,
    // forked from and joined back into `stream` every step
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork;
    double inv_dx[3], dx[3], cell_volume;
    long launches;
};

namespace {

char *interior(const hydro_slabs *S, const Slab &sl, int b)
{
    return static_cast<char *>(sl.buf[b]) + 2 * S->plane * S->bytes_per;
}

StepArgs slab_args(const hydro_slabs *S, const Slab &sl)
{
    StepArgs a{};
    a.U = interior(S, sl, S->cur);
    a.Unew = interior(S, sl, 1 - S->cur);
    for (int d = 0; d < 3; ++d) {
        a.n[d] = d == 2 ? sl.nz : S->g.n[d];
        a.bc_lo[d] = d == 2 ? sl.bc_lo : S->g.bc_lo[d];
        a.bc_hi[d] = d == 2 ? sl.bc_hi : S->g.bc_hi[d];
        a.inv_dx[d] = S->inv_dx[d];
        a.grav[d] = S->g.grav[d];
    }
    a.plane = S->plane;
    a.vstride = sl.vstride;
    a.gamma = S->g.gamma;
    a.cfl = S->g.cfl;
    a.t_end = INFINITY;
    a.step_end = LLONG_MAX;
    a.ctrl = sl.ctrl;
    a.partial = sl.partial;
    a.bgT = nullptr;
    if (S->g.hse_subtract)
        a.bgT = S->g.precision == HYDRO_FP32 ? static_cast<const void *>(sl.bgf) : static_cast<const void *>(sl.bg);
    a.zchunk = S->balanced ? S->balanced : std::min(S->zchunk, sl.nz);   // <= 0: balanced grid
    a.tiles_x = sl.tiles_x;
    fill_fp32_constants(a);
    return a;
}

AuxArgs slab_aux(const hydro_slabs *S, const Slab &sl, void *U)
{
    AuxArgs a{};
    a.U = U;
    a.ndim = 3;
    for (int d = 0; d < 3; ++d) { a.n[d] = d == 2 ? sl.nz : S->g.n[d]; a.inv_dx[d] = S->inv_dx[d]; }
    a.N = sl.N;
    a.vstride = sl.vstride;
    a.plane = S->plane;
    a.gamma = S->g.gamma;
    a.cfl = S->g.cfl;
    a.cell_volume = S->cell_volume;
    a.ctrl = sl.ctrl;
    a.partial = sl.partial;
    a.bg = S->g.hse_subtract ? sl.bg : nullptr;
    a.hse = S->g.hse_subtract;
    a.fp32 = S->g.precision == HYDRO_FP32;
    return a;
}

cudaError_t exchange(hydro_slabs *S)
{
    const size_t pb = (size_t)S->plane * S->bytes_per;
    for (const HaloCopy &c : S->copies) {
        const Slab &src = S->slab[c.src], &dst = S->slab[c.dst];
        const char *s0 = interior(S, src, S->cur) + (long long)c.sp * pb;
        char *d0 = interior(S, dst, S->cur) + (long long)c.dp * pb;
        for (int q = 0; q < S->nvar; ++q) {
            cudaError_t e = cudaMemcpyAsync(d0 + (size_t)q * dst.vstride * S->bytes_per,
                                            s0 + (size_t)q * src.vstride * S->bytes_per, 2 * pb,
                                            cudaMemcpyDeviceToDevice, S->stream);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

void release(hydro_slabs *S)
{
    for (cudaStream_t st : S->side)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : S->done)
        if (ev) cudaEventDestroy(ev);
    if (S->fork) cudaEventDestroy(S->fork);
    delete S;
}

cudaError_t make_streams(hydro_slabs *S)
{
    S->side.assign(S->R, nullptr);
    S->done.assign(S->R, nullptr);
    cudaError_t e = cudaEventCreateWithFlags(&S->fork, cudaEventDisableTiming);
    for (int r = 0; r < S->R && e == cudaSuccess; ++r) {
        e = cudaStreamCreateWithFlags(&S->side[r], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->done[r], cudaEventDisableTiming);
    }
    return e;
}

cudaError_t allreduce_dt(hydro_slabs *S)
{
    dt_allreduce_kernel<<<1, 32, 0, S->stream>>>(S->d_ctrls, S->R, S->g.cfl);
    S->launches += 1;
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int hydro_slab_extent(const hydro_problem *global, int nranks, int rank, int *z0, int *nz)
{
    if (!z0 || !nz || !valid_global(global, nranks)) return HYDRO_ERR_INVALID_ARG;
    return extent(global, nranks, rank, z0, nz) ? HYDRO_OK : HYDRO_ERR_INVALID_ARG;
}

size_t hydro_slab_state_bytes(const hydro_problem *global, int nranks, int rank)
{
    int z0, nz;
    if (!valid_global(global, nranks) || !extent(global, nranks, rank, &z0, &nz)) return 0;
    return (size_t)(global->ndim + 2) * (nz + 4) * global->n[0] * global->n[1] *
           (global->precision == HYDRO_FP32 ? 4 : 8);
}

size_t hydro_slab_workspace_bytes(const hydro_problem *global, int nranks, int rank)
{
    int z0, nz;
    if (!valid_global(global, nranks) || !extent(global, nranks, rank, &z0, &nz)) return 0;
    return slab_layout(global, nz).total + align_up(sizeof(Ctrl *) * (size_t)nranks);
}

int hydro_slabs_exchange_plan(const hydro_problem *global, int nranks, int *out, int max_copies)
{
    if (!valid_global(global, nranks)) return HYDRO_ERR_INVALID_ARG;
    std::vector<HaloCopy> p = plan(global, nranks);
    if (out) {
        if ((int)p.size() > max_copies) return HYDRO_ERR_OOM;
        for (size_t i = 0; i < p.size(); ++i) {
            out[4 * i + 0] = p[i].src;
            out[4 * i + 1] = p[i].sp;
            out[4 * i + 2] = p[i].dst;
            out[4 * i + 3] = p[i].dp;
        }
    }
    return (int)p.size();
}

int hydro_slabs_init(const hydro_problem *global, int nranks, void *const *Ua, void *const *Ub,
                     void *const *work, const double *W0, const double *bg, void *stream,
                     hydro_slabs **out)
{
    if (!out) return HYDRO_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_global(global, nranks) || !Ua || !Ub || !work || !W0) return HYDRO_ERR_INVALID_ARG;
    if (global->hse_subtract && !bg) return HYDRO_ERR_INVALID_ARG;
    if ((global->bc_lo[2] == HYDRO_BC_PERIODIC) != (global->bc_hi[2] == HYDRO_BC_PERIODIC)) return HYDRO_ERR_INVALID_ARG;
    for (int r = 0; r < nranks; ++r)
        if (!Ua[r] || !Ub[r] || !work[r] || !aligned(Ua[r]) || !aligned(Ub[r]) || !aligned(work[r]) || Ua[r] == Ub[r])
            return HYDRO_ERR_INVALID_ARG;
    hydro_slabs *S = new (std::nothrow) hydro_slabs();
    if (!S) return HYDRO_ERR_OOM;
    S->fork = nullptr;
    S->g = *global;
    S->R = nranks;
    S->nvar = 5;
    S->bytes_per = global->precision == HYDRO_FP32 ? 4 : 8;
    S->plane = (long long)global->n[0] * global->n[1];
    S->stream = static_cast<cudaStream_t>(stream);
    S->variant = global->precision == HYDRO_FP32 ? 7 : 6;   // asynchronous staging, 32 x 16 / 16 x 16
    S->cell_volume = 1.0;
    for (int d = 0; d < 3; ++d) {
        S->dx[d] = (global->hi[d] - global->lo[d]) / global->n[d];
        S->inv_dx[d] = 1.0 / S->dx[d];
        S->cell_volume *= S->dx[d];
    }
    S->copies = plan(global, nranks);
    S->slab.resize(nranks);
    const bool per = global->bc_lo[2] == HYDRO_BC_PERIODIC;
    cudaError_t e = cudaSuccess;
    int rc = HYDRO_OK;
    std::vector<Ctrl *> ctrls(nranks);
    if (make_streams(S) != cudaSuccess) rc = HYDRO_ERR_CUDA;
    for (int r = 0; r < nranks && rc == HYDRO_OK; ++r) {
        Slab &sl = S->slab[r];
        extent(global, nranks, r, &sl.z0, &sl.nz);
        sl.N = S->plane * sl.nz;
        sl.vstride = S->plane * (sl.nz + 4);
        sl.buf[0] = Ua[r];
        sl.buf[1] = Ub[r];
        const SlabLayout L = slab_layout(global, sl.nz);
        unsigned char *w = static_cast<unsigned char *>(work[r]);
        sl.ctrl = reinterpret_cast<Ctrl *>(w + L.ctrl);
        sl.partial = reinterpret_cast<double *>(w + L.partial);
        sl.bg = reinterpret_cast<PlaneBG *>(w + L.bg);
        sl.bgf = reinterpret_cast<PlaneBGT<float> *>(w + L.bgf);
        ctrls[r] = sl.ctrl;
        sl.bc_lo = (r == 0 && !per) ? global->bc_lo[2] : BC_HALO;
        sl.bc_hi = (r == nranks - 1 && !per) ? global->bc_hi[2] : BC_HALO;
        sl.tiles_x = tiles_along(global->n[0], TILE3D_SHAPES[S->variant].tx);
        sl.tiles_y = tiles_along(global->n[1], TILE3D_SHAPES[S->variant].ty);
        e = cudaMemsetAsync(w, 0, L.total, S->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(Ua[r], 0, hydro_slab_state_bytes(global, nranks, r), S->stream);
        if (e == cudaSuccess && global->hse_subtract) {
            // this slab's planes -2 .. nz+2 of the global background tables
            const int gnz = global->n[2];
            const double *rc_ = bg, *pc_ = bg + (gnz + 4), *rf_ = bg + 2 * (gnz + 4), *pf_ = bg + 2 * (gnz + 4) + (gnz + 5);
            std::vector<PlaneBG> tb(sl.nz + 5);
            std::vector<PlaneBGT<float>> tf(sl.nz + 5);
            for (int k = -2; k <= sl.nz + 2; ++k) {
                const int gk = sl.z0 + k;             // global plane, in [-2, gnz + 2]
                PlaneBG &q = tb[k + 2];
                const bool has_c = gk <= gnz + 1;
                q.rho_c = has_c ? rc_[gk + 2] : 0.0;
                q.p_c = has_c ? pc_[gk + 2] : 0.0;
                q.rho_f = rf_[gk + 2];
                q.p_f = pf_[gk + 2];
                if (has_c) {
                    q.drho = rf_[gk + 3] - rf_[gk + 2];
                    q.dp = pf_[gk + 3] - pf_[gk + 2];
                    q.B = q.dp / S->dx[2] - q.rho_c * global->grav[2];
                }
                tf[k + 2] = PlaneBGT<float>{(float)q.rho_c, (float)q.p_c, (float)q.rho_f, (float)q.p_f,
                                            (float)q.drho, (float)q.dp, (float)q.B, 0.0f};
            }
            e = cudaMemcpyAsync(sl.bg, tb.data(), sizeof(PlaneBG) * tb.size(), cudaMemcpyHostToDevice, S->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(sl.bgf, tf.data(), sizeof(PlaneBGT<float>) * tf.size(), cudaMemcpyHostToDevice,
                                    S->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
        }
        // interior initial state through the spare buffer
        const long long cap = (long long)(hydro_slab_state_bytes(global, nranks, r) / (sizeof(double) * 5));
        double *stg = static_cast<double *>(sl.buf[1]);
        const long long gN = S->plane * global->n[2];
        AuxArgs a = slab_aux(S, sl, interior(S, sl, 0));
        for (long long c0 = 0; c0 < sl.N && e == cudaSuccess; c0 += cap) {
            const long long m = std::min(cap, sl.N - c0);
            for (int q = 0; q < 5 && e == cudaSuccess; ++q)
                e = cudaMemcpyAsync(stg + (size_t)q * m, W0 + (size_t)q * gN + (size_t)sl.z0 * S->plane + c0,
                                    sizeof(double) * m, cudaMemcpyHostToDevice, S->stream);
            if (e == cudaSuccess) e = launch_init_convert(a, stg, c0, m, S->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
            S->launches += 1;
        }
        if (e == cudaSuccess) e = launch_signal(a, S->stream);
        S->launches += 1;
        if (e != cudaSuccess) rc = HYDRO_ERR_CUDA;
    }
    if (rc == HYDRO_OK) {
        // the control-block pointer table lives after slab 0's work layout
        const SlabLayout L0 = slab_layout(global, S->slab[0].nz);
        S->d_ctrls = reinterpret_cast<Ctrl **>(static_cast<unsigned char *>(work[0]) + L0.total);
        e = cudaMemcpyAsync(S->d_ctrls, ctrls.data(), sizeof(Ctrl *) * nranks, cudaMemcpyHostToDevice, S->stream);
        if (e == cudaSuccess) e = allreduce_dt(S);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
        if (e != cudaSuccess) rc = HYDRO_ERR_CUDA;
    }
    if (rc != HYDRO_OK) {
        release(S);
        return rc;
    }
    S->zchunk = 64;
    *out = S;
    return HYDRO_OK;
}

int hydro_slabs_step(hydro_slabs *S, long nsteps)
{
    nvtxRangePushA("hydro_slabs_step");
    struct Pop { ~Pop() { nvtxRangePop(); } } pop;
    if (!S || nsteps < 0) return HYDRO_ERR_INVALID_ARG;
    const bool fp32 = S->g.precision == HYDRO_FP32;
    for (long i = 0; i < nsteps; ++i) {
        cudaError_t e = exchange(S);
        if (e == cudaSuccess) e = cudaEventRecord(S->fork, S->stream);
        for (int r = 0; r < S->R && e == cudaSuccess; ++r) {
            const Slab &sl = S->slab[r];
            StepArgs a = slab_args(S, sl);
            // (the balanced grid's size is the launcher's)
            const int nch = a.zchunk > 0 ? (sl.nz + a.zchunk - 1) / a.zchunk : 1;
            dim3 grid(sl.tiles_x * sl.tiles_y, nch);
            e = cudaStreamWaitEvent(S->side[r], S->fork, 0);
            if (e == cudaSuccess)
                e = fp32 ? launch_step3d_f32(S->variant, a, grid, S->side[r], S->g.hse_subtract != 0)
                         : launch_step3d_f64(S->variant, a, grid, S->side[r], S->g.hse_subtract != 0);
            S->launches += 1;
            if (e == cudaSuccess) e = cudaEventRecord(S->done[r], S->side[r]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(S->stream, S->done[r], 0);
        }
        if (e == cudaSuccess) e = allreduce_dt(S);
        if (e != cudaSuccess) return HYDRO_ERR_CUDA;
        S->cur = 1 - S->cur;
    }
    return HYDRO_OK;
}

int hydro_slabs_get_state(hydro_slabs *S, void *host_dst)
{
    if (!S || !host_dst) return HYDRO_ERR_INVALID_ARG;
    const size_t b = S->bytes_per;
    const long long gN = S->plane * S->g.n[2];
    for (const Slab &sl : S->slab)
        for (int q = 0; q < S->nvar; ++q) {
            cudaError_t e = cudaMemcpyAsync(static_cast<char *>(host_dst) + ((size_t)q * gN + (size_t)sl.z0 * S->plane) * b,
                                            interior(S, sl, S->cur) + (size_t)q * sl.vstride * b, sl.N * b,
                                            cudaMemcpyDeviceToHost, S->stream);
            if (e != cudaSuccess) return HYDRO_ERR_CUDA;
        }
    return cudaStreamSynchronize(S->stream) == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
}

int hydro_slabs_get_fields(hydro_slabs *S, int what, double *host_dst)
{
    if (!S || !host_dst || (what != 0 && what != 1)) return HYDRO_ERR_INVALID_ARG;
    const long long gN = S->plane * S->g.n[2];
    for (const Slab &sl : S->slab) {
        // staged through this slab's spare buffer (FP64 values, 5 per cell)
        const long long cap = (long long)(sl.vstride * S->nvar * S->bytes_per / (sizeof(double) * S->nvar));
        double *stg = static_cast<double *>(sl.buf[1 - S->cur]);
        AuxArgs a = slab_aux(S, sl, interior(S, sl, S->cur));
        for (long long c0 = 0; c0 < sl.N; c0 += cap) {
            const long long m = std::min(cap, sl.N - c0);
            S->launches += 1;
            cudaError_t e = launch_fields(a, stg, c0, m, what, S->stream);
            for (int q = 0; q < S->nvar && e == cudaSuccess; ++q)
                e = cudaMemcpyAsync(host_dst + (size_t)q * gN + (size_t)sl.z0 * S->plane + c0, stg + (size_t)q * m,
                                    sizeof(double) * m, cudaMemcpyDeviceToHost, S->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
            if (e != cudaSuccess) return HYDRO_ERR_CUDA;
        }
    }
    return HYDRO_OK;
}

int hydro_slabs_reduce(hydro_slabs *S, int what, double *out)
{
    if (!S || !out) return HYDRO_ERR_INVALID_ARG;
    if (what == HYDRO_RED_TOTALS) {
        for (int q = 0; q < S->nvar; ++q) out[q] = 0.0;
        for (const Slab &sl : S->slab) {
            AuxArgs a = slab_aux(S, sl, interior(S, sl, S->cur));
            S->launches += 1;
            if (launch_totals(a, S->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
            Ctrl c;
            if (cudaMemcpyAsync(&c, sl.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, S->stream) != cudaSuccess ||
                cudaStreamSynchronize(S->stream) != cudaSuccess)
                return HYDRO_ERR_CUDA;
            for (int q = 0; q < S->nvar; ++q) out[q] += c.totals[q];
        }
        return HYDRO_OK;
    }
    Ctrl c;
    if (cudaMemcpyAsync(&c, S->slab[0].ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, S->stream) != cudaSuccess ||
        cudaStreamSynchronize(S->stream) != cudaSuccess)
        return HYDRO_ERR_CUDA;
    switch (what) {
    case HYDRO_RED_DT: out[0] = c.dt_next; break;
    case HYDRO_RED_TIME: out[0] = c.t; break;
    case HYDRO_RED_MAXSPEED: out[0] = c.max_speed; break;
    case HYDRO_RED_STEP: out[0] = (double)c.step; break;
    case HYDRO_RED_DT_LAST: out[0] = c.dt_last; break;
    default: return HYDRO_ERR_INVALID_ARG;
    }
    return c.err ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK;
}

int hydro_slabs_configure(hydro_slabs *S, int variant, int zchunk)
{
    if (!S || !tile3d_available(variant, S->g.precision == HYDRO_FP32)) return HYDRO_ERR_INVALID_ARG;
    S->variant = variant;
    S->balanced = zchunk < 0 ? std::max(zchunk, -S->g.n[2]) : 0;   // chunks of at most nz planes
    if (!S->balanced) S->zchunk = zchunk == 0 ? 64 : zchunk;
    for (Slab &sl : S->slab) {
        sl.tiles_x = tiles_along(S->g.n[0], TILE3D_SHAPES[variant].tx);
        sl.tiles_y = tiles_along(S->g.n[1], TILE3D_SHAPES[variant].ty);
    }
    return HYDRO_OK;
}

long hydro_slabs_launch_count(hydro_slabs *S) { return S ? S->launches : -1; }

int hydro_slabs_destroy(hydro_slabs *S)
{
    if (!S) return HYDRO_ERR_INVALID_ARG;
    cudaStreamSynchronize(S->stream);
    release(S);
    return HYDRO_OK;
}

}  // extern "C"
