// hydro_api.cu -- the C ABI declared in include/hydro.h: argument checking,
// workspace layout, launch configuration and host-side time control.
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "../../include/hydro.h"
#include "hydro_internal.h"
#include "launchers.h"
#include "per_device.h"
#include "pieces.h"

using namespace hydro;

struct hydro_sim {
    hydro_problem prob;
    int nvar;
    long long N, plane;
    size_t state_bytes;
    void *buf[2];
    int cur;                 // index of the buffer holding the current state
    int cur0;                // buffer index at step 0: a frozen launch moves nothing, so the state
                             // after s steps is in buf[(cur0 + s) & 1] (re-read with the control block)
    unsigned char *work;
    WorkLayout lay;
    Ctrl *ctrl;
    double *partial;
    PlaneBG *bg;
    PlaneBGT<float> *bgf;
    void *stage;             // first Runge-Kutta stage state (SSP-RK2), in the workspace
    cudaStream_t stream;
    double dx[3], inv_dx[3], cell_volume;
    int tiles_x, tiles_y;
    int variant;             // 3D tile shape (TILE3D_SHAPES index)
    int zchunk;
    int balanced;            // 3D: 0, or the balanced grid's z-chunk setting (-1: whole columns, -Z)
    long launches;
    int err_state;           // sticky host-side copy of a non-physical error
    std::vector<PlaneBG> bg_host;
    std::vector<PlaneBGT<float>> bgf_host;
};

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

bool aligned(const void *p) { return (reinterpret_cast<uintptr_t>(p) % ALIGN) == 0; }

int check_problem(const hydro_problem *p)
{
    if (!p) return HYDRO_ERR_INVALID_ARG;
    if (p->ndim != 2 && p->ndim != 3) return HYDRO_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d) {
        if (d < p->ndim) {
            if (p->n[d] < 2) return HYDRO_ERR_INVALID_ARG;
        } else if (p->n[d] != 1) {
            return HYDRO_ERR_INVALID_ARG;
        }
        if (!(p->hi[d] > p->lo[d]) || !std::isfinite(p->hi[d] - p->lo[d])) return HYDRO_ERR_INVALID_ARG;
        if (p->bc_lo[d] < 0 || p->bc_lo[d] > 2 || p->bc_hi[d] < 0 || p->bc_hi[d] > 2)
            return HYDRO_ERR_INVALID_ARG;
        if ((p->bc_lo[d] == HYDRO_BC_PERIODIC) != (p->bc_hi[d] == HYDRO_BC_PERIODIC))
            return HYDRO_ERR_INVALID_ARG;
        if (!std::isfinite(p->grav[d])) return HYDRO_ERR_INVALID_ARG;
    }
    if (p->ndim == 2 && p->grav[2] != 0.0) return HYDRO_ERR_INVALID_ARG;
    if (!(p->gamma > 1.0) || !(p->cfl > 0.0) || !std::isfinite(p->gamma) || !std::isfinite(p->cfl))
        return HYDRO_ERR_INVALID_ARG;
    if (p->precision != HYDRO_FP64 && p->precision != HYDRO_FP32) return HYDRO_ERR_INVALID_ARG;
    if (p->hse_subtract != 0 && p->hse_subtract != 1) return HYDRO_ERR_INVALID_ARG;
    if (p->scheme != HYDRO_SCHEME_HANCOCK && p->scheme != HYDRO_SCHEME_SSPRK2 && p->scheme != HYDRO_SCHEME_CTU)
        return HYDRO_ERR_INVALID_ARG;
    if (p->scheme == HYDRO_SCHEME_CTU && p->recon != HYDRO_RECON_PLM)
        return HYDRO_ERR_INVALID_ARG;
    if (p->recon != HYDRO_RECON_PLM && p->recon != HYDRO_RECON_PPM) return HYDRO_ERR_INVALID_ARG;
    if (p->recon == HYDRO_RECON_PPM) {
        // three-cell halo: every active axis needs three cells to map into
        if (p->scheme != HYDRO_SCHEME_SSPRK2 || p->hse_subtract) return HYDRO_ERR_INVALID_ARG;
        for (int d = 0; d < p->ndim; ++d)
            if (p->n[d] < 3) return HYDRO_ERR_INVALID_ARG;
    }
    if (p->hse_subtract && (p->ndim != 3 || p->grav[0] != 0.0 || p->grav[1] != 0.0))
        return HYDRO_ERR_INVALID_ARG;
    // 32-bit plane and cell indexing inside a plane; 64-bit across planes
    const long long plane = (long long)p->n[0] * p->n[1];
    if (plane > (1ll << 31) - 1) return HYDRO_ERR_INVALID_ARG;
    return HYDRO_OK;
}

int tiles_along(int n, int t) { return (n + t - 1) / t; }

int step_max_ctas(const hydro_problem *p)
{
    if (p->ndim == 2)
        return tiles_along(p->n[0], STEP2D_TX) * tiles_along(p->n[1], STEP2D_TY);
    // any tile shape, zchunk >= 1: at most nz chunks
    int m = 0;
    for (int v = 0; v < TILE3D_VARIANTS; ++v)
        m = std::max(m, tiles_along(p->n[0], TILE3D_SHAPES[v].tx) * tiles_along(p->n[1], TILE3D_SHAPES[v].ty) *
                            p->n[2]);
    for (int v = 0; v < PAIR_VARIANTS; ++v)
        m = std::max(m, tiles_along(p->n[0], PAIR_SHAPES[v].tx) * tiles_along(p->n[1], PAIR_SHAPES[v].ty) * p->n[2]);
    if (p->scheme == HYDRO_SCHEME_CTU)
        m = std::max(m, (int)ctu3d_blocks(p->n, p->precision == HYDRO_FP32));
    return m;
}

WorkLayout layout(const hydro_problem *p)
{
    WorkLayout L{};
    const long long N = (long long)p->n[0] * p->n[1] * p->n[2];
    const int aux = aux_reduce_blocks(N);
    const int nparts = std::max(step_max_ctas(p), 5 * aux);
    L.max_ctas = nparts;
    size_t off = 0;
    L.ctrl = off;
    off = align_up(off + sizeof(Ctrl));
    L.partial = off;
    off = align_up(off + sizeof(double) * (size_t)nparts);
    L.bg = off;
    off = align_up(off + (p->hse_subtract ? sizeof(PlaneBG) * (size_t)(p->n[2] + 5) : 0));
    L.bgf = off;
    off = align_up(off + (p->hse_subtract ? sizeof(PlaneBGT<float>) * (size_t)(p->n[2] + 5) : 0));
    // the first Runge-Kutta stage's state (SSP-RK2 only)
    L.stage = off;
    if (p->scheme == HYDRO_SCHEME_SSPRK2)
        off = align_up(off + (size_t)N * (p->ndim + 2) * (p->precision == HYDRO_FP32 ? 4 : 8));
    L.red = off;
    L.total = off;
    return L;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA; }

// NVTX range over an API call (visible in Nsight timelines; a no-op when no
// tool is attached)
struct ApiRange {
    explicit ApiRange(const char *name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
};

// Checkpoint file: this header, then the raw stored state.
struct CheckpointHeader {
    char magic[8];            // "HYDROCK1"
    uint32_t version;         // 1
    uint32_t header_bytes;    // sizeof(CheckpointHeader)
    hydro_problem prob;
    double t;
    long long step;
    uint64_t state_bytes;
    uint64_t checksum;        // FNV-1a (64-bit) of the state bytes
};

uint64_t fnv1a64(const unsigned char *p, size_t n)
{
    uint64_t h = 14695981039346656037ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

bool same_problem(const hydro_problem &a, const hydro_problem &b)
{
    if (a.ndim != b.ndim || a.gamma != b.gamma || a.cfl != b.cfl || a.precision != b.precision ||
        a.hse_subtract != b.hse_subtract || a.scheme != b.scheme || a.recon != b.recon)
        return false;
    for (int d = 0; d < 3; ++d)
        if (a.n[d] != b.n[d] || a.lo[d] != b.lo[d] || a.hi[d] != b.hi[d] || a.bc_lo[d] != b.bc_lo[d] ||
            a.bc_hi[d] != b.bc_hi[d] || a.grav[d] != b.grav[d])
            return false;
    return true;
}

AuxArgs aux_args(const hydro_sim *s, void *U)
{
    AuxArgs a{};
    a.U = U;
    a.ndim = s->prob.ndim;
    for (int d = 0; d < 3; ++d) { a.n[d] = s->prob.n[d]; a.inv_dx[d] = s->inv_dx[d]; }
    a.N = s->N;
    a.vstride = s->N;
    a.plane = s->plane;
    a.gamma = s->prob.gamma;
    a.cfl = s->prob.cfl;
    a.cell_volume = s->cell_volume;
    a.ctrl = s->ctrl;
    a.partial = s->partial;
    a.bg = s->prob.hse_subtract ? s->bg : nullptr;
    a.hse = s->prob.hse_subtract;
    a.fp32 = s->prob.precision == HYDRO_FP32;
    return a;
}

int default_zchunk(const hydro_sim *s)
{
    if (s->prob.ndim == 2) return 1;
    const int nz = s->prob.n[2];
    const long long tiles = (long long)s->tiles_x * s->tiles_y;
    // aim for >= 8 CTAs per SM on 152 SMs with chunks of 8..64 planes,
    // split evenly so that no chunk is much shorter than the others
    long long nch = std::max(1ll, (8ll * 152 + tiles - 1) / tiles);
    nch = std::max(nch, (long long)((nz + 63) / 64));
    nch = std::min(nch, std::max(1ll, (long long)(nz / 8)));
    return (int)((nz + nch - 1) / nch);
}

StepArgs step_args(const hydro_sim *s, double t_end)
{
    StepArgs a{};
    a.U = s->buf[s->cur];
    a.Unew = s->buf[1 - s->cur];
    for (int d = 0; d < 3; ++d) {
        a.n[d] = s->prob.n[d];
        a.bc_lo[d] = s->prob.bc_lo[d];
        a.bc_hi[d] = s->prob.bc_hi[d];
        a.inv_dx[d] = d < s->prob.ndim ? s->inv_dx[d] : 0.0;
        a.grav[d] = s->prob.grav[d];
    }
    a.plane = s->plane;
    a.vstride = s->N;
    a.gamma = s->prob.gamma;
    a.cfl = s->prob.cfl;
    a.t_end = t_end;
    a.step_end = LLONG_MAX;
    a.ctrl = s->ctrl;
    a.partial = s->partial;
    a.bgT = nullptr;
    if (s->prob.hse_subtract)
        a.bgT = s->prob.precision == HYDRO_FP32 ? static_cast<const void *>(s->bgf)
                                                : static_cast<const void *>(s->bg);
    a.U0 = nullptr;
    a.zchunk = s->balanced ? s->balanced : s->zchunk;   // <= 0: balanced grid
    a.tiles_x = s->tiles_x;
    fill_fp32_constants(a);
    return a;
}

cudaError_t launch_kernel(hydro_sim *s, const StepArgs &a, int stage)
{
    const bool fp32 = s->prob.precision == HYDRO_FP32;
    const bool hse = s->prob.hse_subtract != 0;
    s->launches += 1;
    const int recon = s->prob.recon;
    if (s->prob.ndim == 2 && s->prob.scheme == HYDRO_SCHEME_CTU)
        return launch_ctu2d(a, dim3(s->tiles_x * s->tiles_y, 1), s->stream, fp32);
    if (s->prob.ndim == 2)
        return launch_step2d(a, dim3(s->tiles_x * s->tiles_y, 1), s->stream, fp32, stage, recon);
    if (s->prob.scheme == HYDRO_SCHEME_CTU) return launch_ctu3d(a, s->stream, fp32, hse);
    const dim3 grid(s->tiles_x * s->tiles_y, (s->prob.n[2] + s->zchunk - 1) / s->zchunk);
    if (stage == STAGE_HANCOCK && pair_variant(s->variant))
        return launch_pair3d(s->variant - PAIR_VARIANT0, a, grid, s->stream, hse);
    if (stage == STAGE_HANCOCK)
        return fp32 ? launch_step3d_f32(s->variant, a, grid, s->stream, hse)
                    : launch_step3d_f64(s->variant, a, grid, s->stream, hse);
    return fp32 ? launch_stage3d_f32(stage, s->variant, a, grid, s->stream, hse, recon)
                : launch_stage3d_f64(stage, s->variant, a, grid, s->stream, hse, recon);
}

int launch_step(hydro_sim *s, double t_end)
{
    StepArgs a = step_args(s, t_end);
    cudaError_t e;
    if (s->prob.scheme == HYDRO_SCHEME_SSPRK2) {
        // U1 = U + dt L(U) into the stage buffer, then
        // U^{n+1} = (U + U1 + dt L(U1)) / 2 into the other state buffer
        StepArgs a1 = a;
        a1.Unew = s->stage;
        e = launch_kernel(s, a1, STAGE_RK1);
        if (e == cudaSuccess) {
            StepArgs a2 = a;
            a2.U = s->stage;
            a2.U0 = s->buf[s->cur];
            e = launch_kernel(s, a2, STAGE_RK2);
        }
    } else {
        e = launch_kernel(s, a, STAGE_HANCOCK);
    }
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    s->cur = 1 - s->cur;
    return HYDRO_OK;
}

int read_ctrl(hydro_sim *s, Ctrl *out)
{
    cudaError_t e = cudaMemcpyAsync(out, s->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    if (out->err) s->err_state = 1;
    s->cur = (int)((s->cur0 + (out->step & 1)) & 1);
    return HYDRO_OK;
}

int recompute_dt(hydro_sim *s)
{
    AuxArgs a = aux_args(s, s->buf[s->cur]);
    s->launches += 1;
    return cuda_status(launch_signal(a, s->stream));
}

// Stage a host FP64 array (nvar planes of N) through the spare buffer in
// chunks; fn(c0, m, staging) is called for each chunk after its upload.
template <typename F>
int staged_upload(hydro_sim *s, const double *host, F fn)
{
    const long long cap = (long long)(s->state_bytes / (sizeof(double) * s->nvar));
    double *stg = static_cast<double *>(s->buf[1 - s->cur]);
    for (long long c0 = 0; c0 < s->N; c0 += cap) {
        const long long m = std::min(cap, s->N - c0);
        for (int q = 0; q < s->nvar; ++q) {
            cudaError_t e = cudaMemcpyAsync(stg + (size_t)q * m, host + (size_t)q * s->N + c0,
                                            sizeof(double) * m, cudaMemcpyHostToDevice, s->stream);
            if (e != cudaSuccess) return HYDRO_ERR_CUDA;
        }
        int rc = fn(c0, m, stg);
        if (rc) return rc;
        // the next chunk's upload must not overwrite staging still being read
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
    }
    return HYDRO_OK;
}

}  // namespace

extern "C" {

size_t hydro_state_bytes(const hydro_problem *prob)
{
    if (check_problem(prob)) return 0;
    const size_t N = (size_t)prob->n[0] * prob->n[1] * prob->n[2];
    return N * (prob->ndim + 2) * (prob->precision == HYDRO_FP32 ? 4 : 8);
}

size_t hydro_workspace_bytes(const hydro_problem *prob)
{
    if (check_problem(prob)) return 0;
    return layout(prob).total;
}

}  // extern "C"

namespace {

// hydro_init and hydro_init_conserved: host0 holds total primitive
// (conserved = false) or total conserved (conserved = true) FP64 variables.
int init_impl(const hydro_problem *prob, void *Ua, void *Ub, void *work, const double *W0,
              const double *bg, void *stream, hydro_sim **out, bool conserved)
{
    if (!out) return HYDRO_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = check_problem(prob);
    if (rc) return rc;
    if (!Ua || !Ub || !work || !W0 || Ua == Ub) return HYDRO_ERR_INVALID_ARG;
    if (!aligned(Ua) || !aligned(Ub) || !aligned(work)) return HYDRO_ERR_INVALID_ARG;
    if (prob->hse_subtract && !bg) return HYDRO_ERR_INVALID_ARG;

    hydro_sim *s = new (std::nothrow) hydro_sim();
    if (!s) return HYDRO_ERR_OOM;
    s->prob = *prob;
    s->nvar = prob->ndim + 2;
    s->plane = (long long)prob->n[0] * prob->n[1];
    s->N = s->plane * prob->n[2];
    s->state_bytes = hydro_state_bytes(prob);
    s->buf[0] = Ua;
    s->buf[1] = Ub;
    s->cur = 0;
    s->cur0 = 0;
    s->work = static_cast<unsigned char *>(work);
    s->lay = layout(prob);
    s->ctrl = reinterpret_cast<Ctrl *>(s->work + s->lay.ctrl);
    s->partial = reinterpret_cast<double *>(s->work + s->lay.partial);
    s->bg = reinterpret_cast<PlaneBG *>(s->work + s->lay.bg);
    s->bgf = reinterpret_cast<PlaneBGT<float> *>(s->work + s->lay.bgf);
    s->stage = s->work + s->lay.stage;
    s->stream = static_cast<cudaStream_t>(stream);
    s->cell_volume = 1.0;
    for (int d = 0; d < 3; ++d) {
        s->dx[d] = (prob->hi[d] - prob->lo[d]) / prob->n[d];
        s->inv_dx[d] = 1.0 / s->dx[d];
        if (d < prob->ndim) s->cell_volume *= s->dx[d];
    }
    if (prob->ndim == 2) {
        s->tiles_x = tiles_along(prob->n[0], STEP2D_TX);
        s->tiles_y = tiles_along(prob->n[1], STEP2D_TY);
    } else {
        // the autotuner's usual choice on GB300: asynchronous staging with
        // 32 x 16 tiles (FP32) or 16 x 16 tiles (FP64)
        s->variant = prob->precision == HYDRO_FP32 ? 7 : 6;
        s->tiles_x = tiles_along(prob->n[0], TILE3D_SHAPES[s->variant].tx);
        s->tiles_y = tiles_along(prob->n[1], TILE3D_SHAPES[s->variant].ty);
    }
    s->zchunk = default_zchunk(s);

    cudaError_t e = cudaMemsetAsync(s->work, 0, s->lay.total, s->stream);
    if (e != cudaSuccess) { delete s; return HYDRO_ERR_CUDA; }

    if (prob->hse_subtract) {
        // per-plane FP64 background constants for planes -2 .. nz+2
        const int nz = prob->n[2];
        const double *rc_ = bg, *pc_ = bg + (nz + 4), *rf_ = bg + 2 * (nz + 4),
                     *pf_ = bg + 2 * (nz + 4) + (nz + 5);
        s->bg_host.assign(nz + 5, PlaneBG{});
        for (int k = -2; k <= nz + 2; ++k) {
            PlaneBG &b = s->bg_host[k + 2];
            const bool has_c = k <= nz + 1;
            b.rho_c = has_c ? rc_[k + 2] : 0.0;
            b.p_c = has_c ? pc_[k + 2] : 0.0;
            b.rho_f = rf_[k + 2];
            b.p_f = pf_[k + 2];
            if (has_c) {
                b.drho = rf_[k + 3] - rf_[k + 2];
                b.dp = pf_[k + 3] - pf_[k + 2];
                b.B = b.dp / s->dx[2] - b.rho_c * prob->grav[2];
            }
            if (!std::isfinite(b.rho_c) || !std::isfinite(b.p_c) || !std::isfinite(b.rho_f) ||
                !std::isfinite(b.p_f)) {
                delete s;
                return HYDRO_ERR_INVALID_ARG;
            }
        }
        e = cudaMemcpyAsync(s->bg, s->bg_host.data(), sizeof(PlaneBG) * s->bg_host.size(),
                            cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) { delete s; return HYDRO_ERR_CUDA; }
        // the same constants rounded once to FP32 for the FP32 step
        s->bgf_host.resize(s->bg_host.size());
        for (size_t i = 0; i < s->bg_host.size(); ++i) {
            const PlaneBG &b = s->bg_host[i];
            s->bgf_host[i] = PlaneBGT<float>{(float)b.rho_c, (float)b.p_c, (float)b.rho_f, (float)b.p_f,
                                             (float)b.drho, (float)b.dp, (float)b.B, 0.0f};
        }
        e = cudaMemcpyAsync(s->bgf, s->bgf_host.data(), sizeof(PlaneBGT<float>) * s->bgf_host.size(),
                            cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) { delete s; return HYDRO_ERR_CUDA; }
    }

    AuxArgs a = aux_args(s, s->buf[s->cur]);
    a.conserved_in = conserved ? 1 : 0;
    rc = staged_upload(s, W0, [&](long long c0, long long m, double *stg) {
        s->launches += 1;
        return cuda_status(launch_init_convert(a, stg, c0, m, s->stream));
    });
    if (rc == HYDRO_OK) rc = recompute_dt(s);
    Ctrl c;
    if (rc == HYDRO_OK) rc = read_ctrl(s, &c);
    if (rc != HYDRO_OK) { delete s; return rc; }
    *out = s;
    return c.err ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK;
}

}  // namespace

extern "C" {

int hydro_init(const hydro_problem *prob, void *Ua, void *Ub, void *work, const double *W0,
               const double *bg, void *stream, hydro_sim **out)
{
    ApiRange range("hydro_init");
    return init_impl(prob, Ua, Ub, work, W0, bg, stream, out, false);
}

int hydro_init_conserved(const hydro_problem *prob, void *Ua, void *Ub, void *work, const double *U0,
                         const double *bg, void *stream, hydro_sim **out)
{
    ApiRange range("hydro_init_conserved");
    return init_impl(prob, Ua, Ub, work, U0, bg, stream, out, true);
}

int hydro_step(hydro_sim *s, double *dt_taken)
{
    ApiRange range("hydro_step");
    if (!s) return HYDRO_ERR_INVALID_ARG;
    if (s->err_state) return HYDRO_ERR_NONPHYSICAL;
    int rc = launch_step(s, INFINITY);
    if (rc) return rc;
    if (dt_taken) {
        Ctrl c;
        rc = read_ctrl(s, &c);
        if (rc) return rc;
        *dt_taken = c.dt_last;
        if (c.err) return HYDRO_ERR_NONPHYSICAL;
    }
    return HYDRO_OK;
}

int hydro_advance_to(hydro_sim *s, double t_end, long max_steps, long *nsteps_out, double *t_out)
{
    ApiRange range("hydro_advance_to");
    if (!s || !std::isfinite(t_end) || max_steps < 0) return HYDRO_ERR_INVALID_ARG;
    if (s->err_state) return HYDRO_ERR_NONPHYSICAL;
    Ctrl c;
    int rc = read_ctrl(s, &c);
    if (rc) return rc;
    const long long step0 = c.step;
    long launched = 0;
    long batch = 4;
    while (c.t < t_end && c.step - step0 < max_steps && !c.err) {
        // launch up to `batch` steps, never more than the steps still allowed;
        // launches after t_end is reached carry the state over unchanged
        const long allowed = max_steps - (long)(c.step - step0);
        const long nb = std::min(batch, allowed);
        for (long i = 0; i < nb; ++i) {
            rc = launch_step(s, t_end);
            if (rc) return rc;
            ++launched;
        }
        rc = read_ctrl(s, &c);
        if (rc) return rc;
        batch = std::min(batch * 2, 64l);
        // estimate of the steps still needed keeps the overshoot small
        if (c.dt_next > 0.0 && c.t < t_end) {
            const double need = std::ceil((t_end - c.t) / c.dt_next);
            if (need < batch) batch = std::max(1l, (long)need);
        }
    }
    if (nsteps_out) *nsteps_out = (long)(c.step - step0);
    if (t_out) *t_out = c.t;
    return c.err ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK;
}

int hydro_reduce(hydro_sim *s, int what, double *out)
{
    ApiRange range("hydro_reduce");
    if (!s || !out) return HYDRO_ERR_INVALID_ARG;
    Ctrl c;
    int rc;
    if (what == HYDRO_RED_TOTALS) {
        AuxArgs a = aux_args(s, s->buf[s->cur]);
        s->launches += 1;
        rc = cuda_status(launch_totals(a, s->stream));
        if (rc) return rc;
    } else if (what < HYDRO_RED_DT || what > HYDRO_RED_DT_LAST) {
        return HYDRO_ERR_INVALID_ARG;
    }
    rc = read_ctrl(s, &c);
    if (rc) return rc;
    switch (what) {
    case HYDRO_RED_TOTALS: for (int q = 0; q < s->nvar; ++q) out[q] = c.totals[q]; break;
    case HYDRO_RED_DT: out[0] = c.dt_next; break;
    case HYDRO_RED_TIME: out[0] = c.t; break;
    case HYDRO_RED_MAXSPEED: out[0] = c.max_speed; break;
    case HYDRO_RED_STEP: out[0] = (double)c.step; break;
    case HYDRO_RED_DT_LAST: out[0] = c.dt_last; break;
    }
    return c.err ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK;
}

void *hydro_current(hydro_sim *s) { return s ? s->buf[s->cur] : nullptr; }

int hydro_get_state(hydro_sim *s, void *host_dst)
{
    if (!s || !host_dst) return HYDRO_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(host_dst, s->buf[s->cur], s->state_bytes, cudaMemcpyDeviceToHost,
                                    s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_status(e);
}

int hydro_set_state(hydro_sim *s, const void *host_src, double t, long step)
{
    if (!s || !host_src || !std::isfinite(t) || step < 0) return HYDRO_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(s->buf[s->cur], host_src, s->state_bytes, cudaMemcpyHostToDevice,
                                    s->stream);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    Ctrl c{};
    c.t = t;
    c.step = step;
    e = cudaMemcpyAsync(s->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    s->err_state = 0;
    s->cur0 = (int)((s->cur + (step & 1)) & 1);
    int rc = recompute_dt(s);
    if (rc) return rc;
    rc = read_ctrl(s, &c);   // also orders the host copies before return
    if (rc) return rc;
    return c.err ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK;
}

int hydro_get_fields(hydro_sim *s, int what, double *host_dst)
{
    if (!s || !host_dst || (what != 0 && what != 1)) return HYDRO_ERR_INVALID_ARG;
    const long long cap = (long long)(s->state_bytes / (sizeof(double) * s->nvar));
    double *stg = static_cast<double *>(s->buf[1 - s->cur]);
    AuxArgs a = aux_args(s, s->buf[s->cur]);
    for (long long c0 = 0; c0 < s->N; c0 += cap) {
        const long long m = std::min(cap, s->N - c0);
        s->launches += 1;
        cudaError_t e = launch_fields(a, stg, c0, m, what, s->stream);
        for (int q = 0; q < s->nvar && e == cudaSuccess; ++q)
            e = cudaMemcpyAsync(host_dst + (size_t)q * s->N + c0, stg + (size_t)q * m,
                                sizeof(double) * m, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    }
    return HYDRO_OK;
}

int hydro_debug_poke(hydro_sim *s, int var, long cell, double v)
{
    if (!s || var < 0 || var >= s->nvar || cell < 0 || cell >= s->N) return HYDRO_ERR_INVALID_ARG;
    AuxArgs a = aux_args(s, s->buf[s->cur]);
    s->launches += 1;
    cudaError_t e = launch_poke(a, var, cell, v, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return cuda_status(e);
}

int hydro_set_zchunk(hydro_sim *s, int zchunk)
{
    if (!s) return HYDRO_ERR_INVALID_ARG;
    if (zchunk < 0) {
        // the balanced grid (HYDRO_ZCHUNK_BALANCED: over whole columns; -Z:
        // over Z-plane chunks): 3D MUSCL-Hancock and SSP-RK2 kernels of tile
        // variants 0..7 only
        if (s->prob.ndim != 3 || s->prob.scheme == HYDRO_SCHEME_CTU || pair_variant(s->variant))
            return HYDRO_ERR_INVALID_ARG;
        s->balanced = std::max(zchunk, -s->prob.n[2]);   // chunks of at most nz planes
        return HYDRO_OK;
    }
    if (s->prob.ndim == 2) return zchunk <= 1 ? HYDRO_OK : HYDRO_ERR_INVALID_ARG;
    s->zchunk = zchunk == 0 ? default_zchunk(s) : std::min(zchunk, s->prob.n[2]);
    s->balanced = 0;
    return HYDRO_OK;
}

int hydro_set_tile(hydro_sim *s, int variant)
{
    if (!s) return HYDRO_ERR_INVALID_ARG;
    if (s->prob.ndim == 2) return variant == 0 ? HYDRO_OK : HYDRO_ERR_INVALID_ARG;
    const bool fp32 = s->prob.precision == HYDRO_FP32;
    if (pair_variant(variant)) {
        // paired-cell tiles: FP32 MUSCL-Hancock only
        if (!fp32 || s->prob.scheme != HYDRO_SCHEME_HANCOCK) return HYDRO_ERR_INVALID_ARG;
    } else if (!tile3d_available(variant, fp32)) {
        return HYDRO_ERR_INVALID_ARG;
    }
    // the other integrators take only the shape of variants 0..7
    if (s->prob.scheme != HYDRO_SCHEME_HANCOCK && pair_variant(variant)) return HYDRO_ERR_INVALID_ARG;
    s->variant = variant;
    if (pair_variant(variant)) s->balanced = 0;   // the paired kernel has z-chunks only
    s->tiles_x = tiles_along(s->prob.n[0], tile_shape(variant).tx);
    s->tiles_y = tiles_along(s->prob.n[1], tile_shape(variant).ty);
    return HYDRO_OK;
}

int hydro_debug_pieces(int zchunk, long long tiles, int nz, int tile, int chunk, long long G, long long b,
                       int *out, int max_pieces)
{
    if (!out || tiles <= 0 || nz <= 0 || max_pieces < 0) return HYDRO_ERR_INVALID_ARG;
    if (zchunk > 0 && (tile < 0 || tile >= tiles || chunk < 0 || (long long)chunk * zchunk >= nz))
        return HYDRO_ERR_INVALID_ARG;
    if (zchunk <= 0 && (G <= 0 || b < 0 || b >= G)) return HYDRO_ERR_INVALID_ARG;
    PieceIter it(zchunk, tiles, nz, tile, chunk, G, b);
    int n = 0, t, z0, z1;
    while (it.next(t, z0, z1)) {
        if (n < max_pieces) {
            out[3 * n] = t;
            out[3 * n + 1] = z0;
            out[3 * n + 2] = z1;
        }
        ++n;
    }
    return n;
}

int hydro_tile_shape(int variant, int *tx, int *ty)
{
    if (!tx || !ty || !(pair_variant(variant) || (variant >= 0 && variant < TILE3D_VARIANTS)))
        return HYDRO_ERR_INVALID_ARG;
    *tx = tile_shape(variant).tx;
    *ty = tile_shape(variant).ty;
    return HYDRO_OK;
}

long hydro_launch_count(hydro_sim *s) { return s ? s->launches : -1; }

int hydro_checkpoint_save(hydro_sim *s, const char *path)
{
    if (!s || !path) return HYDRO_ERR_INVALID_ARG;
    ApiRange range("hydro_checkpoint_save");
    Ctrl c;
    int rc = read_ctrl(s, &c);
    if (rc) return rc;
    std::vector<unsigned char> state(s->state_bytes);
    rc = hydro_get_state(s, state.data());
    if (rc) return rc;
    CheckpointHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "HYDROCK1", 8);
    h.version = 1;
    h.header_bytes = sizeof(CheckpointHeader);
    h.prob = s->prob;
    h.t = c.t;
    h.step = c.step;
    h.state_bytes = s->state_bytes;
    h.checksum = fnv1a64(state.data(), state.size());
    FILE *f = std::fopen(path, "wb");
    if (!f) return HYDRO_ERR_INVALID_ARG;
    const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(state.data(), 1, state.size(), f) == state.size();
    return (std::fclose(f) == 0 && ok) ? HYDRO_OK : HYDRO_ERR_INVALID_ARG;
}

int hydro_checkpoint_load(hydro_sim *s, const char *path)
{
    if (!s || !path) return HYDRO_ERR_INVALID_ARG;
    ApiRange range("hydro_checkpoint_load");
    FILE *f = std::fopen(path, "rb");
    if (!f) return HYDRO_ERR_INVALID_ARG;
    CheckpointHeader h;
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, "HYDROCK1", 8) == 0 && h.version == 1 &&
              h.header_bytes == sizeof(CheckpointHeader) && same_problem(h.prob, s->prob) &&
              h.state_bytes == s->state_bytes && std::isfinite(h.t) && h.step >= 0;
    std::vector<unsigned char> state;
    if (ok) {
        state.resize(h.state_bytes);
        ok = std::fread(state.data(), 1, state.size(), f) == state.size() &&
             fnv1a64(state.data(), state.size()) == h.checksum;
    }
    std::fclose(f);
    if (!ok) return HYDRO_ERR_INVALID_ARG;
    return hydro_set_state(s, state.data(), h.t, (long)h.step);
}

int hydro_selftest_math(int which, const double *x, const double *y, double *out, long n, void *stream)
{
    if (which < 0 || which > 3 || !x || !out || n < 0 || ((which == 1 || which == 3) && !y))
        return HYDRO_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_math(which, x, y, out, n, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

int hydro_selftest_device_once(const int *devs, int n, int fail_dev, int threads, int ndev,
                               int *once_calls, int *value_calls, int *values)
{
    if (!devs || n < 0 || threads < 1 || threads > 64 || ndev < 1 || ndev > MAX_DEVICES || !once_calls ||
        !value_calls || !values)
        return HYDRO_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (devs[i] < 0 || devs[i] >= ndev) return HYDRO_ERR_INVALID_ARG;
    PerDeviceOnce once;
    PerDeviceInt cache;
    std::vector<std::atomic<int>> oc(ndev), vc(ndev);
    for (int d = 0; d < ndev; ++d) { oc[d] = 0; vc[d] = 0; values[d] = 0; }
    std::atomic<int> bad{0};
    auto walk = [&] {
        for (int i = 0; i < n; ++i) {
            const int d = devs[i];
            // the set-up of fail_dev fails on its first attempt and must be retried
            const cudaError_t e = once.run(d, [&] {
                const int attempt = oc[d].fetch_add(1);
                return (d == fail_dev && attempt == 0) ? cudaErrorUnknown : cudaSuccess;
            });
            int v = 0;
            const cudaError_t f = cache.get(d, [&](int *out) {
                const int attempt = vc[d].fetch_add(1);
                if (d == fail_dev && attempt == 0) return cudaErrorUnknown;
                *out = 100 + d;
                return cudaSuccess;
            }, &v);
            if (f == cudaSuccess && v != 100 + d) bad.fetch_add(1);
            if (f == cudaSuccess) values[d] = v;
            (void)e;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(walk);
    walk();
    for (auto &th : pool) th.join();
    for (int d = 0; d < ndev; ++d) { once_calls[d] = oc[d]; value_calls[d] = vc[d]; }
    return bad.load() ? HYDRO_ERR_STATE : HYDRO_OK;
}

int hydro_destroy(hydro_sim *s)
{
    if (!s) return HYDRO_ERR_INVALID_ARG;
    cudaStreamSynchronize(s->stream);
    delete s;
    return HYDRO_OK;
}

const char *hydro_strerror(int status)
{
    switch (status) {
    case HYDRO_OK: return "ok";
    case HYDRO_ERR_INVALID_ARG: return "invalid argument";
    case HYDRO_ERR_OOM: return "buffer too small";
    case HYDRO_ERR_CUDA: return "CUDA error";
    case HYDRO_ERR_NONPHYSICAL: return "non-physical state (density or pressure not positive or not finite)";
    case HYDRO_ERR_TIMEOUT: return "bounded device wait timed out";
    case HYDRO_ERR_STATE: return "call not valid in the current state";
    default: return "unknown status";
    }
}

}  // extern "C"
