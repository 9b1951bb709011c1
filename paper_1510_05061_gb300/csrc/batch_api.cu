// batch_api.cu -- batched solves: many independent, uneven instances
// advanced together, one persistent launch per step over a device work list
// (one launch for the 3D instances, one for the 2D ones), replayed from a
// captured CUDA graph.  Instances may join and leave between steps (the
// continuous-batching server uses that); the work lists and the graph are
// rebuilt lazily when membership or configuration changes.
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

// Largest work-item count of one instance over every tile shape and any
// z-chunk >= 1.
size_t max_items_of(const hydro_problem &p)
{
    if (p.ndim == 2) return (size_t)tiles_along(p.n[0], BATCH2D_TX) * tiles_along(p.n[1], BATCH2D_TY);
    size_t m = 0;
    for (int v = 0; v < TILE3D_VARIANTS; ++v)
        m = std::max(m, (size_t)tiles_along(p.n[0], TILE3D_SHAPES[v].tx) *
                            tiles_along(p.n[1], TILE3D_SHAPES[v].ty) * p.n[2]);
    return m;
}

// Per-instance work buffer: time control, partial slots, background tables.
struct InstLayout {
    size_t ctrl, partial, bg, bgf, total;
};

InstLayout inst_layout(const hydro_problem &p)
{
    InstLayout L{};
    const long long N = (long long)p.n[0] * p.n[1] * p.n[2];
    const size_t nparts = std::max(max_items_of(p), (size_t)5 * aux_reduce_blocks(N));
    size_t off = 0;
    L.ctrl = off;
    off = align_up(off + sizeof(Ctrl));
    L.partial = off;
    off = align_up(off + sizeof(double) * nparts);
    L.bg = L.bgf = 0;
    if (p.hse_subtract) {
        L.bg = off;
        off = align_up(off + sizeof(PlaneBG) * (size_t)(p.n[2] + 5));
        L.bgf = off;
        off = align_up(off + sizeof(PlaneBGT<float>) * (size_t)(p.n[2] + 5));
    }
    L.total = off;
    return L;
}

// Shared work buffer: instance table and the two item lists.
struct BatchLayout {
    size_t insts, items3, items2, total;
};

BatchLayout batch_layout(int max_instances, long long cap3, long long cap2)
{
    BatchLayout L{};
    size_t off = 0;
    L.insts = off;
    off = align_up(off + sizeof(BatchInst) * (size_t)max_instances);
    L.items3 = off;
    off = align_up(off + sizeof(BatchItem) * (size_t)cap3);
    L.items2 = off;
    off = align_up(off + sizeof(BatchItem) * (size_t)cap2);
    L.total = off;
    return L;
}

struct InstInfo {
    bool active;
    hydro_problem prob;
    long long N, plane;
    int nvar;
    size_t state_bytes;
    void *buf[2];
    Ctrl *ctrl;
    double *partial;
    PlaneBG *bg;
    PlaneBGT<float> *bgf;
    double dx[3], inv_dx[3], cell_volume;
    long long step_end;
    size_t items;           // max_items_of(prob)
};

AuxArgs aux_for(const InstInfo &I, void *U)
{
    AuxArgs a{};
    a.U = U;
    a.ndim = I.prob.ndim;
    for (int d = 0; d < 3; ++d) { a.n[d] = I.prob.n[d]; a.inv_dx[d] = I.inv_dx[d]; }
    a.N = I.N;
    a.vstride = I.N;
    a.plane = I.plane;
    a.gamma = I.prob.gamma;
    a.cfl = I.prob.cfl;
    a.cell_volume = I.cell_volume;
    a.ctrl = I.ctrl;
    a.partial = I.partial;
    a.bg = I.prob.hse_subtract ? I.bg : nullptr;
    a.hse = I.prob.hse_subtract;
    a.fp32 = I.prob.precision == HYDRO_FP32;
    return a;
}

}  // namespace

struct hydro_batch {
    int max_instances;
    long long cap3, cap2;
    int precision, hse3;       // hse3 = -1 until the first 3D instance fixes it
    std::vector<InstInfo> inst;
    unsigned char *work;
    BatchLayout lay;
    cudaStream_t stream;
    int parity;                // buffer index holding every instance's current state
    int variant, zchunk;       // zchunk 0 = default
    bool dirty;                // work lists / graph need a rebuild
    bool use_graph;
    std::vector<BatchInst> host_insts;
    std::vector<BatchItem> host_items3, host_items2;
    BatchInst *d_insts;
    BatchItem *d_items3, *d_items2;
    int nitems3, nitems2, grid3, grid2;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool graph_ok;
    long launches;
    std::vector<void *> owned_inst_work;   // convenience init: instance buffers inside `work`
};

namespace {

void drop_graph(hydro_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_ok = false;
}

cudaError_t launch_once(hydro_batch *b, int parity)
{
    cudaError_t e = cudaSuccess;
    if (b->nitems3 > 0)
        e = launch_batch3d(b->variant, b->precision == HYDRO_FP32, b->hse3 == 1, b->d_insts, b->d_items3,
                           b->nitems3, parity, b->grid3, b->stream);
    if (e == cudaSuccess && b->nitems2 > 0)
        e = launch_batch2d(b->precision == HYDRO_FP32, b->d_insts, b->d_items2, b->nitems2, parity,
                           b->grid2, b->stream);
    return e;
}

int effective_zchunk(const hydro_batch *b)
{
    if (b->zchunk > 0) return b->zchunk;
    // a few planes per item keeps the item count high enough for balance
    // across the SMs and the chunk-end overhead (two extra planes) small
    long long cells = 0;
    for (const InstInfo &I : b->inst)
        if (I.active && I.prob.ndim == 3) cells += I.N;
    return cells > (1ll << 24) ? 16 : 8;
}

// Rebuild the work lists and per-instance arguments, upload them and
// capture the two-launch (both parities) graph.
int rebuild(hydro_batch *b)
{
    const TileShape ts = TILE3D_SHAPES[b->variant];
    const int zdef = effective_zchunk(b);
    b->host_insts.assign(b->max_instances, BatchInst{});
    b->host_items3.clear();
    b->host_items2.clear();
    for (int i = 0; i < (int)b->inst.size(); ++i) {
        const InstInfo &I = b->inst[i];
        if (!I.active) continue;
        const hydro_problem &p = I.prob;
        const bool is3 = p.ndim == 3;
        const int tx = is3 ? ts.tx : BATCH2D_TX, ty = is3 ? ts.ty : BATCH2D_TY;
        const int tiles_x = tiles_along(p.n[0], tx), tiles_y = tiles_along(p.n[1], ty);
        const int zc = is3 ? std::min(zdef, p.n[2]) : 1;
        const int nch = is3 ? (p.n[2] + zc - 1) / zc : 1;
        BatchInst &bi = b->host_insts[i];
        bi.nitems = tiles_x * tiles_y * nch;
        for (int par = 0; par < 2; ++par) {
            StepArgs &a = bi.a[par];
            a = StepArgs{};
            a.U = I.buf[par];
            a.Unew = I.buf[1 - par];
            for (int d = 0; d < 3; ++d) {
                a.n[d] = p.n[d];
                a.bc_lo[d] = p.bc_lo[d];
                a.bc_hi[d] = p.bc_hi[d];
                a.inv_dx[d] = d < p.ndim ? I.inv_dx[d] : 0.0;
                a.grav[d] = p.grav[d];
            }
            a.plane = I.plane;
            a.vstride = I.N;
            a.gamma = p.gamma;
            a.cfl = p.cfl;
            a.t_end = INFINITY;
            a.step_end = I.step_end;
            a.ctrl = I.ctrl;
            a.partial = I.partial;
            a.bgT = nullptr;
            if (p.hse_subtract)
                a.bgT = b->precision == HYDRO_FP32 ? static_cast<const void *>(I.bgf)
                                                   : static_cast<const void *>(I.bg);
            a.zchunk = zc;
            a.tiles_x = tiles_x;
            fill_fp32_constants(a);
        }
        std::vector<BatchItem> &lst = is3 ? b->host_items3 : b->host_items2;
        int local = 0;
        for (int c = 0; c < nch; ++c)
            for (int t = 0; t < tiles_x * tiles_y; ++t) lst.push_back(BatchItem{i, t, c, local++});
    }
    if ((long long)b->host_items3.size() > b->cap3 || (long long)b->host_items2.size() > b->cap2)
        return HYDRO_ERR_OOM;
    b->nitems3 = (int)b->host_items3.size();
    b->nitems2 = (int)b->host_items2.size();
    cudaError_t e = cudaMemcpyAsync(b->d_insts, b->host_insts.data(), sizeof(BatchInst) * b->max_instances,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && b->nitems3)
        e = cudaMemcpyAsync(b->d_items3, b->host_items3.data(), sizeof(BatchItem) * b->nitems3,
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && b->nitems2)
        e = cudaMemcpyAsync(b->d_items2, b->host_items2.data(), sizeof(BatchItem) * b->nitems2,
                            cudaMemcpyHostToDevice, b->stream);
    // the host vectors are staging for these copies; they may change on the
    // next rebuild only after the copies are done
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    const bool fp32 = b->precision == HYDRO_FP32;
    b->grid3 = b->nitems3 ? std::max(1, std::min(b->nitems3, batch3d_max_grid(b->variant, fp32, b->hse3 == 1))) : 0;
    b->grid2 = b->nitems2 ? std::max(1, std::min(b->nitems2, batch2d_max_grid(fp32))) : 0;

    drop_graph(b);
    if (b->use_graph && b->stream != nullptr && (b->nitems3 || b->nitems2)) {
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e0 = launch_once(b, 0);
            cudaError_t e1 = e0 == cudaSuccess ? launch_once(b, 1) : e0;
            e = cudaStreamEndCapture(b->stream, &b->graph);
            if (e == cudaSuccess && e1 == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            else if (e == cudaSuccess) e = e1;
            b->graph_ok = e == cudaSuccess;
        }
        if (!b->graph_ok) {
            drop_graph(b);
            cudaGetLastError();   // capture failures are not sticky: launch directly instead
        }
    }
    b->dirty = false;
    return HYDRO_OK;
}

int add_instance(hydro_batch *b, const hydro_problem *prob, void *Ua, void *Ub, void *inst_work,
                 const double *W0, const double *bg, long long step_end, int *id_out)
{
    if (!prob || !Ua || !Ub || !inst_work || !W0 || Ua == Ub) return HYDRO_ERR_INVALID_ARG;
    if (!aligned(Ua) || !aligned(Ub) || !aligned(inst_work)) return HYDRO_ERR_INVALID_ARG;
    if (hydro_state_bytes(prob) == 0 || prob->precision != b->precision) return HYDRO_ERR_INVALID_ARG;
    if (prob->scheme != HYDRO_SCHEME_HANCOCK) return HYDRO_ERR_INVALID_ARG;   // batches step MUSCL-Hancock
    if (prob->hse_subtract && !bg) return HYDRO_ERR_INVALID_ARG;
    if (prob->ndim == 3 && b->hse3 >= 0 && prob->hse_subtract != b->hse3) {
        // one launch serves all 3D instances: one mode per batch
        bool any3 = false;
        for (const InstInfo &J : b->inst) any3 |= J.active && J.prob.ndim == 3;
        if (any3) return HYDRO_ERR_INVALID_ARG;
    }
    int slot = -1;
    for (int i = 0; i < (int)b->inst.size(); ++i)
        if (!b->inst[i].active) { slot = i; break; }
    if (slot < 0) {
        if ((int)b->inst.size() >= b->max_instances) return HYDRO_ERR_OOM;
        b->inst.push_back(InstInfo{});
        slot = (int)b->inst.size() - 1;
    }
    // the new instance's items must fit the work lists together with the others
    long long need3 = 0, need2 = 0;
    for (const InstInfo &J : b->inst)
        if (J.active) (J.prob.ndim == 3 ? need3 : need2) += (long long)J.items;
    (prob->ndim == 3 ? need3 : need2) += (long long)max_items_of(*prob);
    if (need3 > b->cap3 || need2 > b->cap2) return HYDRO_ERR_OOM;

    InstInfo I{};
    I.prob = *prob;
    I.nvar = prob->ndim + 2;
    I.plane = (long long)prob->n[0] * prob->n[1];
    I.N = I.plane * prob->n[2];
    I.state_bytes = hydro_state_bytes(prob);
    // the instance joins at the batch's current parity
    I.buf[b->parity] = Ua;
    I.buf[1 - b->parity] = Ub;
    const InstLayout L = inst_layout(*prob);
    unsigned char *w = static_cast<unsigned char *>(inst_work);
    I.ctrl = reinterpret_cast<Ctrl *>(w + L.ctrl);
    I.partial = reinterpret_cast<double *>(w + L.partial);
    I.bg = reinterpret_cast<PlaneBG *>(w + L.bg);
    I.bgf = reinterpret_cast<PlaneBGT<float> *>(w + L.bgf);
    I.step_end = step_end < 0 ? LLONG_MAX : step_end;
    I.items = max_items_of(*prob);
    I.cell_volume = 1.0;
    for (int d = 0; d < 3; ++d) {
        I.dx[d] = (prob->hi[d] - prob->lo[d]) / prob->n[d];
        I.inv_dx[d] = 1.0 / I.dx[d];
        if (d < prob->ndim) I.cell_volume *= I.dx[d];
    }
    cudaError_t e = cudaMemsetAsync(inst_work, 0, L.total, b->stream);
    std::vector<PlaneBG> tb;
    std::vector<PlaneBGT<float>> tf;
    if (e == cudaSuccess && prob->hse_subtract) {
        const int nz = prob->n[2];
        const double *rc_ = bg, *pc_ = bg + (nz + 4), *rf_ = bg + 2 * (nz + 4), *pf_ = bg + 2 * (nz + 4) + (nz + 5);
        tb.assign(nz + 5, PlaneBG{});
        tf.assign(nz + 5, PlaneBGT<float>{});
        for (int k = -2; k <= nz + 2; ++k) {
            PlaneBG &q = tb[k + 2];
            const bool has_c = k <= nz + 1;
            q.rho_c = has_c ? rc_[k + 2] : 0.0;
            q.p_c = has_c ? pc_[k + 2] : 0.0;
            q.rho_f = rf_[k + 2];
            q.p_f = pf_[k + 2];
            if (has_c) {
                q.drho = rf_[k + 3] - rf_[k + 2];
                q.dp = pf_[k + 3] - pf_[k + 2];
                q.B = q.dp / I.dx[2] - q.rho_c * prob->grav[2];
            }
            if (!std::isfinite(q.rho_c) || !std::isfinite(q.p_c) || !std::isfinite(q.rho_f) || !std::isfinite(q.p_f))
                return HYDRO_ERR_INVALID_ARG;
            tf[k + 2] = PlaneBGT<float>{(float)q.rho_c, (float)q.p_c, (float)q.rho_f, (float)q.p_f,
                                        (float)q.drho, (float)q.dp, (float)q.B, 0.0f};
        }
        e = cudaMemcpyAsync(I.bg, tb.data(), sizeof(PlaneBG) * tb.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(I.bgf, tf.data(), sizeof(PlaneBGT<float>) * tf.size(), cudaMemcpyHostToDevice,
                                b->stream);
    }
    // initial state through the spare buffer, then the first dt
    const long long cap = (long long)(I.state_bytes / (sizeof(double) * I.nvar));
    double *stg = static_cast<double *>(I.buf[1 - b->parity]);
    AuxArgs a = aux_for(I, I.buf[b->parity]);
    for (long long c0 = 0; c0 < I.N && e == cudaSuccess; c0 += cap) {
        const long long m = std::min(cap, I.N - c0);
        for (int q = 0; q < I.nvar && e == cudaSuccess; ++q)
            e = cudaMemcpyAsync(stg + (size_t)q * m, W0 + (size_t)q * I.N + c0, sizeof(double) * m,
                                cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = launch_init_convert(a, stg, c0, m, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    if (e == cudaSuccess) e = launch_signal(a, b->stream);
    Ctrl c{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c, I.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    b->launches += 2;
    I.active = true;
    b->inst[slot] = I;
    if (prob->ndim == 3) b->hse3 = prob->hse_subtract;
    b->dirty = true;
    *id_out = slot;
    return c.err ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK;
}

bool valid_id(const hydro_batch *b, int id)
{
    return b && id >= 0 && id < (int)b->inst.size() && b->inst[id].active;
}

}  // namespace

extern "C" {

size_t hydro_instance_work_bytes(const hydro_problem *prob)
{
    if (!prob || hydro_state_bytes(prob) == 0) return 0;
    return inst_layout(*prob).total;
}

size_t hydro_batch_create_bytes(int max_instances, long max_items3d, long max_items2d)
{
    if (max_instances <= 0 || max_items3d < 0 || max_items2d < 0) return 0;
    return batch_layout(max_instances, max_items3d, max_items2d).total;
}

long hydro_problem_max_items(const hydro_problem *prob)
{
    if (!prob || hydro_state_bytes(prob) == 0) return -1;
    return (long)max_items_of(*prob);
}

int hydro_batch_create(int max_instances, long max_items3d, long max_items2d, int precision, void *work,
                       void *stream, hydro_batch **out)
{
    if (!out) return HYDRO_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_instances <= 0 || max_items3d < 0 || max_items2d < 0 || !work || !aligned(work) ||
        (precision != HYDRO_FP64 && precision != HYDRO_FP32))
        return HYDRO_ERR_INVALID_ARG;
    hydro_batch *b = new (std::nothrow) hydro_batch();
    if (!b) return HYDRO_ERR_OOM;
    b->variant = precision == HYDRO_FP32 ? 7 : 6;   // asynchronous staging, 32 x 16 (FP32) / 16 x 16 (FP64)
    b->max_instances = max_instances;
    b->cap3 = max_items3d;
    b->cap2 = max_items2d;
    b->precision = precision;
    b->hse3 = -1;
    b->work = static_cast<unsigned char *>(work);
    b->lay = batch_layout(max_instances, max_items3d, max_items2d);
    b->stream = static_cast<cudaStream_t>(stream);
    b->d_insts = reinterpret_cast<BatchInst *>(b->work + b->lay.insts);
    b->d_items3 = reinterpret_cast<BatchItem *>(b->work + b->lay.items3);
    b->d_items2 = reinterpret_cast<BatchItem *>(b->work + b->lay.items2);
    b->use_graph = true;
    b->dirty = true;
    *out = b;
    return HYDRO_OK;
}

int hydro_batch_add(hydro_batch *b, const hydro_problem *prob, void *Ua, void *Ub, void *inst_work,
                    const double *W0, const double *bg, long step_end, int *id)
{
    if (!b || !id) return HYDRO_ERR_INVALID_ARG;
    return add_instance(b, prob, Ua, Ub, inst_work, W0, bg, step_end, id);
}

int hydro_batch_remove(hydro_batch *b, int id)
{
    if (!valid_id(b, id)) return HYDRO_ERR_INVALID_ARG;
    // the instance's buffers may be reused by the caller once this returns
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
    b->inst[id].active = false;
    b->dirty = true;
    return HYDRO_OK;
}

int hydro_batch_set_graph(hydro_batch *b, int on)
{
    if (!b) return HYDRO_ERR_INVALID_ARG;
    b->use_graph = on != 0;
    b->dirty = true;
    return HYDRO_OK;
}

size_t hydro_batch_workspace_bytes(const hydro_problem *probs, int count)
{
    if (!probs || count <= 0) return 0;
    long long cap3 = 0, cap2 = 0;
    size_t inst = 0;
    for (int i = 0; i < count; ++i) {
        if (hydro_state_bytes(&probs[i]) == 0 || probs[i].precision != probs[0].precision ||
            probs[i].scheme != HYDRO_SCHEME_HANCOCK)
            return 0;
        (probs[i].ndim == 3 ? cap3 : cap2) += (long long)max_items_of(probs[i]);
        inst += inst_layout(probs[i]).total;
    }
    return batch_layout(count, cap3, cap2).total + inst;
}

int hydro_batch_init(const hydro_problem *probs, int count, void *const *Ua, void *const *Ub, void *work,
                     const double *const *W0, const double *const *bg, void *stream, hydro_batch **out)
{
    if (!out) return HYDRO_ERR_INVALID_ARG;
    *out = nullptr;
    if (hydro_batch_workspace_bytes(probs, count) == 0 || !Ua || !Ub || !W0 || !work) return HYDRO_ERR_INVALID_ARG;
    long long cap3 = 0, cap2 = 0;
    for (int i = 0; i < count; ++i) (probs[i].ndim == 3 ? cap3 : cap2) += (long long)max_items_of(probs[i]);
    hydro_batch *b = nullptr;
    int rc = hydro_batch_create(count, cap3, cap2, probs[0].precision, work, stream, &b);
    if (rc) return rc;
    unsigned char *w = static_cast<unsigned char *>(work) + b->lay.total;
    int err_any = 0;
    for (int i = 0; i < count; ++i) {
        int id = -1;
        rc = add_instance(b, &probs[i], Ua[i], Ub[i], w, W0[i], bg ? bg[i] : nullptr, -1, &id);
        if (rc == HYDRO_ERR_NONPHYSICAL) { err_any = 1; rc = HYDRO_OK; }
        if (rc) break;
        w += inst_layout(probs[i]).total;
    }
    if (rc == HYDRO_OK) rc = rebuild(b);
    if (rc) {
        drop_graph(b);
        delete b;
        return rc;
    }
    *out = b;
    return err_any ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK;
}

int hydro_batch_configure(hydro_batch *b, int variant, int zchunk)
{
    if (!b || !tile3d_available(variant, b->precision == HYDRO_FP32) || zchunk < 0) return HYDRO_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
    b->variant = variant;
    b->zchunk = zchunk;
    return rebuild(b);
}

int hydro_batch_variant_shape(int variant, int *tx, int *ty)
{
    if (variant < 0 || variant >= TILE3D_VARIANTS || !tx || !ty) return HYDRO_ERR_INVALID_ARG;
    *tx = TILE3D_SHAPES[variant].tx;
    *ty = TILE3D_SHAPES[variant].ty;
    return HYDRO_OK;
}

int hydro_batch_step(hydro_batch *b, long nsteps)
{
    nvtxRangePushA("hydro_batch_step");
    struct Pop { ~Pop() { nvtxRangePop(); } } pop;
    if (!b || nsteps < 0) return HYDRO_ERR_INVALID_ARG;
    if (b->dirty) {
        int rc = rebuild(b);
        if (rc) return rc;
    }
    cudaError_t e = cudaSuccess;
    long done = 0;
    const int per = (b->nitems3 > 0) + (b->nitems2 > 0);
    // direct launches until the parity is even, graph replays (two steps
    // each) for the bulk, a direct launch for an odd remainder
    while (done < nsteps && e == cudaSuccess) {
        if (b->graph_ok && b->parity == 0 && nsteps - done >= 2) {
            e = cudaGraphLaunch(b->exec, b->stream);
            done += 2;
            b->launches += 2 * per;
        } else {
            e = launch_once(b, b->parity);
            b->parity ^= 1;
            done += 1;
            b->launches += per;
        }
    }
    return e == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
}

int hydro_batch_reduce(hydro_batch *b, int id, int what, double *out)
{
    if (!valid_id(b, id) || !out) return HYDRO_ERR_INVALID_ARG;
    InstInfo &I = b->inst[id];
    if (what == HYDRO_RED_TOTALS) {
        AuxArgs a = aux_for(I, I.buf[b->parity]);
        b->launches += 1;
        if (launch_totals(a, b->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
    } else if (what < HYDRO_RED_DT || what > HYDRO_RED_DT_LAST) {
        return HYDRO_ERR_INVALID_ARG;
    }
    Ctrl c;
    cudaError_t e = cudaMemcpyAsync(&c, I.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    switch (what) {
    case HYDRO_RED_TOTALS: for (int q = 0; q < I.nvar; ++q) out[q] = c.totals[q]; break;
    case HYDRO_RED_DT: out[0] = c.dt_next; break;
    case HYDRO_RED_TIME: out[0] = c.t; break;
    case HYDRO_RED_MAXSPEED: out[0] = c.max_speed; break;
    case HYDRO_RED_STEP: out[0] = (double)c.step; break;
    case HYDRO_RED_DT_LAST: out[0] = c.dt_last; break;
    }
    return c.err ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK;
}

int hydro_batch_get_fields(hydro_batch *b, int id, int what, double *host_dst)
{
    if (!valid_id(b, id) || !host_dst || (what != 0 && what != 1)) return HYDRO_ERR_INVALID_ARG;
    InstInfo &I = b->inst[id];
    const long long cap = (long long)(I.state_bytes / (sizeof(double) * I.nvar));
    double *stg = static_cast<double *>(I.buf[1 - b->parity]);
    AuxArgs a = aux_for(I, I.buf[b->parity]);
    for (long long c0 = 0; c0 < I.N; c0 += cap) {
        const long long m = std::min(cap, I.N - c0);
        b->launches += 1;
        cudaError_t e = launch_fields(a, stg, c0, m, what, b->stream);
        for (int q = 0; q < I.nvar && e == cudaSuccess; ++q)
            e = cudaMemcpyAsync(host_dst + (size_t)q * I.N + c0, stg + (size_t)q * m, sizeof(double) * m,
                                cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    }
    return HYDRO_OK;
}

int hydro_batch_get_state(hydro_batch *b, int id, void *host_dst)
{
    if (!valid_id(b, id) || !host_dst) return HYDRO_ERR_INVALID_ARG;
    InstInfo &I = b->inst[id];
    cudaError_t e = cudaMemcpyAsync(host_dst, I.buf[b->parity], I.state_bytes, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
}

void *hydro_batch_current(hydro_batch *b, int id)
{
    if (!valid_id(b, id)) return nullptr;
    return b->inst[id].buf[b->parity];
}

long hydro_batch_launch_count(hydro_batch *b) { return b ? b->launches : -1; }

int hydro_batch_items(hydro_batch *b, int *items3d, int *items2d, int *grid3d, int *grid2d)
{
    if (!b) return HYDRO_ERR_INVALID_ARG;
    if (b->dirty) {
        int rc = rebuild(b);
        if (rc) return rc;
    }
    if (items3d) *items3d = b->nitems3;
    if (items2d) *items2d = b->nitems2;
    if (grid3d) *grid3d = b->grid3;
    if (grid2d) *grid2d = b->grid2;
    return HYDRO_OK;
}

int hydro_batch_destroy(hydro_batch *b)
{
    if (!b) return HYDRO_ERR_INVALID_ARG;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    delete b;
    return HYDRO_OK;
}

}  // extern "C"
