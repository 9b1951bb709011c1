// batch_api.cu -- batched solves: many independent, uneven instances
// advanced together, one persistent launch per step (one for the 3D
// instances, one for the 2D ones) whose CTAs claim work items from a
// device-resident queue, replayed from a captured CUDA graph.  Instances may
// join and leave between steps (the continuous-batching server does so
// without synchronising: the queue, the instance table and the item lists
// are rewritten by stream-ordered copies from pinned host memory, and the
// graph, whose launches read them at run time, stays valid).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
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

// Shared work buffer: the queue, the instance table and the two item lists.
struct BatchLayout {
    size_t queue, insts, items3, items2, total;
};

BatchLayout batch_layout(int max_instances, long long cap3, long long cap2)
{
    BatchLayout L{};
    size_t off = 0;
    L.queue = off;
    off = align_up(off + sizeof(BatchQueue));
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
    int join_parity;        // batch parity of the first launch after the join: buf[join_parity] held U^0
    long long launched;     // batched steps launched since the join
};

// Buffer index (into InstInfo::buf) of the state after `steps` steps: a
// frozen instance (step limit reached, or its error state) is skipped by the
// kernels, so its state stays in the buffer of its last step.
int state_index(const InstInfo &I, long long steps) { return (int)((I.join_parity + (steps & 1)) & 1); }

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
    int parity;                // parity of the next launch
    int variant, zchunk;       // zchunk: longest chunk of an instance's column (0 = default)
    bool dirty;                // queue / tables need an upload
    bool use_graph;
    BatchQueue *d_queue;
    BatchInst *d_insts;
    BatchItem *d_items3, *d_items2;
    // two pinned host staging buffers used in turn for the uploads; one is
    // rewritten only after the upload made from it has completed (its event
    // `staged`), i.e. the host waits at most for the upload before the last
    unsigned char *pinned[2];
    size_t pinned_bytes[2];
    cudaEvent_t staged[2];
    bool staged_pending[2];
    int stage_buf;             // buffer the next upload uses
    int nitems3, nitems2, grid3, grid2;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool graph_ok;
    int graph_variant, graph_has3, graph_has2;
    long launches;
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
        e = launch_batch3d(b->variant, b->precision == HYDRO_FP32, b->hse3 == 1, b->d_insts, b->d_queue, parity,
                           b->grid3, b->stream);
    if (e == cudaSuccess && b->nitems2 > 0)
        e = launch_batch2d(b->precision == HYDRO_FP32, b->d_insts, b->d_queue, parity, b->grid2, b->stream);
    return e;
}

// Longest z-chunk of an instance's column: long chunks re-read few halo
// planes (4 per chunk), and the largest-first claim order keeps the SMs
// balanced even when whole columns are single items.
constexpr int BATCH_ZCHUNK_DEFAULT = 64;

int zchunk_of(const hydro_batch *b, const hydro_problem &p)
{
    const int zmax = b->zchunk > 0 ? b->zchunk : BATCH_ZCHUNK_DEFAULT;
    const int nch = (p.n[2] + zmax - 1) / zmax;       // chunks of (nearly) equal length
    return (p.n[2] + nch - 1) / nch;
}

// Staging buffer k ready for rewriting and holding at least `need` bytes.
int ensure_pinned(hydro_batch *b, int k, size_t need)
{
    if (b->staged_pending[k] && cudaEventSynchronize(b->staged[k]) != cudaSuccess) return HYDRO_ERR_CUDA;
    b->staged_pending[k] = false;
    if (need <= b->pinned_bytes[k]) return HYDRO_OK;
    if (b->pinned[k]) cudaFreeHost(b->pinned[k]);
    b->pinned[k] = nullptr;
    b->pinned_bytes[k] = 0;
    size_t cap = 1 << 20;
    while (cap < need) cap *= 2;
    if (cudaHostAlloc(reinterpret_cast<void **>(&b->pinned[k]), cap, cudaHostAllocDefault) != cudaSuccess) {
        b->pinned[k] = nullptr;
        return HYDRO_ERR_OOM;
    }
    b->pinned_bytes[k] = cap;
    return HYDRO_OK;
}

// Rebuild the per-instance arguments and the item lists and upload them
// (with the queue's list lengths) by stream-ordered copies: launches already
// enqueued still see the old ones, later launches the new ones.  Items are
// ordered largest first (3D: by chunk length) for the dynamic claim.  The
// graph (two launches, both parities) is captured again only when the
// kernels or grids change, not when the membership does.
int rebuild(hydro_batch *b)
{
    const TileShape ts = TILE3D_SHAPES[b->variant];
    std::vector<BatchInst> insts(b->max_instances, BatchInst{});
    std::vector<BatchItem> items3, items2;
    std::vector<int> len3;
    for (int i = 0; i < (int)b->inst.size(); ++i) {
        const InstInfo &I = b->inst[i];
        if (!I.active) continue;
        const hydro_problem &p = I.prob;
        const bool is3 = p.ndim == 3;
        const int tx = is3 ? ts.tx : BATCH2D_TX, ty = is3 ? ts.ty : BATCH2D_TY;
        const int tiles_x = tiles_along(p.n[0], tx), tiles_y = tiles_along(p.n[1], ty);
        const int zc = is3 ? zchunk_of(b, p) : 1;
        const int nch = is3 ? (p.n[2] + zc - 1) / zc : 1;
        BatchInst &bi = insts[i];
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
        int local = 0;
        for (int c = 0; c < nch; ++c)
            for (int t = 0; t < tiles_x * tiles_y; ++t) {
                if (is3) {
                    items3.push_back(BatchItem{i, t, c, local++});
                    len3.push_back(std::min(zc, p.n[2] - c * zc));
                } else {
                    items2.push_back(BatchItem{i, t, c, local++});
                }
            }
    }
    if ((long long)items3.size() > b->cap3 || (long long)items2.size() > b->cap2) return HYDRO_ERR_OOM;
    // largest first (stable: an instance's items stay in tile order)
    std::vector<int> order(items3.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return len3[x] > len3[y]; });
    std::vector<BatchItem> sorted3(items3.size());
    for (size_t k = 0; k < order.size(); ++k) sorted3[k] = items3[order[k]];

    b->nitems3 = (int)sorted3.size();
    b->nitems2 = (int)items2.size();
    const size_t bi_bytes = sizeof(BatchInst) * (size_t)b->max_instances;
    const size_t i3_bytes = sizeof(BatchItem) * sorted3.size();
    const size_t i2_bytes = sizeof(BatchItem) * items2.size();
    const size_t q_bytes = offsetof(BatchQueue, next);   // list pointers and lengths, not the counters
    const size_t o_i3 = align_up(bi_bytes), o_i2 = o_i3 + align_up(i3_bytes), o_q = o_i2 + align_up(i2_bytes);
    const int k = b->stage_buf;
    int rc = ensure_pinned(b, k, o_q + align_up(q_bytes));
    if (rc) return rc;
    unsigned char *pin = b->pinned[k];
    std::memcpy(pin, insts.data(), bi_bytes);
    if (i3_bytes) std::memcpy(pin + o_i3, sorted3.data(), i3_bytes);
    if (i2_bytes) std::memcpy(pin + o_i2, items2.data(), i2_bytes);
    BatchQueue qh{};
    qh.items[0] = b->d_items3;
    qh.items[1] = b->d_items2;
    qh.nitems[0] = b->nitems3;
    qh.nitems[1] = b->nitems2;
    std::memcpy(pin + o_q, &qh, q_bytes);
    cudaError_t e = cudaMemcpyAsync(b->d_insts, pin, bi_bytes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && i3_bytes)
        e = cudaMemcpyAsync(b->d_items3, pin + o_i3, i3_bytes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && i2_bytes)
        e = cudaMemcpyAsync(b->d_items2, pin + o_i2, i2_bytes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_queue, pin + o_q, q_bytes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->staged[k], b->stream);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    b->staged_pending[k] = true;
    b->stage_buf = 1 - k;

    // persistent grids: the resident CTAs (the claim loop balances the items)
    const bool fp32 = b->precision == HYDRO_FP32;
    b->grid3 = b->nitems3 ? std::max(1, batch3d_max_grid(b->variant, fp32, b->hse3 == 1)) : 0;
    b->grid2 = b->nitems2 ? std::max(1, batch2d_max_grid(fp32)) : 0;

    const bool has3 = b->nitems3 > 0, has2 = b->nitems2 > 0;
    const bool same_graph = b->graph_ok && b->graph_variant == b->variant && b->graph_has3 == has3 &&
                            b->graph_has2 == has2;
    if (!same_graph) {
        drop_graph(b);
        if (b->use_graph && b->stream != nullptr && (has3 || has2)) {
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
            b->graph_variant = b->variant;
            b->graph_has3 = has3;
            b->graph_has2 = has2;
        }
    }
    b->dirty = false;
    return HYDRO_OK;
}

// Checks and bookkeeping shared by the synchronous and asynchronous adds;
// fills *I (buffers, layout, background tables uploaded on the stream) and
// the slot.  The initial state is converted by the caller.
int prepare_instance(hydro_batch *b, const hydro_problem *prob, void *Ua, void *Ub, void *inst_work,
                     const double *bg, long long step_end, InstInfo *Iout, int *slot_out)
{
    if (!prob || !Ua || !Ub || !inst_work || Ua == Ub) return HYDRO_ERR_INVALID_ARG;
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
    if (slot < 0 && (int)b->inst.size() >= b->max_instances) return HYDRO_ERR_OOM;
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
    // the instance joins at the batch's current parity: the next launch
    // (parity b->parity) reads buf[b->parity] = Ua
    I.join_parity = b->parity;
    I.launched = 0;
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
    if (e == cudaSuccess && prob->hse_subtract) {
        const int nz = prob->n[2];
        const double *rc_ = bg, *pc_ = bg + (nz + 4), *rf_ = bg + 2 * (nz + 4), *pf_ = bg + 2 * (nz + 4) + (nz + 5);
        std::vector<PlaneBG> tb(nz + 5, PlaneBG{});
        std::vector<PlaneBGT<float>> tf(nz + 5, PlaneBGT<float>{});
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
        // (copies from pageable memory have read the vectors when they return)
        e = cudaMemcpyAsync(I.bg, tb.data(), sizeof(PlaneBG) * tb.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(I.bgf, tf.data(), sizeof(PlaneBGT<float>) * tf.size(), cudaMemcpyHostToDevice,
                                b->stream);
    }
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    *Iout = I;
    *slot_out = slot;
    return HYDRO_OK;
}

void commit_instance(hydro_batch *b, const InstInfo &I, int slot, int *id_out)
{
    if (slot < 0) {
        b->inst.push_back(InstInfo{});
        slot = (int)b->inst.size() - 1;
    }
    b->inst[slot] = I;
    b->inst[slot].active = true;
    if (I.prob.ndim == 3) b->hse3 = I.prob.hse_subtract;
    b->dirty = true;
    *id_out = slot;
}

// Synchronous add: the host primitives go through the spare buffer in
// chunks; the first dt is read back.
int add_instance(hydro_batch *b, const hydro_problem *prob, void *Ua, void *Ub, void *inst_work,
                 const double *W0, const double *bg, long long step_end, int *id_out)
{
    if (!W0) return HYDRO_ERR_INVALID_ARG;
    InstInfo I{};
    int slot = -1;
    int rc = prepare_instance(b, prob, Ua, Ub, inst_work, bg, step_end, &I, &slot);
    if (rc) return rc;
    const long long cap = (long long)(I.state_bytes / (sizeof(double) * I.nvar));
    double *stg = static_cast<double *>(I.buf[1 - b->parity]);
    AuxArgs a = aux_for(I, I.buf[b->parity]);
    cudaError_t e = cudaSuccess;
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
    commit_instance(b, I, slot, id_out);
    return c.err ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK;
}

// Asynchronous add: W0dev is a DEVICE array of the FP64 total primitives;
// the conversion and the first dt are enqueued on the batch stream.
int add_instance_async(hydro_batch *b, const hydro_problem *prob, void *Ua, void *Ub, void *inst_work,
                       const double *W0dev, const double *bg, long long step_end, int *id_out)
{
    if (!W0dev) return HYDRO_ERR_INVALID_ARG;
    InstInfo I{};
    int slot = -1;
    int rc = prepare_instance(b, prob, Ua, Ub, inst_work, bg, step_end, &I, &slot);
    if (rc) return rc;
    AuxArgs a = aux_for(I, I.buf[b->parity]);
    cudaError_t e = launch_init_convert(a, W0dev, 0, I.N, b->stream);
    if (e == cudaSuccess) e = launch_signal(a, b->stream);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    b->launches += 2;
    commit_instance(b, I, slot, id_out);
    return HYDRO_OK;
}

bool valid_id(const hydro_batch *b, int id)
{
    return b && id >= 0 && id < (int)b->inst.size() && b->inst[id].active;
}

// Control block of an instance (synchronises) and the buffer of its current state.
int read_inst_ctrl(hydro_batch *b, const InstInfo &I, Ctrl *c)
{
    cudaError_t e = cudaMemcpyAsync(c, I.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
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
    b->d_queue = reinterpret_cast<BatchQueue *>(b->work + b->lay.queue);
    b->d_insts = reinterpret_cast<BatchInst *>(b->work + b->lay.insts);
    b->d_items3 = reinterpret_cast<BatchItem *>(b->work + b->lay.items3);
    b->d_items2 = reinterpret_cast<BatchItem *>(b->work + b->lay.items2);
    b->use_graph = true;
    b->dirty = true;
    b->graph_variant = -1;
    // the queue's claim counters start at zero (the kernels reset them after each launch)
    cudaError_t e = cudaMemsetAsync(b->d_queue, 0, sizeof(BatchQueue), b->stream);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged[1], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete b;
        return HYDRO_ERR_CUDA;
    }
    *out = b;
    return HYDRO_OK;
}

int hydro_batch_add(hydro_batch *b, const hydro_problem *prob, void *Ua, void *Ub, void *inst_work,
                    const double *W0, const double *bg, long step_end, int *id)
{
    if (!b || !id) return HYDRO_ERR_INVALID_ARG;
    return add_instance(b, prob, Ua, Ub, inst_work, W0, bg, step_end, id);
}

int hydro_batch_add_async(hydro_batch *b, const hydro_problem *prob, void *Ua, void *Ub, void *inst_work,
                          const double *W0_device, const double *bg, long step_end, int *id)
{
    if (!b || !id) return HYDRO_ERR_INVALID_ARG;
    return add_instance_async(b, prob, Ua, Ub, inst_work, W0_device, bg, step_end, id);
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

int hydro_batch_remove_async(hydro_batch *b, int id)
{
    if (!valid_id(b, id)) return HYDRO_ERR_INVALID_ARG;
    b->inst[id].active = false;
    b->dirty = true;
    return HYDRO_OK;
}

int hydro_batch_set_graph(hydro_batch *b, int on)
{
    if (!b) return HYDRO_ERR_INVALID_ARG;
    b->use_graph = on != 0;
    drop_graph(b);
    b->graph_variant = -1;
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
        hydro_batch_destroy(b);
        return rc;
    }
    *out = b;
    return err_any ? HYDRO_ERR_NONPHYSICAL : HYDRO_OK;
}

int hydro_batch_configure(hydro_batch *b, int variant, int zchunk)
{
    if (!b || !tile3d_available(variant, b->precision == HYDRO_FP32) || zchunk < 0) return HYDRO_ERR_INVALID_ARG;
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
    for (InstInfo &I : b->inst)
        if (I.active) I.launched += done;
    return e == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
}

int hydro_batch_reduce(hydro_batch *b, int id, int what, double *out)
{
    if (!valid_id(b, id) || !out) return HYDRO_ERR_INVALID_ARG;
    InstInfo &I = b->inst[id];
    if (what < HYDRO_RED_TOTALS || what > HYDRO_RED_DT_LAST) return HYDRO_ERR_INVALID_ARG;
    Ctrl c;
    int rc = read_inst_ctrl(b, I, &c);
    if (rc) return rc;
    if (what == HYDRO_RED_TOTALS) {
        AuxArgs a = aux_for(I, I.buf[state_index(I, c.step)]);
        b->launches += 1;
        if (launch_totals(a, b->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
        rc = read_inst_ctrl(b, I, &c);
        if (rc) return rc;
    }
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
    Ctrl c;
    int rc = read_inst_ctrl(b, I, &c);
    if (rc) return rc;
    const int cur = state_index(I, c.step);
    const long long cap = (long long)(I.state_bytes / (sizeof(double) * I.nvar));
    double *stg = static_cast<double *>(I.buf[1 - cur]);
    AuxArgs a = aux_for(I, I.buf[cur]);
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
    Ctrl c;
    int rc = read_inst_ctrl(b, I, &c);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(host_dst, I.buf[state_index(I, c.step)], I.state_bytes, cudaMemcpyDeviceToHost,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
}

int hydro_batch_get_state_async(hydro_batch *b, int id, void *host_dst)
{
    if (!valid_id(b, id) || !host_dst) return HYDRO_ERR_INVALID_ARG;
    const InstInfo &I = b->inst[id];
    // the steps taken once the enqueued launches have run: every launch
    // steps the instance until its step limit (an instance in its error
    // state stops earlier; its state is then not meaningful)
    const long long steps = std::min(I.launched, I.step_end);
    cudaError_t e = cudaMemcpyAsync(host_dst, I.buf[state_index(I, steps)], I.state_bytes, cudaMemcpyDeviceToHost,
                                    b->stream);
    return e == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
}

void *hydro_batch_current(hydro_batch *b, int id)
{
    if (!valid_id(b, id)) return nullptr;
    Ctrl c;
    if (read_inst_ctrl(b, b->inst[id], &c)) return nullptr;
    return b->inst[id].buf[state_index(b->inst[id], c.step)];
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
    for (int k = 0; k < 2; ++k) {
        if (b->staged[k]) cudaEventDestroy(b->staged[k]);
        if (b->pinned[k]) cudaFreeHost(b->pinned[k]);
    }
    delete b;
    return HYDRO_OK;
}

}  // extern "C"
