// noalloc.cu -- conserved totals of a caller's state with no allocation.
//
// hydro_totals_noalloc runs the same deterministic FP64 totals kernel as
// hydro_reduce(HYDRO_RED_TOTALS), but its scratch (the arrival counter, the
// per-CTA partial sums and the background table) lives in one file-scope
// __device__ array of fixed size instead of a caller workspace.  The host
// needs that array's device address: in host code the symbol name only
// stands in for it, so every call looks the address up on the current
// device with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/hydro.h"
#include "hydro_internal.h"
#include "launchers.h"

using namespace hydro;

namespace {

// capacity of the static scratch
constexpr int NOALLOC_MAX_PARTIALS = 4096 * 5;   // aux_reduce_blocks(N) <= 4096 CTAs x 5 sums
constexpr int NOALLOC_MAX_BG_PLANES = 4096;      // hse background entries: nz + 5 <= 4096

struct NoallocScratch {
    Ctrl ctrl;
    double partial[NOALLOC_MAX_PARTIALS];
    PlaneBG bg[NOALLOC_MAX_BG_PLANES];
};

constexpr size_t NOALLOC_SCRATCH_BYTES = (sizeof(NoallocScratch) + 255) / 256 * 256;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch on the current device.  Looked up on every
// call (cudaGetSymbolAddress allocates nothing): a cached address could
// outlive the context it belongs to (after cudaDeviceReset, or when the
// primary context is released and created again).
int scratch_for_current_device(NoallocScratch **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess || !p) return HYDRO_ERR_CUDA;
    *out = static_cast<NoallocScratch *>(p);
    return HYDRO_OK;
}

}  // namespace

extern "C" int hydro_totals_noalloc(const hydro_problem *prob, const void *U, const double *bg,
                                    void *stream, double *out)
{
    if (!prob || !U || !out) return HYDRO_ERR_INVALID_ARG;
    if (hydro_state_bytes(prob) == 0) return HYDRO_ERR_INVALID_ARG;
    const int nz = prob->n[2];
    if (prob->hse_subtract) {
        if (nz + 5 > NOALLOC_MAX_BG_PLANES || !bg) return HYDRO_ERR_INVALID_ARG;
        // the four tables (2 (nz + 4) centre and 2 (nz + 5) face entries) must be finite
        for (int i = 0; i < 4 * nz + 18; ++i)
            if (!std::isfinite(bg[i])) return HYDRO_ERR_INVALID_ARG;
    }
    const long long plane = (long long)prob->n[0] * prob->n[1];
    const long long N = plane * nz;
    if (5 * aux_reduce_blocks(N) > NOALLOC_MAX_PARTIALS) return HYDRO_ERR_INVALID_ARG;

    NoallocScratch *S = nullptr;
    int rc = scratch_for_current_device(&S);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // the arrival counter must start at zero; everything else is overwritten
    cudaError_t e = cudaMemsetAsync(&S->ctrl, 0, sizeof(Ctrl), s);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;

    double dx[3];
    double vol = 1.0;
    for (int d = 0; d < 3; ++d) {
        dx[d] = (prob->hi[d] - prob->lo[d]) / prob->n[d];
        if (d < prob->ndim) vol *= dx[d];
    }
    if (prob->hse_subtract) {
        // per-plane background constants, staged through a small stack block
        // (a copy from pageable memory has read the block when it returns)
        const double *rc_ = bg, *pc_ = bg + (nz + 4), *rf_ = bg + 2 * (nz + 4),
                     *pf_ = bg + 2 * (nz + 4) + (nz + 5);
        PlaneBG block[64];
        for (int k0 = -2; k0 <= nz + 2; k0 += 64) {
            const int cnt = (k0 + 64 <= nz + 3) ? 64 : nz + 3 - k0;
            for (int i = 0; i < cnt; ++i) {
                const int k = k0 + i;
                PlaneBG b{};
                const bool has_c = k <= nz + 1;
                b.rho_c = has_c ? rc_[k + 2] : 0.0;
                b.p_c = has_c ? pc_[k + 2] : 0.0;
                b.rho_f = rf_[k + 2];
                b.p_f = pf_[k + 2];
                if (has_c) {
                    b.drho = rf_[k + 3] - rf_[k + 2];
                    b.dp = pf_[k + 3] - pf_[k + 2];
                    b.B = b.dp / dx[2] - b.rho_c * prob->grav[2];
                }
                block[i] = b;
            }
            e = cudaMemcpyAsync(S->bg + (k0 + 2), block, sizeof(PlaneBG) * cnt,
                                cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return HYDRO_ERR_CUDA;
        }
    }

    AuxArgs a{};
    a.U = const_cast<void *>(U);
    a.ndim = prob->ndim;
    for (int d = 0; d < 3; ++d) { a.n[d] = prob->n[d]; a.inv_dx[d] = 1.0 / dx[d]; }
    a.N = N;
    a.vstride = N;
    a.plane = plane;
    a.gamma = prob->gamma;
    a.cfl = prob->cfl;
    a.cell_volume = vol;
    a.ctrl = &S->ctrl;
    a.partial = S->partial;
    a.bg = prob->hse_subtract ? S->bg : nullptr;
    a.hse = prob->hse_subtract;
    a.fp32 = prob->precision == HYDRO_FP32;
    e = launch_totals(a, s);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    e = cudaMemcpyAsync(out, S->ctrl.totals, sizeof(double) * (prob->ndim + 2),
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
}
