// step2d.cu -- FP64 and FP32 instantiations of the fused 2D step and of
// the two Runge-Kutta stages.
#include "launchers.h"
#include "per_device.h"
#include "step2d.cuh"

namespace hydro {

template <typename T, int ST, int RC = RECON_PLM>
static cudaError_t launch2d(const StepArgs &a, dim3 grid, cudaStream_t s)
{
    constexpr int TX = STEP2D_TX, TY = STEP2D_TY;
    auto k = step2d_kernel<T, TX, TY, ST, RC>;
    constexpr size_t smem = Step2DSmem<T, TX, TY, RC>::bytes;
    static PerDeviceOnce configured;   // the attribute is per function and device
    const cudaError_t e = ensure_smem_limit(configured, k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, TX * TY, smem, s>>>(a);
    return cudaGetLastError();
}

template <int ST, int RC>
static cudaError_t launch2d_p(const StepArgs &a, dim3 grid, cudaStream_t s, bool fp32)
{
    return fp32 ? launch2d<float, ST, RC>(a, grid, s) : launch2d<double, ST, RC>(a, grid, s);
}

cudaError_t launch_step2d(const StepArgs &a, dim3 grid, cudaStream_t s, bool fp32, int stage, int recon)
{
    if (recon == RECON_PPM) {
        if (stage == STAGE_RK1) return launch2d_p<STAGE_RK1, RECON_PPM>(a, grid, s, fp32);
        if (stage == STAGE_RK2) return launch2d_p<STAGE_RK2, RECON_PPM>(a, grid, s, fp32);
        return cudaErrorInvalidValue;
    }
    switch (stage) {
    case STAGE_HANCOCK: return launch2d_p<STAGE_HANCOCK, RECON_PLM>(a, grid, s, fp32);
    case STAGE_RK1: return launch2d_p<STAGE_RK1, RECON_PLM>(a, grid, s, fp32);
    case STAGE_RK2: return launch2d_p<STAGE_RK2, RECON_PLM>(a, grid, s, fp32);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hydro
