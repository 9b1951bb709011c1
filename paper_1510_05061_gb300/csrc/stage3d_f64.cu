// stage3d_f64.cu -- FP64 instantiations of the two stages of the SSP-RK2
// method of lines (3D, every tile shape; PLM with and without background
// subtraction, PPM without).
#include "launchers.h"
#include "per_device.h"
#include "step3d.cuh"

namespace hydro {

namespace {

template <int ST, int RC, bool HSE, int TX, int TY>
cudaError_t launch3d(const StepArgs &a, dim3 grid, cudaStream_t s)
{
    auto k = step3d_kernel<double, HSE, TX, TY, ST, RC>;
    constexpr size_t smem = Step3DSmem<double, HSE, TX, TY, RC>::bytes;
    static PerDeviceOnce configured;   // the attribute is per function and device
    static PerDeviceInt resident;      // balanced grid size, per device
    return launch_step_grid<TX, TY>(k, smem, configured, resident, a, grid, s);
}

template <int ST, int RC, bool HSE>
cudaError_t launch_v(int v, const StepArgs &a, dim3 grid, cudaStream_t s)
{
    switch (v % 4) {   // the stages use the precision's default staging
    case 0: return launch3d<ST, RC, HSE, 32, 8>(a, grid, s);
    case 1: return launch3d<ST, RC, HSE, 32, 4>(a, grid, s);
    case 2: return launch3d<ST, RC, HSE, 16, 16>(a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int ST>
cudaError_t launch_h(int v, const StepArgs &a, dim3 grid, cudaStream_t s, bool hse, int recon)
{
    if (recon == RECON_PPM)
        return hse ? cudaErrorInvalidValue : launch_v<ST, RECON_PPM, false>(v, a, grid, s);
    return hse ? launch_v<ST, RECON_PLM, true>(v, a, grid, s) : launch_v<ST, RECON_PLM, false>(v, a, grid, s);
}

}  // namespace

cudaError_t launch_stage3d_f64(int stage, int v, const StepArgs &a, dim3 grid, cudaStream_t s, bool hse, int recon)
{
    if (stage == STAGE_RK1) return launch_h<STAGE_RK1>(v, a, grid, s, hse, recon);
    if (stage == STAGE_RK2) return launch_h<STAGE_RK2>(v, a, grid, s, hse, recon);
    return cudaErrorInvalidValue;
}

}  // namespace hydro
