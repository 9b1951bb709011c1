// step3d_f64.cu -- FP64 instantiations of the fused single-solve 3D step
// for every tile shape and
// staging depth.
#include "launchers.h"
#include "per_device.h"
#include "step3d.cuh"

namespace hydro {

namespace {

template <typename T, bool HSE, int TX, int TY, bool AS, bool GZ>
cudaError_t launch3d_g(const StepArgs &a, dim3 grid, cudaStream_t s)
{
    auto k = step3d_kernel<T, HSE, TX, TY, STAGE_HANCOCK, RECON_PLM, AS, GZ>;
    constexpr size_t smem = Step3DSmem<T, HSE, TX, TY, RECON_PLM, AS>::bytes;
    static PerDeviceOnce configured;   // the attribute is per function and device
    static PerDeviceInt resident;      // balanced grid size, per device
    return launch_step_grid<TX, TY>(k, smem, configured, resident, a, grid, s);
}

// Gravity along z only (always so with the hydrostatic background) takes the
// kernel without the x and y gravity terms.
template <typename T, bool HSE, int TX, int TY, bool AS>
cudaError_t launch3d(const StepArgs &a, dim3 grid, cudaStream_t s)
{
    if constexpr (HSE) {
        return launch3d_g<T, HSE, TX, TY, AS, true>(a, grid, s);
    } else {
        if (a.grav[0] == 0.0 && a.grav[1] == 0.0) return launch3d_g<T, HSE, TX, TY, AS, true>(a, grid, s);
        return launch3d_g<T, HSE, TX, TY, AS, false>(a, grid, s);
    }
}

template <bool HSE>
cudaError_t launch_v(int v, const StepArgs &a, dim3 grid, cudaStream_t s)
{
    switch (v) {
    case 0: return launch3d<double, HSE, 32, 8, false>(a, grid, s);
    case 1: return launch3d<double, HSE, 32, 4, false>(a, grid, s);
    case 2: return launch3d<double, HSE, 16, 16, false>(a, grid, s);
    case 4: return launch3d<double, HSE, 32, 8, true>(a, grid, s);
    case 5: return launch3d<double, HSE, 32, 4, true>(a, grid, s);
    case 6: return launch3d<double, HSE, 16, 16, true>(a, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_step3d_f64(int v, const StepArgs &a, dim3 grid, cudaStream_t s, bool hse)
{
    return hse ? launch_v<true>(v, a, grid, s) : launch_v<false>(v, a, grid, s);
}

}  // namespace hydro
