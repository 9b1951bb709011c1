// ctu2d.cu -- FP64 and FP32 instantiations of the fused 2D corner transport
// upwind step.
#include "ctu2d.cuh"
#include "launchers.h"
#include "per_device.h"

namespace hydro {

template <typename T>
static cudaError_t launch_ctu(const StepArgs &a, dim3 grid, cudaStream_t s)
{
    constexpr int TX = STEP2D_TX, TY = STEP2D_TY;
    auto k = ctu2d_kernel<T, TX, TY>;
    constexpr size_t smem = Ctu2DSmem<T, TX, TY>::bytes;
    static PerDeviceOnce configured;   // the attribute is per function and device
    const cudaError_t e = ensure_smem_limit(configured, k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, TX * TY, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ctu2d(const StepArgs &a, dim3 grid, cudaStream_t s, bool fp32)
{
    return fp32 ? launch_ctu<float>(a, grid, s) : launch_ctu<double>(a, grid, s);
}

}  // namespace hydro
