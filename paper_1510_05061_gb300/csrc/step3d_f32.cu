// step3d_f64.cu -- FP32 instantiations of the fused 3D step.
#include "launchers.h"
#include "step3d.cuh"

namespace hydro {

template <typename T, bool HSE>
static cudaError_t launch3d(const StepArgs &a, dim3 grid, cudaStream_t s)
{
    constexpr int TX = STEP3D_TX, TY = STEP3D_TY;
    auto k = step3d_kernel<T, HSE, TX, TY>;
    constexpr size_t smem = Step3DSmem<T, HSE, TX, TY>::bytes;
    static bool configured = false;   // per process; the attribute is per function
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k<<<grid, TX * TY, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_step3d_f32(const StepArgs &a, dim3 grid, cudaStream_t s, bool hse)
{
    return hse ? launch3d<float, true>(a, grid, s) : launch3d<float, false>(a, grid, s);
}

}  // namespace hydro
