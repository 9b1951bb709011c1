// ctu3d.cu -- FP64 and FP32 instantiations of the fused 3D corner transport
// upwind step.  Blocks: FP32 8 x 8 x 4 cells (256 threads, 127 KB of shared
// memory), FP64 8 x 4 x 4 (128 threads, 154 KB).
#include "ctu3d.cuh"
#include "launchers.h"

namespace hydro {

template <typename T, int TX, int TY, int TZ>
static cudaError_t launch_ctu(const StepArgs &a, cudaStream_t s)
{
    auto k = ctu3d_kernel<T, TX, TY, TZ>;
    constexpr size_t smem = Ctu3DSmem<T, TX, TY, TZ>::bytes;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const long long blocks = (long long)((a.n[0] + TX - 1) / TX) * ((a.n[1] + TY - 1) / TY) * ((a.n[2] + TZ - 1) / TZ);
    k<<<(unsigned)blocks, TX * TY * TZ, smem, s>>>(a);
    return cudaGetLastError();
}

long long ctu3d_blocks(const int n[3], bool fp32)
{
    const int tx = 8, ty = fp32 ? 8 : 4, tz = 4;
    return (long long)((n[0] + tx - 1) / tx) * ((n[1] + ty - 1) / ty) * ((n[2] + tz - 1) / tz);
}

cudaError_t launch_ctu3d(const StepArgs &a, cudaStream_t s, bool fp32)
{
    return fp32 ? launch_ctu<float, 8, 8, 4>(a, s) : launch_ctu<double, 8, 4, 4>(a, s);
}

}  // namespace hydro
