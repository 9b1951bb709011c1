// pair3d_f32.cu -- instantiations of the paired-cell FP32 MUSCL-Hancock step
// (two x-adjacent cells per thread, packed f32x2 arithmetic) for its tile
// shapes, both modes, and gravity along z only or not.
#include "launchers.h"
#include "pair3d.cuh"
#include "per_device.h"

namespace hydro {

namespace {

template <bool HSE, int TXP, int TY, int MINB, bool GZ>
cudaError_t launch_pair(const StepArgs &a, dim3 grid, cudaStream_t s)
{
    auto k = step3d_pair_kernel<HSE, TXP, TY, GZ, MINB>;
    constexpr size_t smem = Pair3DSmem<HSE, TXP, TY, MINB>::bytes;
    static PerDeviceOnce configured;   // the attribute is per function and device
    const cudaError_t e = ensure_smem_limit(configured, k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, TXP * TY, smem, s>>>(a);
    return cudaGetLastError();
}

template <bool HSE, int TXP, int TY, int MINB>
cudaError_t launch_g(const StepArgs &a, dim3 grid, cudaStream_t s)
{
    // gravity along z only (always so with the background) leaves out the
    // x and y gravity terms
    if (HSE || (a.grav[0] == 0.0 && a.grav[1] == 0.0)) return launch_pair<HSE, TXP, TY, MINB, true>(a, grid, s);
    return launch_pair<HSE, TXP, TY, MINB, false>(a, grid, s);
}

template <bool HSE>
cudaError_t launch_v(int pv, const StepArgs &a, dim3 grid, cudaStream_t s)
{
    switch (pv) {
    // (threads x, threads y, CTAs per SM asked of the register allocation)
    case 0: return launch_g<HSE, 16, 16, 2>(a, grid, s);   // 32 x 16 cells, 256 threads, 2 CTAs per SM
    case 1: return launch_g<HSE, 16, 8, 3>(a, grid, s);    // 32 x 8 cells, 128 threads, 3 CTAs per SM
    case 2: return launch_g<HSE, 8, 16, 3>(a, grid, s);    // 16 x 16 cells, 128 threads, 3 CTAs per SM
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_pair3d(int pv, const StepArgs &a, dim3 grid, cudaStream_t s, bool hse)
{
    return hse ? launch_v<true>(pv, a, grid, s) : launch_v<false>(pv, a, grid, s);
}

}  // namespace hydro
