// ctu3d.cu -- FP64 and FP32 instantiations of the fused 3D corner transport
// upwind step.  Tiles: FP32 16 x 16 (256 threads, 152 KB of shared memory),
// FP64 16 x 8 (128 threads, 171 KB); FP32 z-chunks sized for several waves
// of the 152 SMs (one CTA per SM), FP64 the balanced grid.
#include <algorithm>

#include "ctu3d.cuh"
#include "launchers.h"
#include "per_device.h"

namespace hydro {

namespace {

constexpr int CTU_TX = 16;
int ctu_ty(bool fp32) { return fp32 ? 16 : 8; }

// planes per CTA: at least 8 waves of one CTA per SM, chunks of 8 or more
int ctu_zchunk(const int n[3], bool fp32)
{
    const long long tiles = (long long)((n[0] + CTU_TX - 1) / CTU_TX) * ((n[1] + ctu_ty(fp32) - 1) / ctu_ty(fp32));
    long long nch = (8ll * 152 + tiles - 1) / tiles;
    nch = std::min(nch, std::max(1ll, (long long)(n[2] / 8)));
    return (int)((n[2] + nch - 1) / nch);
}

template <typename T, bool HSE, int TX, int TY>
cudaError_t launch_ctu(const StepArgs &a0, cudaStream_t s)
{
    auto k = ctu3d_kernel<T, HSE, TX, TY>;
    constexpr size_t smem = Ctu3DSmem<T, TX, TY>::bytes;
    static PerDeviceInt resident;   // resident CTAs of the balanced grid, per device
    int g = 0;
    const cudaError_t e = persistent_grid(resident, k, smem, TX * TY, &g);
    if (e != cudaSuccess) return e;
    StepArgs a = a0;
    a.tiles_x = (a.n[0] + TX - 1) / TX;
    if constexpr (sizeof(T) == 8) {
        // FP64: the balanced grid, every resident CTA marching an equal share
        // of the plane-tiles (no partial last wave; measured +8 % at RT 256^3).
        // FP32 keeps z-chunks: the same speed there, and neighbouring tiles
        // marched at the same heights keep their halo rows in L2
        a.zchunk = 0;
        const long long W = (long long)a.tiles_x * ((a.n[1] + TY - 1) / TY) * a.n[2];
        k<<<(int)std::min<long long>(g, W), TX * TY, smem, s>>>(a);
    } else {
        a.zchunk = ctu_zchunk(a.n, sizeof(T) == 4);
        const dim3 grid(a.tiles_x * ((a.n[1] + TY - 1) / TY), (a.n[2] + a.zchunk - 1) / a.zchunk);
        k<<<grid, TX * TY, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

long long ctu3d_blocks(const int n[3], bool fp32)
{
    // upper bound over chunk lengths (at least one plane per chunk)
    return (long long)((n[0] + CTU_TX - 1) / CTU_TX) * ((n[1] + ctu_ty(fp32) - 1) / ctu_ty(fp32)) * n[2];
}

cudaError_t launch_ctu3d(const StepArgs &a, cudaStream_t s, bool fp32, bool hse)
{
    if (hse) return fp32 ? launch_ctu<float, true, 16, 16>(a, s) : launch_ctu<double, true, 16, 8>(a, s);
    return fp32 ? launch_ctu<float, false, 16, 16>(a, s) : launch_ctu<double, false, 16, 8>(a, s);
}

}  // namespace hydro
