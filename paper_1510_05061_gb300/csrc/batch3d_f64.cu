// batch3d_f64.cu -- FP64 instantiations of the persistent batched 3D step
// for every tile shape the autotuner may choose, both modes.
#include "launchers.h"
#include "per_device.h"
#include "step3d.cuh"

namespace hydro {

namespace {

template <typename T, bool HSE, int TX, int TY, bool AS>
struct Batch3D {
    static cudaError_t ensure(int *grid)
    {
        static PerDeviceInt cache;   // per device: shared-memory limit and resident grid
        return persistent_grid(cache, step3d_batch_kernel<T, HSE, TX, TY, AS>,
                               Step3DSmem<T, HSE, TX, TY, RECON_PLM, AS>::bytes, TX * TY, grid);
    }
    static cudaError_t launch(const BatchInst *insts, BatchQueue *q, int parity, int grid, cudaStream_t s)
    {
        int cap = 0;
        cudaError_t e = ensure(&cap);
        if (e != cudaSuccess) return e;
        step3d_batch_kernel<T, HSE, TX, TY, AS>
            <<<grid, TX * TY, Step3DSmem<T, HSE, TX, TY, RECON_PLM, AS>::bytes, s>>>(insts, q, parity);
        return cudaGetLastError();
    }
    static int max_grid()
    {
        int cap = 0;
        return ensure(&cap) == cudaSuccess ? cap : 0;
    }
};

template <bool HSE>
cudaError_t launch_v(int v, const BatchInst *insts, BatchQueue *q, int parity, int grid, cudaStream_t s)
{
    switch (v) {
    case 0: return Batch3D<double, HSE, 32, 8, false>::launch(insts, q, parity, grid, s);
    case 1: return Batch3D<double, HSE, 32, 4, false>::launch(insts, q, parity, grid, s);
    case 2: return Batch3D<double, HSE, 16, 16, false>::launch(insts, q, parity, grid, s);
    case 4: return Batch3D<double, HSE, 32, 8, true>::launch(insts, q, parity, grid, s);
    case 5: return Batch3D<double, HSE, 32, 4, true>::launch(insts, q, parity, grid, s);
    case 6: return Batch3D<double, HSE, 16, 16, true>::launch(insts, q, parity, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <bool HSE>
int grid_v(int v)
{
    switch (v) {
    case 0: return Batch3D<double, HSE, 32, 8, false>::max_grid();
    case 1: return Batch3D<double, HSE, 32, 4, false>::max_grid();
    case 2: return Batch3D<double, HSE, 16, 16, false>::max_grid();
    case 4: return Batch3D<double, HSE, 32, 8, true>::max_grid();
    case 5: return Batch3D<double, HSE, 32, 4, true>::max_grid();
    case 6: return Batch3D<double, HSE, 16, 16, true>::max_grid();
    default: return 0;
    }
}

}  // namespace

cudaError_t launch_batch3d_f64(int variant, bool hse, const BatchInst *insts, BatchQueue *q, int parity,
                               int grid, cudaStream_t s)
{
    return hse ? launch_v<true>(variant, insts, q, parity, grid, s) : launch_v<false>(variant, insts, q, parity, grid, s);
}

int batch3d_max_grid_f64(int variant, bool hse)
{
    return hse ? grid_v<true>(variant) : grid_v<false>(variant);
}

}  // namespace hydro
