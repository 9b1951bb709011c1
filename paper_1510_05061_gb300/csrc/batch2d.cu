// batch2d.cu -- the persistent batched 2D step, both precisions.
#include "launchers.h"
#include "per_device.h"
#include "step2d.cuh"

namespace hydro {

namespace {

template <typename T>
struct Batch2D {
    static cudaError_t ensure(int *grid)
    {
        static PerDeviceInt cache;   // per device: shared-memory limit and resident grid
        return persistent_grid(cache, step2d_batch_kernel<T, BATCH2D_TX, BATCH2D_TY>,
                               Step2DSmem<T, BATCH2D_TX, BATCH2D_TY>::bytes, BATCH2D_TX * BATCH2D_TY, grid);
    }
    static int max_grid()
    {
        int cap = 0;
        return ensure(&cap) == cudaSuccess ? cap : 0;
    }
};

}  // namespace

cudaError_t launch_batch2d(bool fp32, const BatchInst *insts, BatchQueue *q, int parity, int grid,
                           cudaStream_t s)
{
    constexpr int NT = BATCH2D_TX * BATCH2D_TY;
    if (fp32) {
        int cap = 0;
        cudaError_t e = Batch2D<float>::ensure(&cap);
        if (e != cudaSuccess) return e;
        step2d_batch_kernel<float, BATCH2D_TX, BATCH2D_TY>
            <<<grid, NT, Step2DSmem<float, BATCH2D_TX, BATCH2D_TY>::bytes, s>>>(insts, q, parity);
    } else {
        int cap = 0;
        cudaError_t e = Batch2D<double>::ensure(&cap);
        if (e != cudaSuccess) return e;
        step2d_batch_kernel<double, BATCH2D_TX, BATCH2D_TY>
            <<<grid, NT, Step2DSmem<double, BATCH2D_TX, BATCH2D_TY>::bytes, s>>>(insts, q, parity);
    }
    return cudaGetLastError();
}

int batch2d_max_grid(bool fp32)
{
    return fp32 ? Batch2D<float>::max_grid() : Batch2D<double>::max_grid();
}

}  // namespace hydro
