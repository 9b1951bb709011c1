// batch2d.cu -- the persistent batched 2D step, both precisions.
#include "launchers.h"
#include "step2d.cuh"

namespace hydro {

namespace {

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <typename K>
cudaError_t prepare(K kernel, size_t smem, int threads, int *max_grid)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    *max_grid = (nb > 0 ? nb : 1) * sm_count();
    return cudaSuccess;
}

template <typename T>
struct Batch2D {
    static int &grid_cap() { static int g = 0; return g; }
    static cudaError_t ensure()
    {
        if (grid_cap()) return cudaSuccess;
        return prepare(step2d_batch_kernel<T, BATCH2D_TX, BATCH2D_TY>, Step2DSmem<T, BATCH2D_TX, BATCH2D_TY>::bytes,
                       BATCH2D_TX * BATCH2D_TY, &grid_cap());
    }
};

}  // namespace

cudaError_t launch_batch2d(bool fp32, const BatchInst *insts, const BatchItem *items, int nitems,
                           int parity, int grid, cudaStream_t s)
{
    constexpr int NT = BATCH2D_TX * BATCH2D_TY;
    if (fp32) {
        cudaError_t e = Batch2D<float>::ensure();
        if (e != cudaSuccess) return e;
        step2d_batch_kernel<float, BATCH2D_TX, BATCH2D_TY>
            <<<grid, NT, Step2DSmem<float, BATCH2D_TX, BATCH2D_TY>::bytes, s>>>(insts, items, nitems, parity);
    } else {
        cudaError_t e = Batch2D<double>::ensure();
        if (e != cudaSuccess) return e;
        step2d_batch_kernel<double, BATCH2D_TX, BATCH2D_TY>
            <<<grid, NT, Step2DSmem<double, BATCH2D_TX, BATCH2D_TY>::bytes, s>>>(insts, items, nitems, parity);
    }
    return cudaGetLastError();
}

int batch2d_max_grid(bool fp32)
{
    if (fp32) return Batch2D<float>::ensure() == cudaSuccess ? Batch2D<float>::grid_cap() : 0;
    return Batch2D<double>::ensure() == cudaSuccess ? Batch2D<double>::grid_cap() : 0;
}

}  // namespace hydro
