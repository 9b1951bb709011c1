// probe.cu -- throughput probe of the fused multiply-add pipe, the
// denominator of the step kernels' arithmetic roofline.
//
// Every thread runs NCHAIN independent chains x <- x * a + b (one FMA each,
// 2 flops) for `iters` rounds and stores the chains' sum, so that no FMA is
// dead code.  With enough resident warps and independent chains the pipe,
// not latency, bounds the kernel; its time then measures the FMA rate the
// step kernels' FP64 (or FP32) arithmetic competes for.
#include <cuda_runtime.h>

#include "../../include/hydro.h"

namespace {

constexpr int NCHAIN = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(long long iters, T a, T b, T *__restrict__ out)
{
    T x[NCHAIN];
#pragma unroll
    for (int i = 0; i < NCHAIN; ++i) x[i] = T(threadIdx.x % 7 + i) * T(1e-3);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < NCHAIN; ++i) x[i] = fma(x[i], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < NCHAIN; ++i) s += x[i];
    out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int hydro_fma_probe(int precision, long long iters, int ctas, int threads, void *out,
                               void *stream)
{
    if ((precision != HYDRO_FP64 && precision != HYDRO_FP32) || iters < 1 || ctas < 1 ||
        threads < 32 || threads > 256 || threads % 32 != 0 || !out)
        return HYDRO_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // a slightly contracting map keeps every chain bounded for any iters
    if (precision == HYDRO_FP64)
        fma_probe_kernel<double><<<ctas, threads, 0, s>>>(iters, 0.999999, 1e-7, static_cast<double *>(out));
    else
        fma_probe_kernel<float><<<ctas, threads, 0, s>>>(iters, 0.9999f, 1e-4f, static_cast<float *>(out));
    return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
}

extern "C" double hydro_fma_probe_flops(long long iters, int ctas, int threads)
{
    return 2.0 * NCHAIN * (double)iters * (double)ctas * (double)threads;
}
