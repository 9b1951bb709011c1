// aux.cu -- initial-state conversion, CFL signal speed, conserved totals,
// field export and the fault-injection poke.
#include <cuda_runtime.h>

#include "hydro_device.cuh"
#include "launchers.h"

namespace hydro {

namespace {

template <typename T>
__device__ __forceinline__ T *state(const AuxArgs &a) { return static_cast<T *>(a.U); }

// total primitives (FP64) -> stored conserved state
template <typename T, int ND, bool HSE>
__global__ void init_convert_kernel(const AuxArgs a, const double *__restrict__ W,
                                    long long c0, long long m)
{
    constexpr int NV = ND + 2;
    T *U = state<T>(a);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x) {
        const long long c = c0 + i;
        double u[NV];
        if (a.conserved_in) {
            // total conserved variables as given
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] = W[q * m + i];
        } else {
            const double rho = W[i];
            double ke = 0.0;
            u[0] = rho;
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const double v = W[(1 + d) * m + i];
                u[1 + d] = rho * v;
                ke += v * v;
            }
            const double p = W[(NV - 1) * m + i];
            u[NV - 1] = p / (a.gamma - 1.0) + 0.5 * rho * ke;
        }
        if (HSE) {
            const int k = (int)(c / a.plane);
            u[0] -= a.bg[k + 2].rho_c;
            u[NV - 1] -= a.bg[k + 2].p_c / (a.gamma - 1.0);
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) U[q * a.vstride + c] = T(u[q]);
    }
}

// stored state of one cell -> total primitives in T (velocity, pressure)
template <typename T, int ND, bool HSE>
__device__ __forceinline__ void cell_prims(const AuxArgs &a, const T *U, long long c, T &rho,
                                           T (&v)[3], T &p)
{
    constexpr int NV = ND + 2;
    const T gam = T(a.gamma);
    T r = U[c];
    T bgr = T(0), bgp = T(0);
    if (HSE) {
        const int k = (int)(c / a.plane);
        bgr = T(a.bg[k + 2].rho_c);
        bgp = T(a.bg[k + 2].p_c);
    }
    rho = bgr + r;
    const T rinv = T(1) / rho;
    T m2 = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = T(0);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const T m = U[(1 + d) * a.vstride + c];
        v[d] = m * rinv;
        m2 += m * m;
    }
    p = bgp + (gam - T(1)) * (U[(NV - 1) * a.vstride + c] - T(0.5) * m2 * rinv);
}

template <typename T, int ND, bool HSE>
__global__ void __launch_bounds__(AUX_THREADS) signal_kernel(const AuxArgs a)
{
    __shared__ double red[32];
    __shared__ int s_last;
    const T *U = state<T>(a);
    const T gam = T(a.gamma);
    double smax = 0.0;
    bool bad = false;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        T rho, v[3], p;
        cell_prims<T, ND, HSE>(a, U, c, rho, v, p);
        const T cs = sqrt(gam * p / rho);
        T s = T(0);
#pragma unroll
        for (int d = 0; d < ND; ++d) s += (fabs(v[d]) + cs) * T(a.inv_dx[d]);
        if (!(rho > T(0)) || !(p > T(0)) || !isfinite(s)) bad = true;
        else smax = fmax(smax, double(s));
    }
    const bool bad_cta = __syncthreads_or(bad) != 0;
    const double m = block_max<AUX_THREADS>(smax, red);
    StepArgs sa{};
    sa.ctrl = a.ctrl;
    sa.partial = a.partial;
    sa.cfl = a.cfl;
    sa.t_end = 0.0;
    finish_step<AUX_THREADS>(m, bad_cta, sa, gridDim.x, blockIdx.x, 0.0, false, &s_last);
}

// Deterministic FP64 totals: CTA b sums cells c = b*blockDim + t + j*stride
// in a fixed per-thread order, then a fixed shuffle tree; the last CTA adds
// the per-CTA partials in index order.
template <typename T, int ND, bool HSE>
__global__ void __launch_bounds__(AUX_THREADS) totals_kernel(const AuxArgs a)
{
    constexpr int NV = ND + 2;
    __shared__ double red[NV][AUX_THREADS / 32];
    __shared__ int s_last;
    const T *U = state<T>(a);
    double acc[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        double bgr = 0.0, bge = 0.0;
        if (HSE) {
            const int k = (int)(c / a.plane);
            bgr = a.bg[k + 2].rho_c;
            bge = a.bg[k + 2].p_c / (a.gamma - 1.0);
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double v = double(U[q * a.vstride + c]);
            if (q == 0) v += bgr;
            if (q == NV - 1) v += bge;
            acc[q] += v;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < AUX_THREADS / 32; ++w) s += red[q][w];
            a.partial[(size_t)blockIdx.x * NV + q] = s;
        }
        __threadfence();
        const unsigned prev = atomicAdd(&a.ctrl->counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(a.partial + (size_t)b * NV + threadIdx.x);
        a.ctrl->totals[threadIdx.x] = s * a.cell_volume;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.ctrl->counter = 0u;
        __threadfence();
    }
}

template <typename T, int ND, bool HSE>
__global__ void fields_kernel(const AuxArgs a, double *__restrict__ out, long long c0, long long m,
                              int what)
{
    constexpr int NV = ND + 2;
    const T *U = state<T>(a);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x) {
        const long long c = c0 + i;
        if (what == 0) {
            double bgr = 0.0, bge = 0.0;
            if (HSE) {
                const int k = (int)(c / a.plane);
                bgr = a.bg[k + 2].rho_c;
                bge = a.bg[k + 2].p_c / (a.gamma - 1.0);
            }
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                double v = double(U[q * a.vstride + c]);
                if (q == 0) v += bgr;
                if (q == NV - 1) v += bge;
                out[q * m + i] = v;
            }
        } else {
            // primitives in FP64 from the stored values
            double bgr = 0.0, bgp = 0.0;
            if (HSE) {
                const int k = (int)(c / a.plane);
                bgr = a.bg[k + 2].rho_c;
                bgp = a.bg[k + 2].p_c;
            }
            const double rho = bgr + double(U[c]);
            double m2 = 0.0;
            out[i] = rho;
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const double mv = double(U[(1 + d) * a.vstride + c]);
                out[(1 + d) * m + i] = mv / rho;
                m2 += mv * mv;
            }
            out[(NV - 1) * m + i] = bgp + (a.gamma - 1.0) * (double(U[(NV - 1) * a.vstride + c]) - 0.5 * m2 / rho);
        }
    }
}

__global__ void math_kernel(int which, const double *__restrict__ x, const double *__restrict__ y,
                            double *__restrict__ out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (which == 0) out[i] = rcp_t(x[i]);
        else if (which == 1) out[i] = div_t(y[i], x[i]);
        else if (which == 2) out[i] = rsqrt_t(x[i]);
        else out[i] = mc_slope(x[i], y[i]);
    }
}

template <typename T>
__global__ void poke_kernel(const AuxArgs a, int var, long long cell, double v)
{
    state<T>(a)[var * a.vstride + cell] = T(v);
}

int grid_for(long long m)
{
    long long b = (m + 255) / 256;
    if (b > 8192) b = 8192;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int aux_reduce_blocks(long long N)
{
    long long b = (N + 4 * AUX_THREADS - 1) / (4 * AUX_THREADS);
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return (int)b;
}

#define HYDRO_DISPATCH(KERNEL, GRID, BLOCK, STREAM, ...)                                  \
    do {                                                                                  \
        if (a.fp32) {                                                                     \
            if (a.ndim == 2) KERNEL<float, 2, false><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); \
            else if (a.hse) KERNEL<float, 3, true><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__);   \
            else KERNEL<float, 3, false><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__);             \
        } else {                                                                          \
            if (a.ndim == 2) KERNEL<double, 2, false><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); \
            else if (a.hse) KERNEL<double, 3, true><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__);   \
            else KERNEL<double, 3, false><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__);             \
        }                                                                                 \
    } while (0)

cudaError_t launch_init_convert(const AuxArgs &a, const double *staging, long long c0,
                                long long m, cudaStream_t s)
{
    HYDRO_DISPATCH(init_convert_kernel, grid_for(m), 256, s, a, staging, c0, m);
    return cudaGetLastError();
}

cudaError_t launch_signal(const AuxArgs &a, cudaStream_t s)
{
    HYDRO_DISPATCH(signal_kernel, aux_reduce_blocks(a.N), AUX_THREADS, s, a);
    return cudaGetLastError();
}

cudaError_t launch_totals(const AuxArgs &a, cudaStream_t s)
{
    HYDRO_DISPATCH(totals_kernel, aux_reduce_blocks(a.N), AUX_THREADS, s, a);
    return cudaGetLastError();
}

cudaError_t launch_fields(const AuxArgs &a, double *staging, long long c0, long long m, int what,
                          cudaStream_t s)
{
    HYDRO_DISPATCH(fields_kernel, grid_for(m), 256, s, a, staging, c0, m, what);
    return cudaGetLastError();
}

cudaError_t launch_math(int which, const double *x, const double *y, double *out, long long n,
                        cudaStream_t s)
{
    math_kernel<<<grid_for(n), 256, 0, s>>>(which, x, y, out, n);
    return cudaGetLastError();
}

cudaError_t launch_poke(const AuxArgs &a, int var, long long cell, double v, cudaStream_t s)
{
    if (a.fp32) poke_kernel<float><<<1, 1, 0, s>>>(a, var, cell, v);
    else poke_kernel<double><<<1, 1, 0, s>>>(a, var, cell, v);
    return cudaGetLastError();
}

}  // namespace hydro
