// per_device.h -- one-time set-up per CUDA device.
//
// Kernel attributes such as the dynamic shared-memory limit belong to the
// device context a kernel is launched in, and occupancy-derived grid sizes
// depend on the device's SM count.  One process may drive several devices
// (for instance one host thread per GPU, or a slab decomposition spread over
// GPUs), so the "already configured" state is kept per device ordinal, and
// set-ups running on different host threads at the same time are serialised.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

namespace hydro {

constexpr int MAX_DEVICES = 64;

// Runs a set-up function at most once with success per device ordinal.  A
// failed set-up is not remembered: the next call for that device retries it.
class PerDeviceOnce {
public:
    template <typename F>
    cudaError_t run(int dev, F &&setup)
    {
        if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
        if (done_[dev].load(std::memory_order_acquire)) return cudaSuccess;
        std::lock_guard<std::mutex> lock(mutex_);
        if (done_[dev].load(std::memory_order_relaxed)) return cudaSuccess;
        const cudaError_t e = setup();
        if (e == cudaSuccess) done_[dev].store(true, std::memory_order_release);
        return e;
    }

private:
    std::mutex mutex_;
    std::atomic<bool> done_[MAX_DEVICES] = {};
};

// An int computed once with success per device ordinal (a resident grid
// size, an SM count); 0 means "not yet computed".
class PerDeviceInt {
public:
    template <typename F>
    cudaError_t get(int dev, F &&compute, int *out)
    {
        if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
        int v = value_[dev].load(std::memory_order_acquire);
        if (v == 0) {
            std::lock_guard<std::mutex> lock(mutex_);
            v = value_[dev].load(std::memory_order_relaxed);
            if (v == 0) {
                const cudaError_t e = compute(&v);
                if (e != cudaSuccess) return e;
                value_[dev].store(v, std::memory_order_release);
            }
        }
        *out = v;
        return cudaSuccess;
    }

private:
    std::mutex mutex_;
    std::atomic<int> value_[MAX_DEVICES] = {};
};

// Sets kernel k's dynamic shared-memory limit to smem on the current device,
// once per device.  `once` must be specific to the kernel.
template <typename K>
cudaError_t ensure_smem_limit(PerDeviceOnce &once, K k, size_t smem)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    return once.run(dev, [&] { return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); });
}

// SM count of the current device.
inline cudaError_t current_sm_count(int *out)
{
    static PerDeviceInt cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    return cache.get(dev, [&](int *v) {
        cudaError_t r = cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev);
        if (r == cudaSuccess && *v <= 0) *v = 1;
        return r;
    }, out);
}

// Resident grid (CTAs per SM at full occupancy x SMs) of a persistent kernel
// on the current device; the kernel's shared-memory limit is set on the way,
// both once per device.  `cache` must be specific to the kernel.
template <typename K>
cudaError_t persistent_grid(PerDeviceInt &cache, K kernel, size_t smem, int threads, int *max_grid)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    return cache.get(dev, [&](int *v) {
        cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r != cudaSuccess) return r;
        int nb = 0;
        r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem);
        if (r != cudaSuccess) return r;
        int sms = 0;
        r = current_sm_count(&sms);
        if (r != cudaSuccess) return r;
        *v = (nb > 0 ? nb : 1) * sms;
        return cudaSuccess;
    }, max_grid);
}

}  // namespace hydro
