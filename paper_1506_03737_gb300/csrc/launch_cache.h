// Host-side launch helpers of the persistent FFT kernels: the dynamic shared-memory attribute
// and the persistent grid size (resident CTAs per SM x SMs), cached per device.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

namespace colapm {

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Persistent grid: resident CTAs per SM x SMs.
template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    if (per < 1) per = 1;
    return per * sms;
}

// Launch configuration of one kernel on each device: its dynamic shared-memory attribute (set
// once per device, raised when a larger size is asked for) and the persistent grid for that size.
// A mutex guards it, so launchers may run from several host threads and on several devices.
constexpr int kMaxDevices = 64;
struct GridCache {
    std::mutex mu;
    int grid[kMaxDevices] = {};
    size_t smem[kMaxDevices] = {};
};

template <typename K>
static cudaError_t cached_grid(GridCache& c, K kernel, int threads, size_t smem, int* grid) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(c.mu);
    if (!c.grid[dev] || smem > c.smem[dev]) {
        e = set_smem(kernel, smem);
        if (e != cudaSuccess) return e;
        if (smem > c.smem[dev]) c.smem[dev] = smem;
        c.grid[dev] = persistent_grid(kernel, threads, c.smem[dev]);
    }
    *grid = c.grid[dev];
    return cudaSuccess;
}

}  // namespace colapm
