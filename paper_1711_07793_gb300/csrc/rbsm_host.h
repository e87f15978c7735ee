// Host helpers shared by the translation units of the RBSM library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "rbsm.h"
#include "rbsm_device.cuh"

namespace rbsm {

int cuda_fail(cudaError_t e);
int check_map(const rbsm_map *m);
int check_frags(const rbsm_frags *f);
int check_params(const rbsm_params *p, int *max_dist);
// True when [out, out + bytes) overlaps the fragment planes or the map.
bool overlaps_inputs(const rbsm_map &m, const rbsm_frags &f, const void *out, size_t bytes);
bool aligned16(const void *p);
int device_sm_count();
MapDev to_dev(const rbsm_map &m);

// Per-device cache of "dynamic shared memory attribute set + occupancy" for
// one kernel.  The attribute is a per-device property, so it is set once on
// every device the kernel is launched on.  Host threads may race on the
// first launch: each computes the same value, and the slots are atomics.
struct KernelSetup {
    static constexpr int kMaxDevices = 64;
    std::atomic<int> occupancy[kMaxDevices] = {};

    template <typename Kernel>
    int get(Kernel kern, int threads, size_t smem, int *occ)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess)
            return cuda_fail(e);
        if (dev < 0 || dev >= kMaxDevices)
            return cuda_fail(cudaErrorInvalidDevice);
        int known = occupancy[dev].load(std::memory_order_acquire);
        if (known == 0) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess)
                return cuda_fail(e);
            int o = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, threads, smem);
            if (e != cudaSuccess)
                return cuda_fail(e);
            if (o < 1)
                return cuda_fail(cudaErrorInvalidConfiguration);
            occupancy[dev].store(o, std::memory_order_release);
            known = o;
        }
        *occ = known;
        return RBSM_OK;
    }
};

}  // namespace rbsm
