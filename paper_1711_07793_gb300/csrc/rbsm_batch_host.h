// Host side of a batched launch, shared by rbsm_batch.cu (the batch entry
// points) and rbsm_stager.cu (host-resident batches).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "rbsm.h"
#include "rbsm_batch_kernel.cuh"

namespace rbsm {

// Launch shape of a batched launch: kernel variant, grid and dynamic shared
// memory.  Kept apart from the launch itself so that it runs before any
// stream capture (it sets a function attribute and queries occupancy).
struct LaunchShape {
    BatchKernelFn kernel;
    int threads;
    unsigned grid;
    size_t smem;
    int chunk;                      // warp tiles per claim (BatchArgs::chunk_tiles)
};

// Validate a batch and fill the kernel arguments (everything but the
// workspace pointers).  Returns RBSM_OK or RBSM_ERR_ARG.
int prepare_batch(const rbsm_batch *b, BatchArgs &a, int *threads);
// Kernel variant, grid and shared memory for a prepared batch; chunk = warp
// tiles per claim (1, 2, 4, 8), 0 = chosen from the batch size.
int launch_shape(const BatchArgs &args, int threads, int ctas_per_sm, int chunk, LaunchShape *out);
int check_workspace(const void *ws, size_t bytes);
// Point the kernel arguments at the counter, status word and statistics of
// a workspace.
void bind_workspace(BatchArgs &a, void *ws);
// Enqueue the workspace memset and the kernel (nothing for an empty batch);
// sets a.chunk_tiles from the shape.
int enqueue_batch(BatchArgs &a, const LaunchShape &sh, void *ws, cudaStream_t s);

}  // namespace rbsm
