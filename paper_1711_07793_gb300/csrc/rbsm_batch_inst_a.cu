// Instantiations of batch_kernel: 256 threads, 4 CTAs per SM (64 registers),
// exact and learned, run-time and batch-uniform modes.
#include "rbsm_batch_kernel.cuh"

namespace rbsm {

BatchKernelFn batch_kernel_256_4(bool learned, int umode)
{
    if (learned) {
        switch (umode) {
        case 3: return batch_kernel<256, true, 4, 3>;
        case 4: return batch_kernel<256, true, 4, 4>;
        default: return batch_kernel<256, true, 4, 0>;
        }
    }
    switch (umode) {
    case 1: return batch_kernel<256, false, 4, 1>;
    case 2: return batch_kernel<256, false, 4, 2>;
    case 3: return batch_kernel<256, false, 4, 3>;
    case 4: return batch_kernel<256, false, 4, 4>;
    case 5: return batch_kernel<256, false, 4, 5>;
    case 6: return batch_kernel<256, false, 4, 6>;
    default: return batch_kernel<256, false, 4, 0>;
    }
}

}  // namespace rbsm
