// Instantiations of batch_kernel: 256 threads, 5 CTAs per SM (48 registers;
// the next tile waits in shared memory, not in registers).
#include "rbsm_batch_kernel.cuh"

namespace rbsm {

BatchKernelFn batch_kernel_256_5(int umode)
{
    switch (umode) {
    case 1: return batch_kernel<256, false, 5, 1>;
    case 2: return batch_kernel<256, false, 5, 2>;
    case 3: return batch_kernel<256, false, 5, 3>;
    case 4: return batch_kernel<256, false, 5, 4>;
    case 5: return batch_kernel<256, false, 5, 5>;
    case 6: return batch_kernel<256, false, 5, 6>;
    default: return batch_kernel<256, false, 5, 0>;
    }
}

}  // namespace rbsm
