// Instantiations of batch_kernel: 256 threads, 3 CTAs per SM (80 registers).
#include "rbsm_batch_kernel.cuh"

namespace rbsm {

BatchKernelFn batch_kernel_256_3(int umode)
{
    switch (umode) {
    case 1: return batch_kernel<256, false, 3, 1>;
    case 2: return batch_kernel<256, false, 3, 2>;
    case 3: return batch_kernel<256, false, 3, 3>;
    case 4: return batch_kernel<256, false, 3, 4>;
    case 5: return batch_kernel<256, false, 3, 5>;
    case 6: return batch_kernel<256, false, 3, 6>;
    default: return batch_kernel<256, false, 3, 0>;
    }
}

}  // namespace rbsm
