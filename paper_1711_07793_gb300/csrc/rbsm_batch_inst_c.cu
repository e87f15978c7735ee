// Instantiations of batch_kernel: 128 and 512 threads (run-time modes).
#include "rbsm_batch_kernel.cuh"

namespace rbsm {

BatchKernelFn batch_kernel_misc(int threads, bool learned)
{
    if (threads == 128)
        return learned ? batch_kernel<128, true, 8, 0> : batch_kernel<128, false, 8, 0>;
    return learned ? batch_kernel<512, true, 2, 0> : batch_kernel<512, false, 2, 0>;
}

}  // namespace rbsm
