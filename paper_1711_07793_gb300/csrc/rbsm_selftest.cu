// Diagnostic of the bounded mbarrier wait that every tensor-core kernel of
// the library uses (tc::mbar_wait): run on a barrier that nothing arrives
// at, it must give up after its limit and let the kernel return, so that a
// lost completion shows up as RBSM_ERR_TIMEOUT on the host instead of a
// hung GPU.  The kernel also checks the other side: after one arrival the
// same wait completes.
#include <cuda_runtime.h>

#include <cstdint>

#include "rbsm.h"
#include "rbsm_host.h"
#include "rbsm_tc.cuh"

namespace rbsm {
namespace {

__global__ void bounded_wait_kernel(uint64_t limit_ns, unsigned long long *out)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0)
        return;
    tc::mbar_init(&bar, 1);
    const uint64_t t0 = tc::global_ns();
    const bool first = tc::mbar_wait(&bar, 0, limit_ns);      // phase 0 has no arrival
    const uint64_t t1 = tc::global_ns();
    tc::mbar_arrive(&bar);                                     // completes phase 0
    const bool second = tc::mbar_wait(&bar, 0, limit_ns);
    out[0] = first ? 0ull : 1ull;
    out[1] = second ? 1ull : 0ull;
    out[2] = (unsigned long long)(t1 - t0);
}

}  // namespace
}  // namespace rbsm

extern "C" int rbsm_selftest_bounded_wait(uint64_t limit_ns, uint64_t *out, void *stream)
{
    using namespace rbsm;
    if (!out || limit_ns < 1000ull || limit_ns > 1000000000ull)
        return RBSM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(out) & 7u) != 0)
        return RBSM_ERR_ARG;
    bounded_wait_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        limit_ns, reinterpret_cast<unsigned long long *>(out));
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RBSM_OK : cuda_fail(e);
}
