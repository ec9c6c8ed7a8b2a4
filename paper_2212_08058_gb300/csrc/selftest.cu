// selftest.cu -- a check of the failure-reporting path that every bounded wait in this library
// takes (TMA completion in the stencil, TMA and MMA completion in the network): a kernel waits on
// an mbarrier that nothing will ever complete, gives up after a bounded number of try_wait
// attempts, raises the timeout flag and returns; the host then reports TIMEOUT and the context
// stays usable.  No copy or MMA is in flight, so nothing has to be drained.
#include "../../include/sfseg.h"
#include "common.cuh"
#include "launch.h"

namespace sfseg {

__global__ void wait_probe_kernel(long long spins, int* flags) {
    __shared__ uint64_t bar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool done = false;
    for (long long i = 0; i < spins && !done; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(0)
            : "memory");
        done = ok != 0;
    }
    if (!done && threadIdx.x == 0) atomicOr(flags, kFlagTimeout);
}

void launch_wait_probe(long long spins, int* flags, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(spins, flags);
    count_launches(1);
}

}  // namespace sfseg
