// A device-side wait that must run out: one CTA waits, through the same
// bounded mbarrier wait every kernel of the library uses, for an mbarrier
// phase that nothing completes, then polls a word that nothing sets. Both
// waits give up after `polls` tries, and the kernel records DEV_ERR_TIMEOUT
// in the status word the host reads: no trap, no hang, and the context stays
// usable. It exercises the failure path of the library's waits without
// faulting a GPU.
#include "../fa_internal.h"
#include "tc_util.cuh"

namespace fa {

__global__ void k_wait_nothing(uint32_t polls, const volatile uint32_t *flag, uint32_t *err) {
    __shared__ __align__(8) uint64_t mb;
    if (threadIdx.x == 0) tc::mbar_init(&mb, 1);
    __syncthreads();
    bool ok = tc::mbar_wait(&mb, 0u, polls);  // no thread ever arrives
    uint32_t i = 0;
    while (i < polls && *flag == 0u) ++i;     // no one ever writes the flag
    ok = ok && i < polls;
    if (!ok && threadIdx.x == 0) atomicOr(err, DEV_ERR_TIMEOUT);
}

void launch_wait_nothing(uint32_t polls, const uint32_t *flag, uint32_t *err, cudaStream_t st) {
    k_wait_nothing<<<1, 32, 0, st>>>(polls, flag, err);
    FA_CHECK_CUDA(cudaGetLastError());
}

}  // namespace fa
