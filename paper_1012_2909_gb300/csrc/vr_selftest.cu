// Failure-detection self-test of the bounded device waits.
//
// The brick pass waits on an mbarrier for each TMA copy, with a bounded number
// of polls; on expiry it records a status word in mapped host memory and its
// CTA returns, and the next call reports VR_ERR_INTERNAL.  A real expiry needs
// a copy that never completes, which does not happen.  This probe reaches the
// same code without any copy: one thread arms a barrier phase with a
// transaction count that nothing will deliver and waits on it with the same
// bounded wait (a shorter time bound), which gives up and records the status.
// No asynchronous copy is ever in flight, so the kernel exits cleanly.
#include "vr_internal.cuh"
#include "vr_tma.cuh"

namespace vr {

namespace {

__global__ void k_wait_probe(int* status, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, 16u);  // 16 bytes that no copy will bring: phase 0 stays open
    mbar_wait(&bar, 0u, status, limit_ns);
}

}  // namespace

cudaError_t launch_wait_probe(int* status, unsigned long long limit_ns, cudaStream_t s) {
    k_wait_probe<<<1, 32, 0, s>>>(status, limit_ns);
    return cudaGetLastError();
}

}  // namespace vr
