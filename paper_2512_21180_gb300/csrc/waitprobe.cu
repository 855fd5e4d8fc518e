// Probe of the bounded-wait path every pipelined kernel of the library relies on:
// a kernel whose warps wait on a shared-memory barrier that nothing completes, with
// the caller's time limit. It exercises exactly the library's mbar_wait (timeout,
// status word, early return), so the path a real kernel takes when its pipeline
// stalls can be tested without a stalled pipeline.
#include "common.cuh"
#include "geom_impl.h"
#include "tma.cuh"

namespace cbct {
namespace {

// One CTA: thread 0 initialises a barrier expecting one arrival that never comes;
// every warp's lane 0 then waits on phase 0 with the limit. The abort flag mirrors
// what the pipelined kernels do: the first warp to give up tells the others.
__global__ void k_wait_probe(int *status, uint64_t limit_ns, int *waited_ok) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        bool ok = false;
        if (!abort_flag) ok = mbar_wait(&bar, 0u, status, limit_ns);
        if (!ok) abort_flag = 1;
        if (ok) atomicAdd(waited_ok, 1);
    }
    __syncthreads();
}

}  // namespace
}  // namespace cbct

using namespace cbct;

extern "C" int cbct_wait_probe(const cbct_geom *g, long long limit_ns, int *waited_ok, void *stream) {
    if (!g || !waited_ok || limit_ns < 1 || limit_ns > 100000000LL)
        return fail(CBCT_EINVAL, "cbct_wait_probe: need a geometry, a device counter and 1 <= limit_ns <= 1e8");
    k_wait_probe<<<1, 64, 0, (cudaStream_t)stream>>>(g->status, (uint64_t)limit_ns, waited_ok);
    CBCT_LAUNCH_CHECK("cbct_wait_probe");
    return 0;
}
