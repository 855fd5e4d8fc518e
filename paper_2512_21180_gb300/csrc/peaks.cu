// Shared-memory read bandwidth of the GPU, measured: the roofline denominator of the
// projector kernels, whose bilinear samples are read from shared memory (their
// binding level is the SM's L1/shared-memory datapath, not HBM).
//
// Every thread of many resident CTAs reads 16-byte words of a 16 KB shared buffer,
// lane-consecutive (a warp's read is 512 contiguous bytes: four wavefronts, no bank
// conflict), four independent accumulators, `iters` rounds of four reads. The loads are
// ld.volatile.shared, which the compiler may neither merge nor hoist out of the loop
// (a plain load of a loop-invariant address could be read once), and the adds keep
// them live.
#include "common.cuh"

namespace cbct {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeWords = 1024;  // float4 words = 16 KB

__global__ void __launch_bounds__(kProbeThreads) k_smem_probe(int iters, float *sink) {
    __shared__ __align__(16) float4 buf[kProbeWords];
    for (int i = threadIdx.x; i < kProbeWords; i += kProbeThreads)
        buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf) + 16u * threadIdx.x;
    float4 acc[4] = {};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 v;
            asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                         : "r"(base + (uint32_t)(k * kProbeThreads * 16)));
            acc[k].x += v.x; acc[k].y += v.y; acc[k].z += v.z; acc[k].w += v.w;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += acc[k].x + acc[k].y + acc[k].z + acc[k].w;
    if (s == -1.f) sink[blockIdx.x] = s;  // never true; keeps the sums live
}

}  // namespace
}  // namespace cbct

using namespace cbct;

extern "C" int cbct_smem_probe(int ctas_per_sm, int iters, float *sink, long long *bytes, void *stream) {
    if (ctas_per_sm < 1 || ctas_per_sm > 8 || iters < 1 || iters > (1 << 20) || !sink || !bytes)
        return fail(CBCT_EINVAL, "cbct_smem_probe: need 1 <= ctas_per_sm <= 8, 1 <= iters <= 2^20, sink, bytes");
    int dev = 0, nsm = 0;
    CBCT_CUDA_TRY(cudaGetDevice(&dev));
    CBCT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = nsm * ctas_per_sm;
    k_smem_probe<<<grid, kProbeThreads, 0, (cudaStream_t)stream>>>(iters, sink);
    CBCT_LAUNCH_CHECK("cbct_smem_probe");
    *bytes = (long long)grid * kProbeThreads * iters * 4LL * 16LL;
    return 0;
}
