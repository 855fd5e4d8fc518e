// Resampling between the levels of the multiscale reconstruction (a11; paper Sec. 2.6,
// the multiscale scheme: the coarse level works on half-resolution volumes and on
// projections with every second angle and 2 x 2 binned pixels, and its result is
// carried to the fine level by upsampling).
//
// Both kernels act on nch independent 3-D arrays [n0][n1][n2] (channels or batch
// first, the last index fastest):
//  down: out[c][i][j][k] = scale * sum over the box (i f0 + a, j f1 + b, k f2 + d),
//        a < f0 (or only a = 0 with pick0: axis 0 subsampled instead of summed),
//        b < f1, d < f2 — average pooling (scale 1/f0f1f2), the 2 x 2 pixel binning of
//        every second angle (pick0, scale 1/4) and the adjoint of nearest upsampling
//        (scale 1);
//  up:   out[c][i][j][k] = in[c][i / f0][j / f1][k / f2] (nearest neighbour).
#include "common.cuh"
#include "geom_impl.h"

namespace cbct {

__global__ void k_resample_down(const float *__restrict__ in, long long nch, int n0, int n1, int n2, int f0, int f1,
                                int f2, int pick0, float scale, float *__restrict__ out) {
    const int m0 = n0 / f0, m1 = n1 / f1, m2 = n2 / f2;
    const long long total = nch * m0 * m1 * m2;
    const int a_end = pick0 ? 1 : f0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % m2);
        long long t = e / m2;
        const int j = (int)(t % m1);
        t /= m1;
        const int i = (int)(t % m0);
        const long long c = t / m0;
        const float *src = in + ((c * n0 + (long long)i * f0) * n1 + (long long)j * f1) * n2 + (long long)k * f2;
        float s = 0.f;
        for (int a = 0; a < a_end; ++a)
            for (int b = 0; b < f1; ++b)
                for (int d = 0; d < f2; ++d) s += src[((long long)a * n1 + b) * n2 + d];
        out[e] = s * scale;
    }
}

__global__ void k_resample_up(const float *__restrict__ in, long long nch, int n0, int n1, int n2, int f0, int f1, int f2,
                              float *__restrict__ out) {
    const int m0 = n0 * f0, m1 = n1 * f1, m2 = n2 * f2;
    const long long total = nch * m0 * m1 * m2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % m2);
        long long t = e / m2;
        const int j = (int)(t % m1);
        t /= m1;
        const int i = (int)(t % m0);
        const long long c = t / m0;
        out[e] = in[((c * n0 + i / f0) * n1 + j / f1) * n2 + k / f2];
    }
}

static int grid_for(long long n) {
    const long long b = (n + 255) / 256;
    const long long cap = 32LL * sm_count();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace cbct

using namespace cbct;

extern "C" int cbct_resample_down(const float *in, long long nch, int n0, int n1, int n2, int f0, int f1, int f2,
                                  int pick0, float scale, float *out, void *stream) {
    if (!in || !out || nch < 1 || n0 < 1 || n1 < 1 || n2 < 1 || f0 < 1 || f1 < 1 || f2 < 1 || n0 % f0 || n1 % f1 ||
        n2 % f2)
        return fail(CBCT_EINVAL, "cbct_resample_down: sizes must be positive and divisible by the factors");
    const long long total = nch * (n0 / f0) * (long long)(n1 / f1) * (n2 / f2);
    k_resample_down<<<grid_for(total), 256, 0, (cudaStream_t)stream>>>(in, nch, n0, n1, n2, f0, f1, f2, pick0 ? 1 : 0,
                                                                       scale, out);
    CBCT_LAUNCH_CHECK("cbct_resample_down");
    return 0;
}

extern "C" int cbct_resample_up(const float *in, long long nch, int n0, int n1, int n2, int f0, int f1, int f2, float *out,
                                void *stream) {
    if (!in || !out || nch < 1 || n0 < 1 || n1 < 1 || n2 < 1 || f0 < 1 || f1 < 1 || f2 < 1)
        return fail(CBCT_EINVAL, "cbct_resample_up: sizes and factors must be positive");
    const long long total = nch * (long long)n0 * f0 * n1 * f1 * n2 * f2;
    k_resample_up<<<grid_for(total), 256, 0, (cudaStream_t)stream>>>(in, nch, n0, n1, n2, f0, f1, f2, out);
    CBCT_LAUNCH_CHECK("cbct_resample_up");
    return 0;
}
