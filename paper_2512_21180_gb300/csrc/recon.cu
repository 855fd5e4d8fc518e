// Classical reconstructions: the learned method's start and the baseline it is compared with:
//  - FDK with redundancy weighting (paper Algorithm 1 initialisation "FDK_w",
//    Sec. 2.6; Feldkamp, Davis, Kress 1984): cosine and redundancy weights, Ram-Lak
//    ramp filter along detector rows at the isocentre pitch, distance-weighted
//    voxel backprojection. An offset panel's rows are zero-padded on the short side
//    to the mirror image of the long edge before filtering.
//  - PDHG (Chambolle-Pock 2011) for 1/2 ||P x - y||^2 + lam TV(x), x >= 0, isotropic
//    TV by forward differences (the paper's TV baseline, Sec. 2.5), on K = [P; gamma grad]
//    with the TV ball radius lam / gamma.
//  - Landweber iterations x <- x - tau P^T (P x - y) (the gradient term of Algorithm 1).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "geom_impl.h"

namespace cbct {

static int grid1(long long n) {
    long long b = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 32LL * sm_count()));
}

// ---- FDK ---------------------------------------------------------------------------

// q0[b][k][v][e] = proj * w(u) * sdd / sqrt(sdd^2 + u^2 + v^2) on the extended row
// (e = iu + lo), zero in the padding.
__global__ void k_fdk_weight(const float *__restrict__ proj, const float *__restrict__ w, float *__restrict__ q0,
                             int nu, int nv, int nue, int lo, int rows, float du, float dv, float uoff,
                             float voff, float sdd) {
    const int ie = blockIdx.x * blockDim.x + threadIdx.x, iu = ie - lo;
    if (ie >= nue) return;
    const float u = ((float)iu - 0.5f * (float)(nu - 1)) * du + uoff;
    const float wu = (iu >= 0 && iu < nu) ? w[iu] * sdd : 0.f;
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {
        const int iv = row % nv;
        const float v = ((float)iv - 0.5f * (float)(nv - 1)) * dv + voff;
        q0[(long long)row * nue + ie] =
            wu != 0.f ? proj[(long long)row * nu + iu] * wu * rsqrtf(sdd * sdd + u * u + v * v) : 0.f;
    }
}

// Ram-Lak filter of each extended row: q[e] = h(0) q0[e] + sum over m of the other
// parity of h(e - m) q0[m], h(d) = -1 / (pi^2 tau d^2) for odd d (zero for even d != 0).
// Per parity the sum is a Toeplitz product on the compact arrays x_j = q0[2 j + p_m]:
// out_i = sum_j g[i - j + c] x_j with g[t] = h(2 t + 1). A thread computes kRampB
// consecutive outputs of one parity and slides a window of kRampB filter taps held in
// registers along j: two shared loads per kRampB multiply-adds.
constexpr int kRampB = 8;
__global__ void __launch_bounds__(128) k_fdk_ramp(const float *__restrict__ q0, float *__restrict__ q, int nue, int nv,
                                                  float tau) {
    extern __shared__ float sm[];
    const int half = (nue + 1) / 2;                         // compact length bound, both parities
    const int npad = (half + kRampB - 1) / kRampB * kRampB;  // compact arrays padded to a block multiple
    float *xs = sm;                                          // [2][npad]: x of parity 0, then parity 1
    float *gs = xs + 2 * npad;                               // g[t] at gs[t + goff], t = -goff .. goff + ...
    float *os = gs + 2 * npad + 2 * kRampB + 2;              // [nue] filtered row
    const int goff = npad + kRampB;
    const long long r = blockIdx.x;
    const float *src = q0 + r * nue;
    const float c1 = -1.0f / (3.14159265358979f * 3.14159265358979f * tau), h0 = 1.0f / (4.0f * tau);
    for (int i = threadIdx.x; i < 2 * npad; i += blockDim.x) {
        const int p = i >= npad, j = i - p * npad, e = 2 * j + p;
        xs[i] = e < nue ? src[e] : 0.f;
    }
    for (int k = threadIdx.x; k < 2 * npad + 2 * kRampB + 2; k += blockDim.x) {
        const float d = (float)(2 * (k - goff) + 1);
        gs[k] = c1 / (d * d);
    }
    __syncthreads();
    const int nb = npad / kRampB;  // output blocks per parity
    for (int wk = threadIdx.x; wk < 2 * nb; wk += blockDim.x) {
        const int pe = wk >= nb, i0 = (wk - pe * nb) * kRampB, pm = 1 - pe;
        const int c = pe - 1;  // e - m = 2 (i - j + c) + 1
        const float *x = xs + pm * npad;
        const float *xe = xs + pe * npad;
        float acc[kRampB], R[kRampB];
#pragma unroll
        for (int b = 0; b < kRampB; ++b) {
            acc[b] = h0 * xe[i0 + b];
            R[b] = gs[goff + i0 + b + c];  // window at j = 0: win_b = g[i0 + b + c]
        }
        for (int j = 0; j < npad; j += kRampB) {
#pragma unroll
            for (int jj = 0; jj < kRampB; ++jj) {
                const float xv = x[j + jj];
#pragma unroll
                for (int b = 0; b < kRampB; ++b) acc[b] = fmaf(R[(b - jj + kRampB) % kRampB], xv, acc[b]);
                // slide: the tap that fell off becomes g[i0 + c - (j + jj) - 1]
                R[(kRampB - 1 - jj) % kRampB] = gs[goff + i0 + c - (j + jj) - 1];
            }
        }
#pragma unroll
        for (int b = 0; b < kRampB; ++b) {
            const int e = 2 * (i0 + b) + pe;
            if (e < nue) os[e] = acc[b];
        }
    }
    __syncthreads();
    // output row of the zero-padded layout [na][nv + 2][nue + 2] (one zero row and column each side)
    const long long kk = r / nv, iv = r - kk * nv;
    float *dst = q + (kk * (nv + 2) + iv + 1) * (nue + 2) + 1;
    for (int e = threadIdx.x; e < nue; e += blockDim.x) dst[e] = os[e];
}

// vol(P) (+)= (2 pi / n_angles) sum_k (sid / U)^2 bilinear(q_k, u(P), v(P)). A thread
// owns a run of kFdkZ voxels along z: the source distance U, the magnification, the
// detector column and the weight depend only on (x, y, angle) and are computed once
// per angle; the detector row is linear in z.
constexpr int kFdkZ = 8;
__global__ void __launch_bounds__(256) k_fdk_backproject(const float *__restrict__ q, const double2 *__restrict__ cs,
                                                         float *__restrict__ vol, int nx, int ny, int nz, int na, int nue,
                                                         int nv, int lo, int nu, float vx, float vy, float vz, float cx,
                                                         float cy, float cz, float sid, float sdd, float rdu, float rdv,
                                                         float uoff, float voff, int accumulate) {
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y;
    const int nzr = (nz + kFdkZ - 1) / kFdkZ;
    const int iz0 = (blockIdx.z % nzr) * kFdkZ, b = blockIdx.z / nzr;
    if (ix >= nx || iy >= ny) return;
    const float px = (ix - 0.5f * (nx - 1)) * vx + cx;
    const float py = (iy - 0.5f * (ny - 1)) * vy + cy;
    const float pz0 = (iz0 - 0.5f * (nz - 1)) * vz + cz;
    const float hu = 0.5f * (nu - 1) + lo, hv = 0.5f * (nv - 1);
    const int pitch = nue + 2;  // zero-padded rows: every bilinear neighbour is in bounds
    const float *qb = q + (long long)b * na * (nv + 2) * pitch;
    float acc[kFdkZ];
#pragma unroll
    for (int j = 0; j < kFdkZ; ++j) acc[j] = 0.f;
    for (int k = 0; k < na; ++k) {
        const double2 t = cs[k];
        const float c = (float)t.x, s = (float)t.y;
        const float U = sid - (px * c + py * s);
        if (!(U > 0.f)) continue;
        const float rU = __frcp_rn(U), m = sdd * rU;
        const float fu = (m * (-px * s + py * c) - uoff) * rdu + hu;
        const float u0 = floorf(fu), au = fu - u0;
        const int ju = (int)u0;
        if (ju < -1 || ju >= nue) continue;
        const float r = sid * rU, w = r * r;
        // the detector row coordinate is affine along the z-run
        const float fv0 = (m * pz0 - voff) * rdv + hv, dfv = m * vz * rdv;
        const float *qk = qb + ((long long)k * (nv + 2) + 1) * pitch + 1 + ju;  // (row 0, column ju)
#pragma unroll
        for (int j = 0; j < kFdkZ; ++j) {
            const float fv = fmaf((float)j, dfv, fv0);
            const float v0 = floorf(fv), av = fv - v0;
            const int jv = (int)v0;
            if (jv < -1 || jv >= nv) continue;
            const float *r0 = qk + (long long)jv * pitch;
            const float q00 = __ldg(r0), q10 = __ldg(r0 + 1), q01 = __ldg(r0 + pitch), q11 = __ldg(r0 + pitch + 1);
            const float a0 = fmaf(au, q10 - q00, q00), a1 = fmaf(au, q11 - q01, q01);
            acc[j] = fmaf(w, fmaf(av, a1 - a0, a0), acc[j]);
        }
    }
    const float sc = 6.28318530717958647f / na;
#pragma unroll
    for (int j = 0; j < kFdkZ; ++j) {
        if (iz0 + j < nz) {
            float *o = vol + (((long long)b * nz + iz0 + j) * ny + iy) * nx + ix;
            *o = accumulate ? *o + acc[j] * sc : acc[j] * sc;
        }
    }
}

// ---- PDHG-TV pieces -------------------------------------------------------------------

// z1 <- (z1 + sigma (p - y)) / (1 + sigma)
__global__ void k_pdhg_dual1(float *__restrict__ z1, const float *__restrict__ p, const float *__restrict__ y,
                             long long n, float sigma) {
    const float inv = 1.0f / (1.0f + sigma);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        z1[e] = (z1[e] + sigma * (p[e] - y[e])) * inv;
}

// z2 <- project_{|.| <= rad}(z2 + sigma gamma grad xbar), grad = forward differences
// (zero on the last index of each axis); z2 layout [3][B][nz][ny][nx]
__global__ void k_pdhg_dual2(float *__restrict__ z2, const float *__restrict__ xb, int nx, int ny, int nz, int batch,
                             float sg, float rad) {
    const long long N = (long long)batch * nx * ny * nz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(e % nx), iy = (int)((e / nx) % ny), iz = (int)((e / ((long long)nx * ny)) % nz);
        const float x = xb[e];
        const float gx = ix < nx - 1 ? xb[e + 1] - x : 0.f;
        const float gy = iy < ny - 1 ? xb[e + nx] - x : 0.f;
        const float gz = iz < nz - 1 ? xb[e + (long long)nx * ny] - x : 0.f;
        const float a0 = z2[e] + sg * gx, a1 = z2[N + e] + sg * gy, a2 = z2[2 * N + e] + sg * gz;
        const float nrm = sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
        const float sc = nrm > rad ? rad / nrm : 1.0f;
        z2[e] = a0 * sc;
        z2[N + e] = a1 * sc;
        z2[2 * N + e] = a2 * sc;
    }
}

// x+ = max(0, x - tau (bt - gamma div z2)); xbar = 2 x+ - x; x = x+
__global__ void k_pdhg_primal(float *__restrict__ x, float *__restrict__ xb, const float *__restrict__ bt,
                              const float *__restrict__ z2, int nx, int ny, int nz, int batch, float tau, float gamma,
                              int nonneg) {
    const long long N = (long long)batch * nx * ny * nz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(e % nx), iy = (int)((e / nx) % ny), iz = (int)((e / ((long long)nx * ny)) % nz);
        const long long sxy = (long long)nx * ny;
        float dv = 0.f;
        dv += (ix < nx - 1 ? z2[e] : 0.f) - (ix > 0 ? z2[e - 1] : 0.f);
        dv += (iy < ny - 1 ? z2[N + e] : 0.f) - (iy > 0 ? z2[N + e - nx] : 0.f);
        dv += (iz < nz - 1 ? z2[2 * N + e] : 0.f) - (iz > 0 ? z2[2 * N + e - sxy] : 0.f);
        const float xo = x[e];
        float xn = xo - tau * (bt[e] - gamma * dv);
        if (nonneg && xn < 0.f) xn = 0.f;
        xb[e] = 2.f * xn - xo;
        x[e] = xn;
    }
}

// r = p - y
// r = p - y elementwise; r may alias p (in-place residual), so no restrict on those two
__global__ void k_sub(const float *p, const float *__restrict__ y, float *r, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        r[e] = p[e] - y[e];
}

// x <- x - tau g  (optionally clamped at 0)
__global__ void k_axpy_clamp(float *__restrict__ x, const float *__restrict__ gr, long long n, float tau, int nonneg) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float v = x[e] - tau * gr[e];
        if (nonneg && v < 0.f) v = 0.f;
        x[e] = v;
    }
}

// out = P^T P x - gamma^2 div grad x  (operator of the power iteration for ||K||)
__global__ void k_tv_normal(const float *__restrict__ x, float *__restrict__ out, int nx, int ny, int nz, int batch,
                            float g2) {
    const long long N = (long long)batch * nx * ny * nz, sxy = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(e % nx), iy = (int)((e / nx) % ny), iz = (int)((e / sxy) % nz);
        const float c = x[e];
        // -div grad x = sum over axes of (x - x_prev) contributions, Neumann
        float l = 0.f;
        if (ix < nx - 1) l += c - x[e + 1];
        if (ix > 0) l += c - x[e - 1];
        if (iy < ny - 1) l += c - x[e + nx];
        if (iy > 0) l += c - x[e - nx];
        if (iz < nz - 1) l += c - x[e + sxy];
        if (iz > 0) l += c - x[e - sxy];
        out[e] += g2 * l;
    }
}

__global__ void k_sumsq_d(const float *__restrict__ x, long long n, double *out) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        s += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void k_scale_inv_sqrt(float *x, long long n, const double *sumsq) {
    const float s = (float)(1.0 / sqrt(*sumsq));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] *= s;
}

__global__ void k_fill1(float *x, long long n, float v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

}  // namespace cbct

using namespace cbct;

extern "C" int cbct_fdk_pad(const cbct_geom *g) {
    if (!g) return fail(CBCT_EINVAL, "cbct_fdk_pad: NULL geometry");
    return (int)ceil(2.0 * fabs(g->desc.u_offset) / g->desc.du - 1e-9);
}

extern "C" int cbct_fdk(const cbct_geom *g, const float *proj, float *vol, int batch, int accumulate, void *stream) {
    if (!g || !proj || !vol || batch < 1 || (accumulate != 0 && accumulate != 1))
        return fail(CBCT_EINVAL, "cbct_fdk: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const cbct_geom_desc &d = g->desc;
    const int npad = cbct_fdk_pad(g), nue = d.nu + npad, lo = d.u_offset > 0 ? npad : 0;
    const long long rows = (long long)batch * d.n_angles * d.nv;
    if (rows > 0x7fffffffLL) return fail(CBCT_EINVAL, "cbct_fdk: too many detector rows");
    const int ramp_pad = ((nue + 1) / 2 + kRampB - 1) / kRampB * kRampB;
    const size_t smem = sizeof(float) * (4 * (size_t)ramp_pad + 2 * kRampB + 2 + nue);
    if (smem > 200 * 1024) return fail(CBCT_EINVAL, "cbct_fdk: extended detector row too long");
    // q0: weighted extended rows [rows][nue]; q: filtered rows, zero-padded [batch na][nv + 2][nue + 2]
    const long long nq0 = rows * nue, nq = (long long)batch * d.n_angles * (d.nv + 2) * (nue + 2);
    float *q0 = nullptr, *q = nullptr, *w = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&q0, sizeof(float) * (nq0 + nq + d.nu), st));
    q = q0 + nq0;
    w = q + nq;
    cudaError_t e = cudaMemsetAsync(q, 0, sizeof(float) * nq, st);
    int rc = 0;
    if (e == cudaSuccess) rc = cbct_redundancy_weight(g, w, stream);
    if (e == cudaSuccess && rc == 0) {
        dim3 gw((nue + 127) / 128, (unsigned)std::min<long long>(rows, 65535));
        k_fdk_weight<<<gw, 128, 0, st>>>(proj, w, q0, d.nu, d.nv, nue, lo, (int)rows, (float)d.du, (float)d.dv,
                                         (float)d.u_offset, (float)d.v_offset, (float)d.sdd);
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_fdk_ramp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_fdk_ramp<<<(unsigned)rows, 128, smem, st>>>(q0, q, nue, d.nv, (float)(d.du * d.sid / d.sdd));
        dim3 grd((d.nx + 31) / 32, (d.ny + 7) / 8, ((d.nz + kFdkZ - 1) / kFdkZ) * batch);
        k_fdk_backproject<<<grd, dim3(32, 8), 0, st>>>(
            q, g->cs, vol, d.nx, d.ny, d.nz, d.n_angles, nue, d.nv, lo, d.nu, (float)d.vox[0], (float)d.vox[1],
            (float)d.vox[2], (float)d.center[0], (float)d.center[1], (float)d.center[2], (float)d.sid, (float)d.sdd,
            (float)(1.0 / d.du), (float)(1.0 / d.dv), (float)d.u_offset, (float)d.v_offset, accumulate);
        e = cudaGetLastError();
    }
    cudaFreeAsync(q0, st);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cbct_fdk");
    return 0;
}

extern "C" int cbct_opnorm(const cbct_geom *g, double gamma, int iters, double *out, void *stream) {
    if (!g || !out || iters < 1) return fail(CBCT_EINVAL, "cbct_opnorm: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const GeomDev &d = g->dev;
    const long long nvox = (long long)d.n[0] * d.n[1] * d.n[2], nproj = (long long)d.na * d.nv * d.nu;
    float *x = nullptr, *p = nullptr, *y = nullptr;
    double *acc = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&x, sizeof(float) * (2 * nvox + nproj) + 16, st));
    y = x + nvox;
    p = y + nvox;
    acc = reinterpret_cast<double *>(p + nproj + (nproj & 1));
    int rc = 0;
    k_fill1<<<grid1(nvox), 256, 0, st>>>(x, nvox, 1.0f);
    double nrm2 = 0.0;
    for (int it = 0; it < iters && rc == 0; ++it) {
        cudaMemsetAsync(acc, 0, sizeof(double), st);
        k_sumsq_d<<<grid1(nvox), 256, 0, st>>>(x, nvox, acc);
        k_scale_inv_sqrt<<<grid1(nvox), 256, 0, st>>>(x, nvox, acc);
        rc = forward_project(g, x, p, 1, 0, stream);
        if (rc == 0) rc = back_project(g, p, y, 1, 0, stream);
        if (rc == 0 && gamma != 0.0)
            k_tv_normal<<<grid1(nvox), 256, 0, st>>>(x, y, d.n[0], d.n[1], d.n[2], 1, (float)(gamma * gamma));
        std::swap(x, y);
    }
    cudaError_t e = cudaSuccess;
    if (rc == 0) {
        cudaMemsetAsync(acc, 0, sizeof(double), st);
        k_sumsq_d<<<grid1(nvox), 256, 0, st>>>(x, nvox, acc);
        e = cudaMemcpyAsync(&nrm2, acc, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFreeAsync(std::min(x, y), st);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cbct_opnorm");
    *out = sqrt(sqrt(nrm2));
    return 0;
}

extern "C" int cbct_pdhg(const cbct_geom *g, const float *y, const float *x0, float *x, int batch, int niter,
                         double lam, double gamma, double sigma, double tau, int nonneg, void *stream) {
    if (!g || !y || !x0 || !x || batch < 1 || niter < 0 || !(gamma > 0) || !(sigma > 0) || !(tau > 0) || lam < 0)
        return fail(CBCT_EINVAL, "cbct_pdhg: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const GeomDev &d = g->dev;
    const long long N = (long long)batch * d.n[0] * d.n[1] * d.n[2], M = (long long)batch * d.na * d.nv * d.nu;
    float *buf = nullptr;
    // xbar, bt (N each), z2 (3N), z1, p (M each)
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&buf, sizeof(float) * (5 * N + 2 * M), st));
    float *xb = buf, *bt = xb + N, *z2 = bt + N, *z1 = z2 + 3 * N, *p = z1 + M;
    if (x != x0) cudaMemcpyAsync(x, x0, sizeof(float) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(xb, x0, sizeof(float) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(z2, 0, sizeof(float) * (3 * N + M), st);
    int rc = 0;
    const float rad = (float)(lam / gamma);
    for (int it = 0; it < niter && rc == 0; ++it) {
        rc = forward_project(g, xb, p, batch, 0, stream);
        if (rc) break;
        k_pdhg_dual1<<<grid1(M), 256, 0, st>>>(z1, p, y, M, (float)sigma);
        k_pdhg_dual2<<<grid1(N), 256, 0, st>>>(z2, xb, d.n[0], d.n[1], d.n[2], batch, (float)(sigma * gamma), rad);
        rc = back_project(g, z1, bt, batch, 0, stream);
        if (rc) break;
        k_pdhg_primal<<<grid1(N), 256, 0, st>>>(x, xb, bt, z2, d.n[0], d.n[1], d.n[2], batch, (float)tau,
                                                 (float)gamma, nonneg);
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(buf, st);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cbct_pdhg");
    return 0;
}

extern "C" int cbct_landweber(const cbct_geom *g, const float *y, float *x, int batch, int niter, double tau,
                              int nonneg, void *stream) {
    if (!g || !y || !x || batch < 1 || niter < 0) return fail(CBCT_EINVAL, "cbct_landweber: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const GeomDev &d = g->dev;
    const long long N = (long long)batch * d.n[0] * d.n[1] * d.n[2], M = (long long)batch * d.na * d.nv * d.nu;
    float *buf = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&buf, sizeof(float) * (N + M), st));
    float *gr = buf, *r = buf + N;
    int rc = 0;
    for (int it = 0; it < niter && rc == 0; ++it) {
        rc = forward_project(g, x, r, batch, 0, stream);
        if (rc) break;
        k_sub<<<grid1(M), 256, 0, st>>>(r, y, r, M);
        rc = back_project(g, r, gr, batch, 0, stream);
        if (rc) break;
        k_axpy_clamp<<<grid1(N), 256, 0, st>>>(x, gr, N, (float)tau, nonneg);
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(buf, st);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cbct_landweber");
    return 0;
}
