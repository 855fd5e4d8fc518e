// Shared definitions of the GB300 cone-beam library: status handling, the device
// geometry view and the canonical per-ray setup used by every projector kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/cbct.h"

namespace cbct {

// ---- status / error reporting ------------------------------------------------

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define CBCT_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return ::cbct::cuda_fail(_e, #expr); \
    } while (0)

#define CBCT_LAUNCH_CHECK(what)                                  \
    do {                                                         \
        cudaError_t _e = cudaGetLastError();                     \
        if (_e != cudaSuccess) return ::cbct::cuda_fail(_e, what); \
    } while (0)

// ---- geometry ----------------------------------------------------------------

// Per-angle ray frame in continuous voxel-index coordinates (FP32 copy).
// S: source; D0S: pixel (0,0) minus source; EU/EV: step per detector column/row.
// ux_lo..ux_hi: smallest/largest column whose rays are x-principal (empty when
// ux_lo > ux_hi), likewise uy_* for y-principal rays. Used only to prune
// candidate columns; every kernel re-checks the principal axis per ray.
struct __align__(16) Frame32 {
    float S[3];
    float D0S[3];
    float EU[3];
    float EV[3];
    int ux_lo, ux_hi, uy_lo, uy_hi;
};

struct Frame64 {
    double S[3];
    double D0S[3];
    double EU[3];
    double EV[3];
};

// Per-(angle, column) ray parameters, computed in FP64 on the host and rounded
// once. With a the column's principal axis, b = 1 - a, c_a = (n_a - 1)/2 the
// central plane and r = D0S + iu EU the direction:
//   dqb = r_b / r_a             in-plane slope along b per plane
//   qcb = S_b + tc r_b          in-plane b coordinate on the central plane
//   tc  = (c_a - S_a) / r_a     source-to-pixel parameter at the central plane
//   inv = 1 / r_a
template <typename T>
struct ColT {
    T dqb, qcb, tc, inv;
};
using Col32 = ColT<float>;
using Col64 = ColT<double>;

// Device view of a geometry (passed by value to kernels).
struct GeomDev {
    int n[3];          // nx, ny, nz
    int nu, nv, na;
    float vox[3];
    double voxd[3];
    float scale;       // operator scale (1/||P|| or 1)
    double scaled;
    float Sz;          // source z coordinate (index space), the same at every angle
    double Szd;
    const Frame32 *f32;
    const Frame64 *f64;
    const Col32 *col32;  // [na][nu]
    const Col64 *col64;
    const float *rz32;   // [nv]: z direction component of row iv, D0S_z + iv EV_z
    const double *rz64;
};

template <typename T> struct FrameOf;
template <> struct FrameOf<float> { using type = Frame32; };
template <> struct FrameOf<double> { using type = Frame64; };

template <typename T> __device__ __forceinline__ const typename FrameOf<T>::type &frame_of(const GeomDev &g, int k);
template <> __device__ __forceinline__ const Frame32 &frame_of<float>(const GeomDev &g, int k) { return g.f32[k]; }
template <> __device__ __forceinline__ const Frame64 &frame_of<double>(const GeomDev &g, int k) { return g.f64[k]; }

// Principal axis of ray (iu, iv) at angle frame f: 0 (x) if |r_x| >= |r_y| else
// 1 (y), on the FP32 direction r = fmaf(iu, EU, D0S) (EV has no x/y component,
// so the row does not enter). Identical in every kernel and in the host checks.
__host__ __device__ __forceinline__ int principal_axis(const Frame32 &f, int iu) {
#ifdef __CUDA_ARCH__
    float rx = __fmaf_rn((float)iu, f.EU[0], f.D0S[0]);
    float ry = __fmaf_rn((float)iu, f.EU[1], f.D0S[1]);
#else
    float rx = fmaf((float)iu, f.EU[0], f.D0S[0]);
    float ry = fmaf((float)iu, f.EU[1], f.D0S[1]);
#endif
    return fabsf(rx) >= fabsf(ry) ? 0 : 1;
}

// Canonical per-ray quantities. A ray (k, iu, iv) with principal axis a samples
// plane i at di = i - c_a from the central plane:
//   t   = fma(di, inv, tc)                 source-to-pixel parameter
//   q_b = fma(di, dqb, qcb)                in-plane coordinate along b = 1 - a
//   q_z = fma(di, dqz, qcz), dqz = rz * inv, qcz = fma(tc, rz, Sz)
// Centring the parametrisation on the volume keeps every FP32 intermediate
// within the volume's coordinate range (the source itself is hundreds of voxels
// away). Forward and backward kernels use exactly these operations, so their
// sample positions agree bit for bit.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T> __device__ __forceinline__ ColT<T> col_of(const GeomDev &g, int k, int iu);
template <> __device__ __forceinline__ ColT<float> col_of<float>(const GeomDev &g, int k, int iu) {
    const float4 c = __ldg(reinterpret_cast<const float4 *>(g.col32) + (long long)k * g.nu + iu);
    return ColT<float>{c.x, c.y, c.z, c.w};
}
template <> __device__ __forceinline__ ColT<double> col_of<double>(const GeomDev &g, int k, int iu) {
    return g.col64[(long long)k * g.nu + iu];
}
template <typename T> __device__ __forceinline__ T rz_of(const GeomDev &g, int iv);
template <> __device__ __forceinline__ float rz_of<float>(const GeomDev &g, int iv) { return __ldg(g.rz32 + iv); }
template <> __device__ __forceinline__ double rz_of<double>(const GeomDev &g, int iv) { return g.rz64[iv]; }
template <typename T> __device__ __forceinline__ T sz_of(const GeomDev &g);
template <> __device__ __forceinline__ float sz_of<float>(const GeomDev &g) { return g.Sz; }
template <> __device__ __forceinline__ double sz_of<double>(const GeomDev &g) { return g.Szd; }

// Row part of a ray: dqz and qcz.
template <typename T>
__device__ __forceinline__ void ray_row(const GeomDev &g, const ColT<T> &c, T rz, T &dqz, T &qcz) {
    dqz = mul_rn(rz, c.inv);
    qcz = fma_rn(c.tc, rz, sz_of<T>(g));
}

// World step length (mm) between consecutive planes: |(vox_a, dqb vox_b, dqz vox_z)|.
template <typename T>
__device__ __forceinline__ T ray_step(const GeomDev &g, int a, T dqb, T dqz) {
    T vx, vy, vz;
    if constexpr (sizeof(T) == 4) { vx = g.vox[0]; vy = g.vox[1]; vz = g.vox[2]; }
    else { vx = g.voxd[0]; vy = g.voxd[1]; vz = g.voxd[2]; }
    const T va = a == 0 ? vx : vy, vb = a == 0 ? vy : vx;
    const T eb = dqb * vb, ez = dqz * vz;
    return sqrt(va * va + eb * eb + ez * ez);
}

// Index of voxel (ix, iy, iz) in a [nz][ny][nx] volume.
__device__ __forceinline__ long long vox_index(const GeomDev &g, int ix, int iy, int iz) {
    return ((long long)iz * g.n[1] + iy) * g.n[0] + ix;
}

// Streaming multiprocessors of the current device (queried once per device): the unit
// of the grid-size heuristics.
int sm_count();

// Host-side geometry object.
struct Geom;
GeomDev dev_view(const cbct_geom *g);

}  // namespace cbct
