// Cone-beam projector pair (a2, a3): Joseph-style forward projection P and its
// exact transpose P* as an atomic-free voxel-driven gather (paper Sec. 2.2,
// projection operator and its adjoint, the backprojection).
//
// Forward (k_forward): one thread per ray; the ray visits every voxel-centre plane
// of its principal axis between source and pixel and accumulates the bilinear
// sample of that plane (zero outside the grid) times the step length.
//
// Backward (k_backproject): one thread per voxel run along z. For each angle and
// each principal axis it finds the detector columns whose rays cross the voxel's
// own plane within one voxel of it (a closed-form interval), then the rows, and
// gathers step * bilinear weight * projection over exactly the (ray, plane,
// neighbour) triples the forward visits. The per-ray step is folded into the
// projection beforehand (k_weight_rays) so the gather needs no square root.
// This kernel serves the FP64 instantiation and geometries whose principal-axis
// columns do not form intervals; FP32 calls otherwise use the segment gather
// k_backproject_v3 further down, which visits the same triples.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "common.cuh"
#include "geom_impl.h"

namespace cbct {

// Conservative plane interval for q0 + i dq in (L, H); intersects [lo, hi].
template <typename T>
__device__ __forceinline__ void lin_range(T q0, T dq, T L, T H, T &lo, T &hi) {
    if (dq == T(0)) {
        if (!(q0 > L && q0 < H)) { lo = T(1); hi = T(0); }
        return;
    }
    T i1 = (L - q0) / dq, i2 = (H - q0) / dq;
    lo = fmax(lo, fmin(i1, i2));
    hi = fmin(hi, fmax(i1, i2));
}

// ---- forward projection -------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(256) k_forward(GeomDev g, const T *__restrict__ vol, T *__restrict__ proj,
                                                 int accumulate) {
    const int iu = blockIdx.x * 32 + threadIdx.x;
    const int iv = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z % g.na, b = blockIdx.z / g.na;
    if (iu >= g.nu || iv >= g.nv) return;
    const int a = principal_axis(g.f32[k], iu);
    const ColT<T> c = col_of<T>(g, k, iu);
    const T rz = rz_of<T>(g, iv);
    T dqz, qcz;
    ray_row(g, c, rz, dqz, qcz);
    const int na = g.n[a], nb = g.n[1 - a], nz = g.n[2];
    const T ca = T(0.5) * T(na - 1);
    const long long nx = g.n[0], nxy = (long long)g.n[0] * g.n[1];
    const long long sa = a == 0 ? 1 : nx, sb = a == 0 ? nx : 1;
    const T *V = vol + (long long)b * nxy * nz;

    // planes with t in (0, 1) and the in-plane point in (-1, n): conservative range
    // in di = i - ca, the exact tests are repeated per sample
    T lo = -ca, hi = ca;
    lin_range(c.tc, c.inv, T(0), T(1), lo, hi);
    lin_range(c.qcb, c.dqb, T(-1), T(nb), lo, hi);
    lin_range(qcz, dqz, T(-1), T(nz), lo, hi);
    const int ilo = max(0, (int)floor(lo + ca) - 1), ihi = min(na - 1, (int)ceil(hi + ca) + 1);

    T acc = T(0);
    for (int i = ilo; i <= ihi; ++i) {
        const T di = T(i) - ca;
        const T t = fma_rn(di, c.inv, c.tc);
        if (!(t > T(0) && t < T(1))) continue;
        const T qb = fma_rn(di, c.dqb, c.qcb);
        const T qz = fma_rn(di, dqz, qcz);
        if (!(qb > T(-1) && qb < T(nb) && qz > T(-1) && qz < T(nz))) continue;
        const T fb0 = floor(qb), fz0 = floor(qz);
        const int jb = (int)fb0, jz = (int)fz0;
        const T fb = qb - fb0, fz = qz - fz0;
        const T *P = V + i * sa;
        const bool b0 = jb >= 0, b1 = jb + 1 < nb, z0 = jz >= 0, z1 = jz + 1 < nz;
        const long long o = (long long)jb * sb + (long long)jz * nxy;
        const T v00 = (b0 && z0) ? __ldg(P + o) : T(0);
        const T v10 = (b1 && z0) ? __ldg(P + o + sb) : T(0);
        const T v01 = (b0 && z1) ? __ldg(P + o + nxy) : T(0);
        const T v11 = (b1 && z1) ? __ldg(P + o + sb + nxy) : T(0);
        acc += (T(1) - fz) * ((T(1) - fb) * v00 + fb * v10) + fz * ((T(1) - fb) * v01 + fb * v11);
    }
    T scale;
    if constexpr (sizeof(T) == 4) scale = g.scale; else scale = g.scaled;
    acc *= ray_step<T>(g, a, c.dqb, dqz) * scale;
    T *out = proj + (((long long)b * g.na + k) * g.nv + iv) * g.nu + iu;
    *out = accumulate ? *out + acc : acc;
}

// ---- backprojection -------------------------------------------------------------

// pw = proj * step(ray) * scale (* colw[column] when colw is given)
template <typename T>
__global__ void k_weight_rays(GeomDev g, const T *__restrict__ proj, T *__restrict__ pw, const T *__restrict__ colw) {
    const int iu = blockIdx.x * 32 + threadIdx.x;
    const int iv = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z % g.na, b = blockIdx.z / g.na;
    if (iu >= g.nu || iv >= g.nv) return;
    const int a = principal_axis(g.f32[k], iu);
    const ColT<T> c = col_of<T>(g, k, iu);
    T dqz, qcz;
    ray_row(g, c, rz_of<T>(g, iv), dqz, qcz);
    T scale;
    if constexpr (sizeof(T) == 4) scale = g.scale; else scale = g.scaled;
    const long long o = (((long long)b * g.na + k) * g.nv + iv) * g.nu + iu;
    const T v = proj[o] * ray_step<T>(g, a, c.dqb, dqz) * scale;
    pw[o] = colw ? v * colw[iu] : v;
}

// Detector column (continuous) hit by the ray from the source through the xy
// index-space point (px, py): D0S + u EU parallel to P - S.
__device__ __forceinline__ float column_of(const Frame32 &F, float px, float py) {
    const float dx = px - F.S[0], dy = py - F.S[1];
    const float num = F.D0S[0] * dy - F.D0S[1] * dx;
    const float den = F.EU[0] * dy - F.EU[1] * dx;
    return -num / den;
}

// column_of with the approximate division: for candidate ranges that carry a margin of a
// column or more (relative error a few ulp; non-finite where column_of is)
__device__ __forceinline__ float column_of_approx(const Frame32 &F, float px, float py) {
    const float dx = px - F.S[0], dy = py - F.S[1];
    const float num = F.D0S[0] * dy - F.D0S[1] * dx;
    const float den = F.EU[0] * dy - F.EU[1] * dx;
    return -__fdividef(num, den);
}

template <typename T, int ZS>
__global__ void __launch_bounds__(256) k_backproject(GeomDev g, const T *__restrict__ pw, T *__restrict__ vol,
                                                     int accumulate) {
    const int ix = blockIdx.x * 32 + threadIdx.x;
    const int iy = blockIdx.y * 8 + threadIdx.y;
    const int nzs = (g.n[2] + ZS - 1) / ZS;
    const int z0 = (blockIdx.z % nzs) * ZS, b = blockIdx.z / nzs;
    if (ix >= g.n[0] || iy >= g.n[1]) return;
    const int nz = g.n[2];
    T acc[ZS];
#pragma unroll
    for (int j = 0; j < ZS; ++j) acc[j] = T(0);
    const T *PB = pw + (long long)b * g.na * g.nv * g.nu;
    const T Sz = sz_of<T>(g);
    // rows: q_z = Sz + t rz(v) and rz(v) = rz0 + v drz
    const float rz0 = g.rz32[0], drz = g.nv > 1 ? g.rz32[1] - g.rz32[0] : 1.0f;

    for (int k = 0; k < g.na; ++k) {
        const Frame32 &F = g.f32[k];
        const T *Pk = PB + (long long)k * g.nv * g.nu;
        for (int a = 0; a < 2; ++a) {
            const int alo = a == 0 ? F.ux_lo : F.uy_lo, ahi = a == 0 ? F.ux_hi : F.uy_hi;
            if (alo > ahi) continue;
            const int i = a == 0 ? ix : iy;   // the voxel's plane on axis a
            const int j = a == 0 ? iy : ix;   // its in-plane coordinate along b
            const T di = T(i) - T(0.5) * T(g.n[a] - 1);
            // columns whose rays meet plane i inside (j - 1, j + 1)
            float u1, u2;
            if (a == 0) { u1 = column_of(F, (float)ix, (float)(iy - 1)); u2 = column_of(F, (float)ix, (float)(iy + 1)); }
            else { u1 = column_of(F, (float)(ix - 1), (float)iy); u2 = column_of(F, (float)(ix + 1), (float)iy); }
            int ulo = alo, uhi = ahi;
            if (isfinite(u1) && isfinite(u2)) {
                const float lo_f = fmaxf(fminf(u1, u2), -1.0e6f), hi_f = fminf(fmaxf(u1, u2), 1.0e6f);
                ulo = max(ulo, (int)floorf(lo_f) - 1);
                uhi = min(uhi, (int)ceilf(hi_f) + 1);
            }
            for (int u = ulo; u <= uhi; ++u) {
                if (principal_axis(F, u) != a) continue;
                const ColT<T> c = col_of<T>(g, k, u);
                const T t = fma_rn(di, c.inv, c.tc);
                if (!(t > T(0) && t < T(1))) continue;
                const T qb = fma_rn(di, c.dqb, c.qcb);
                const T wb = T(1) - fabs(qb - T(j));
                if (!(wb > T(0))) continue;
                // rows whose sample on plane i lies within one voxel of [z0, z0+ZS-1]
                const float tf = (float)t;
                float v1 = ((float)(z0 - 1) - (float)Sz) / tf, v2 = ((float)(z0 + ZS) - (float)Sz) / tf;
                v1 = (v1 - rz0) / drz;
                v2 = (v2 - rz0) / drz;
                if (!(v1 == v1) || !(v2 == v2)) continue;
                const float vmin = fmaxf(fminf(v1, v2), -1.0e6f), vmax = fminf(fmaxf(v1, v2), 1.0e6f);
                const int vlo = max(0, (int)floorf(vmin) - 1);
                const int vhi = min(g.nv - 1, (int)ceilf(vmax) + 1);
                for (int v = vlo; v <= vhi; ++v) {
                    T dqz, qcz;
                    ray_row(g, c, rz_of<T>(g, v), dqz, qcz);
                    const T qz = fma_rn(di, dqz, qcz);
                    const T p = wb * __ldg(Pk + (long long)v * g.nu + u);
#pragma unroll
                    for (int jj = 0; jj < ZS; ++jj) {
                        const T wz = T(1) - fabs(qz - T(z0 + jj));
                        if (wz > T(0)) acc[jj] += wz * p;
                    }
                }
            }
        }
    }
    const long long nxy = (long long)g.n[0] * g.n[1];
    T *out = vol + (long long)b * nxy * nz + ((long long)z0 * g.n[1] + iy) * g.n[0] + ix;
#pragma unroll
    for (int jj = 0; jj < ZS; ++jj) {
        if (z0 + jj < nz) {
            T *o = out + (long long)jj * nxy;
            *o = accumulate ? *o + acc[jj] : acc[jj];
        }
    }
}

// Segment gather (FP32, geometries whose x- and y-principal columns form intervals).
// CTA = brick of 16 x 16 voxel columns x 8 voxels in z, 288 threads. For the rays
// of principal axis a at angle k, plane i of the brick is crossed at
// q_b(u) = fma(di, dqb(u), qcb(u)), monotone in the detector column u. The columns
// with floor(q_b) = s form segment s of the plane; their samples lie between voxels
// s and s + 1 with weights 1 - frac(q_b) and frac(q_b). Thread (segment, plane)
// sweeps the rows of each of its columns once, summing the rows of every unit
// z-interval (L, L + 1] as S0 = sum p and S1 = sum p (q_z - L) (lower voxel
// S0 - S1, upper voxel S1), and accumulates SA[z] for voxel s and SB[z] for voxel
// s + 1. A thread's two voxel runs depend on the axis only, so the angles run inside
// one sweep per principal axis and SA, SB stay in registers over all of them; after
// each sweep every voxel adds the SA of its own segment, then (after a barrier) the SB
// of the segment below, to its shared accumulator — a fixed order, so the result does
// not depend on scheduling, and no barrier or shared-memory traffic per angle.
// The kernel is bound by load latency, which shapes the loops: a thread first
// narrows its candidate columns to the first and last column of its segment (so
// the lanes of a warp run their useful columns in the same iterations); a row's
// z-coordinate is the affine q_z(v) = voff + v step of the row index (rz(v) =
// rz_0 + v EV_z), so no table load sits between two intervals; and the rows of
// an interval go through a fixed block of five predicated loads (3 to 5 rows per
// interval at these magnifications) plus a loop for longer intervals, which makes
// the (kZ3 + 1)-interval sweep straight-line code whose loads overlap.
// The panel width is a template parameter for common widths (256, 512, 1024 columns): the five
// row loads of an interval then sit at constant offsets from one row pointer, which took the
// clinical adjoint from 23.3 to 19.6 ms (CUDA events, bit-identical output).
// Bricks 8 voxels tall with four CTAs per SM (registers capped at 56, no spills): with the
// width-specialised loads the kernel is bound by load latency more than by issue, and the
// fourth CTA's warps hide it. Clinical adjoint (CUDA events): 18.3 ms, against 19.6 with
// 12-voxel bricks at three CTAs, 19.7 with 8-voxel bricks at three, 19.0 with 10 at four,
// 20.0 with 6 at four, 28.4 with 12 at four and 23.3 with 8 at five (spills). Before the
// width-specialised loads 12-voxel bricks at three CTAs had been best (23.7 ms; 24.5 with 8,
// 26.0 with 6, 31.5 with 4, 26.8 with 16; capped registers slower).
constexpr int kB3 = 16, kZ3 = 8, kThreads3 = 288;
constexpr int kVacc3 = kZ3 * kB3 * (kB3 + 1);  // [z][y][x], y stride 17 (bank-conflict free both ways)
constexpr size_t kSmem3 = sizeof(float) * kVacc3;

// NU > 0 fixes the panel width at compile time, so the rows of an interval are loaded at
// constant offsets (rr NU floats) from one row pointer; NU = 0 reads it from the geometry.
template <int NU>
__global__ void __launch_bounds__(kThreads3, 4) k_backproject_v3(GeomDev g, const float *__restrict__ pw,
                                                                 float *__restrict__ vol, int accumulate,
                                                                 int nparts, float *__restrict__ partial) {
    extern __shared__ float sm3[];
    float *vacc = sm3;
    const int tid = threadIdx.x;
    const int il = tid & 15, seg = tid >> 4;  // plane il of the brick; segment j0 - 1 + seg
    const bool item = seg <= kB3;             // 17 segments x 16 planes
    const int x0 = blockIdx.x * kB3, y0 = blockIdx.y * kB3;
    const int nzb = (g.n[2] + kZ3 - 1) / kZ3;
    const int part = blockIdx.z % nparts, zb = blockIdx.z / nparts;
    const int z0 = (zb % nzb) * kZ3, b = zb / nzb;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nu = NU > 0 ? NU : g.nu, nv = g.nv;
    const int k_begin = (int)((long long)g.na * part / nparts);
    int k_end = (int)((long long)g.na * (part + 1) / nparts);
    __shared__ int s_reach;
    if (tid == 0) s_reach = 0;
    for (int e = tid; e < kVacc3; e += kThreads3) vacc[e] = 0.f;
    __syncthreads();
    const float Sz = g.Sz;
    const float rz0 = g.rz32[0], drz = g.f32[0].EV[2], inv_drz = 1.0f / drz;
    const float *PB = pw + (long long)b * g.na * nv * nu;
    {
        // Does any panel row reach the brick's support (the brick and one voxel around it)
        // at an angle of this part? The source-to-panel parameter t of a point is affine in
        // its (x, y), so over the support it lies between its values at the four corners;
        // the rows that meet z in (zlo, zhi) at t lie between zlo / t and zhi / t, and
        // those are monotone in t. Two rows of margin, as in the per-column test below; a
        // non-finite value counts as reachable. Bricks no row reaches skip the angle loop
        // and write zeros.
        const float zlo = (float)(z0 - 1) - Sz, zhi = (float)(z0 + kZ3) - Sz;
        const float cx[2] = {(float)(x0 - 1), (float)(x0 + kB3)}, cy[2] = {(float)(y0 - 1), (float)(y0 + kB3)};
        bool any = false;
        for (int k = k_begin + tid; k < k_end && !any; k += kThreads3) {
            const Frame32 &F = g.f32[k];
            const float den = F.EU[0] * F.D0S[1] - F.EU[1] * F.D0S[0];
            float tmin = INFINITY, tmax = -INFINITY;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float t = __fdividef(F.EU[0] * (cy[c >> 1] - F.S[1]) - F.EU[1] * (cx[c & 1] - F.S[0]), den);
                tmin = fminf(tmin, t);
                tmax = fmaxf(tmax, t);
            }
            if (tmax <= 0.f) continue;  // behind the source
            const float t1 = fmaxf(tmin, 1e-6f);
            const float rlo = fminf(__fdividef(zlo, t1), __fdividef(zlo, tmax));
            const float rhi = fmaxf(__fdividef(zhi, t1), __fdividef(zhi, tmax));
            const float va = (rlo - rz0) * inv_drz, vb = (rhi - rz0) * inv_drz;
            if (!(fmaxf(va, vb) + 2.f < 0.f || fminf(va, vb) - 2.f > (float)(nv - 1))) any = true;
        }
        if (any) s_reach = 1;
    }
    __syncthreads();
    if (!s_reach) k_end = k_begin;

#pragma unroll 1
    for (int a = 0; a < 2; ++a) {
        const int j0 = a == 0 ? y0 : x0;
        const int i = (a == 0 ? x0 : y0) + il, s = j0 - 1 + seg;
        const bool mine = item && i < g.n[a] && s < g.n[1 - a];
        const float di = (float)i - 0.5f * (float)(g.n[a] - 1);
        float SA[kZ3], SB[kZ3];
#pragma unroll
        for (int m = 0; m < kZ3; ++m) SA[m] = SB[m] = 0.f;
#pragma unroll 1
        for (int k = k_begin; k < k_end; ++k) {
            const Frame32 &F = g.f32[k];
            const int alo = a == 0 ? F.ux_lo : F.uy_lo, ahi = a == 0 ? F.ux_hi : F.uy_hi;
            if (alo > ahi || !mine) continue;
            const float *Pk = PB + (long long)k * nv * nu;
            // candidate columns for q_b in [s, s + 1), one column of margin (which also covers
            // the approximate divisions here and in the z-run test below: the exact test on
            // floor(q_b) decides which columns contribute)
            float u1, u2;
            if (a == 0) { u1 = column_of_approx(F, (float)i, (float)s); u2 = column_of_approx(F, (float)i, (float)(s + 1)); }
            else { u1 = column_of_approx(F, (float)s, (float)i); u2 = column_of_approx(F, (float)(s + 1), (float)i); }
            int ulo = alo, uhi = ahi;
            if (isfinite(u1) && isfinite(u2)) {
                ulo = max(ulo, (int)floorf(fmaxf(fminf(u1, u2), -1.0e6f)) - 1);
                uhi = min(uhi, (int)ceilf(fminf(fmaxf(u1, u2), 1.0e6f)) + 1);
            }
            if (ulo <= uhi) {
                // skip the columns when no row of the panel reaches the z-run
                const ColT<float> cl = col_of<float>(g, k, ulo), ch = col_of<float>(g, k, uhi);
                const float tl = fma_rn(di, cl.inv, cl.tc), th = fma_rn(di, ch.inv, ch.tc);
                const float tmin = fminf(tl, th), tmax = fmaxf(tl, th);
                const float zlo = (float)(z0 - 1) - Sz, zhi = (float)(z0 + kZ3) - Sz;
                const float t1 = fmaxf(tmin, 1e-6f);
                const float rlo = fminf(__fdividef(zlo, t1), __fdividef(zlo, tmax));
                const float rhi = fmaxf(__fdividef(zhi, t1), __fdividef(zhi, tmax));
                const float vlo = (rlo - rz0) * inv_drz - 2.f, vhi = (rhi - rz0) * inv_drz + 2.f;
                if (!(tmax > 0.f) || vhi < 0.f || vlo > (float)(nv - 1)) uhi = ulo - 1;
            }
            {  // first and last column of the segment
                int ua = uhi + 1, ub = uhi;
#pragma unroll 1
                for (int u = ulo; u <= uhi; ++u) {
                    const ColT<float> c = col_of<float>(g, k, u);
                    const float t = fma_rn(di, c.inv, c.tc);
                    const float qb = fma_rn(di, c.dqb, c.qcb);
                    if (t > 0.f && t < 1.f && floorf(qb) == (float)s) { ua = min(ua, u); ub = u; }
                }
                ulo = ua;
                uhi = ub;
            }
#pragma unroll 1
            for (int u = ulo; u <= uhi; ++u) {
                const ColT<float> c = col_of<float>(g, k, u);
                const float t = fma_rn(di, c.inv, c.tc);
                if (!(t > 0.f && t < 1.f)) continue;
                const float qb = fma_rn(di, c.dqb, c.qcb);
                const float fb = floorf(qb);
                if (fb != (float)s) continue;  // the column belongs to another segment
                const float wu = qb - fb, wl = 1.0f - wu;
                const float step = t * drz, irs = 1.0f / step, voff = fmaf(t, rz0, Sz);
                // sample z of row v relative to z0 - 1: v step + voffz; the first row whose
                // sample lies above z0 - 1 + m is floor((m - voffz) / step) + 1, and clamping
                // the quotient to [-1, nv - 1] before the floor keeps it in [0, nv]
                const float voffz = voff - (float)(z0 - 1), vbase = -voffz * irs;
                const float vmax = (float)(nv - 1);
                auto row_above = [&](int m) {
                    return __float2int_rd(fminf(fmaxf(fmaf((float)m, irs, vbase), -1.0f), vmax)) + 1;
                };
                const float *Pu = Pk + u;
                int va = row_above(0);
                float carry = 0.f;  // upper-voxel share of the previous interval
#pragma unroll
                for (int m = 0; m < kZ3 + 1; ++m) {
                    const int ve = row_above(m + 1);
                    float S0 = 0.f, S1 = 0.f;
                    if (va < ve) {
                        float qf = fmaf((float)va, step, voffz) - (float)m;
                        const float *pp = Pu + (long long)va * nu;
                        const int n = ve - va;
                        float T = 0.f;  // sum of rr p: S1 = qf S0 + step T
#pragma unroll
                        for (int rr = 0; rr < 5; ++rr) {
                            const float p = rr < n ? __ldg(pp + rr * nu) : 0.f;
                            S0 += p;
                            if (rr > 0) T = fmaf((float)rr, p, T);
                        }
#pragma unroll 1
                        for (int rr = 5; rr < n; ++rr) {
                            const float p = __ldg(pp + rr * nu);
                            S0 += p;
                            T = fmaf((float)rr, p, T);
                        }
                        S1 = fmaf(qf, S0, step * T);
                    }
                    // voxel z0 - 1 + m: upper share of interval m - 1, lower share of interval m
                    if (m >= 1) {
                        const float R = carry + S0 - S1;
                        SA[m - 1] = fmaf(wl, R, SA[m - 1]);
                        SB[m - 1] = fmaf(wu, R, SB[m - 1]);
                    }
                    carry = S1;
                    va = ve;
                }
            }
        }
        // voxel (plane il, local index seg - 1): its own segment's lower shares, then the
        // upper shares of the segment below it
        if (mine && seg >= 1) {
            const int vl = seg - 1;
            float *v = vacc + (a == 0 ? vl * (kB3 + 1) + il : il * (kB3 + 1) + vl);
#pragma unroll
            for (int m = 0; m < kZ3; ++m) v[m * kB3 * (kB3 + 1)] += SA[m];
        }
        __syncthreads();
        if (mine && seg < kB3) {
            float *v = vacc + (a == 0 ? seg * (kB3 + 1) + il : il * (kB3 + 1) + seg);
#pragma unroll
            for (int m = 0; m < kZ3; ++m) v[m * kB3 * (kB3 + 1)] += SB[m];
        }
        __syncthreads();
    }
    const long long nxy = (long long)nx * ny;
    const int nbatch = (int)(gridDim.z / nparts / nzb);
    float *out = nparts > 1 ? partial + ((long long)part * nbatch + b) * nxy * nz : vol + (long long)b * nxy * nz;
    const int acc_mode = nparts > 1 ? 0 : accumulate;
    for (int e = tid; e < kZ3 * kB3 * kB3; e += kThreads3) {
        const int xl = e & (kB3 - 1), yl = (e / kB3) & (kB3 - 1), zl = e / (kB3 * kB3);
        const int ix = x0 + xl, iy = y0 + yl, iz = z0 + zl;
        if (ix < nx && iy < ny && iz < nz) {
            float *o = out + ((long long)iz * ny + iy) * nx + ix;
            const float v = vacc[zl * kB3 * (kB3 + 1) + yl * (kB3 + 1) + xl];
            *o = acc_mode ? *o + v : v;
        }
    }
}

// vol (+)= sum over parts of partial[part], in part order (deterministic)
__global__ void k_sum_parts(const float *__restrict__ partial, int nparts, long long n, float *__restrict__ vol,
                            int accumulate) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float s = accumulate ? vol[e] : 0.f;
        for (int p = 0; p < nparts; ++p) s += partial[(long long)p * n + e];
        vol[e] = s;
    }
}

// ---- sample count -----------------------------------------------------------------

__global__ void __launch_bounds__(256) k_count(GeomDev g, unsigned long long *total) {
    const int iu = blockIdx.x * 32 + threadIdx.x;
    const int iv = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    unsigned long long cnt = 0;
    if (iu < g.nu && iv < g.nv) {
        const int a = principal_axis(g.f32[k], iu);
        const ColT<float> c = col_of<float>(g, k, iu);
        float dqz, qcz;
        ray_row(g, c, rz_of<float>(g, iv), dqz, qcz);
        const int na = g.n[a], nb = g.n[1 - a], nz = g.n[2];
        const float ca = 0.5f * (float)(na - 1);
        for (int i = 0; i < na; ++i) {
            const float di = (float)i - ca;
            const float t = fma_rn(di, c.inv, c.tc);
            if (!(t > 0.0f && t < 1.0f)) continue;
            const float qb = fma_rn(di, c.dqb, c.qcb);
            const float qz = fma_rn(di, dqz, qcz);
            if (qb > -1.0f && qb < float(nb) && qz > -1.0f && qz < float(nz)) cnt++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(total, cnt);
}

// ---- FP64 norms for the power iteration ------------------------------------------

__global__ void k_sumsq(const float *__restrict__ x, long long n, double *out) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = x[i];
        s += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void k_scale_by(float *x, long long n, const double *sumsq) {
    const float s = (float)(1.0 / sqrt(*sumsq));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] *= s;
}

__global__ void k_fill(float *x, long long n, float v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

// ---- launchers ------------------------------------------------------------------------

static int check_common(const cbct_geom *g, const void *a, const void *b, int batch, int accumulate) {
    if (!g || !a || !b) return fail(CBCT_EINVAL, "NULL geometry or buffer");
    if (batch < 1) return fail(CBCT_EINVAL, "batch must be >= 1");
    if (accumulate != 0 && accumulate != 1) return fail(CBCT_EINVAL, "accumulate must be 0 or 1");
    if ((long long)batch * g->dev.na > 65535) return fail(CBCT_EINVAL, "batch * n_angles must be <= 65535");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != g->device) return fail(CBCT_EINVAL, "current device differs from the geometry's device");
    return 0;
}

template <typename T>
static int forward_impl(const cbct_geom *g, const T *vol, T *proj, int batch, int accumulate, cudaStream_t st) {
    int rc = check_common(g, vol, proj, batch, accumulate);
    if (rc) return rc;
    if constexpr (sizeof(T) == 4) {
        rc = forward_staged(g, vol, proj, batch, accumulate, st);
        if (rc < 0) return rc;
        if (rc == 1) return 0;
    }
    const GeomDev &d = g->dev;
    dim3 blk(32, 8), grd((d.nu + 31) / 32, (d.nv + 7) / 8, d.na * batch);
    k_forward<T><<<grd, blk, 0, st>>>(d, vol, proj, accumulate);
    CBCT_LAUNCH_CHECK("forward_project launch");
    return 0;
}

constexpr int kZS = 4;

template <typename T>
static int backward_impl(const cbct_geom *g, const T *proj, T *vol, int batch, int accumulate, cudaStream_t st,
                         const T *colw = nullptr) {
    int rc = check_common(g, proj, vol, batch, accumulate);
    if (rc) return rc;
    const GeomDev &d = g->dev;
    const long long nproj = (long long)batch * d.na * d.nv * d.nu;
    const int nzs = (d.n[2] + kZS - 1) / kZS;
    if ((long long)nzs * batch > 65535) return fail(CBCT_EINVAL, "back_project: batch too large");
    T *pw = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&pw, sizeof(T) * nproj, st));
    dim3 blk(32, 8), gw((d.nu + 31) / 32, (d.nv + 7) / 8, d.na * batch);
    k_weight_rays<T><<<gw, blk, 0, st>>>(d, proj, pw, colw);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        if constexpr (sizeof(T) == 4) {
            if (g->axis_contiguous) {
                const int nzb = (d.n[2] + kZ3 - 1) / kZ3;
                const long long base = (long long)((d.n[0] + kB3 - 1) / kB3) * ((d.n[1] + kB3 - 1) / kB3) * nzb * batch;
                // split the angles so that about 9 CTAs per SM are available (4 resident, 2+ waves)
                const long long want = 9LL * sm_count();
                int nparts = (int)std::min<long long>(16, std::max<long long>(1, (want + base - 1) / base));
                nparts = std::min(nparts, d.na);
                while (nparts > 1 && (long long)nzb * batch * nparts > 65535) --nparts;
                if ((long long)nzb * batch * nparts > 65535) e = cudaErrorInvalidConfiguration;
                float *partial = nullptr;
                const long long nvol = (long long)batch * d.n[0] * d.n[1] * d.n[2];
                if (e == cudaSuccess && nparts > 1) e = cudaMallocAsync((void **)&partial, sizeof(float) * nvol * nparts, st);
                // panel widths of common flat panels get a kernel with the width built in
                auto kern = d.nu == 256 ? k_backproject_v3<256>
                          : d.nu == 512 ? k_backproject_v3<512>
                          : d.nu == 1024 ? k_backproject_v3<1024> : k_backproject_v3<0>;
                if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem3);
                if (e == cudaSuccess) {
                    dim3 gb3((d.n[0] + kB3 - 1) / kB3, (d.n[1] + kB3 - 1) / kB3, nzb * batch * nparts);
                    kern<<<gb3, kThreads3, kSmem3, st>>>(d, pw, vol, accumulate, nparts, partial);
                    e = cudaGetLastError();
                    if (e == cudaSuccess && nparts > 1) {
                        k_sum_parts<<<8 * sm_count(), 256, 0, st>>>(partial, nparts, nvol, vol, accumulate);
                        e = cudaGetLastError();
                    }
                }
                if (partial) cudaFreeAsync(partial, st);
                cudaFreeAsync(pw, st);
                if (e != cudaSuccess) return cuda_fail(e, "back_project launch");
                return 0;
            }
        }
        dim3 gb((d.n[0] + 31) / 32, (d.n[1] + 7) / 8, nzs * batch);
        k_backproject<T, kZS><<<gb, blk, 0, st>>>(d, pw, vol, accumulate);
        e = cudaGetLastError();
    }
    cudaFreeAsync(pw, st);
    if (e != cudaSuccess) return cuda_fail(e, "back_project launch");
    return 0;
}

// P^T (colw x proj): the adjoint of a projection scaled per detector column (the
// redundancy weight of the learned primal block), the scaling folded into the
// per-ray weighting pass.
int back_project_colw(const cbct_geom *g, const float *proj, const float *colw, float *vol, int batch, int accumulate,
                      cudaStream_t st) {
    return backward_impl<float>(g, proj, vol, batch, accumulate, st, colw);
}

int operator_norm(cbct_geom *g, int iters, double *out) {
    const GeomDev &d = g->dev;
    const long long nvox = (long long)d.n[0] * d.n[1] * d.n[2], nproj = (long long)d.na * d.nv * d.nu;
    float *x = nullptr, *p = nullptr;
    double *acc = nullptr;
    cudaError_t e = cudaMalloc(&x, sizeof(float) * nvox);
    if (e == cudaSuccess) e = cudaMalloc(&p, sizeof(float) * nproj);
    if (e == cudaSuccess) e = cudaMalloc(&acc, sizeof(double));
    double nrm2 = 0.0;
    int rc = 0;
    if (e == cudaSuccess) {
        k_fill<<<1024, 256>>>(x, nvox, 1.0f);
        for (int it = 0; it < iters && rc == 0; ++it) {
            cudaMemset(acc, 0, sizeof(double));
            k_sumsq<<<1024, 256>>>(x, nvox, acc);
            k_scale_by<<<1024, 256>>>(x, nvox, acc);
            rc = forward_impl<float>(g, x, p, 1, 0, 0);
            if (rc == 0) rc = backward_impl<float>(g, p, x, 1, 0, 0);
        }
        if (rc == 0) {
            cudaMemset(acc, 0, sizeof(double));
            k_sumsq<<<1024, 256>>>(x, nvox, acc);
            e = cudaMemcpy(&nrm2, acc, sizeof(double), cudaMemcpyDeviceToHost);
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(x);
    cudaFree(p);
    cudaFree(acc);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "operator norm");
    *out = sqrt(sqrt(nrm2));  // ||P^T P x|| with ||x|| = 1 -> ||P||^2
    return 0;
}

}  // namespace cbct

using namespace cbct;

extern "C" int forward_project(const cbct_geom *g, const float *vol, float *proj, int batch, int accumulate,
                               void *stream) {
    return forward_impl<float>(g, vol, proj, batch, accumulate, (cudaStream_t)stream);
}

extern "C" int back_project(const cbct_geom *g, const float *proj, float *vol, int batch, int accumulate,
                            void *stream) {
    return backward_impl<float>(g, proj, vol, batch, accumulate, (cudaStream_t)stream);
}

extern "C" int forward_project_f64(const cbct_geom *g, const double *vol, double *proj, int batch, int accumulate,
                                   void *stream) {
    return forward_impl<double>(g, vol, proj, batch, accumulate, (cudaStream_t)stream);
}

extern "C" int back_project_f64(const cbct_geom *g, const double *proj, double *vol, int batch, int accumulate,
                                void *stream) {
    return backward_impl<double>(g, proj, vol, batch, accumulate, (cudaStream_t)stream);
}

extern "C" int cbct_count_samples(const cbct_geom *g, long long *out, void *stream) {
    if (!g || !out) return fail(CBCT_EINVAL, "cbct_count_samples: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *d = nullptr, h = 0;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&d, sizeof(unsigned long long), st));
    cudaMemsetAsync(d, 0, sizeof(unsigned long long), st);
    const GeomDev &v = g->dev;
    dim3 blk(32, 8), grd((v.nu + 31) / 32, (v.nv + 7) / 8, v.na);
    k_count<<<grd, blk, 0, st>>>(v, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cbct_count_samples");
    *out = (long long)h;
    return 0;
}

// ---- backprojection without allocation --------------------------------------------
//
// back_project needs a scratch copy of the projections with the per-ray step
// length folded in, which it takes from the stream-ordered pool. Some callers
// cannot allocate device memory at call time: a host framework that owns the
// whole device memory budget through its own allocator, or a latency-critical
// loop that must not enter the CUDA allocator (which may take locks or wait on
// the device). back_project_noalloc serves them: its scratch is the fixed
// device array below, and it processes the angles in chunks that fit it.

namespace cbct {

// 8 Mi floats (32 MiB). The CUDA runtime places it on every GPU that loads this
// library, for the lifetime of the process.
constexpr long long kNoAllocScratchFloats = 8ll * 1024 * 1024;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

static std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 256;
static float *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (the current device). Looked up
// once per device: in host code the array's name is only a host-side stand-in.
static int noalloc_scratch(int dev, float **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (dev < 0 || dev >= kMaxDevices) return fail(CBCT_EINVAL, "back_project_noalloc: device index out of range");
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "back_project_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return 0;
}

int noalloc_prime(int dev) {
    float *p = nullptr;
    return noalloc_scratch(dev, &p);
}

}  // namespace cbct

extern "C" int back_project_noalloc(const cbct_geom *g, const float *proj, float *vol, int batch, int accumulate,
                                    void *stream) {
    int rc = check_common(g, proj, vol, batch, accumulate);
    if (rc) return rc;
    const GeomDev &d = g->dev;
    const long long per_angle = (long long)d.nv * d.nu;
    if (per_angle > kNoAllocScratchFloats)
        return fail(CBCT_EINVAL, "back_project_noalloc: one projection (nu * nv = " + std::to_string(per_angle) +
                                     " floats) exceeds the fixed scratch of " +
                                     std::to_string(kNoAllocScratchFloats) + " floats");
    float *scratch = nullptr;
    rc = noalloc_scratch(g->device, &scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int chunk = (int)std::min<long long>(d.na, kNoAllocScratchFloats / per_angle);
    const int nzs = (d.n[2] + kZS - 1) / kZS;
    const long long nvox = (long long)d.n[0] * d.n[1] * d.n[2];
    dim3 blk(32, 8);
    for (int b = 0; b < batch; ++b) {
        for (int k0 = 0; k0 < d.na; k0 += chunk) {
            const int kc = std::min(chunk, d.na - k0);
            // the same kernels on the angle sub-range [k0, k0 + kc)
            GeomDev v = d;
            v.na = kc;
            v.f32 = d.f32 + k0;
            v.f64 = d.f64 + k0;
            v.col32 = d.col32 + (long long)k0 * d.nu;
            v.col64 = d.col64 + (long long)k0 * d.nu;
            const float *pb = proj + ((long long)b * d.na + k0) * per_angle;
            dim3 gw((d.nu + 31) / 32, (d.nv + 7) / 8, kc);
            k_weight_rays<float><<<gw, blk, 0, st>>>(v, pb, scratch, nullptr);
            dim3 gb((d.n[0] + 31) / 32, (d.n[1] + 7) / 8, nzs);
            k_backproject<float, kZS><<<gb, blk, 0, st>>>(v, scratch, vol + b * nvox, k0 == 0 ? accumulate : 1);
            CBCT_LAUNCH_CHECK("back_project_noalloc launch");
        }
    }
    return 0;
}
