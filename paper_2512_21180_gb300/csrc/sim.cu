// Data simulation and per-geometry tensors (a5, a6):
//  - ellipsoid phantom voxeliser (stand-in for the paper's CT volumes, Sec. 2.4)
//  - photon counts N ~ Poisson(I0 exp(-p)) (paper Sec. 2.2, primary model, one
//    energy) from a Philox4x32-10 counter stream (Salmon et al., SC'11), sampled by
//    inversion for means below 10 and by Hoermann's PTRS transformed rejection
//    (1993) above
//  - normalised log transform y = -log(min(max(N, 1) / I0, 1)) (Sec. 2.4)
//  - polychromatic primary (Sec. 2.1): water-bone split of the mu_60 volume, the
//    resp-weighted sum over energy bins of Poisson draws from two line integrals
//    per pixel (water and bone), normalised by the expected air reading
//  - offset-detector redundancy weight w (Sec. 2.6; Wang's sin^2 weight over the
//    overlap band, 1/2 for a centred panel)
//  - field-of-view tensor V = (angles seeing the voxel centre) / (all angles)
//    (Sec. 2.6, definition of V)
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "geom_impl.h"

namespace cbct {

// ---- phantom ---------------------------------------------------------------------

// World coordinate (mm) of sub-sample s of voxel i along one axis:
// ((i - (n-1)/2) + (s + 1/2)/ss - 1/2) vox + c, rounded step by step (no FMA
// contraction) so that every FP64 evaluation of the definition agrees.
__device__ __forceinline__ double sub_point(int i, int n, int s, int ss, double vox, double c) {
    const double t1 = __dsub_rn((double)i, __dmul_rn(0.5, (double)(n - 1)));
    const double t2 = __ddiv_rn(__dadd_rn((double)s, 0.5), (double)ss);
    const double t3 = __dsub_rn(__dadd_rn(t1, t2), 0.5);
    return __dadd_rn(__dmul_rn(t3, vox), c);
}

// ell rows: centre (3, mm), semi-axes (3, mm), rotation (9, rows = ellipsoid axes),
// value, mode (0 add, 1 overwrite). FP64 inside test so that voxels on a boundary
// fall on the same side as in any other FP64 evaluation.
__global__ void k_phantom(GeomDev g, const double *__restrict__ ell, int nell, int ss, double cx, double cy,
                          double cz, float *__restrict__ vol) {
    const long long nvox = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nvox;
         q += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(q % g.n[0]), iy = (int)((q / g.n[0]) % g.n[1]);
        const int iz = (int)(q / ((long long)g.n[0] * g.n[1]));
        double acc = 0.0;
        for (int sz = 0; sz < ss; ++sz)
            for (int sy = 0; sy < ss; ++sy)
                for (int sx = 0; sx < ss; ++sx) {
                    const double P[3] = {sub_point(ix, g.n[0], sx, ss, g.voxd[0], cx),
                                         sub_point(iy, g.n[1], sy, ss, g.voxd[1], cy),
                                         sub_point(iz, g.n[2], sz, ss, g.voxd[2], cz)};
                    double val = 0.0;
                    for (int e = 0; e < nell; ++e) {
                        const double *E = ell + 17 * e;
                        const double d0 = __dsub_rn(P[0], E[0]), d1 = __dsub_rn(P[1], E[1]), d2 = __dsub_rn(P[2], E[2]);
                        double r = 0.0;
                        for (int i = 0; i < 3; ++i) {
                            double l = __dadd_rn(__dadd_rn(__dmul_rn(E[6 + 3 * i], d0), __dmul_rn(E[7 + 3 * i], d1)),
                                                 __dmul_rn(E[8 + 3 * i], d2));
                            double h = __ddiv_rn(l, E[3 + i]);
                            r = __dadd_rn(r, __dmul_rn(h, h));
                        }
                        if (r <= 1.0) val = (E[16] != 0.0) ? E[15] : __dadd_rn(val, E[15]);
                    }
                    acc += val;
                }
        vol[q] = (float)(acc / ((double)ss * ss * ss));
    }
}

// ---- Philox4x32-10 and Poisson -----------------------------------------------------

__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

// One Poisson(lam) draw for element e: key (seed lo, seed hi), counter
// (e lo, e hi, block, 0x50303031); block 0 word 0 for inversion (lam < 10); blocks
// 0, 1, ... two words per attempt for PTRS (lam >= 10).
__device__ int32_t poisson_draw(double lam, unsigned long long e, unsigned long long seed) {
    if (!(lam > 0.0)) return 0;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint4 ctr = make_uint4((uint32_t)e, (uint32_t)(e >> 32), 0u, 0x50303031u);
    // every step rounded as written (no FMA contraction), as in the definition
    if (lam < 10.0) {
        const uint4 r = philox(ctr, k0, k1);
        const double u = u01(r.x);
        double p = exp(-lam), F = p;
        int32_t k = 0;
        while (u > F && k < 1000) {
            k++;
            p = __dmul_rn(p, __ddiv_rn(lam, (double)k));
            F = __dadd_rn(F, p);
        }
        return k;
    }
    const double slam = sqrt(lam), loglam = log(lam);
    const double b = __dadd_rn(0.931, __dmul_rn(2.53, slam));
    const double a = __dadd_rn(-0.059, __dmul_rn(0.02483, b));
    const double inv_alpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dsub_rn(b, 3.4)));
    const double vr = __dsub_rn(0.9277, __ddiv_rn(3.6224, __dsub_rn(b, 2.0)));
    const double twoa = __dmul_rn(2.0, a);
    for (uint32_t j = 0; j < 4096u; ++j) {
        ctr.z = j;
        const uint4 r = philox(ctr, k0, k1);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double U = __dsub_rn(u01(w[2 * h]), 0.5), V = u01(w[2 * h + 1]);
            const double us = __dsub_rn(0.5, fabs(U));
            const double kf = floor(__dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(twoa, us), b), U), lam), 0.43));
            if (us >= 0.07 && V <= vr) return (int32_t)kf;
            if (kf < 0.0 || (us < 0.013 && V > us)) continue;
            const double lhs = log(__ddiv_rn(__dmul_rn(V, inv_alpha), __dadd_rn(__ddiv_rn(a, __dmul_rn(us, us)), b)));
            const double rhs = __dsub_rn(__dadd_rn(-lam, __dmul_rn(kf, loglam)), lgamma(__dadd_rn(kf, 1.0)));
            if (lhs <= rhs) return (int32_t)kf;
        }
    }
    return (int32_t)floor(lam + 0.5);
}

__global__ void k_poisson(const float *__restrict__ p, long long n, double I0, unsigned long long seed,
                          int32_t *__restrict__ counts) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        counts[e] = poisson_draw(__dmul_rn(I0, exp(-(double)p[e])), (unsigned long long)e, seed);
}

__global__ void k_neglog(const int32_t *__restrict__ counts, long long n, float I0, float *__restrict__ y) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float c = counts[e] < 1 ? 1.0f : (float)counts[e];
        y[e] = -logf(fminf(c / I0, 1.0f));
    }
}

// fused: counts from line integrals, then -log, without storing counts
__global__ void k_poisson_neglog(const float *__restrict__ p, long long n, double I0, unsigned long long seed,
                                 float *__restrict__ y) {
    const float I0f = (float)I0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int32_t N = poisson_draw(__dmul_rn(I0, exp(-(double)p[e])), (unsigned long long)e, seed);
        const float c = N < 1 ? 1.0f : (float)N;
        y[e] = -logf(fminf(c / I0f, 1.0f));
    }
}

// ---- polychromatic primary (Sec. 2.1, "Primary simulation") --------------------------

constexpr int kPolyMaxBins = 16;

struct PolyTab {
    int ne;
    double muw[kPolyMaxBins], mub[kPolyMaxBins], resp[kPolyMaxBins];
    double rmin;  // smallest resp_j: the reading of one photon in the least responsive bin
};

// Water-bone split of mu_60 volumes into rho[b][0][.] (water) and rho[b][1][.] (bone):
// rho_hat = mu / mu_w60 (= 0.001 HU + 1); rho_w = rho_hat below tau1 = 1.2, falling
// linearly to 0 at tau2 = 1.6, 0 above (and 0 for rho_hat < 0); rho_b = 0 below tau1,
// rising linearly to kappa_b tau2 at tau2, kappa_b rho_hat above (kappa_b = 0.409).
__global__ void k_water_bone(const float *__restrict__ mu, long long nvox, long long n, float mu_w60,
                             float *__restrict__ rho) {
    const float t1 = 1.2f, t2 = 1.6f, kb = 0.409f;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / nvox, i = e - b * nvox;
        const float r = __fdiv_rn(mu[e], mu_w60);
        float w, bn;
        if (r < t1) {
            w = r < 0.0f ? 0.0f : r;
            bn = 0.0f;
        } else if (r < t2) {
            const float f = (t2 - r) / (t2 - t1);
            w = t1 * f;
            bn = kb * t2 * (1.0f - f);
        } else {
            w = 0.0f;
            bn = kb * r;
        }
        rho[(2 * b) * nvox + i] = w;
        rho[(2 * b + 1) * nvox + i] = bn;
    }
}

// Per detector element (all batch items, angles and pixels): mean counts of bin j
// lam_j = I0[j][pix] exp(-(mu_w[j] L_w + mu_b[j] L_b)) from the water and bone line
// integrals L[b][0 / 1][angle][pixel]; reading = sum_j resp_j N_j with N_j ~
// Poisson(lam_j) drawn on the counter of element e ne + j (lam_j itself when noise
// is 0); y = -log(min(max(reading, rmin) / air, 1)) with the expected air reading
// air = sum_j resp_j I0[j][pix] (a reading of zero photons is taken as one photon of
// the least responsive bin, as the monochromatic path clamps counts to one). FP64
// throughout, each operation rounded as written.
__global__ void k_poly_reading(const float *__restrict__ L, long long per_item, long long n, int npix,
                               const float *__restrict__ I0, PolyTab t, unsigned long long seed, int noise,
                               float *__restrict__ reading, float *__restrict__ y, int32_t *__restrict__ counts) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / per_item, r = e - b * per_item;
        const int pix = (int)(r % npix);
        const double Lw = (double)L[(2 * b) * per_item + r], Lb = (double)L[(2 * b + 1) * per_item + r];
        double acc = 0.0, air = 0.0;
        for (int j = 0; j < t.ne; ++j) {
            const double i0 = (double)I0[(long long)j * npix + pix];
            const double a = __dadd_rn(__dmul_rn(t.muw[j], Lw), __dmul_rn(t.mub[j], Lb));
            const double lam = __dmul_rn(i0, exp(-a));
            double v = lam;
            if (noise) {
                const int32_t c = poisson_draw(lam, (unsigned long long)e * (unsigned long long)t.ne + j, seed);
                if (counts) counts[e * t.ne + j] = c;
                v = (double)c;
            }
            acc = __dadd_rn(acc, __dmul_rn(t.resp[j], v));
            air = __dadd_rn(air, __dmul_rn(t.resp[j], i0));
        }
        if (reading) reading[e] = (float)acc;
        if (y) y[e] = (float)(-log(fmin(__ddiv_rn(fmax(acc, t.rmin), air), 1.0)));
    }
}

// resp(e) for e in keV: piecewise linear through (20, 5), (60, 20), (120, 10),
// constant outside [20, 120].
static double detector_response(double e) {
    if (e <= 20.0) return 5.0;
    if (e <= 60.0) return 5.0 + (e - 20.0) * (20.0 - 5.0) / (60.0 - 20.0);
    if (e <= 120.0) return 20.0 + (e - 60.0) * (10.0 - 20.0) / (120.0 - 60.0);
    return 10.0;
}

static int poly_table(int n_e, const double *energies, const double *mu_w, const double *mu_b, PolyTab *t,
                      const char *who) {
    if (n_e < 1 || n_e > kPolyMaxBins || !energies || !mu_w || !mu_b)
        return fail(CBCT_EINVAL, std::string(who) + ": need 1 <= n_e <= 16 and host tables");
    t->ne = n_e;
    t->rmin = detector_response(energies[0]);
    for (int j = 0; j < n_e; ++j) {
        if (!(energies[j] > 0.0) || !std::isfinite(energies[j]) || !(mu_w[j] >= 0.0) || !std::isfinite(mu_w[j]) ||
            !(mu_b[j] >= 0.0) || !std::isfinite(mu_b[j]))
            return fail(CBCT_EINVAL, std::string(who) + ": energies must be > 0 and attenuations finite and >= 0");
        t->muw[j] = mu_w[j];
        t->mub[j] = mu_b[j];
        t->resp[j] = detector_response(energies[j]);
        t->rmin = fmin(t->rmin, t->resp[j]);
    }
    return 0;
}

// ---- redundancy weight and field of view ---------------------------------------------

__global__ void k_redundancy(int nu, double du, double uoff, float *__restrict__ w) {
    const int iu = blockIdx.x * blockDim.x + threadIdx.x;
    if (iu >= nu) return;
    const double PI = 3.14159265358979323846;
    const double u = (iu - 0.5 * (nu - 1)) * du + uoff;
    double val;
    if (uoff == 0.0) val = 0.5;
    else {
        const double D = 0.5 * nu * du - fabs(uoff);
        const double us = uoff > 0 ? u : -u;
        if (us < -D) val = 0.0;
        else if (us > D) val = 1.0;
        else { const double s = sin(0.25 * PI * (us + D) / D); val = s * s; }
    }
    w[iu] = (float)val;
}

// V: one thread per voxel, counts angles whose projection of the voxel centre lies on
// the panel (continuous pixel coordinates in [-1/2, n - 1/2]); FP64 geometry.
__global__ void k_fov(GeomDev g, const double *__restrict__ cs, double sid, double sdd, double du, double dv,
                      double uoff, double voff, double cx, double cy, double cz, float *__restrict__ V) {
    const long long nvox = (long long)g.n[0] * g.n[1] * g.n[2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nvox;
         q += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(q % g.n[0]), iy = (int)((q / g.n[0]) % g.n[1]);
        const int iz = (int)(q / ((long long)g.n[0] * g.n[1]));
        const double px = __dadd_rn(__dmul_rn(__dsub_rn((double)ix, __dmul_rn(0.5, (double)(g.n[0] - 1))), g.voxd[0]), cx);
        const double py = __dadd_rn(__dmul_rn(__dsub_rn((double)iy, __dmul_rn(0.5, (double)(g.n[1] - 1))), g.voxd[1]), cy);
        const double pz = __dadd_rn(__dmul_rn(__dsub_rn((double)iz, __dmul_rn(0.5, (double)(g.n[2] - 1))), g.voxd[2]), cz);
        const double hu = __dmul_rn(0.5, (double)(g.nu - 1)), hv = __dmul_rn(0.5, (double)(g.nv - 1));
        int cnt = 0;
        for (int k = 0; k < g.na; ++k) {
            const double c = cs[2 * k], s = cs[2 * k + 1];
            const double U = __dsub_rn(sid, __dadd_rn(__dmul_rn(px, c), __dmul_rn(py, s)));
            if (!(U > 0.0)) continue;
            const double m = __ddiv_rn(sdd, U);
            const double u = __dmul_rn(m, __dadd_rn(__dmul_rn(-px, s), __dmul_rn(py, c)));
            const double fu = __dadd_rn(__ddiv_rn(__dsub_rn(u, uoff), du), hu);
            const double fv = __dadd_rn(__ddiv_rn(__dsub_rn(__dmul_rn(m, pz), voff), dv), hv);
            if (fu >= -0.5 && fu <= g.nu - 0.5 && fv >= -0.5 && fv <= g.nv - 0.5) cnt++;
        }
        V[q] = (float)((double)cnt / g.na);
    }
}

static int grid_for(long long n) {
    long long b = (n + 255) / 256;
    const long long cap = 16LL * sm_count();
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

}  // namespace cbct

using namespace cbct;

extern "C" int cbct_phantom(const cbct_geom *g, const double *ell_host, int n_ell, int supersample, float *vol,
                            void *stream) {
    if (!g || !vol || (n_ell > 0 && !ell_host) || n_ell < 0 || supersample < 1 || supersample > 8)
        return fail(CBCT_EINVAL, "cbct_phantom: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    double *d = nullptr;
    if (n_ell > 0) {
        CBCT_CUDA_TRY(cudaMallocAsync((void **)&d, sizeof(double) * 17 * n_ell, st));
        cudaError_t e = cudaMemcpyAsync(d, ell_host, sizeof(double) * 17 * n_ell, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { cudaFreeAsync(d, st); return cuda_fail(e, "cbct_phantom: upload"); }
    }
    const GeomDev &v = g->dev;
    const long long nvox = (long long)v.n[0] * v.n[1] * v.n[2];
    k_phantom<<<grid_for(nvox), 256, 0, st>>>(v, d, n_ell, supersample, g->desc.center[0], g->desc.center[1],
                                              g->desc.center[2], vol);
    cudaError_t e = cudaGetLastError();
    if (d) cudaFreeAsync(d, st);
    if (e != cudaSuccess) return cuda_fail(e, "cbct_phantom launch");
    // the host array may be reused as soon as this call returns
    CBCT_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

extern "C" int cbct_poisson(const float *line_integrals, long long n, double I0, unsigned long long seed,
                            int32_t *counts, void *stream) {
    if (!line_integrals || !counts || n < 0 || !(I0 > 0)) return fail(CBCT_EINVAL, "cbct_poisson: invalid argument");
    if (n == 0) return 0;
    k_poisson<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(line_integrals, n, I0, seed, counts);
    CBCT_LAUNCH_CHECK("cbct_poisson launch");
    return 0;
}

extern "C" int cbct_neglog(const int32_t *counts, long long n, double I0, float *y, void *stream) {
    if (!counts || !y || n < 0 || !(I0 > 0)) return fail(CBCT_EINVAL, "cbct_neglog: invalid argument");
    if (n == 0) return 0;
    k_neglog<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(counts, n, (float)I0, y);
    CBCT_LAUNCH_CHECK("cbct_neglog launch");
    return 0;
}

extern "C" int cbct_simulate(const cbct_geom *g, const float *vol, int batch, double I0, unsigned long long seed,
                             float *line_integrals, float *y, void *stream) {
    if (!g || !vol || !line_integrals || !y || batch < 1 || !(I0 > 0))
        return fail(CBCT_EINVAL, "cbct_simulate: invalid argument");
    int rc = forward_project(g, vol, line_integrals, batch, 0, stream);
    if (rc) return rc;
    const GeomDev &v = g->dev;
    const long long n = (long long)batch * v.na * v.nv * v.nu;
    k_poisson_neglog<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(line_integrals, n, I0, seed, y);
    CBCT_LAUNCH_CHECK("cbct_simulate launch");
    return 0;
}

extern "C" int cbct_redundancy_weight(const cbct_geom *g, float *w, void *stream) {
    if (!g || !w) return fail(CBCT_EINVAL, "cbct_redundancy_weight: invalid argument");
    const cbct_geom_desc &d = g->desc;
    k_redundancy<<<(d.nu + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d.nu, d.du, d.u_offset, w);
    CBCT_LAUNCH_CHECK("cbct_redundancy_weight launch");
    return 0;
}

extern "C" int cbct_fov(const cbct_geom *g, float *V, void *stream) {
    if (!g || !V) return fail(CBCT_EINVAL, "cbct_fov: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const cbct_geom_desc &d = g->desc;
    const double PI = 3.14159265358979323846;
    std::vector<double> cs(2 * (size_t)d.n_angles);
    for (int k = 0; k < d.n_angles; ++k) {
        const double th = g->angles.empty() ? 2.0 * PI * k / d.n_angles : g->angles[k];
        cs[2 * k] = cos(th);
        cs[2 * k + 1] = sin(th);
    }
    double *dcs = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&dcs, sizeof(double) * cs.size(), st));
    cudaError_t e = cudaMemcpyAsync(dcs, cs.data(), sizeof(double) * cs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const long long nvox = (long long)d.nx * d.ny * d.nz;
        k_fov<<<grid_for(nvox), 256, 0, st>>>(g->dev, dcs, d.sid, d.sdd, d.du, d.dv, d.u_offset, d.v_offset,
                                              d.center[0], d.center[1], d.center[2], V);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host table must outlive the copy
    cudaFreeAsync(dcs, st);
    if (e != cudaSuccess) return cuda_fail(e, "cbct_fov");
    return 0;
}

extern "C" int cbct_detector_response(const double *energies_kev, int n_e, double *resp) {
    if (!energies_kev || !resp || n_e < 0) return fail(CBCT_EINVAL, "cbct_detector_response: invalid argument");
    for (int j = 0; j < n_e; ++j) resp[j] = detector_response(energies_kev[j]);
    return 0;
}

extern "C" int cbct_water_bone(const float *mu, long long n_vox, int batch, double mu_water60, float *rho,
                               void *stream) {
    if (!mu || !rho || n_vox < 0 || batch < 1 || !(mu_water60 > 0) || !std::isfinite(mu_water60))
        return fail(CBCT_EINVAL, "cbct_water_bone: invalid argument");
    const long long n = n_vox * batch;
    if (n == 0) return 0;
    k_water_bone<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(mu, n_vox, n, (float)mu_water60, rho);
    CBCT_LAUNCH_CHECK("cbct_water_bone launch");
    return 0;
}

extern "C" int cbct_poly_reading(const float *line_integrals, int batch, long long n_per_item, int npix, int n_e,
                                 const double *energies_kev, const double *mu_water, const double *mu_bone,
                                 const float *I0, unsigned long long seed, int noise, float *reading, float *y,
                                 int32_t *counts, void *stream) {
    PolyTab t;
    int rc = poly_table(n_e, energies_kev, mu_water, mu_bone, &t, "cbct_poly_reading");
    if (rc) return rc;
    if (!line_integrals || !I0 || batch < 1 || n_per_item < 0 || npix < 1 || n_per_item % npix != 0 ||
        (!reading && !y && !counts) || (counts && !noise))
        return fail(CBCT_EINVAL, "cbct_poly_reading: invalid argument");
    const long long n = n_per_item * batch;
    if (n == 0) return 0;
    k_poly_reading<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(line_integrals, n_per_item, n, npix, I0, t, seed,
                                                                  noise ? 1 : 0, reading, y, counts);
    CBCT_LAUNCH_CHECK("cbct_poly_reading launch");
    return 0;
}

extern "C" int cbct_poly_simulate(const cbct_geom *g, const float *mu, int batch, double mu_water60, int n_e,
                                  const double *energies_kev, const double *mu_water, const double *mu_bone,
                                  const float *I0, unsigned long long seed, int noise, float *line_integrals, float *y,
                                  void *stream) {
    PolyTab t;
    int rc = poly_table(n_e, energies_kev, mu_water, mu_bone, &t, "cbct_poly_simulate");
    if (rc) return rc;
    if (!g || !mu || !I0 || !line_integrals || !y || batch < 1 || !(mu_water60 > 0) || !std::isfinite(mu_water60))
        return fail(CBCT_EINVAL, "cbct_poly_simulate: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const GeomDev &v = g->dev;
    const long long nvox = (long long)v.n[0] * v.n[1] * v.n[2];
    const long long per_item = (long long)v.na * v.nv * v.nu;
    float *rho = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&rho, sizeof(float) * 2 * nvox * batch, st));
    k_water_bone<<<grid_for(nvox * batch), 256, 0, st>>>(mu, nvox, nvox * batch, (float)mu_water60, rho);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFreeAsync(rho, st);
        return cuda_fail(e, "cbct_poly_simulate: water-bone launch");
    }
    rc = forward_project(g, rho, line_integrals, 2 * batch, 0, stream);
    cudaFreeAsync(rho, st);
    if (rc) return rc;
    k_poly_reading<<<grid_for(per_item * batch), 256, 0, st>>>(line_integrals, per_item, per_item * batch,
                                                              v.nv * v.nu, I0, t, seed, noise ? 1 : 0, nullptr, y,
                                                              nullptr);
    CBCT_LAUNCH_CHECK("cbct_poly_simulate: reading launch");
    return 0;
}
