// Geometry object of the cone-beam library (a1): per-angle ray tables in voxel-index
// coordinates, validation, status reporting.
//
// The frame of angle theta (paper Sec. 2.2 scanner: source on a circle of radius
// SID about z, flat panel at SDD, panel offset along the direction of rotation):
//   S   = ((sid cos - cx)/vx + (nx-1)/2, (sid sin - cy)/vy + (ny-1)/2, -cz/vz + (nz-1)/2)
//   D0S = ((-sdd cos - a sin)/vx, (-sdd sin + a cos)/vy, b/vz)      pixel (0,0) - source
//   EU  = (-du sin/vx, du cos/vy, 0),  EV = (0, 0, dv/vz)
// with a = -(nu-1)/2 du + u_offset and b = -(nv-1)/2 dv + v_offset, evaluated in
// FP64 on the host in this order and rounded once to FP32 for the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "geom_impl.h"

namespace cbct {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(e == cudaErrorMemoryAllocation ? CBCT_ENOMEM : CBCT_ECUDA, m);
}

GeomDev dev_view(const cbct_geom *g) { return g->dev; }

int sm_count() {
    constexpr int kMaxDev = 64;
    static int cached[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 152;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
        cached[dev] = n;
    }
    return cached[dev];
}

}  // namespace cbct

using namespace cbct;

extern "C" const char *cbct_last_error(void) { return g_last_error.c_str(); }

static void build_frames(const cbct_geom_desc &d, const std::vector<double> &ang, std::vector<Frame32> &f32,
                         std::vector<Frame64> &f64) {
    const double PI = 3.14159265358979323846;
    int na = d.n_angles;
    f32.resize(na);
    f64.resize(na);
    for (int k = 0; k < na; ++k) {
        double th = ang.empty() ? 2.0 * PI * k / na : ang[k];
        double c = cos(th), s = sin(th);
        double a = -0.5 * (d.nu - 1) * d.du + d.u_offset;
        double b = -0.5 * (d.nv - 1) * d.dv + d.v_offset;
        Frame64 F;
        F.S[0] = (d.sid * c - d.center[0]) / d.vox[0] + 0.5 * (d.nx - 1);
        F.S[1] = (d.sid * s - d.center[1]) / d.vox[1] + 0.5 * (d.ny - 1);
        F.S[2] = (0.0 - d.center[2]) / d.vox[2] + 0.5 * (d.nz - 1);
        F.D0S[0] = (-d.sdd * c - a * s) / d.vox[0];
        F.D0S[1] = (-d.sdd * s + a * c) / d.vox[1];
        F.D0S[2] = b / d.vox[2];
        F.EU[0] = -d.du * s / d.vox[0];
        F.EU[1] = d.du * c / d.vox[1];
        F.EU[2] = 0.0;
        F.EV[0] = 0.0;
        F.EV[1] = 0.0;
        F.EV[2] = d.dv / d.vox[2];
        f64[k] = F;
        Frame32 G;
        for (int i = 0; i < 3; ++i) {
            G.S[i] = (float)F.S[i];
            G.D0S[i] = (float)F.D0S[i];
            G.EU[i] = (float)F.EU[i];
            G.EV[i] = (float)F.EV[i];
        }
        G.ux_lo = d.nu; G.ux_hi = -1; G.uy_lo = d.nu; G.uy_hi = -1;
        for (int iu = 0; iu < d.nu; ++iu) {
            if (principal_axis(G, iu) == 0) {
                if (iu < G.ux_lo) G.ux_lo = iu;
                G.ux_hi = iu;
            } else {
                if (iu < G.uy_lo) G.uy_lo = iu;
                G.uy_hi = iu;
            }
        }
        f32[k] = G;
    }
}

// Per-column ray parameters (see ColT in common.cuh), FP64, from the FP64 frames
// and the FP32 principal-axis decision.
static void build_columns(const cbct_geom_desc &d, const std::vector<Frame32> &f32, const std::vector<Frame64> &f64,
                          std::vector<Col32> &c32, std::vector<Col64> &c64, std::vector<float> &rz32,
                          std::vector<double> &rz64) {
    const int na = d.n_angles, nu = d.nu;
    const int n[2] = {d.nx, d.ny};
    c32.resize((size_t)na * nu);
    c64.resize((size_t)na * nu);
    for (int k = 0; k < na; ++k) {
        const Frame64 &F = f64[k];
        for (int iu = 0; iu < nu; ++iu) {
            const int a = principal_axis(f32[k], iu), b = 1 - a;
            const double ra = F.D0S[a] + iu * F.EU[a];
            const double rb = F.D0S[b] + iu * F.EU[b];
            const double ca = 0.5 * (n[a] - 1);
            Col64 c;
            c.inv = 1.0 / ra;
            c.dqb = rb / ra;
            c.tc = (ca - F.S[a]) / ra;
            c.qcb = F.S[b] + c.tc * rb;
            c64[(size_t)k * nu + iu] = c;
            c32[(size_t)k * nu + iu] = Col32{(float)c.dqb, (float)c.qcb, (float)c.tc, (float)c.inv};
        }
    }
    rz32.resize(d.nv);
    rz64.resize(d.nv);
    for (int iv = 0; iv < d.nv; ++iv) {
        rz64[iv] = f64[0].D0S[2] + iv * f64[0].EV[2];
        rz32[iv] = (float)rz64[iv];
    }
}

// Bounds on the footprint of a 32 x 8 ray tile over one 8-plane chunk (the staged
// forward's TMA box must hold it): per-column changes of the central-plane
// parameters times the tile width, plane slopes times the chunk depth, plus
// neighbour, floor and alignment margins. Also checks that at every angle the
// x- and y-principal columns form intervals.
static void forward_bounds(const cbct_geom_desc &d, const std::vector<Frame32> &f32, const std::vector<Col64> &c64,
                           const std::vector<double> &rz64, double &need_b, double &need_z, bool &contiguous) {
    const int TU = 32, TV = 8, P = 8;
    const int n[2] = {d.nx, d.ny};
    double rzmax = 0.0;
    for (double r : rz64) rzmax = std::max(rzmax, std::fabs(r));
    const double drz = d.nv > 1 ? std::fabs(rz64[1] - rz64[0]) : 0.0;
    double Mb = 0, Mzu = 0, Dq = 0, Dz = 0, tmax = 0;
    contiguous = true;
    for (int k = 0; k < d.n_angles; ++k) {
        const Frame32 &F = f32[k];
        for (int u = F.ux_lo; u <= F.ux_hi; ++u)
            if (principal_axis(F, u) != 0) contiguous = false;
        for (int u = F.uy_lo; u <= F.uy_hi; ++u)
            if (principal_axis(F, u) != 1) contiguous = false;
        for (int u = 0; u < d.nu; ++u) {
            const int a = principal_axis(F, u);
            const double ca = 0.5 * (n[a] - 1);
            const Col64 &c = c64[(size_t)k * d.nu + u];
            Dq = std::max(Dq, std::fabs(c.dqb));
            Dz = std::max(Dz, rzmax * std::fabs(c.inv));
            tmax = std::max(tmax, std::fabs(c.tc) + ca * std::fabs(c.inv));
            if (u + 1 < d.nu && principal_axis(F, u + 1) == a) {
                const Col64 &e = c64[(size_t)k * d.nu + u + 1];
                Mb = std::max(Mb, std::fabs(e.qcb - c.qcb) + ca * std::fabs(e.dqb - c.dqb));
                Mzu = std::max(Mzu, rzmax * (std::fabs(e.tc - c.tc) + ca * std::fabs(e.inv - c.inv)));
            }
        }
    }
    need_b = (TU - 1) * Mb + (P - 1) * Dq + 8.0;
    need_z = (TV - 1) * tmax * drz + (TU - 1) * Mzu + (P - 1) * Dz + 5.0;
}

// No ray may have z as its principal axis: at every angle the smallest
// max(|r_x|, |r_y|) over columns must exceed the largest |r_z| over rows (r_x, r_y
// depend on the column only and r_z on the row only), on the FP32 directions.
static bool z_principal_free(const cbct_geom_desc &d, const std::vector<Frame32> &f32) {
    for (const Frame32 &f : f32) {
        float mxy = INFINITY, mz = 0.0f;
        for (int iu = 0; iu < d.nu; ++iu) {
            float rx = fabsf(fmaf((float)iu, f.EU[0], f.D0S[0]));
            float ry = fabsf(fmaf((float)iu, f.EU[1], f.D0S[1]));
            mxy = fminf(mxy, fmaxf(rx, ry));
        }
        for (int iv = 0; iv < d.nv; ++iv) mz = fmaxf(mz, fabsf(fmaf((float)iv, f.EV[2], f.D0S[2])));
        if (!(mz < mxy)) return false;
    }
    return true;
}

extern "C" int geometry_create(const cbct_geom_desc *desc, cbct_geom **out) {
    if (!desc || !out) return fail(CBCT_EINVAL, "geometry_create: NULL argument");
    *out = nullptr;
    const cbct_geom_desc &d = *desc;
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nu < 1 || d.nv < 1 || d.n_angles < 1)
        return fail(CBCT_EINVAL, "geometry_create: sizes must be >= 1");
    if (!(d.vox[0] > 0 && d.vox[1] > 0 && d.vox[2] > 0 && d.du > 0 && d.dv > 0 && d.sid > 0 && d.sdd > 0))
        return fail(CBCT_EINVAL, "geometry_create: pitches and distances must be > 0");
    if ((double)d.nx * d.ny * d.nz >= 2147483647.0 || (double)d.nu * d.nv * d.n_angles >= 2147483647.0)
        return fail(CBCT_EINVAL, "geometry_create: volume or projection larger than 2^31 elements");
    if (d.n_angles > 65535) return fail(CBCT_EINVAL, "geometry_create: more than 65535 angles");
    if (d.normalize != 0 && d.normalize != 1) return fail(CBCT_EINVAL, "geometry_create: normalize must be 0 or 1");
    std::vector<double> ang;
    if (d.angles) ang.assign(d.angles, d.angles + d.n_angles);
    std::vector<Frame32> f32;
    std::vector<Frame64> f64;
    build_frames(d, ang, f32, f64);
    if (!z_principal_free(d, f32))
        return fail(CBCT_EINVAL, "geometry_create: some rays would have z as principal axis (cone too wide)");

    cbct_geom *g = new (std::nothrow) cbct_geom();
    if (!g) return fail(CBCT_ENOMEM, "geometry_create: host allocation failed");
    g->desc = d;
    g->angles = ang;
    g->desc.angles = nullptr;
    g->h32 = f32;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "cudaGetDevice"); }
    g->device = dev;
    std::vector<Col32> c32;
    std::vector<Col64> c64;
    std::vector<float> rz32;
    std::vector<double> rz64;
    build_columns(d, f32, f64, c32, c64, rz32, rz64);
    const size_t ncol = (size_t)d.n_angles * d.nu;
    forward_bounds(d, f32, c64, rz64, g->fwd_need_b, g->fwd_need_z, g->axis_contiguous);
    g->fwd_cfg = g->axis_contiguous ? choose_forward_cfg(g->fwd_need_b, g->fwd_need_z) : -1;
    e = cudaMalloc(&g->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(g->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&g->f32, sizeof(Frame32) * d.n_angles);
    if (e == cudaSuccess) e = cudaMalloc(&g->f64, sizeof(Frame64) * d.n_angles);
    if (e == cudaSuccess) e = cudaMalloc(&g->col32, sizeof(Col32) * ncol);
    if (e == cudaSuccess) e = cudaMalloc(&g->col64, sizeof(Col64) * ncol);
    if (e == cudaSuccess) e = cudaMalloc(&g->rz32, sizeof(float) * d.nv);
    if (e == cudaSuccess) e = cudaMalloc(&g->rz64, sizeof(double) * d.nv);
    std::vector<double2> cs(d.n_angles);
    for (int k = 0; k < d.n_angles; ++k) {
        const double th = ang.empty() ? 2.0 * 3.14159265358979323846 * k / d.n_angles : ang[k];
        cs[k] = make_double2(cos(th), sin(th));
    }
    if (e == cudaSuccess) e = cudaMalloc(&g->cs, sizeof(double2) * d.n_angles);
    if (e == cudaSuccess) e = cudaMemcpy(g->cs, cs.data(), sizeof(double2) * d.n_angles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->f32, f32.data(), sizeof(Frame32) * d.n_angles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->f64, f64.data(), sizeof(Frame64) * d.n_angles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->col32, c32.data(), sizeof(Col32) * ncol, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->col64, c64.data(), sizeof(Col64) * ncol, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->rz32, rz32.data(), sizeof(float) * d.nv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->rz64, rz64.data(), sizeof(double) * d.nv, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        geometry_destroy(g);
        return cuda_fail(e, "geometry_create: table upload");
    }
    GeomDev &v = g->dev;
    v.n[0] = d.nx; v.n[1] = d.ny; v.n[2] = d.nz;
    v.nu = d.nu; v.nv = d.nv; v.na = d.n_angles;
    for (int i = 0; i < 3; ++i) { v.vox[i] = (float)d.vox[i]; v.voxd[i] = d.vox[i]; }
    v.scale = 1.0f;
    v.scaled = 1.0;
    v.f32 = g->f32;
    v.f64 = g->f64;
    v.col32 = g->col32;
    v.col64 = g->col64;
    v.rz32 = g->rz32;
    v.rz64 = g->rz64;
    v.Szd = f64[0].S[2];
    v.Sz = (float)v.Szd;
    if (d.normalize) {
        double nrm = 0.0;
        int rc = cbct::operator_norm(g, 30, &nrm);
        if (rc != 0) { geometry_destroy(g); return rc; }
        if (!(nrm > 0.0)) { geometry_destroy(g); return fail(CBCT_EINVAL, "geometry_create: ||P|| is zero"); }
        v.scaled = 1.0 / nrm;
        v.scale = (float)v.scaled;
    }
    // resolve the fixed scratch array of back_project_noalloc on this device now: the
    // lookup loads the projector module (and so places the array) here, so that the
    // no-allocation entry point itself never reaches the allocator
    {
        int rc = cbct::noalloc_prime(dev);
        if (rc != 0) { geometry_destroy(g); return rc; }
    }
    *out = g;
    return 0;
}

extern "C" void geometry_destroy(cbct_geom *g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    if (g->f32) cudaFree(g->f32);
    if (g->f64) cudaFree(g->f64);
    if (g->col32) cudaFree(g->col32);
    if (g->col64) cudaFree(g->col64);
    if (g->rz32) cudaFree(g->rz32);
    if (g->rz64) cudaFree(g->rz64);
    if (g->cs) cudaFree(g->cs);
    if (g->status) cudaFree(g->status);
    cudaSetDevice(cur);
    delete g;
}

extern "C" double geometry_scale(const cbct_geom *g) { return g ? g->dev.scaled : 0.0; }

extern "C" int cbct_device_status(const cbct_geom *g, int *out, int clear) {
    if (!g || !out) return fail(CBCT_EINVAL, "cbct_device_status: NULL argument");
    int v = 0;
    CBCT_CUDA_TRY(cudaMemcpy(&v, g->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (clear && v) CBCT_CUDA_TRY(cudaMemset(g->status, 0, sizeof(int)));
    *out = v;
    return 0;
}

extern "C" int cbct_forward_config(const cbct_geom *g, int *cfg, double *need_b, double *need_z) {
    if (!g) return fail(CBCT_EINVAL, "cbct_forward_config: NULL geometry");
    if (cfg) *cfg = g->fwd_cfg;
    if (need_b) *need_b = g->fwd_need_b;
    if (need_z) *need_z = g->fwd_need_z;
    return 0;
}
