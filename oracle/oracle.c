/*
 * FP64 CPU oracle for the cone-beam projector pair and the data simulation.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg call this code; the GPU library never links or calls it, and
 * it shares no code with the GPU library. It is written to be read against its
 * definitions, not to be fast: plain loops, FP64 throughout.
 *
 * What is computed (citations are to the paper, arXiv 2512.21180):
 *  - the cone-beam transform P(mu)(t,u) = integral of mu along the line from the
 *    source to detector element u at time t, and its adjoint P* (Sec. 2.2, the
 *    projection-operator equation). The paper does not say how P is discretised;
 *    this oracle fixes the Joseph-style reading: for each ray choose the principal
 *    axis, sample the volume on every voxel-centre plane perpendicular to it by
 *    bilinear interpolation (zero outside the grid) and sum with the step length.
 *    The adjoint scatters with exactly the same weights.
 *  - the circular-orbit, laterally offset flat-panel geometry (Sec. 2.2: SID 1000,
 *    isocentre-detector 536 mm, panel offset in the direction of rotation).
 *  - the field-of-view tensor V (Sec. 2.6, definition of V).
 *  - the offset-detector redundancy weight w (Sec. 2.6; the paper names no scheme,
 *    the reading used is Wang's smooth sin^2 weight over the overlap band).
 *  - FDK with redundancy weighting (Sec. 2.6, Algorithm 1 initialisation; Feldkamp
 *    et al. 1984).
 *  - PDHG with isotropic TV and x >= 0 (Sec. 2.5 baseline; Chambolle-Pock 2011).
 *  - Poisson photon counts and the normalised -log transform (Sec. 2.2 primary
 *    model, Sec. 2.4 normalisation equations), monochromatic.
 *  - Philox4x32-10 (Salmon et al., SC'11), the counter-based generator that feeds
 *    the Poisson sampler on both sides; Poisson sampling by inversion for small
 *    means and Hoermann's PTRS transformed rejection (1993) otherwise.
 *  - ellipsoid phantom voxelisation (point and supersampled).
 *  - the polychromatic primary (Sec. 2.1): water-bone decomposition, detector
 *    response and the resp-weighted sum of per-energy Poisson draws.
 *
 * The one FP32 computation in this file is the principal-axis choice of a ray:
 * it is defined on the FP32 ray direction (see paxis32) so that the CPU and GPU
 * choose the same axis on near-diagonal rays.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* dims = {nx, ny, nz, nu, nv, n_angles};
 * par  = {vox_x, vox_y, vox_z, cx, cy, cz, du, dv, u_offset, v_offset, sid, sdd} */
typedef struct {
    int n[3];
    int nu, nv, na;
    double vox[3], ctr[3];
    double du, dv, uoff, voff, sid, sdd;
    const double *ang;
} ogeom;

static ogeom mk(const int *dims, const double *par, const double *ang)
{
    ogeom g;
    g.n[0] = dims[0]; g.n[1] = dims[1]; g.n[2] = dims[2];
    g.nu = dims[3]; g.nv = dims[4]; g.na = dims[5];
    for (int c = 0; c < 3; ++c) { g.vox[c] = par[c]; g.ctr[c] = par[3 + c]; }
    g.du = par[6]; g.dv = par[7]; g.uoff = par[8]; g.voff = par[9];
    g.sid = par[10]; g.sdd = par[11];
    g.ang = ang;
    return g;
}

static double angle_of(const ogeom *g, int k)
{
    return g->ang ? g->ang[k] : 2.0 * M_PI * k / g->na;
}

/* Per-angle ray frame in continuous voxel-index coordinates.
 * World frame: isocentre at the origin, rotation axis z. At angle th the source is
 * s = sid (cos th, sin th, 0); the detector centre is s + sdd (-cos th, -sin th, 0);
 * the detector axes are e_u = (-sin th, cos th, 0) (direction of rotation) and
 * e_v = (0, 0, 1). Pixel (iu, iv) sits at ((iu - (nu-1)/2) du + u_offset) e_u +
 * ((iv - (nv-1)/2) dv + v_offset) e_v from the detector centre. A world point P has
 * index coordinates (P_c - center_c)/vox_c + (n_c - 1)/2.
 * Outputs: S = source, D0S = pixel(0,0) - source, EU/EV = per-pixel steps. */
static void frame(const ogeom *g, int k, double S[3], double D0S[3], double EU[3], double EV[3])
{
    double th = angle_of(g, k);
    double c = cos(th), s = sin(th);
    double a = -0.5 * (g->nu - 1) * g->du + g->uoff;
    double b = -0.5 * (g->nv - 1) * g->dv + g->voff;
    S[0] = (g->sid * c - g->ctr[0]) / g->vox[0] + 0.5 * (g->n[0] - 1);
    S[1] = (g->sid * s - g->ctr[1]) / g->vox[1] + 0.5 * (g->n[1] - 1);
    S[2] = (0.0 - g->ctr[2]) / g->vox[2] + 0.5 * (g->n[2] - 1);
    D0S[0] = (-g->sdd * c - a * s) / g->vox[0];
    D0S[1] = (-g->sdd * s + a * c) / g->vox[1];
    D0S[2] = b / g->vox[2];
    EU[0] = -g->du * s / g->vox[0];
    EU[1] = g->du * c / g->vox[1];
    EU[2] = 0.0;
    EV[0] = 0.0;
    EV[1] = 0.0;
    EV[2] = g->dv / g->vox[2];
}

/* Principal axis of ray (iu, iv): the axis of largest |direction| component, ties
 * to x before y before z. Decided on the FP32 direction
 * r_c = fmaf(iv, EV_c, fmaf(iu, EU_c, D0S_c)) built from the FP32-rounded frame, so
 * that every implementation takes the same decision on near-diagonal rays. */
static int paxis32(const double D0S[3], const double EU[3], const double EV[3], int iu, int iv)
{
    float r[3];
    for (int c = 0; c < 3; ++c)
        r[c] = fmaf((float)iv, (float)EV[c], fmaf((float)iu, (float)EU[c], (float)D0S[c]));
    float ax = fabsf(r[0]), ay = fabsf(r[1]), az = fabsf(r[2]);
    if (ax >= ay && ax >= az) return 0;
    if (ay >= az) return 1;
    return 2;
}

static long vidx(const ogeom *g, const int p[3])
{
    return ((long)p[2] * g->n[1] + p[1]) * g->n[0] + p[0];
}

/* Walk one ray: for every plane i of the principal axis a with source-to-pixel
 * parameter t in (0, 1) and in-plane point inside (-1, n) x (-1, n), visit the four
 * bilinear neighbours (weights (1-fb)(1-fc), ...; neighbours outside the grid are
 * skipped, i.e. the volume is zero there). mode 0: return w * sum of samples of vol;
 * mode 1: scatter w * weight * pval into vol. Counts visited samples in *ns. */
static double walk(const ogeom *g, double *vol, const double *cvol, int k, int iu, int iv,
                   int mode, double pval, long *ns)
{
    double S[3], D0S[3], EU[3], EV[3], R[3];
    frame(g, k, S, D0S, EU, EV);
    for (int c = 0; c < 3; ++c) R[c] = D0S[c] + iu * EU[c] + iv * EV[c];
    int a = paxis32(D0S, EU, EV, iu, iv);
    int b = (a == 0) ? 1 : 0;
    int c2 = (a == 2) ? 1 : 2;
    double len = sqrt(R[0] * g->vox[0] * R[0] * g->vox[0] + R[1] * g->vox[1] * R[1] * g->vox[1] +
                      R[2] * g->vox[2] * R[2] * g->vox[2]);
    double w = len / fabs(R[a]); /* world length of the ray between consecutive planes */
    double sum = 0.0;
    for (int i = 0; i < g->n[a]; ++i) {
        double t = (i - S[a]) / R[a];
        if (!(t > 0.0 && t < 1.0)) continue;
        double qb = S[b] + t * R[b];
        double qc = S[c2] + t * R[c2];
        if (!(qb > -1.0 && qb < g->n[b] && qc > -1.0 && qc < g->n[c2])) continue;
        if (ns) (*ns)++;
        double fb0 = floor(qb), fc0 = floor(qc);
        double fb = qb - fb0, fc = qc - fc0;
        int ib = (int)fb0, ic = (int)fc0;
        for (int db = 0; db < 2; ++db) {
            for (int dc = 0; dc < 2; ++dc) {
                int jb = ib + db, jc = ic + dc;
                if (jb < 0 || jb >= g->n[b] || jc < 0 || jc >= g->n[c2]) continue;
                double wt = (db ? fb : 1.0 - fb) * (dc ? fc : 1.0 - fc);
                int p[3];
                p[a] = i; p[b] = jb; p[c2] = jc;
                long q = vidx(g, p);
                if (mode == 0) sum += w * wt * cvol[q];
                else vol[q] += w * wt * pval;
            }
        }
    }
    return sum;
}

/* ---- exported: geometry ---- */

void o_frame(const int *dims, const double *par, const double *ang, int k, double *out12)
{
    ogeom g = mk(dims, par, ang);
    frame(&g, k, out12, out12 + 3, out12 + 6, out12 + 9);
}

int o_principal_axis(const int *dims, const double *par, const double *ang, int k, int iu, int iv)
{
    ogeom g = mk(dims, par, ang);
    double S[3], D0S[3], EU[3], EV[3];
    frame(&g, k, S, D0S, EU, EV);
    return paxis32(D0S, EU, EV, iu, iv);
}

/* ---- exported: projector pair (P: Sec. 2.2; discretisation as described above) ---- */

/* proj[k][iv][iu] = (P vol); returns the number of samples in *nsamples. */
void o_forward(const int *dims, const double *par, const double *ang, const double *vol,
               double *proj, long *nsamples)
{
    ogeom g = mk(dims, par, ang);
    long nray = (long)g.na * g.nv * g.nu, total = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : total)
    for (long r = 0; r < nray; ++r) {
        int iu = (int)(r % g.nu), iv = (int)((r / g.nu) % g.nv), k = (int)(r / ((long)g.nu * g.nv));
        long ns = 0;
        proj[r] = walk(&g, NULL, vol, k, iu, iv, 0, 0.0, &ns);
        total += ns;
    }
    if (nsamples) *nsamples = total;
}

/* Selected rays only: out[j] = (P vol)[ray_ids[j]], ray id = (k*nv + iv)*nu + iu. */
void o_forward_rays(const int *dims, const double *par, const double *ang, const double *vol,
                    const long *ray_ids, long n, double *out)
{
    ogeom g = mk(dims, par, ang);
#pragma omp parallel for schedule(dynamic, 16)
    for (long j = 0; j < n; ++j) {
        long r = ray_ids[j];
        int iu = (int)(r % g.nu), iv = (int)((r / g.nu) % g.nv), k = (int)(r / ((long)g.nu * g.nv));
        out[j] = walk(&g, NULL, vol, k, iu, iv, 0, 0.0, NULL);
    }
}

/* vol = (P* proj), ray-driven scatter of the forward's weights. Each thread
 * scatters a block of angles into a private volume; the private volumes are
 * summed at the end. */
void o_adjoint(const int *dims, const double *par, const double *ang, const double *proj,
               double *vol)
{
    ogeom g = mk(dims, par, ang);
    long nvox = (long)g.n[0] * g.n[1] * g.n[2];
    memset(vol, 0, sizeof(double) * nvox);
#pragma omp parallel
    {
        double *priv = (double *)calloc(nvox, sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < g.na; ++k)
            for (int iv = 0; iv < g.nv; ++iv)
                for (int iu = 0; iu < g.nu; ++iu) {
                    double p = proj[((long)k * g.nv + iv) * g.nu + iu];
                    if (p != 0.0) walk(&g, priv, NULL, k, iu, iv, 1, p, NULL);
                }
#pragma omp critical
        for (long q = 0; q < nvox; ++q) vol[q] += priv[q];
        free(priv);
    }
}

/* Brute-force adjoint at selected voxels: for every ray of every angle, the ray's
 * sample on the voxel's own principal-axis plane contributes
 * w * (1 - |qb - vb|)(1 - |qc - vc|) * proj when both distances are below 1. */
void o_adjoint_voxels(const int *dims, const double *par, const double *ang, const double *proj,
                      const long *vox_ids, long n, double *out)
{
    ogeom g = mk(dims, par, ang);
#pragma omp parallel for schedule(dynamic, 1)
    for (long j = 0; j < n; ++j) {
        long q = vox_ids[j];
        int p[3] = {(int)(q % g.n[0]), (int)((q / g.n[0]) % g.n[1]), (int)(q / ((long)g.n[0] * g.n[1]))};
        double acc = 0.0;
        for (int k = 0; k < g.na; ++k) {
            double S[3], D0S[3], EU[3], EV[3], R[3];
            frame(&g, k, S, D0S, EU, EV);
            for (int iv = 0; iv < g.nv; ++iv)
                for (int iu = 0; iu < g.nu; ++iu) {
                    for (int c = 0; c < 3; ++c) R[c] = D0S[c] + iu * EU[c] + iv * EV[c];
                    int a = paxis32(D0S, EU, EV, iu, iv);
                    int b = (a == 0) ? 1 : 0, c2 = (a == 2) ? 1 : 2;
                    double t = (p[a] - S[a]) / R[a];
                    if (!(t > 0.0 && t < 1.0)) continue;
                    double db = fabs(S[b] + t * R[b] - p[b]);
                    double dc = fabs(S[c2] + t * R[c2] - p[c2]);
                    if (db >= 1.0 || dc >= 1.0) continue;
                    double len = sqrt(R[0] * g.vox[0] * R[0] * g.vox[0] + R[1] * g.vox[1] * R[1] * g.vox[1] +
                                      R[2] * g.vox[2] * R[2] * g.vox[2]);
                    acc += len / fabs(R[a]) * (1.0 - db) * (1.0 - dc) * proj[((long)k * g.nv + iv) * g.nu + iu];
                }
        }
        out[j] = acc;
    }
}

/* ---- exported: field-of-view tensor V (Sec. 2.6) ----
 * V[voxel] = (number of angles whose projection of the voxel centre falls on the
 * panel, i.e. continuous pixel coordinates in [-1/2, n - 1/2]) / n_angles. */
void o_fov(const int *dims, const double *par, const double *ang, double *V)
{
    ogeom g = mk(dims, par, ang);
    long nvox = (long)g.n[0] * g.n[1] * g.n[2];
#pragma omp parallel for schedule(static)
    for (long q = 0; q < nvox; ++q) {
        int ix = (int)(q % g.n[0]), iy = (int)((q / g.n[0]) % g.n[1]), iz = (int)(q / ((long)g.n[0] * g.n[1]));
        double P[3] = {(ix - 0.5 * (g.n[0] - 1)) * g.vox[0] + g.ctr[0],
                       (iy - 0.5 * (g.n[1] - 1)) * g.vox[1] + g.ctr[1],
                       (iz - 0.5 * (g.n[2] - 1)) * g.vox[2] + g.ctr[2]};
        int cnt = 0;
        for (int k = 0; k < g.na; ++k) {
            double th = angle_of(&g, k), c = cos(th), s = sin(th);
            double U = g.sid - (P[0] * c + P[1] * s);  /* depth along the central ray */
            if (!(U > 0.0)) continue;
            double m = g.sdd / U;
            double u = m * (-P[0] * s + P[1] * c), v = m * P[2];
            double fu = (u - g.uoff) / g.du + 0.5 * (g.nu - 1);
            double fv = (v - g.voff) / g.dv + 0.5 * (g.nv - 1);
            if (fu >= -0.5 && fu <= g.nu - 0.5 && fv >= -0.5 && fv <= g.nv - 0.5) cnt++;
        }
        V[q] = (double)cnt / g.na;
    }
}

/* ---- exported: offset-detector redundancy weight w (Sec. 2.6) ----
 * u' = (iu - (nu-1)/2) du + u_offset is the signed distance of the pixel column
 * from the central ray. Overlap half-width D = nu du / 2 - |u_offset|. For a
 * positive offset w = 0 below -D, sin^2(pi/4 (u' + D)/D) on [-D, D], 1 above D
 * (mirrored for a negative offset), so that w(u') + w(-u') = 1. A centred panel
 * measures every line twice over a full orbit: w = 1/2. */
void o_redundancy(const int *dims, const double *par, double *w)
{
    ogeom g = mk(dims, par, NULL);
    double D = 0.5 * g.nu * g.du - fabs(g.uoff);
    for (int iu = 0; iu < g.nu; ++iu) {
        double u = (iu - 0.5 * (g.nu - 1)) * g.du + g.uoff;
        if (g.uoff == 0.0) { w[iu] = 0.5; continue; }
        double us = g.uoff > 0 ? u : -u;
        double val;
        if (us < -D) val = 0.0;
        else if (us > D) val = 1.0;
        else { double sv = sin(0.25 * M_PI * (us + D) / D); val = sv * sv; }
        w[iu] = val;
    }
}

/* ---- exported: FDK with redundancy weighting (Feldkamp 1984; Sec. 2.6 FDK_w) ----
 * 1. q0 = proj * w(u') * sdd / sqrt(sdd^2 + u'^2 + v'^2)      (redundancy, cosine)
 * 2. q  = tau * sum_m h(e - m) q0[m] along each detector row, with the Ram-Lak
 *    kernel at the isocentre pitch tau = du sid/sdd: h(0) = 1/(4 tau^2),
 *    h(odd j) = -1/(pi^2 j^2 tau^2), h(even j != 0) = 0.
 *    For an offset panel the row is extended on its short side by
 *    npad = ceil(2 |u_offset| / du) columns of zero weighted data (w = 0 there), so
 *    that the filtered row is also known at the mirror image of the long side:
 *    voxels seen by one side of the panel only need it.
 * 3. vol(P) = sum_k (2 pi / n_angles) (sid/U)^2 q_k(u(P), v(P)), U the depth of P
 *    along the central ray, (u, v) its projection, bilinear on the (extended)
 *    row grid, zero off it. */
int o_fdk_pad(const int *dims, const double *par)
{
    ogeom g = mk(dims, par, NULL);
    return (int)ceil(2.0 * fabs(g.uoff) / g.du - 1e-9);
}

void o_fdk(const int *dims, const double *par, const double *ang, const double *proj, double *vol)
{
    ogeom g = mk(dims, par, ang);
    int npad = o_fdk_pad(dims, par);
    int nue = g.nu + npad;
    int lo = g.uoff > 0 ? npad : 0;   /* extended column of detector column 0 */
    long nq = (long)nue * g.nv * g.na;
    double *q = (double *)malloc(sizeof(double) * nq);
    double *w = (double *)malloc(sizeof(double) * g.nu);
    o_redundancy(dims, par, w);
    double tau = g.du * g.sid / g.sdd;
#pragma omp parallel for schedule(static)
    for (long row = 0; row < (long)g.na * g.nv; ++row) {
        int iv = (int)(row % g.nv);
        double v = (iv - 0.5 * (g.nv - 1)) * g.dv + g.voff;
        double *q0 = (double *)calloc(nue, sizeof(double));
        for (int iu = 0; iu < g.nu; ++iu) {
            double u = (iu - 0.5 * (g.nu - 1)) * g.du + g.uoff;
            q0[lo + iu] = proj[row * g.nu + iu] * w[iu] * g.sdd / sqrt(g.sdd * g.sdd + u * u + v * v);
        }
        for (int e = 0; e < nue; ++e) {
            double acc = 0.0;
            for (int m = 0; m < nue; ++m) {
                int j = e - m;
                double h;
                if (j == 0) h = 1.0 / (4.0 * tau * tau);
                else if (j % 2 != 0) h = -1.0 / (M_PI * M_PI * (double)j * j * tau * tau);
                else h = 0.0;
                acc += h * q0[m];
            }
            q[row * nue + e] = tau * acc;
        }
        free(q0);
    }
    long nvox = (long)g.n[0] * g.n[1] * g.n[2];
#pragma omp parallel for schedule(static)
    for (long p = 0; p < nvox; ++p) {
        int ix = (int)(p % g.n[0]), iy = (int)((p / g.n[0]) % g.n[1]), iz = (int)(p / ((long)g.n[0] * g.n[1]));
        double P[3] = {(ix - 0.5 * (g.n[0] - 1)) * g.vox[0] + g.ctr[0],
                       (iy - 0.5 * (g.n[1] - 1)) * g.vox[1] + g.ctr[1],
                       (iz - 0.5 * (g.n[2] - 1)) * g.vox[2] + g.ctr[2]};
        double acc = 0.0;
        for (int k = 0; k < g.na; ++k) {
            double th = angle_of(&g, k), c = cos(th), s = sin(th);
            double U = g.sid - (P[0] * c + P[1] * s);
            if (!(U > 0.0)) continue;
            double m = g.sdd / U;
            double fu = (m * (-P[0] * s + P[1] * c) - g.uoff) / g.du + 0.5 * (g.nu - 1) + lo;
            double fv = (m * P[2] - g.voff) / g.dv + 0.5 * (g.nv - 1);
            double u0 = floor(fu), v0 = floor(fv);
            double au = fu - u0, av = fv - v0;
            double val = 0.0;
            for (int du_ = 0; du_ < 2; ++du_)
                for (int dv_ = 0; dv_ < 2; ++dv_) {
                    int ju = (int)u0 + du_, jv = (int)v0 + dv_;
                    if (ju < 0 || ju >= nue || jv < 0 || jv >= g.nv) continue;
                    val += (du_ ? au : 1.0 - au) * (dv_ ? av : 1.0 - av) * q[((long)k * g.nv + jv) * nue + ju];
                }
            acc += (g.sid / U) * (g.sid / U) * val;
        }
        vol[p] = acc * 2.0 * M_PI / g.na;
    }
    free(q);
    free(w);
}

/* ---- exported: TV pieces and PDHG (Chambolle-Pock 2011; Sec. 2.5 baseline) ----
 * grad: forward differences in voxel units, zero on the last index (Neumann).
 * div = -grad^T. */
void o_grad(const int *n, const double *x, double *g3)
{
    long nx = n[0], ny = n[1], nz = n[2], N = nx * ny * nz;
    for (long iz = 0; iz < nz; ++iz)
        for (long iy = 0; iy < ny; ++iy)
            for (long ix = 0; ix < nx; ++ix) {
                long p = (iz * ny + iy) * nx + ix;
                g3[p] = ix < nx - 1 ? x[p + 1] - x[p] : 0.0;
                g3[N + p] = iy < ny - 1 ? x[p + nx] - x[p] : 0.0;
                g3[2 * N + p] = iz < nz - 1 ? x[p + nx * ny] - x[p] : 0.0;
            }
}

void o_div(const int *n, const double *g3, double *d)
{
    long nx = n[0], ny = n[1], nz = n[2], N = nx * ny * nz;
    for (long iz = 0; iz < nz; ++iz)
        for (long iy = 0; iy < ny; ++iy)
            for (long ix = 0; ix < nx; ++ix) {
                long p = (iz * ny + iy) * nx + ix;
                double v = 0.0;
                v += (ix < nx - 1 ? g3[p] : 0.0) - (ix > 0 ? g3[p - 1] : 0.0);
                v += (iy < ny - 1 ? g3[N + p] : 0.0) - (iy > 0 ? g3[N + p - nx] : 0.0);
                v += (iz < nz - 1 ? g3[2 * N + p] : 0.0) - (iz > 0 ? g3[2 * N + p - nx * ny] : 0.0);
                d[p] = v;
            }
}

/* min_x 1/2 ||P x - y||^2 + lam ||grad x||_{2,1}  s.t. x >= 0, solved as
 * Chambolle-Pock on K = [P; gamma grad] with F2(g) = (lam/gamma) ||g||_{2,1}
 * (the same problem; gamma balances the two blocks of K):
 *   z1 <- (z1 + sigma (P xbar - y)) / (1 + sigma)
 *   z2 <- project_{|.| <= lam/gamma}(z2 + sigma gamma grad xbar)   (per voxel)
 *   x+ <- max(0, x - tau (P* z1 - gamma div z2));  xbar <- 2 x+ - x;  x <- x+ */
void o_pdhg(const int *dims, const double *par, const double *ang, const double *y,
            const double *x0, int niter, double lam, double gamma, double sigma, double tau, double *x)
{
    ogeom g = mk(dims, par, ang);
    long N = (long)g.n[0] * g.n[1] * g.n[2], M = (long)g.na * g.nv * g.nu;
    double *xb = (double *)malloc(sizeof(double) * N), *z1 = (double *)calloc(M, sizeof(double));
    double *z2 = (double *)calloc(3 * N, sizeof(double)), *px = (double *)malloc(sizeof(double) * M);
    double *g3 = (double *)malloc(sizeof(double) * 3 * N), *bt = (double *)malloc(sizeof(double) * N);
    double *dv = (double *)malloc(sizeof(double) * N);
    double rad = lam / gamma;
    memcpy(x, x0, sizeof(double) * N);
    memcpy(xb, x0, sizeof(double) * N);
    for (int it = 0; it < niter; ++it) {
        o_forward(dims, par, ang, xb, px, NULL);
        for (long r = 0; r < M; ++r) z1[r] = (z1[r] + sigma * (px[r] - y[r])) / (1.0 + sigma);
        o_grad(g.n, xb, g3);
        for (long p = 0; p < N; ++p) {
            double a0 = z2[p] + sigma * gamma * g3[p], a1 = z2[N + p] + sigma * gamma * g3[N + p];
            double a2 = z2[2 * N + p] + sigma * gamma * g3[2 * N + p];
            double nrm = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
            double sc = nrm > rad ? rad / nrm : 1.0;
            z2[p] = a0 * sc; z2[N + p] = a1 * sc; z2[2 * N + p] = a2 * sc;
        }
        o_adjoint(dims, par, ang, z1, bt);
        o_div(g.n, z2, dv);
        for (long p = 0; p < N; ++p) {
            double xn = x[p] - tau * (bt[p] - gamma * dv[p]);
            if (xn < 0.0) xn = 0.0;
            xb[p] = 2.0 * xn - x[p];
            x[p] = xn;
        }
    }
    free(xb); free(z1); free(z2); free(px); free(g3); free(bt); free(dv);
}

/* ---- exported: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ----
 * Ten rounds of: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (32x32 -> 64-bit),
 * c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by the Weyl
 * constants (W0, W1) before every round after the first. */
void o_philox(const uint32_t *ctr_in, const uint32_t *key_in, uint32_t *out)
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* Uniform variate strictly inside (0, 1) from a 32-bit word. */
static double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* One Poisson(lam) draw for element e. Random words come from Philox4x32-10 with
 * key (seed lo, seed hi) and counter (e lo, e hi, block j, 0x50303031), blocks
 * j = 0, 1, ... consumed in order, two words per attempt.
 *  lam < 10: inversion by sequential search on the first word.
 *  lam >= 10: PTRS (Hoermann 1993): U = u - 1/2, us = 1/2 - |U|,
 *   k = floor((2a/us + b) U + lam + 0.43); quick accept if us >= 0.07 and V <= v_r;
 *   reject if k < 0 or (us < 0.013 and V > us); else accept iff
 *   log(V inv_alpha / (a/us^2 + b)) <= -lam + k log(lam) - lgamma(k + 1),
 *   with b = 0.931 + 2.53 sqrt(lam), a = -0.059 + 0.02483 b,
 *   inv_alpha = 1.1239 + 1.1328/(b - 3.4), v_r = 0.9277 - 3.6224/(b - 2). */
static int32_t poisson_one(double lam, uint64_t e, uint64_t seed)
{
    if (!(lam > 0.0)) return 0;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)e, (uint32_t)(e >> 32), 0u, 0x50303031u};
    uint32_t r[4];
    if (lam < 10.0) {
        o_philox(ctr, key, r);
        double u = u01(r[0]);
        double p = exp(-lam), F = p;
        int32_t k = 0;
        while (u > F && k < 1000) { k++; p *= lam / k; F += p; }
        return k;
    }
    double slam = sqrt(lam), loglam = log(lam);
    double b = 0.931 + 2.53 * slam;
    double a = -0.059 + 0.02483 * b;
    double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
    double vr = 0.9277 - 3.6224 / (b - 2.0);
    for (uint32_t j = 0; j < 4096u; ++j) {
        ctr[2] = j;
        o_philox(ctr, key, r);
        for (int h = 0; h < 2; ++h) {
            double U = u01(r[2 * h]) - 0.5, V = u01(r[2 * h + 1]);
            double us = 0.5 - fabs(U);
            double kf = floor((2.0 * a / us + b) * U + lam + 0.43);
            if (us >= 0.07 && V <= vr) return (int32_t)kf;
            if (kf < 0.0 || (us < 0.013 && V > us)) continue;
            if (log(V * inv_alpha / (a / (us * us) + b)) <= -lam + kf * loglam - lgamma(kf + 1.0))
                return (int32_t)kf;
        }
    }
    return (int32_t)floor(lam + 0.5);
}

/* counts[e] ~ Poisson(I0 exp(-p[e])), the monochromatic primary model (Sec. 2.2). */
void o_poisson(const float *p, long n, double I0, uint64_t seed, int32_t *counts)
{
#pragma omp parallel for schedule(static)
    for (long e = 0; e < n; ++e) counts[e] = poisson_one(I0 * exp(-(double)p[e]), (uint64_t)e, seed);
}

void o_poisson_lam(const double *lam, long n, uint64_t seed, int32_t *counts)
{
#pragma omp parallel for schedule(static)
    for (long e = 0; e < n; ++e) counts[e] = poisson_one(lam[e], (uint64_t)e, seed);
}

/* y = -log(min(max(N, 1) / I0, 1)): the normalised log transform (Sec. 2.4), with
 * zero counts clamped to one so the logarithm stays finite. */
void o_neglog(const int32_t *counts, long n, double I0, double *y)
{
    for (long e = 0; e < n; ++e) {
        double c = counts[e] < 1 ? 1.0 : (double)counts[e];
        double r = c / I0;
        y[e] = -log(r < 1.0 ? r : 1.0);
    }
}

/* ---- exported: ellipsoid phantom ----
 * ell rows (17 doubles): centre (3, mm), semi-axes (3, mm), rotation R (9,
 * row-major, rows are the ellipsoid's axes in world coordinates), value, mode.
 * A point P is inside when sum_i ((R (P - c))_i / a_i)^2 <= 1; mode 0 adds the
 * value there, mode 1 overwrites. With ss > 1 each voxel is the mean over an
 * ss^3 grid of sub-points at offsets ((j + 1/2)/ss - 1/2) vox. */
void o_phantom(const int *dims, const double *par, const double *ell, int nell, int ss, double *vol)
{
    ogeom g = mk(dims, par, NULL);
    long nvox = (long)g.n[0] * g.n[1] * g.n[2];
#pragma omp parallel for schedule(static)
    for (long q = 0; q < nvox; ++q) {
        int ix = (int)(q % g.n[0]), iy = (int)((q / g.n[0]) % g.n[1]), iz = (int)(q / ((long)g.n[0] * g.n[1]));
        double acc = 0.0;
        for (int sz = 0; sz < ss; ++sz)
            for (int sy = 0; sy < ss; ++sy)
                for (int sx = 0; sx < ss; ++sx) {
                    double P[3] = {(ix - 0.5 * (g.n[0] - 1) + (sx + 0.5) / ss - 0.5) * g.vox[0] + g.ctr[0],
                                   (iy - 0.5 * (g.n[1] - 1) + (sy + 0.5) / ss - 0.5) * g.vox[1] + g.ctr[1],
                                   (iz - 0.5 * (g.n[2] - 1) + (sz + 0.5) / ss - 0.5) * g.vox[2] + g.ctr[2]};
                    double val = 0.0;
                    for (int e = 0; e < nell; ++e) {
                        const double *E = ell + 17 * e;
                        double d[3] = {P[0] - E[0], P[1] - E[1], P[2] - E[2]};
                        double r = 0.0;
                        for (int i = 0; i < 3; ++i) {
                            double l = E[6 + 3 * i] * d[0] + E[7 + 3 * i] * d[1] + E[8 + 3 * i] * d[2];
                            r += (l / E[3 + i]) * (l / E[3 + i]);
                        }
                        if (r <= 1.0) val = (E[16] != 0.0) ? E[15] : val + E[15];
                    }
                    acc += val;
                }
        vol[q] = acc / ((double)ss * ss * ss);
    }
}

int o_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- polychromatic primary simulation (Sec. 2.1, "Primary simulation") ----
 *
 * Water-bone decomposition (the paper adopts Wang et al. 2018): HU values become
 * modified CT numbers rho_hat = 0.001 HU + 1, and with tau1 = 1.2, tau2 = 1.6,
 * kappa_b = 0.409
 *   rho_w = 0 (rho_hat < tau0), rho_hat (tau0 <= rho_hat < tau1),
 *           tau1 (tau2 - rho_hat) / (tau2 - tau1) (tau1 <= rho_hat < tau2), 0 above;
 *   rho_b = 0 (rho_hat < tau1), kappa_b tau2 (rho_hat - tau1) / (tau2 - tau1)
 *           (tau1 <= rho_hat < tau2), kappa_b rho_hat above.
 * The CT scan is mu = mu_tot,60 in 1/mm, so HU = 1000 (mu - mu_w60) / mu_w60 with
 * mu_w60 the attenuation of water at 60 keV. The paper does not state tau0; it
 * calls both densities continuous functions of rho_hat, and rho_w is continuous at
 * tau0 only for tau0 = 0, which is the reading taken here. */
void o_water_bone(const double *mu, long n, double mu_w60, double *rho_w, double *rho_b)
{
    const double tau0 = 0.0, tau1 = 1.2, tau2 = 1.6, kappa_b = 0.409;
    for (long i = 0; i < n; ++i) {
        double hu = 1000.0 * (mu[i] - mu_w60) / mu_w60;
        double r = 0.001 * hu + 1.0;
        double w, b;
        if (r < tau0) w = 0.0;
        else if (r < tau1) w = r;
        else if (r < tau2) w = tau1 * (tau2 - r) / (tau2 - tau1);
        else w = 0.0;
        if (r < tau1) b = 0.0;
        else if (r < tau2) b = kappa_b * tau2 * (r - tau1) / (tau2 - tau1);
        else b = kappa_b * r;
        rho_w[i] = w;
        rho_b[i] = b;
    }
}

/* Detector response resp(e), e in keV: linear between the key points
 * (20, 5), (60, 20) and (120, 10) (Sec. 2.1, after Poludniowski 2009); held at the
 * end values outside [20, 120] (the paper's bins 25 ... 115 keV lie inside). */
double o_resp(double e)
{
    if (e <= 20.0) return 5.0;
    if (e <= 60.0) return 5.0 + (e - 20.0) * (20.0 - 5.0) / (60.0 - 20.0);
    if (e <= 120.0) return 20.0 + (e - 60.0) * (10.0 - 20.0) / (120.0 - 60.0);
    return 10.0;
}

/* Mean photon counts of each energy bin from water and bone line integrals:
 * lam[i ne + j] = I0[j][i mod npix] exp(-(mu_w[j] Lw[i] + mu_b[j] Lb[i])), which is
 * I0 exp(-P(mu_tilde_e)) of the primary model with P(rho_w mu_w + rho_b mu_b) =
 * mu_w P(rho_w) + mu_b P(rho_b) (P is linear). Element i runs over [n_angles][nv][nu]
 * (times the batch); npix = nv nu. */
void o_poly_lam(const float *Lw, const float *Lb, long n, long npix, int ne, const double *mu_w,
                const double *mu_b, const float *I0, double *lam)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i)
        for (int j = 0; j < ne; ++j) {
            double a = mu_w[j] * (double)Lw[i] + mu_b[j] * (double)Lb[i];
            lam[i * ne + j] = (double)I0[(long)j * npix + i % npix] * exp(-a);
        }
}

/* Polychromatic primary reading (Sec. 2.1, primary-model equation):
 * reading[i] = sum over bins j (in order) of resp(E_j) Poisson(lam[i ne + j]), the
 * draw of bin j taken from the Philox counter of element i ne + j (the same
 * sampler as o_poisson). With noise = 0 the mean lam replaces the draw (the
 * expected reading). counts (may be NULL) receives the draws, [n][ne]. */
void o_poly_reading(const double *lam, long n, int ne, const double *energies, uint64_t seed, int noise,
                    double *reading, int32_t *counts)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < ne; ++j) {
            double v;
            if (noise) {
                int32_t c = poisson_one(lam[i * ne + j], (uint64_t)(i * ne + j), seed);
                if (counts) counts[i * ne + j] = c;
                v = (double)c;
            } else {
                v = lam[i * ne + j];
            }
            acc += o_resp(energies[j]) * v;
        }
        reading[i] = acc;
    }
}
