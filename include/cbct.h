/*
 * cbct.h — C ABI of the GB300 (sm_103a) cone-beam CT library.
 *
 * The library computes the discretised cone-beam transform P and its exact
 * adjoint P* (paper: "Equivariant Multiscale Learned Invertible Reconstruction
 * for Cone Beam CT", arXiv 2512.21180, Sec. 2.2, projection-operator equation:
 * P(mu)(t,u) is the integral of mu along the line from the source to detector
 * element u at time t, and P* is its adjoint, the backprojection), the
 * field-of-view tensor V and redundancy weight w used by the reconstruction
 * (Sec. 2.6), FDK with redundancy weighting, PDHG-TV (Sec. 2.5 baselines), the
 * primary-signal simulation (Sec. 2.2 primary model with Poisson noise, Sec. 2.4
 * log normalisation; monochromatic, and polychromatic with the water-bone split of
 * Sec. 2.1) and the learned primal-dual reconstruction (Sec. 2.6,
 * Algorithm 1).
 *
 * Conventions for every call
 *  - Pointers named vol/proj/... are DEVICE pointers on the device that was current
 *    when the geometry was created; the caller owns them. They must be contiguous
 *    and 16-byte aligned, in these layouts (fastest index last):
 *        volume      [batch][nz][ny][nx]       (x fastest)
 *        projection  [batch][n_angles][nv][nu] (u fastest)
 *  - The library owns geometry tables, weights and workspaces behind opaque
 *    handles. Scratch memory is taken from the CUDA stream-ordered pool on the
 *    caller's stream (cudaMallocAsync) and returned on the same stream.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; 0 = legacy default) and
 *    never synchronise the device.
 *  - Return value: 0 on success, negative on error; cbct_last_error() returns a
 *    thread-local message for the last failing call on this thread.
 *        CBCT_EINVAL  -1  invalid argument (nothing was launched)
 *        CBCT_ECUDA   -2  CUDA runtime error (launch or allocation)
 *        CBCT_ENOMEM  -3  out of device memory
 *        CBCT_EDEVICE -4  reserved: kernels report a bounded wait that gave up through
 *                         a device status word the caller reads (cbct_device_status,
 *                         lpd_device_status, the status argument of cbct_conv and
 *                         cbct_conv_wgrad), not through a return code
 *
 * Geometry (the paper's scanner, Sec. 2.2: circular orbit, offset flat panel):
 * isocentre at the origin, rotation axis z. At angle theta the source sits at
 * sid (cos theta, sin theta, 0), the panel centre at sid - sdd along that
 * direction, the panel axes are e_u = (-sin theta, cos theta, 0) (the direction
 * of rotation) and e_v = z. Pixel (iu, iv) is at ((iu - (nu-1)/2) du + u_offset)
 * e_u + ((iv - (nv-1)/2) dv + v_offset) e_v from the panel centre; voxel
 * (ix, iy, iz) is centred at ((ix - (nx-1)/2) vox_x + center_x, ...). A positive
 * u_offset moves the panel in the direction of rotation.
 *
 * Discretisation (the paper defines only the continuous P): Joseph-style ray
 * sums. For the ray from the source to a pixel centre the principal axis a is x
 * if |r_x| >= |r_y| else y, decided on the FP32 ray direction
 * r = fmaf(iv, EV, fmaf(iu, EU, D0S)) of the FP32 geometry table; every
 * voxel-centre plane i of axis a between source and pixel contributes
 * (step length) x (bilinear interpolation of the volume on that plane, zero
 * outside the grid). Rays whose principal axis would be z are not supported and
 * such geometries are rejected at creation.
 */
#ifndef CBCT_H
#define CBCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CBCT_EINVAL (-1)
#define CBCT_ECUDA (-2)
#define CBCT_ENOMEM (-3)
#define CBCT_EDEVICE (-4)

typedef struct cbct_geom cbct_geom; /* opaque: geometry tables on one device */

typedef struct {
    int nx, ny, nz;          /* volume grid */
    double vox[3];           /* voxel pitch, mm */
    double center[3];        /* volume centre relative to the isocentre, mm */
    int nu, nv;              /* panel columns (along e_u) and rows (along z) */
    double du, dv;           /* pixel pitch, mm */
    double u_offset, v_offset; /* panel offset, mm; +u = direction of rotation */
    double sid, sdd;         /* source-isocentre and source-detector distances, mm */
    int n_angles;            /* projections over the orbit */
    const double *angles;    /* host array of n_angles radians, or NULL for 2 pi k / n_angles */
    int normalize;           /* 1: scale P and P* by 1/||P|| (Sec. 2.6, "normalized
                                operators"); ||P|| from 30 FP64-accumulated power
                                iterations at creation. 0: unscaled. */
} cbct_geom_desc;

/* Last error message of this thread (static storage, never NULL). */
const char *cbct_last_error(void);

/* Build the per-angle ray tables on the current device (a1). The descriptor and
 * its angle array are copied. Synchronises the current device once (table
 * upload; with normalize = 1 also the power iteration). Errors: CBCT_EINVAL for
 * non-positive sizes/pitches/distances, sizes whose index products exceed 2^31,
 * or a geometry with z-principal rays; CBCT_ECUDA/ENOMEM on CUDA failures. */
int geometry_create(const cbct_geom_desc *desc, cbct_geom **out);

/* Free the device tables (synchronises with the device). NULL is a no-op. */
void geometry_destroy(cbct_geom *g);

/* Operator scale applied by forward_project/back_project (1/||P|| when the
 * geometry was created with normalize = 1, else 1). */
double geometry_scale(const cbct_geom *g);

/* Read (and with clear = 1 reset) the geometry's device status word: 0 = ok,
 * 1 = a kernel gave up waiting on a shared-memory barrier (it then left its
 * outputs unwritten). Synchronises the device. */
int cbct_device_status(const cbct_geom *g, int *out, int clear);

/* Staged-forward configuration chosen for this geometry: *cfg = index of the
 * shared-memory box (0..3) or -1 for the direct kernel; *need_b / *need_z = host
 * bounds of a 32 x 8 ray tile's footprint over 8 planes (voxels). Any pointer may
 * be NULL. */
int cbct_forward_config(const cbct_geom *g, int *cfg, double *need_b, double *need_z);

/* Forward projection (a2, Sec. 2.2): proj[b] (+)= P vol[b] for b < batch.
 * accumulate = 0 overwrites proj, 1 adds to it. FP32 in, FP32 accumulation.
 * batch >= 1; batch * n_angles <= 65535. Scratch: two plane-major copies of the
 * volumes (2 * batch * nx * ny * nz floats, rows padded to 4), from the
 * stream-ordered pool. Errors: CBCT_EINVAL (before any launch) for a NULL pointer,
 * batch < 1, accumulate not 0 or 1, batch * n_angles > 65535 or a current device
 * other than the geometry's; CBCT_ENOMEM when the scratch cannot be allocated;
 * CBCT_ECUDA for a failed launch. */
int forward_project(const cbct_geom *g, const float *vol, float *proj, int batch, int accumulate,
                    void *stream);

/* Backprojection (a3, Sec. 2.2): vol[b] (+)= P* proj[b], the exact transpose of
 * forward_project (same rays, planes and bilinear weights), computed as an
 * atomic-free voxel-driven gather. Scratch: batch * n_angles * nv * nu floats
 * (the ray-weighted projections, plus up to 16 partial volumes when small volumes
 * split the angles), from the stream-ordered pool. The split follows the size of the
 * grid (volume and batch), so a volume's result in a batch can differ from its
 * single-volume result by FP32 summation order; a given geometry and batch size
 * always give the same bits. Errors: as forward_project, and
 * CBCT_EINVAL when batch * ceil(nz / 4) exceeds 65535 (a grid dimension limit). */
int back_project(const cbct_geom *g, const float *proj, float *vol, int batch, int accumulate,
                 void *stream);

/* FP64 instantiations of the same operators (tests and finite-difference checks;
 * the principal-axis decision stays the FP32 one). Same arguments, layouts and
 * errors as the FP32 calls, with double buffers. */
int forward_project_f64(const cbct_geom *g, const double *vol, double *proj, int batch,
                        int accumulate, void *stream);
int back_project_f64(const cbct_geom *g, const double *proj, double *vol, int batch,
                     int accumulate, void *stream);

/* back_project without any device allocation (the paper has no counterpart; this
 * serves callers that cannot allocate device memory during the call, e.g. a host
 * framework that owns the whole device memory budget through its own allocator,
 * or a latency-critical loop that must not enter the CUDA allocator). Same
 * arguments and result as back_project, up to FP32 summation order. Its scratch
 * is a fixed 8 Mi-float (32 MiB) device array inside the library, placed on a GPU
 * when geometry_create first runs there (it looks up the array's device address with
 * cudaGetSymbolAddress, which loads the library's projector module on that device)
 * and held until the process exits; this call itself neither allocates nor loads
 * anything. The angles are processed in chunks that fit the array. Limit: nu * nv <=
 * 8388608 (one projection must fit), else CBCT_EINVAL before any launch. All calls
 * share the one array: calls whose executions overlap on the GPU (different streams,
 * or different host threads) race and give wrong results. Nothing in the array needs
 * to start at zero. */
int back_project_noalloc(const cbct_geom *g, const float *proj, float *vol, int batch, int accumulate,
                         void *stream);

/* Number of samples of one forward projection: (ray, plane) pairs with the
 * source-to-pixel parameter in (0, 1) and the in-plane point inside the
 * (-1, n) x (-1, n) extended grid. The throughput unit. Writes one int64 to the
 * host pointer *out; synchronises `stream`. */
int cbct_count_samples(const cbct_geom *g, long long *out, void *stream);


/* ---- simulation and per-geometry tensors (a5, a6) ---- */

/* Ellipsoid phantom on the geometry's voxel grid. ell_host: n_ell rows of 17
 * doubles in host memory: centre (3, mm), semi-axes (3, mm), rotation (9,
 * row-major; rows are the ellipsoid axes in world coordinates), value (1/mm),
 * mode (0: add the value inside, 1: overwrite with it). Rows apply in order. A
 * point P is inside when sum_i ((R (P - c))_i / a_i)^2 <= 1 (FP64). With
 * supersample = s in [1, 8] each voxel is the mean over s^3 sub-points at offsets
 * ((j + 1/2)/s - 1/2) vox. Writes one volume [nz][ny][nx]. Synchronises `stream`
 * before returning (the host rows may be reused at once). Stand-in for the
 * paper's CT volumes (Sec. 2.4). */
int cbct_phantom(const cbct_geom *g, const double *ell_host, int n_ell, int supersample, float *vol,
                 void *stream);

/* Photon counts (Sec. 2.2, primary model, one energy): counts[e] ~
 * Poisson(I0 exp(-line_integrals[e])) for e < n, device arrays. Random words come
 * from Philox4x32-10 (Salmon et al., SC'11) with key (seed lo, seed hi) and counter
 * (e lo, e hi, block, 0x50303031); means below 10 are sampled by inversion, others
 * by Hoermann's PTRS (1993); decisions in FP64. Deterministic for a given seed. */
int cbct_poisson(const float *line_integrals, long long n, double I0, unsigned long long seed, int32_t *counts,
                 void *stream);

/* Normalised log transform (Sec. 2.4): y[e] = -log(min(max(counts[e], 1) / I0, 1)). */
int cbct_neglog(const int32_t *counts, long long n, double I0, float *y, void *stream);

/* Simulated measurement of `batch` volumes: line_integrals = P vol (forward_project),
 * then y = -log(min(max(N, 1)/I0, 1)) with N ~ Poisson(I0 exp(-line_integrals)),
 * the counter e running over the whole [batch][n_angles][nv][nu] array. */
int cbct_simulate(const cbct_geom *g, const float *vol, int batch, double I0, unsigned long long seed,
                  float *line_integrals, float *y, void *stream);

/* ---- polychromatic primary (Sec. 2.1, "Primary simulation", primary-model
 * equation; Sec. 2.4, normalised primary data) ----
 * The paper's primary model is a sum over energy bins e (ten 10 keV bins centred at
 * 25 ... 115 keV) of resp(e) Poisson(I0_e exp(-P(mu_w(e) rho_w + mu_b(e) rho_b))),
 * with rho_w, rho_b the water and bone relative densities of the CT scan and
 * mu_w(e), mu_b(e) the attenuation of water and bone at e. P is linear, so the
 * library projects rho_w and rho_b once each and forms every bin's exponent as
 * mu_w(e) P(rho_w) + mu_b(e) P(rho_b): two projections per volume for any number
 * of bins. The attenuation tables (the paper takes them from xraylib) and the
 * per-pixel intensity maps I0_e (from the paper's phase file) are inputs. At most
 * 16 bins. */

/* Detector response resp(e) for n_e energies in keV (host arrays): linear between
 * (20 keV, 5), (60 keV, 20) and (120 keV, 10), constant outside [20, 120]
 * (Sec. 2.1, after Poludniowski 2009). Host only; launches nothing. */
int cbct_detector_response(const double *energies_kev, int n_e, double *resp);

/* Water-bone decomposition (Sec. 2.1, after Wang et al. 2018) of `batch` volumes
 * mu[batch][n_vox] of mu_tot,60 (1/mm) into rho[batch][2][n_vox] (water, then bone,
 * relative densities): rho_hat = 0.001 HU + 1 = mu / mu_water60; with tau1 = 1.2,
 * tau2 = 1.6, kappa_b = 0.409, rho_w = rho_hat on [0, tau1), tau1 (tau2 - rho_hat) /
 * (tau2 - tau1) on [tau1, tau2), 0 elsewhere; rho_b = 0 below tau1, kappa_b tau2
 * (rho_hat - tau1) / (tau2 - tau1) on [tau1, tau2), kappa_b rho_hat above. The paper
 * leaves tau0 unstated; 0 makes rho_w continuous, as the paper says it is. FP32. */
int cbct_water_bone(const float *mu, long long n_vox, int batch, double mu_water60, float *rho, void *stream);

/* Polychromatic reading from line integrals. line_integrals[batch][2][n_per_item]
 * (water P(rho_w), then bone P(rho_b); n_per_item = n_angles nv nu), I0[n_e][npix]
 * (device, npix = nv nu, the same map for every angle), energies_kev, mu_water,
 * mu_bone: host arrays of n_e entries (1/mm). Per element e (over all items):
 * lam_j = I0[j][pixel] exp(-(mu_water[j] L_w + mu_bone[j] L_b)); N_j ~ Poisson(lam_j)
 * drawn as in cbct_poisson on the counter of element e n_e + j (lam_j itself when
 * noise is 0); reading[e] = sum_j resp_j N_j (bins in order, FP64, rounded once);
 * y[e] = -log(min(max(reading, r_min) / air, 1)) with the expected air reading
 * air = sum_j resp_j I0[j][pixel] (the paper's normalisation by an air scan, here
 * noise-free) and r_min = min_j resp_j (a reading of no photons counts as one photon
 * of the least responsive bin, so y stays finite, as cbct_neglog clamps counts to 1).
 * Any of reading, y, counts ([n][n_e] draws; needs noise) may be NULL, not all. */
int cbct_poly_reading(const float *line_integrals, int batch, long long n_per_item, int npix, int n_e,
                      const double *energies_kev, const double *mu_water, const double *mu_bone,
                      const float *I0, unsigned long long seed, int noise, float *reading, float *y,
                      int32_t *counts, void *stream);

/* Polychromatic simulated measurement of `batch` mu_60 volumes (Sec. 2.1 and 2.4):
 * cbct_water_bone, one forward projection of the 2 batch density volumes into
 * line_integrals[batch][2][n_angles][nv][nu] (output), then y[batch][n_angles][nv][nu]
 * as in cbct_poly_reading. Scratch for the densities (8 bytes per voxel) comes from
 * the stream-ordered pool. */
int cbct_poly_simulate(const cbct_geom *g, const float *mu, int batch, double mu_water60, int n_e,
                       const double *energies_kev, const double *mu_water, const double *mu_bone,
                       const float *I0, unsigned long long seed, int noise, float *line_integrals, float *y,
                       void *stream);

/* Offset-detector redundancy weight w[nu] (device), Sec. 2.6 (the paper names no
 * scheme; this is Wang's): u' = (iu - (nu-1)/2) du + u_offset, D = nu du/2 -
 * |u_offset|; for u_offset > 0 w = 0 below -D, sin^2(pi/4 (u' + D)/D) on [-D, D],
 * 1 above D (mirrored for u_offset < 0); w = 1/2 for a centred panel, so that
 * conjugate rays sum to one. */
int cbct_redundancy_weight(const cbct_geom *g, float *w, void *stream);

/* Field-of-view tensor V[nz][ny][nx] (device), Sec. 2.6: the fraction of angles at
 * which the voxel centre projects onto the panel (continuous pixel coordinates in
 * [-1/2, n - 1/2]), FP64. Synchronises `stream`. */
int cbct_fov(const cbct_geom *g, float *V, void *stream);

/* ---- classical reconstructions (a5 FDK_w, a10 PDHG-TV and Landweber) ---- */

/* Columns of zero padding FDK adds on the short side of an offset panel:
 * ceil(2 |u_offset| / du). */
int cbct_fdk_pad(const cbct_geom *g);

/* FDK with redundancy weighting (Algorithm 1 initialisation, Sec. 2.6; Feldkamp
 * 1984): rows weighted by w(u') sdd / sqrt(sdd^2 + u'^2 + v'^2), zero-padded on the
 * short side (cbct_fdk_pad), filtered by the Ram-Lak kernel at the isocentre pitch
 * tau = du sid / sdd (tau h(0) = 1/(4 tau), tau h(odd j) = -1/(pi^2 j^2 tau)), then
 * vol(P) (+)= (2 pi / n_angles) sum_k (sid / U_k)^2 q_k(u_k(P), v_k(P)) with bilinear
 * sampling (zero off the extended panel), U_k the depth of P along the central ray.
 * Scratch: 2 batch n_angles nv (nu + pad) floats. Synchronises `stream`. */
int cbct_fdk(const cbct_geom *g, const float *proj, float *vol, int batch, int accumulate, void *stream);

/* ||K|| for K = [P; gamma grad] by `iters` power iterations on K^T K from the
 * all-ones volume (FP32 operators, FP64 norms); gamma = 0 gives ||P||.
 * Synchronises `stream`. */
int cbct_opnorm(const cbct_geom *g, double gamma, int iters, double *out, void *stream);

/* PDHG (Chambolle-Pock 2011) for min_x 1/2 ||P x - y||^2 + lam ||grad x||_{2,1}
 * (+ x >= 0 when nonneg), the paper's TV baseline (Sec. 2.5), on K = [P; gamma grad]
 * with F2 = (lam/gamma) ||.||_{2,1}: per iteration
 *   z1 <- (z1 + sigma (P xbar - y)) / (1 + sigma)
 *   z2 <- project_{|.| <= lam/gamma}(z2 + sigma gamma grad xbar)
 *   x+ <- max(0, x - tau (P^T z1 - gamma div z2)); xbar <- 2 x+ - x; x <- x+
 * grad = forward differences in voxel units, zero on the last index (Neumann),
 * div = -grad^T. Convergence needs sigma tau ||K||^2 < 1 (cbct_opnorm). y, x0 and x
 * are device arrays of `batch` items; x0 and x may alias. Scratch: 5 volumes and 2
 * projections per item. */
int cbct_pdhg(const cbct_geom *g, const float *y, const float *x0, float *x, int batch, int niter, double lam,
              double gamma, double sigma, double tau, int nonneg, void *stream);

/* Landweber iterations x <- x - tau P^T (P x - y) (clamped at 0 when nonneg), in place
 * on x. Scratch: one volume and one projection per item. */
int cbct_landweber(const cbct_geom *g, const float *y, float *x, int batch, int niter, double tau, int nonneg,
                   void *stream);

/* ---- convolutions of the learned blocks (a7, a8) ---- */

/* One 3x3 (taps3d = 0: over (H, W) of each of nimg * D images) or 3x3x3 (taps3d = 1)
 * "same" cross-correlation, stride 1, on the tensor cores (tcgen05.mma, BF16
 * operands, FP32 accumulation in TMEM): the learned blocks of Sec. 2.6 (Algorithm 1,
 * Gamma and Lambda). Activations are BF16 "row-blocked": image row (img, d, h) holds
 * its channel groups one after the other, element (img, d, h, w, c) at
 * ((((img * D + d) * H + h) * (cp / 8) + c / 8) * W + w) * 8 + c % 8 for cp channel
 * slots per pixel. x: cpin = 8, 16, 32 or 64 slots (slots >= cin zero); w: FP32
 * [cout][taps][cin]; bias: FP32 [cout] or NULL.
 * flip = 0: y = conv(x) with cout outputs; flip = 1: the input-gradient convolution
 * (x holds cout channels, mirrored taps, cin outputs). At most 64 outputs: more than
 * 32 run as two launches of at most 32 outputs each, over the same input.
 * epi 0: y = BF16 LeakyReLU(acc + bias), row-blocked with cpout slots (padding 0)
 * epi 1: state[c * sstride + pixel] += acc + bias (FP32, channel-first), c < outputs
 * epi 2: y = BF16 acc * (mask > 0 ? 1 : slope), mask BF16 row-blocked like y (the
 *        LeakyReLU derivative from the forward activation).
 * status: device int, set to 1 if a kernel gives up waiting on its tensor cores.
 * Errors: CBCT_EINVAL for cpin not in {8, 16, 32, 64}, cpin below the input channels,
 * more than 64 outputs, a LeakyReLU slope outside [0, 1], a missing output buffer, or
 * a shape whose weights and two input stages do not fit in shared memory (64 slots
 * need 3x3 over at least 2 rows, or 3x3x3 at 32 outputs per launch: both fit).
 * Scratch: the packed weights. */
int cbct_conv(const void *x, int nimg, int D, int H, int W, int cpin, int taps3d, const float *w,
              const float *bias, int cin, int cout, int flip, int epi, float slope, void *y, int cpout,
              const void *mask, float *state, long long sstride, int *status, void *stream);

/* Tile plan cbct_conv uses for a convolution of this shape (host only: no GPU call):
 * output rows per tile (rpt), bytes of the packed weights (B operand in row units),
 * input stages in shared memory and TMEM accumulators per CTA — of the first launch
 * (its first 32 outputs) when there are more than 32 outputs. Arguments as for
 * cbct_conv; any output pointer may be NULL. Errors: CBCT_EINVAL for an invalid shape. */
int cbct_conv_plan(int taps3d, int H, int cpin, int cin, int cout, int flip, int *rpt, long long *packed_bytes,
                   int *stages, int *accumulators);

/* Weight and bias gradients of the convolution above: dw[co][tap][ci] (+)=
 * sum_p dy[p][co] x[p + tap][ci], db[co] (+)= sum_p dy[p][co]; x BF16 row-blocked
 * with cpin slots, dy BF16 row-blocked with cpout slots (both multiples of 8). With
 * cpin 8, 32 or 64 and cpout 8, 16, 32 or 64 the weight gradient runs on the tensor
 * cores (BF16 operands, FP32 accumulation in TMEM; one partial per CTA; 64 slots as
 * blocks of 32 x 32 channels), otherwise on the CUDA cores (FP32); partials are
 * reduced in a fixed order (deterministic). status:
 * device int, set to 1 if a tensor-core kernel gives up waiting on its pipeline (its
 * partial is then written as zero). Errors: CBCT_EINVAL for NULL pointers (status
 * included) or non-positive channel counts. Scratch: the partial sums. */
int cbct_conv_wgrad(const void *x, int cpin, int cin, const void *dy, int cpout, int cout, int nimg, int D, int H,
                    int W, int taps3d, float *dw, float *db, int accumulate, int *status, void *stream);

/* ---- resampling between multiscale levels (a11; Sec. 2.6, multiscale scheme) ---- */

/* nch independent 3-D FP32 arrays [n0][n1][n2] (last index fastest), device.
 * cbct_resample_down: out[c][i][j][k] = scale * sum of in over the box
 * (i f0 + a, j f1 + b, k f2 + d), b < f1, d < f2, a < f0 — or a = 0 only when pick0
 * (axis 0 subsampled). Average pooling of a volume: f = (2, 2, 2), scale 1/8; the
 * coarse level's projections (every second angle, 2 x 2 binned pixels): f = (2, 2, 2),
 * pick0, scale 1/4; adjoint of nearest upsampling: scale 1. out has
 * (n0 / f0) x (n1 / f1) x (n2 / f2) per array; each n must be divisible by its f.
 * cbct_resample_up: out[c][i][j][k] = in[c][i / f0][j / f1][k / f2] (nearest), out of
 * size n0 f0 x n1 f1 x n2 f2. Errors: CBCT_EINVAL for NULL pointers or bad sizes. */
int cbct_resample_down(const float *in, long long nch, int n0, int n1, int n2, int f0, int f1, int f2, int pick0,
                       float scale, float *out, void *stream);
int cbct_resample_up(const float *in, long long nch, int n0, int n1, int n2, int f0, int f1, int f2, float *out,
                     void *stream);

/* ---- learned primal-dual reconstruction (a7-a9, a12; Sec. 2.6, Algorithm 1) ---- */

typedef struct cbct_lpd cbct_lpd; /* opaque: weights (FP32 master), gradients, Adam moments, workspaces */

typedef struct {
    int n_iter;                  /* unrolled iterations (8 in the learned workload) */
    int n_mem;                   /* primal / dual memory channels, 2..6 (5) */
    int width;                   /* hidden channels of every block: 32 or 64 (P4 primal blocks: 32) */
    float slope;                 /* LeakyReLU slope (0.2), in [0, 1] */
    float mu_ref;                /* volume unit (1/mm): f' = f / mu_ref internally (0.02) */
    float bp_scale;              /* scale of P^T (w h_1) in the primal input; <= 0: 1 / max P^T(w 1) */
    unsigned long long seed;     /* initial weights (He normal; last layer of a block x 0.1; zero bias) */
    int residual_input;          /* 1: the dual block also receives mu_ref P f_1 - y, formed in FP32
                                    before its BF16 rounding (n_mem <= 5); 0: not */
    int max_batch;               /* volumes per lpd_forward call the workspaces hold (0 means 1) */
    int reversible;              /* 1: additive coupling with channel permutations (Sec. 2.6,
                                    Algorithm 1 split / update / combine / permute; n_mem even):
                                    the backward recovers every iterate from the final states
                                    instead of storing them. 0: Adler-style memory update. */
    int lire;                    /* 1 (needs reversible = 1, residual_input = 0): the iteration of
                                    Algorithm 1 at one resolution, see below. 0: off. */
    int p4;                      /* 1: P4-equivariant primal blocks (Sec. 2.6), see below. 0: plain */
    int unet;                    /* 1 (needs p4): the primal block is a P4 U-Net of depth 1, see below */
    int weight_norm;             /* 1: forced weight normalisation of every convolution, see below */
} cbct_lpd_desc;

/* Network on geometry g (which must outlive it): per iteration n a dual block
 * Gamma_n (3x3 convs over each projection image: n_mem + 2 (+ 1 with residual_input)
 * -> width -> width -> n_mem) and a primal block Lambda_n (3x3x3: n_mem + 1 -> width ->
 * width -> n_mem), LeakyReLU between convs; parameters flat FP32 per iteration [dual w1
 * b1 w2 b2 w3 b3, primal ...], w as [cout][taps][cin]. Memory, for max_batch volumes:
 * (n_iter + 1) iterates of n_mem volumes and n_mem projections plus ~4 x width-channel
 * BF16 activations per block. Synchronises. Errors: CBCT_EINVAL unless 1 <= n_iter <= 64,
 * 2 <= n_mem <= 6 (<= 5 with residual_input), width 32 or 64, mu_ref > 0, 0 <= slope <= 1,
 * residual_input is 0 or 1, max_batch <= 64 and max_batch * n_angles <= 65535 (2 *
 * max_batch * n_angles with lire = 1), and the constraints of the modes below. */
int lpd_create(const cbct_geom *g, const cbct_lpd_desc *desc, cbct_lpd **out);
void lpd_destroy(cbct_lpd *m);

/* Reversible mode (desc.reversible = 1), per iteration n with halves of K = n_mem / 2
 * channels, f = [p1, p2], h = [d1, d2]:
 *   d2 <- d2 + Gamma_n([d1, mu_ref P p2[0], y (, mu_ref P p2[0] - y)])
 *   p2 <- p2 + Lambda_n([p1, bp_scale P^T(w d2[0])])
 *   f <- f[perm_f[n]],  h <- h[perm_h[n]]        (new channel c = old channel perm[c])
 * output mu_ref f[0]. Blocks: dual K + 2 (+ 1) -> width -> width -> K, primal K + 1 ->
 * width -> width -> K. The permutations are drawn from desc.seed at creation so that each
 * mixes the halves (the new first half takes a channel of the old second half); a
 * training forward keeps only the final states, and lpd_backward undoes the iterations
 * one by one (p2 -= Lambda_n(..), d2 -= Gamma_n(..)), exact up to one FP32 rounding of each
 * state update. The latent-state entries below refuse a reversible model.
 * lpd_get_perms / lpd_set_perms copy the n_iter x 2 x n_mem permutation table (per
 * iteration perm_f then perm_h) to / from host memory; set checks that each row is a
 * permutation that mixes the halves. Errors: CBCT_EINVAL for a model that is not
 * reversible, NULL pointers or (set) an invalid table. */
int lpd_get_perms(const cbct_lpd *m, int *host);

/* LIRE mode (desc.lire = 1; Sec. 2.6, Algorithm 1 at one resolution; the paper's dual block is
 * width 64 with n_mem = 8: K + 4 -> 64 -> 64 -> 4):
 * a separate FP32 reconstruction x next to the reversible latents (halves of K =
 * n_mem / 2 channels), x <- x0, f <- [x0 / mu_ref, s P^T(w y), x0 / mu_ref, ...],
 * h <- y in every channel (s = bp_scale), then per iteration n:
 *   p_op = [mu_ref P p2[0], P x]
 *   d2 <- d2 + Gamma_n([d1, p_op, y, P x - y])        3x3x3 convs over (angle, v, u)
 *   p2 <- p2 + Lambda_n([p1, s P^T(w d2[0]), x / mu_ref, s P^T(P x - y), V])
 *   x  <- x + mu_ref (beta_n + sum_c omega_n[c] f[c])  1x1x1 output convolution
 *   f <- f[perm_f[n]],  h <- h[perm_h[n]]
 * with V the FoV tensor; x_out = x. Blocks: K + 4 -> width -> width -> K, all 3x3x3;
 * parameters per iteration: dual layers, primal layers (as above), then omega [n_mem]
 * and beta. The backward undoes x, p2 and d2 in reverse order, like the reversible mode. */
int lpd_set_perms(cbct_lpd *m, const int *host);

/* P4-equivariant primal blocks (desc.p4 = 1; Sec. 2.6: the primal block's convolutions are
 * equivariant to 90-degree rotations about z). Each primal block is lift -> LReLU -> group ->
 * LReLU -> group averaged over the four rotations, 3x3x3, 8 base filters (32 group channels,
 * channel 4 c + r for filter c rotated r quarter turns). The learnable parameters are base
 * filters: lifting [8][27][cin] + bias [8], group [8][4][27][8] + bias [8], averaged
 * [K][4][27][8] + bias [K] (the 4 is the relative rotation (s - r) mod 4 between input and
 * output group channel); they are expanded into full weights before each pass, and the full
 * weight gradients are gathered back onto them after each backward. With a square x-y
 * grid the block then commutes with the quarter turn v'[z][y][x] = v[z][x][n-1-y]. */

/* P4 U-Net primal blocks (desc.unet = 1, needs p4 and even volume sizes; Sec. 2.6: a U-Net
 * of depth 1 of six P4-equivariant 3x3x3 layers, LeakyReLU after all but the last, averaged
 * over the rotations). With F = 4 base filters:
 *   a = L(lift(x)) [4F],  s = L(g2(a)) [4F],  q = L(g3(pool(s))) [8F, half resolution],
 *   r = L(g4(q)) [8F, half],  t = L(g5([up(r), s])) [4F],  out = avg6(t) [K]
 * (pool: mean of 2 x 2 x 2 blocks; up: nearest; [ , ]: channel concatenation, up(r) first).
 * Base filters per layer, each + bias: lift [F][27][cin], g2 [F][4][27][F], g3 [2F][4][27][F],
 * g4 [2F][4][27][2F], g5 [F][4][27][3F], avg [K][4][27][F]. The paper's 48 / 96 filters
 * (F = 12) would give 144 concatenated channels; F = 4 keeps the concatenation within the
 * convolution's 64 input slots.
 *
 * Forced weight normalisation (desc.weight_norm = 1; Sec. 2.6, after Karras et al. 2024):
 * every layer's learnable parameters are [w][b][g] — g one gain per layer after the bias —
 * and the convolution uses g (w_c - mean w_c) / ||w_c - mean w_c|| for each output filter c
 * (for P4 layers each base filter, normalised before the rotation expansion); biases are used
 * as they are. lpd_adam_step then re-projects every raw filter to zero mean and norm
 * sqrt(filter length), which leaves the effective weights unchanged. A filter of zero norm
 * gives zero effective weights. */

/* Parameter count and device pointers to the parameters and the gradient buffer. */
int lpd_info(const cbct_lpd *m, long long *nparams, float **params, float **grads, float *bp_scale);

/* x_out = LPD(y, x0) for `batch` volumes at once (1 <= batch <= max_batch; y
 * [batch][n_angles][nv][nu], x0 and x_out [batch][nz][ny][nx]): f <- x0 / mu_ref
 * repeated, h <- 0; for n < n_iter:
 *   h <- h + Gamma_n([h, mu_ref P f_1, y (, mu_ref P f_1 - y)]);
 *   f <- f + Lambda_n([f, bp_scale P^T(w h_1)])
 * (w = the redundancy weight per detector column), x_out = mu_ref f_0. Every projector
 * call and convolution runs on the whole batch. save_for_backward = 1 keeps the iterates
 * for lpd_backward. Errors: CBCT_EINVAL for NULL pointers or a batch out of range. */
int lpd_forward(cbct_lpd *m, const float *y, const float *x0, float *x_out, int batch, int save_for_backward,
                void *stream);

/* Reverse sweep for dL/dx_out = grad_x (the last forward's batch): recomputes each
 * block's activations from the saved iterate, ADDS the parameter gradients (summed over
 * the batch) to the model's gradient buffer, writes dL/dy and dL/dx0 when those pointers
 * are not NULL. */
int lpd_backward(cbct_lpd *m, const float *grad_x, float *grad_y, float *grad_x0, void *stream);

/* Latent-state variants for the multiscale scheme (a11; Sec. 2.6: a coarser level's
 * result initialises the next level), one volume per call. The primal state f is [n_mem][nvox] FP32 in units
 * of mu_ref, the dual state h is [n_mem][nproj] FP32 (y's units), both device.
 * lpd_forward_latent: f_0 = f0 (NULL: x0 / mu_ref in every channel, then x0 is
 * required), h_0 = h0 (NULL: zero); x_out (nullable) = mu_ref f_N[0].
 * lpd_get_state: copies the final f_N / h_N of the last forward pass (either nullable);
 * for a reversible model, the states it holds in logical channel order: f_N / h_N after
 * a forward pass, the recovered f_0 / h_0 after lpd_backward.
 * lpd_backward_latent: upstream dL/dx_out (grad_x) and/or dL/df_N, dL/dh_N (each
 * nullable, at least one given; needs save_for_backward); accumulates parameter
 * gradients; writes dL/dy, dL/dx0, dL/df_0, dL/dh_0 where non-NULL. Errors: CBCT_EINVAL
 * for missing inputs or no saved forward pass. */
int lpd_forward_latent(cbct_lpd *m, const float *y, const float *x0, const float *f0, const float *h0, float *x_out,
                       int save_for_backward, void *stream);
int lpd_get_state(const cbct_lpd *m, float *f_out, float *h_out, void *stream);
int lpd_backward_latent(cbct_lpd *m, const float *grad_x, const float *grad_fN, const float *grad_hN, float *grad_y,
                        float *grad_x0, float *grad_f0, float *grad_h0, void *stream);

int lpd_zero_grad(cbct_lpd *m, void *stream);

/* Global gradient-norm clipping before lpd_adam_step (unrolled networks are trained
 * with it; without it the lpd128 training diverged after ~190 steps): n = ||grad_scale
 * * g|| (FP64, fixed-order reduction); g *= min(1, max_norm / n), or g = 0 when n is not
 * finite (the step is skipped). norm_out (host, nullable) receives n; giving it
 * synchronises the stream. Errors: CBCT_EINVAL for max_norm <= 0. */
int lpd_clip_grads(cbct_lpd *m, float max_norm, float grad_scale, double *norm_out, void *stream);

/* Adam (Kingma & Ba) on the gradient buffer times grad_scale, bias-corrected for step
 * number `step` (>= 1). */
int lpd_adam_step(cbct_lpd *m, float lr, float beta1, float beta2, float eps, int step, float grad_scale,
                  void *stream);

/* Measured shared-memory read bandwidth (the paper has no counterpart: it gives the
 * roofline denominator of the projector kernels, which read their bilinear samples from
 * shared memory). Launches ctas_per_sm (1..8) CTAs of 256 threads per SM; each thread
 * makes iters (1..2^20) rounds of four conflict-free 16-byte shared-memory loads. *bytes
 * (host) receives the bytes the launch reads; the caller times the launch on `stream`
 * (CUDA events) and divides. sink: a device float per CTA (never written in practice).
 * Asynchronous. Errors: CBCT_EINVAL for arguments out of range. */
int cbct_smem_probe(int ctas_per_sm, int iters, float *sink, long long *bytes, void *stream);

/* Test of the library's bounded waits (the paper has no counterpart: this checks the
 * failure handling of the pipelined kernels). Launches one CTA whose two warps wait on
 * a shared-memory barrier that nothing completes, each for at most limit_ns
 * nanoseconds (1 .. 1e8) of the GPU's global timer: the same wait the TMA and
 * tensor-core pipelines use, with a short limit instead of their 2 s. When a wait
 * runs out the kernel sets the geometry's device status word to 1, the timeout code
 * the projector kernels write (read and cleared by cbct_device_status), and returns;
 * *waited_ok (device int) is incremented once per wait that completed (none do).
 * Asynchronous on `stream`. Errors: CBCT_EINVAL for NULL pointers or a limit out of
 * range. */
int cbct_wait_probe(const cbct_geom *g, long long limit_ns, int *waited_ok, void *stream);

/* Read (and with clear = 1 reset) the model's device status word: 0 = ok, 1 = one of
 * its convolution kernels (forward, input-gradient or weight-gradient) gave up waiting
 * on its tensor-core pipeline (it then left its outputs unwritten, or wrote a zero
 * weight-gradient partial). Synchronises the device. Errors: CBCT_EINVAL for NULL. */
int lpd_device_status(const cbct_lpd *m, int *out, int clear);

/* Copy the n FP32 parameters to / from host memory (checkpoints). Synchronous. */
int lpd_set_params(cbct_lpd *m, const float *host, long long n);
int lpd_get_params(const cbct_lpd *m, float *host, long long n);
/* Copy the n accumulated parameter gradients to host memory. Synchronous. */
int lpd_get_grads(const cbct_lpd *m, float *host, long long n);

/* Masked mean squared error on the device: over elements with V[i] >= thr (all if V is
 * NULL), *loss = mean (x - ref)^2 and grad = 2 (x - ref) / count there, 0 elsewhere
 * (grad may be NULL). loss is a device float. Deterministic (fixed-order reduction). */
int cbct_masked_mse(const float *x, const float *ref, const float *V, float thr, long long n, float *loss,
                    float *grad, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CBCT_H */
