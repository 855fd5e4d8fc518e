// Learned primal-dual reconstruction (paper Sec. 2.6, Algorithm 1; the unrolled
// primal-dual network with additive primal and dual updates), in the form of the
// learned-primal-dual workload: n_iter iterations of
//     h <- h + Gamma_n([h, P f_1, y (, P f_1 - y)])  dual block, 2D convs per projection
//     f <- f + Lambda_n([f, P^T (w h_1)])            primal block, 3D convs
// with n_mem-channel primal/dual memories, f starting from the FDK-style initial
// volume repeated, h from zero, output f_0. Every block is conv3x3(x3) -> LReLU ->
// conv -> LReLU -> conv at width `width`, BF16 operands on the tensor cores, FP32
// states. Internally volumes are in units of mu_ref (f' = f / mu_ref, so mu_ref P f'
// is in the units of y) and the backprojection is scaled by bp_scale. The optional
// data-residual channel mu_ref P f_1 - y is formed in FP32 before its BF16 rounding:
// the projection-domain counterpart of the paper's Landweber input P*(P x - y)
// (Algorithm 1), which a block could otherwise only form from two BF16-rounded
// operands. A batch of volumes runs through every kernel at once: states are laid
// out [channel][batch][pixels].
//
// Backward: the iterates (f_n, h_n) are the only saved tensors; each block's
// activations are recomputed from its saved input during the reverse sweep
// (activation recomputation), and the projector's adjoint carries gradients through
// P and P^T.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "geom_impl.h"

namespace cbct {

// from conv.cu
struct ConvArgs;
int conv_wgrad(const __nv_bfloat16 *x, int cpin, int cin, const __nv_bfloat16 *dy, int cpout, int cout, int nimg,
               int D, int H, int W, int taps3d, float *dw, float *db, int accumulate, int *status, cudaStream_t st);

}  // namespace cbct

extern "C" int cbct_conv(const void *x, int nimg, int D, int H, int W, int cpin, int taps3d, const float *w,
                         const float *bias, int cin, int cout, int flip, int epi, float slope, void *y, int cpout,
                         const void *mask, float *state, long long sstride, int *status, void *stream);

using namespace cbct;

struct LayerSpec {
    int cin, cout, taps3d;   // of the convolution as run (full channel counts)
    int H;                   // rows of an image / plane (the tile plan depends on it)
    long long w_off, b_off;  // offsets of the layer's parameters in the flat array
    long long pk_off = 0;    // forward B operand within cbct_lpd::wpk
    // P4 weight tying: kind 0 = plain (the convolution reads w_off / b_off); 1 = lifting,
    // 2 = group, 3 = group averaged over rotations, whose parameters are base filters
    // (cb outputs, cib inputs) expanded into full weights at fw_off / fb_off
    int kind = 0, cb = 0, cib = 0;
    long long fw_off = 0, fb_off = 0;
    int cpin = 32;  // channel slots of the layer's input activation
    int last = 0;   // the block's output layer (initialised 10x smaller)
    // weight normalisation: gain at g_off (learnable), normalised filters at nw_off (the
    // convolution's weights for a plain layer, the expanded base for a P4 layer)
    long long g_off = -1, nw_off = 0;
};

// one P4 layer for the expansion / contraction kernels
struct P4Job {
    int kind, cb, cib, cout, cin;  // cout, cin: full
    long long w_off, b_off, fw_off, fb_off;
    int assign;  // 1: the contraction writes the base weights' gradients (normalised filters) instead of adding
};

struct cbct_lpd {
    const cbct_geom *g = nullptr;
    cbct_lpd_desc d{};
    int maxb = 1;    // largest batch the workspaces hold
    int batch = 1;   // batch of the last forward pass (the backward uses the same)
    int nd = 7;      // dual input channels: n_mem + 2 (+ 1 with the residual channel); half of n_mem when reversible
    // reversible mode: fixed channel permutations per iteration (new[c] = old[perm[c]]) and
    // the plane of each logical channel after the last forward pass
    std::vector<std::vector<int>> perm_f, perm_h;
    // LIRE mode: per-iteration offset of the output convolution's parameters (omega [n_mem],
    // beta) in the flat array, the reconstruction x [batch][nvox], the FoV tensor repeated
    // per batch item, and two-item scratch for batched projector calls
    std::vector<long long> out_off;
    // P4 primal layers: jobs (device) and the size of the expansion area that follows the
    // nparams learnable parameters in params (full weights) and grads (full gradients)
    P4Job *p4_jobs = nullptr;
    int n_p4 = 0;
    long long nexp = 0, p4_max = 0;
    float *x = nullptr, *Vb = nullptr, *t2v = nullptr, *t2p = nullptr, *gx = nullptr, *opart = nullptr;
    int fin_f[8] = {}, fin_h[8] = {};
    int cur_f[8] = {}, cur_h[8] = {};  // plane of each logical channel of the states held now
    std::vector<LayerSpec> layers;  // per iteration: 3 dual layers, then the primal block's (3, or 6 for the U-Net)
    std::vector<int> dual_at, prim_at;  // index of each iteration's first dual / primal layer
    int unet = 0;                       // primal block: P4 U-Net of depth 1 (Sec. 2.6)
    int wn = 0;                         // forced weight normalisation of every layer
    struct WnJob *wn_jobs = nullptr;    // device [n_wn]
    int n_wn = 0;
    long long wn_lo = 0, wn_hi = 0;     // the normalised filters' area (gradients reset each pass)
    // U-Net activations (BF16 row-blocked): a (full, 4F), C = [up(r), s] (full, 64 slots),
    // p = pool(s) (half, 4F), q, r (half, 8F), t (full, 4F); uh1, uh2: half-resolution gradients
    __nv_bfloat16 *u_a = nullptr, *u_C = nullptr, *u_p = nullptr, *u_q = nullptr, *u_r = nullptr, *u_t = nullptr;
    __nv_bfloat16 *u_h1 = nullptr, *u_h2 = nullptr;
    __nv_bfloat16 *u_ga = nullptr, *u_gb = nullptr;  // 16-channel gradients (full resolution, 32 slots)
    long long nparams = 0;
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    float *wred = nullptr;  // redundancy weight [nu]
    float bp_scale = 1.f;
    int last = -1;  // slot of the final states after a forward pass
    // saved iterates: f[n_iter + 1][n_mem][batch][nvox], h[n_iter + 1][n_mem][batch][nproj]
    float *f = nullptr, *h = nullptr;
    float *y = nullptr;  // the data of the last forward (copied)
    int saved = 0;
    // workspaces
    float *tproj = nullptr, *tproj2 = nullptr, *tvol = nullptr;
    // projector outputs of each iteration kept by a training forward pass (so the
    // backward does not recompute them): P f_1 [n_iter][nproj], P^T (w h_1) [n_iter][nvox]
    float *pf_saved = nullptr, *bp_saved = nullptr;
    double *clip = nullptr;  // gradient-norm scratch: per-block partial sums, then norm and factor
    __nv_bfloat16 *din = nullptr, *a1 = nullptr, *a2 = nullptr, *pin = nullptr, *b1 = nullptr, *b2 = nullptr;
    __nv_bfloat16 *g32a = nullptr, *g32b = nullptr, *gsmall = nullptr;  // gradient buffers
    float *gf = nullptr, *gh = nullptr;  // [n_mem + 1][batch][nvox], [nd][batch][nproj]
    int *status = nullptr;
    long long nvox = 0, nproj = 0;  // per volume
    // every forward layer's weights packed as tensor-core B operands, refreshed by one
    // launch at the start of each forward and backward pass
    uint8_t *wpk = nullptr;
    ConvPackJob *pack_jobs = nullptr;  // device [n_pack_jobs]: one per launch of 32 outputs
    int n_pack_jobs = 0;
    long long pack_max_nelem = 0;
};

namespace {

// SplitMix64 + Box-Muller: deterministic initial weights on every platform.
struct InitRng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() {
        const double u1 = uniform(), u2 = uniform();
        return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    }
};

__global__ void k_fill_f(float *x, long long n, float v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

// f[c][i] = x0[i] * s for c < n_mem
__global__ void k_init_f(const float *__restrict__ x0, float *__restrict__ f, long long n, int n_mem, float s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = x0[i] * s;
        for (int c = 0; c < n_mem; ++c) f[c * n + i] = v;
    }
}

// channels-last BF16 [n][8] from up to 8 FP32 channel-first planes: channel c =
// s[c] p[c][i] - q[c][i] (p null: 0; q null: no subtrahend), formed in FP32 and rounded
// once to BF16
struct Planes {
    const float *p[8];
    float s[8];
    const float *q[8];
};
__global__ void k_pack8(Planes pl, long long n, __nv_bfloat16 *__restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float x = pl.p[c] ? pl.p[c][i] * pl.s[c] : 0.f;
            if (pl.q[c]) x -= pl.q[c][i];
            v[c] = __float2bfloat16_rn(x);
        }
        *reinterpret_cast<uint4 *>(out + i * 8) = *reinterpret_cast<const uint4 *>(v);
    }
}

// acc[i] += a[i] - b[i]
__global__ void k_add_diff(float *__restrict__ acc, const float *__restrict__ a, const float *__restrict__ b,
                           long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc[i] += a[i] - b[i];
}

// out[k][v][u] = w[u] * in[k][v][u] * s
__global__ void k_scale_cols(const float *__restrict__ in, const float *__restrict__ w, long long n, int nu, float s,
                             float *__restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = in[i] * w[i % nu] * s;
}

// acc[i] += s * src[i]
__global__ void k_axpy(float *__restrict__ acc, const float *__restrict__ src, long long n, float s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc[i] += s * src[i];
}

// out[i] = s * sum_c g[c][i]
__global__ void k_sum_channels(const float *__restrict__ g, int nc, long long n, float s, float *__restrict__ out,
                               int accumulate) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int c = 0; c < nc; ++c) v += g[c * n + i];
        out[i] = accumulate ? out[i] + s * v : s * v;
    }
}

__global__ void k_max_reduce(const float *__restrict__ x, long long n, float *out) {
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, x[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(m));  // m >= 0
}

// Adam (Kingma & Ba 2014) with bias correction.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2, float gs) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i] * gs;
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// masked mean squared error: loss = sum_{mask} (x - r)^2 / count, grad = 2 (x - r) / count on
// the mask (mask: voxels with V >= thr). Deterministic: per-block partials, fixed-order sum.
__global__ void k_mse_partial(const float *__restrict__ x, const float *__restrict__ r, const float *__restrict__ V,
                              float thr, long long n, double *part, double *pcount) {
    double s = 0.0, c = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (V && V[i] < thr) continue;
        const double d = (double)x[i] - (double)r[i];
        s += d * d;
        c += 1.0;
    }
    __shared__ double ss[256], sc[256];
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ss[0];
        pcount[blockIdx.x] = sc[0];
    }
}

__global__ void k_mse_final(const double *part, const double *pcount, int nb, float *loss, float *count) {
    double s = 0.0, c = 0.0;
    for (int b = 0; b < nb; ++b) {
        s += part[b];
        c += pcount[b];
    }
    *loss = (float)(c > 0 ? s / c : 0.0);
    *count = (float)c;
}

__global__ void k_mse_grad(const float *__restrict__ x, const float *__restrict__ r, const float *__restrict__ V,
                           float thr, long long n, const float *count, float *__restrict__ g) {
    const float inv = *count > 0.f ? 2.f / *count : 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        g[i] = (V && V[i] < thr) ? 0.f : inv * (x[i] - r[i]);
}

// ---- output convolution of the LIRE mode (1x1x1, n_mem channels -> 1) ----

constexpr int kOutBlocks = 304;

struct PlanesW {
    float *p[8];
};

// x[i] += sign * mu * (beta + sum_c omega[c] f_c[i]), omega = om[0..M), beta = om[M]. The
// inverse update (sign -1) recomputes the same term, so it undoes the forward one up to
// one FP32 rounding of x.
__global__ void k_outconv(float *__restrict__ x, Planes fp, const float *__restrict__ om, float mu, long long n, int M,
                          float sign) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v = om[M];
        for (int c = 0; c < M; ++c) v = fmaf(om[c], fp.p[c][i], v);
        x[i] = x[i] + sign * (mu * v);
    }
}

// Backward of k_outconv: g_f_c[i] += mu omega[c] g_x[i]; partial[blk][c] = mu sum_i g_x[i]
// f_c[i] (c < M) and partial[blk][M] = mu sum_i g_x[i], over the block's grid-stride share
// (fixed-order tree in shared memory).
__global__ void __launch_bounds__(256) k_outconv_grad(const float *__restrict__ gx, Planes fp, PlanesW gp,
                                                      const float *__restrict__ om, float mu, long long n, int M,
                                                      float *__restrict__ partial) {
    float acc[9] = {};
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float g = gx[i];
        for (int c = 0; c < M; ++c) {
            acc[c] = fmaf(g, fp.p[c][i], acc[c]);
            gp.p[c][i] += mu * om[c] * g;
        }
        acc[M] += g;
    }
    __shared__ float red[256];
    for (int c = 0; c <= M; ++c) {
        red[threadIdx.x] = acc[c];
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(long long)blockIdx.x * (M + 1) + c] = mu * red[0];
        __syncthreads();
    }
}

// f[c][i] = c even ? x0[i] * inv_mu : xbp[i] * s (the initial primal latents of Algorithm 1)
__global__ void k_lire_init_f(const float *__restrict__ x0, const float *__restrict__ xbp, float *__restrict__ f,
                              long long n, int M, float inv_mu, float s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float a = x0[i] * inv_mu, b = xbp[i] * s;
        for (int c = 0; c < M; ++c) f[c * n + i] = (c & 1) ? b : a;
    }
}

// ---- P4 weight tying (Sec. 2.6: P4-equivariant primal layers) ----
//
// A full 3x3x3 weight [cout][27][cin] is built from base filters. Rotating a filter r
// quarter turns about z (the rotation that maps a volume v to v'[z][y][x] = v[z][x][n-1-y])
// puts at tap (z, y, x) the base entry at p4_tap(tap, r). Lifting layer: full[(co, r)][t][ci]
// = base[co][p4_tap(t, r)][ci]; group layer: full[(co, r)][t][(ci, s)] =
// base[co][(s - r) mod 4][p4_tap(t, r)][ci]; averaged group layer: full[c][t][(ci, s)] =
// 1/4 sum_r base[c][(s - r) mod 4][p4_tap(t, r)][ci]; group channel (c, r) is index 4 c + r.

__host__ __device__ __forceinline__ int p4_tap(int t, int r) {
    const int z = t / 9, y = (t / 3) % 3, x = t % 3;
    int by, bx;
    switch (r & 3) {
        case 0: by = y; bx = x; break;
        case 1: by = x; bx = 2 - y; break;
        case 2: by = 2 - y; bx = 2 - x; break;
        default: by = 2 - x; bx = y; break;
    }
    return z * 9 + by * 3 + bx;
}

// params[fw_off..] = full weights (and biases) of job blockIdx.y from its base filters
__global__ void k_p4_expand(const P4Job *__restrict__ jobs, float *__restrict__ params) {
    const P4Job J = jobs[blockIdx.y];
    const long long n = (long long)J.cout * 27 * J.cin;
    const float *bw = params + J.w_off;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n + J.cout;
         e += (long long)gridDim.x * blockDim.x) {
        if (e >= n) {  // bias
            const int co = (int)(e - n);
            params[J.fb_off + co] = params[J.b_off + (J.kind == 3 ? co : co / 4)];
            continue;
        }
        const int ci_f = (int)(e % J.cin), t = (int)((e / J.cin) % 27), co_f = (int)(e / ((long long)J.cin * 27));
        float v;
        if (J.kind == 1) {
            const int co = co_f / 4, r = co_f % 4;
            v = bw[((long long)co * 27 + p4_tap(t, r)) * J.cib + ci_f];
        } else if (J.kind == 2) {
            const int co = co_f / 4, r = co_f % 4, ci = ci_f / 4, sg = ci_f % 4;
            v = bw[(((long long)co * 4 + ((sg - r) & 3)) * 27 + p4_tap(t, r)) * J.cib + ci];
        } else {
            const int ci = ci_f / 4, sg = ci_f % 4;
            float a = 0.f;
            for (int r = 0; r < 4; ++r) a += bw[(((long long)co_f * 4 + ((sg - r) & 3)) * 27 + p4_tap(t, r)) * J.cib + ci];
            v = 0.25f * a;
        }
        params[J.fw_off + e] = v;
    }
}

// grads[w_off..] += the full gradients of job blockIdx.y gathered back onto its base
// filters (each base entry sums the full entries it was copied to, in a fixed order)
__global__ void k_p4_contract(const P4Job *__restrict__ jobs, float *__restrict__ grads) {
    const P4Job J = jobs[blockIdx.y];
    const long long nb = (long long)J.cb * (J.kind == 1 ? 1 : 4) * 27 * J.cib;  // base weights
    const float *gf = grads + J.fw_off;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nb + J.cb;
         e += (long long)gridDim.x * blockDim.x) {
        float a = 0.f;
        if (e >= nb) {  // bias
            const int co = (int)(e - nb);
            if (J.kind == 3) a = grads[J.fb_off + co];
            else for (int r = 0; r < 4; ++r) a += grads[J.fb_off + 4 * co + r];
            grads[J.b_off + co] += a;
            continue;
        }
        if (J.kind == 1) {
            const int ci = (int)(e % J.cib), tb = (int)((e / J.cib) % 27), co = (int)(e / ((long long)J.cib * 27));
            for (int r = 0; r < 4; ++r)
                a += gf[((long long)(4 * co + r) * 27 + p4_tap(tb, 4 - r)) * J.cin + ci];
        } else {
            const int ci = (int)(e % J.cib), tb = (int)((e / J.cib) % 27), g = (int)((e / ((long long)J.cib * 27)) % 4);
            const int co = (int)(e / ((long long)J.cib * 27 * 4));
            for (int r = 0; r < 4; ++r) {
                const int co_f = J.kind == 3 ? co : 4 * co + r;
                const float v = gf[((long long)co_f * 27 + p4_tap(tb, 4 - r)) * J.cin + 4 * ci + ((g + r) & 3)];
                a += J.kind == 3 ? 0.25f * v : v;
            }
        }
        if (J.assign) grads[J.w_off + e] = a;
        else grads[J.w_off + e] += a;
    }
}

// out[i] += sum_b partial[b][i] (fixed order)
__global__ void k_sum_partials(const float *__restrict__ partial, int nblk, int n, float *__restrict__ out) {
    const int i = threadIdx.x;
    if (i >= n) return;
    float s = out[i];
    for (int b = 0; b < nblk; ++b) s += partial[(long long)b * n + i];
    out[i] = s;
}

// out[i] = a[i] - b[i]
__global__ void k_diff(float *__restrict__ out, const float *__restrict__ a, const float *__restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

// a permutation of 2K channels mixes the halves when the new first half takes at least
// one channel of the old second half
bool perm_mixes(const int *p, int M) {
    for (int c = 0; c < M / 2; ++c)
        if (p[c] >= M / 2) return true;
    return false;
}

int grid_n(long long n) {
    long long b = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 32LL * sm_count()));
}

}  // namespace

// ---- U-Net primal block: 2 x 2 x 2 resampling of BF16 row-blocked activations ----------------
// A row-blocked tensor with cp slots holds (img, d, h, w, channel c) at
// ((((img D + d) H + h) (cp / 8) + c / 8) W + w) 8 + c % 8; g0 selects a run of channel
// groups inside a wider tensor. One thread moves one pixel's 8-channel group (16 bytes).
struct Rb {
    __nv_bfloat16 *p;
    int cp, g0;  // slots per pixel, first channel group
};

__device__ __forceinline__ uint4 *rb_at(const Rb &t, long long row, int g, int W, int w) {
    return reinterpret_cast<uint4 *>(t.p + ((row * (t.cp / 8) + t.g0 + g) * (long long)W + w) * 8);
}

__device__ __forceinline__ void rb_unpack(const uint4 &v, float *f) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 t = __bfloat1622float2(h[j]);
        f[2 * j] = t.x;
        f[2 * j + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 rb_pack(const float *f) {
    uint4 v;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&v);
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
    return v;
}

// dst (half resolution) = scale x the sum of src over each 2 x 2 x 2 block (scale 1/8: the
// mean, the pooling; scale 1: the adjoint of nearest upsampling). D, H, W: the fine sizes (even).
__global__ void k_pool2_rb(Rb src, Rb dst, int ng, int nimg, int D, int H, int W, float scale) {
    const int D2 = D / 2, H2 = H / 2, W2 = W / 2;
    const long long n = (long long)nimg * D2 * H2 * ng * W2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int w2 = (int)(e % W2), g = (int)((e / W2) % ng);
        const long long row2 = e / ((long long)W2 * ng);
        const int h2 = (int)(row2 % H2), d2 = (int)((row2 / H2) % D2), img = (int)(row2 / ((long long)H2 * D2));
        float acc[8] = {};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long row = ((long long)img * D + 2 * d2 + (k >> 2)) * H + 2 * h2 + ((k >> 1) & 1);
            float f[8];
            rb_unpack(*rb_at(src, row, g, W, 2 * w2 + (k & 1)), f);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += f[j];
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] *= scale;
        *rb_at(dst, row2, g, W2, w2) = rb_pack(acc);
    }
}

// dst (full resolution, D, H, W) = nearest upsampling of src (half resolution)
__global__ void k_up2_rb(Rb src, Rb dst, int ng, int nimg, int D, int H, int W) {
    const long long n = (long long)nimg * D * H * ng * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(e % W), g = (int)((e / W) % ng);
        const long long row = e / ((long long)W * ng);
        const int h = (int)(row % H), d = (int)((row / H) % D), img = (int)(row / ((long long)H * D));
        const long long row2 = ((long long)img * (D / 2) + d / 2) * (H / 2) + h / 2;
        *rb_at(dst, row, g, W, w) = *rb_at(src, row2, g, W / 2, w / 2);
    }
}

// Gradient of the skip activation s (full resolution): the concatenation's share gc (already
// multiplied by the LeakyReLU derivative at s) plus that derivative times the pooling's
// adjoint of gp (half resolution): out = gc + (s > 0 ? 1 : slope) gp[coarse] / 8.
__global__ void k_skip_grad_rb(Rb gc, Rb s, Rb gp, Rb out, int ng, int nimg, int D, int H, int W, float slope) {
    const long long n = (long long)nimg * D * H * ng * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(e % W), g = (int)((e / W) % ng);
        const long long row = e / ((long long)W * ng);
        const int h = (int)(row % H), d = (int)((row / H) % D), img = (int)(row / ((long long)H * D));
        const long long row2 = ((long long)img * (D / 2) + d / 2) * (H / 2) + h / 2;
        float a[8], m[8], q[8];
        rb_unpack(*rb_at(gc, row, g, W, w), a);
        rb_unpack(*rb_at(s, row, g, W, w), m);
        rb_unpack(*rb_at(gp, row2, g, W / 2, w / 2), q);
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] += (m[j] > 0.f ? 1.f : slope) * (0.125f * q[j]);
        *rb_at(out, row, g, W, w) = rb_pack(a);
    }
}

// ---- forced weight normalisation ------------------------------------------------------------
// One job per layer: rows filters of len weights at raw_off (the learnable values), their
// effective values g (w - mean w) / ||w - mean w|| at dst_off, g the layer's gain at g_off.
// One CTA per job walks the rows with fixed-order block reductions (deterministic).
struct WnJob {
    long long raw_off, dst_off, g_off;
    int rows, len;
    long long b_raw, b_dst;  // a plain layer's biases, copied (and their gradients added back)
    int nb;                  // 0 for P4 layers (their expansion moves the biases)
};

// sum over the block of v (double), fixed order; every thread gets the result
__device__ double wn_block_sum(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// mean and 1 / norm of the centred row (a zero row gives 1 / norm = 0: zero effective weights)
__device__ void wn_row_stats(const float *w, int len, double *red, double &mean, double &inv) {
    double a = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) a += w[i];
    mean = wn_block_sum(a, red) / len;
    double q = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const double v = w[i] - mean;
        q += v * v;
    }
    const double n = sqrt(wn_block_sum(q, red));
    inv = n > 0.0 ? 1.0 / n : 0.0;
}

__global__ void __launch_bounds__(256) k_wn_fwd(const WnJob *__restrict__ jobs, float *__restrict__ params) {
    __shared__ double red[256];
    const WnJob J = jobs[blockIdx.x];
    const double g = params[J.g_off];
    for (int r = 0; r < J.rows; ++r) {
        const float *w = params + J.raw_off + (long long)r * J.len;
        double mean, inv;
        wn_row_stats(w, J.len, red, mean, inv);
        float *e = params + J.dst_off + (long long)r * J.len;
        for (int i = threadIdx.x; i < J.len; i += blockDim.x) e[i] = (float)(g * (w[i] - mean) * inv);
    }
    for (int i = threadIdx.x; i < J.nb; i += blockDim.x) params[J.b_dst + i] = params[J.b_raw + i];
}

// grads at dst_off (of the effective weights) -> raw weights and gain (added):
// u = (w - mean) / n, dL/dg = sum G u, dv = g (G - u (u . G)) / n, dw = dv - mean dv
__global__ void __launch_bounds__(256) k_wn_bwd(const WnJob *__restrict__ jobs, const float *__restrict__ params,
                                                float *__restrict__ grads) {
    __shared__ double red[256];
    const WnJob J = jobs[blockIdx.x];
    const double g = params[J.g_off];
    double gg = 0.0;
    for (int r = 0; r < J.rows; ++r) {
        const float *w = params + J.raw_off + (long long)r * J.len;
        const float *G = grads + J.dst_off + (long long)r * J.len;
        double mean, inv;
        wn_row_stats(w, J.len, red, mean, inv);
        double a = 0.0;
        for (int i = threadIdx.x; i < J.len; i += blockDim.x) a += G[i] * ((w[i] - mean) * inv);
        const double uG = wn_block_sum(a, red);
        gg += uG;
        double b = 0.0;
        for (int i = threadIdx.x; i < J.len; i += blockDim.x) b += G[i] - ((w[i] - mean) * inv) * uG;
        const double mdv = wn_block_sum(b, red) / J.len;  // mean of (G - u uG)
        float *dw = grads + J.raw_off + (long long)r * J.len;
        for (int i = threadIdx.x; i < J.len; i += blockDim.x)
            dw[i] += (float)(g * inv * (G[i] - ((w[i] - mean) * inv) * uG - mdv));
    }
    if (threadIdx.x == 0) grads[J.g_off] += (float)gg;
    for (int i = threadIdx.x; i < J.nb; i += blockDim.x) grads[J.b_raw + i] += grads[J.b_dst + i];
}

// the forced step: every raw filter becomes its centred, normalised self times sqrt(len)
__global__ void __launch_bounds__(256) k_wn_force(const WnJob *__restrict__ jobs, float *__restrict__ params) {
    __shared__ double red[256];
    const WnJob J = jobs[blockIdx.x];
    const double s = sqrt((double)J.len);
    for (int r = 0; r < J.rows; ++r) {
        float *w = params + J.raw_off + (long long)r * J.len;
        double mean, inv;
        wn_row_stats(w, J.len, red, mean, inv);
        for (int i = threadIdx.x; i < J.len; i += blockDim.x) w[i] = (float)((w[i] - mean) * inv * s);
        __syncthreads();  // the next row's statistics read only their own row, but keep the phases apart
    }
}

// effective weights of every layer from the learnable ones: normalisation, then P4 expansion
static void p4_expand(cbct_lpd *m, cudaStream_t st);
static void weights_expand(cbct_lpd *m, cudaStream_t st) {
    if (m->n_wn) k_wn_fwd<<<m->n_wn, 256, 0, st>>>(m->wn_jobs, m->params);
    p4_expand(m, st);
}

static void p4_contract(cbct_lpd *m, cudaStream_t st);
// gradients of the effective weights back onto the learnable ones (after every weight gradient
// of the pass): P4 contraction into the normalised filters' area, then through the normalisation
static void weights_contract(cbct_lpd *m, cudaStream_t st) {
    p4_contract(m, st);  // with normalisation it assigns the normalised base filters' gradients
    if (m->n_wn) k_wn_bwd<<<m->n_wn, 256, 0, st>>>(m->wn_jobs, m->params, m->grads);
}

static void p4_expand(cbct_lpd *m, cudaStream_t st) {
    if (!m->n_p4) return;
    dim3 grd((unsigned)std::min<long long>(64, (m->p4_max + 255) / 256 + 1), (unsigned)m->n_p4);
    k_p4_expand<<<grd, 256, 0, st>>>(m->p4_jobs, m->params);
}

static void p4_contract(cbct_lpd *m, cudaStream_t st) {
    if (!m->n_p4) return;
    dim3 grd((unsigned)std::min<long long>(64, (m->p4_max + 255) / 256 + 1), (unsigned)m->n_p4);
    k_p4_contract<<<grd, 256, 0, st>>>(m->p4_jobs, m->grads);
}

// weight gradients add up across backward passes only where the convolution reads the
// learnable weights themselves (plain layers without normalisation); elsewhere the pass
// writes the effective weights' gradients, which the contraction maps back
static inline int wacc(const cbct_lpd *m, const LayerSpec &L) { return (L.kind || m->wn) ? 0 : 1; }

// channel slots of a hidden activation (or its gradient) with c channels: 32, or 64 for
// the wider blocks
static inline int hs(int c) { return c > 32 ? 64 : 32; }

// forward conv of layer L; the residual epilogue (epi 1) writes state = state_in + conv
static int conv_fwd(cbct_lpd *m, const LayerSpec &L, const __nv_bfloat16 *x, int cpin, int nimg, int D, int H, int W,
                    int epi, __nv_bfloat16 *y, float *state, long long sstride, cudaStream_t st,
                    const float *state_in = nullptr, int zero_state_in = 0, int cpout = 0) {
    return conv_apply(x, nimg, D, H, W, cpin, L.taps3d, m->params + L.fw_off, m->params + L.fb_off, L.cin, L.cout, 0, epi,
                      m->d.slope, y, cpout ? cpout : hs(L.cout), nullptr, state_in, state, sstride, m->status, st,
                      m->wpk + L.pk_off, zero_state_in);
}

// input-gradient conv of layer L: dy (BF16 [..][cp_dy], L.cout channels) -> L.cin outputs
static int conv_dx(cbct_lpd *m, const LayerSpec &L, const __nv_bfloat16 *dy, int cp_dy, int nimg, int D, int H, int W,
                   int epi, __nv_bfloat16 *y, const __nv_bfloat16 *mask, float *state, long long sstride,
                   cudaStream_t st, int cpout = 0, float slope = -1.f) {
    return cbct_conv(dy, nimg, D, H, W, cp_dy, L.taps3d, m->params + L.fw_off, nullptr, L.cin, L.cout, 1, epi,
                     slope < 0.f ? m->d.slope : slope, y, cpout ? cpout : hs(L.cin), mask, state, sstride, m->status, st);
}

// geometry of the two blocks' tensors for a batch of B volumes: dual = B na images of nv x nu
// (2D), primal = B volumes nz x ny x nx (3D)
#define DUAL_DIMS B * m->g->dev.na, 1, m->g->dev.nv, m->g->dev.nu
#define PRIM_DIMS B, m->g->dev.n[2], m->g->dev.n[1], m->g->dev.n[0]

// dual block input [h (M), mu_ref pf, y (, mu_ref pf - y)] of a batch: planes of n elements
static Planes dual_planes(const cbct_lpd *m, const float *h, const float *pf, const float *y) {
    const int M = m->d.n_mem;
    Planes pl{};
    for (int c = 0; c < M; ++c) { pl.p[c] = h ? h + c * (long long)m->batch * m->nproj : nullptr; pl.s[c] = 1.f; }
    pl.p[M] = pf; pl.s[M] = m->d.mu_ref;
    pl.p[M + 1] = y; pl.s[M + 1] = 1.f;
    if (m->d.residual_input) { pl.p[M + 2] = pf; pl.s[M + 2] = m->d.mu_ref; pl.q[M + 2] = y; }
    return pl;
}

// One forward iteration n: (f_in, h_in) -> (f_out, h_out); activations left in the
// workspaces (a1, a2, b1, b2, din, pin).
// pf, bp: where the iteration's P f_1 and P^T (w h_1) go (workspaces, or the per-
// iteration buffers of a training forward). h_zero: h_in is zero and is not read.
// ---- primal block: the three-layer block or the P4 U-Net, from the packed input m->pin ----
// U-Net sizes (full resolution nz x ny x nx, half resolution each halved)
#define UNET_HALF B, m->g->dev.n[2] / 2, m->g->dev.n[1] / 2, m->g->dev.n[0] / 2
#define UNET_FULL_N B, m->g->dev.n[2], m->g->dev.n[1], m->g->dev.n[0]

static int rb_grid(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 32LL * sm_count())); }

// activations of every layer but the last (3-layer block: b1, b2; U-Net: a, s in C, pool(s),
// q, r, up(r) into C, t)
static int prim_hidden(cbct_lpd *m, const LayerSpec *Lp, int B, cudaStream_t st) {
    int rc;
    if (!m->unet) {
        if ((rc = conv_fwd(m, Lp[0], m->pin, 8, PRIM_DIMS, 0, m->b1, nullptr, 0, st))) return rc;
        return conv_fwd(m, Lp[1], m->b1, hs(Lp[1].cin), PRIM_DIMS, 0, m->b2, nullptr, 0, st);
    }
    const int nx = m->g->dev.n[0];
    const long long nvh = (long long)B * m->nvox / 8;
    if ((rc = conv_fwd(m, Lp[0], m->pin, 8, PRIM_DIMS, 0, m->u_a, nullptr, 0, st))) return rc;
    // s = g2(a) into channel groups 4, 5 of C (the epilogue writes groups from the pointer on)
    if ((rc = conv_fwd(m, Lp[1], m->u_a, 32, PRIM_DIMS, 0, m->u_C + 32LL * nx, nullptr, 0, st, nullptr, 0, 64))) return rc;
    k_pool2_rb<<<rb_grid(nvh * 2), 256, 0, st>>>(Rb{m->u_C, 64, 4}, Rb{m->u_p, 32, 0}, 2, UNET_FULL_N, 0.125f);
    if ((rc = conv_fwd(m, Lp[2], m->u_p, 32, UNET_HALF, 0, m->u_q, nullptr, 0, st))) return rc;
    if ((rc = conv_fwd(m, Lp[3], m->u_q, 32, UNET_HALF, 0, m->u_r, nullptr, 0, st))) return rc;
    k_up2_rb<<<rb_grid(nvh * 8 * 4), 256, 0, st>>>(Rb{m->u_r, 32, 0}, Rb{m->u_C, 64, 0}, 4, UNET_FULL_N);
    return conv_fwd(m, Lp[4], m->u_C, 64, PRIM_DIMS, 0, m->u_t, nullptr, 0, st);
}

// the block's output layer and the activation it reads
static const LayerSpec &prim_out(const cbct_lpd *m, const LayerSpec *Lp) { return Lp[m->unet ? 5 : 2]; }
static const __nv_bfloat16 *prim_out_in(const cbct_lpd *m, const LayerSpec *Lp) { return m->unet ? m->u_t : m->b2; }
static int prim_out_cp(const cbct_lpd *m, const LayerSpec *Lp) { return m->unet ? 32 : hs(Lp[2].cin); }

// Backward through the block (activations from prim_hidden): upstream gradient of its
// output in m->gsmall (8 slots); weight and bias gradients into dW; the gradient of the
// block input added to the FP32 planes gdst (channel c into plane map[c], or c).
static int prim_bwd(cbct_lpd *m, const LayerSpec *Lp, int B, float *gdst, long long sstride, const int *map,
                    float *dW, cudaStream_t st) {
    int rc;
    const __nv_bfloat16 *gin;  // gradient at the first layer's output (pre-activation)
    int gcp;
    if (!m->unet) {
        if ((rc = conv_wgrad(m->b2, hs(Lp[2].cin), Lp[2].cin, m->gsmall, 8, Lp[2].cout, PRIM_DIMS, 1, dW + Lp[2].fw_off,
                             dW + Lp[2].fb_off, wacc(m, Lp[2]), m->status, st))) return rc;
        if ((rc = conv_dx(m, Lp[2], m->gsmall, 8, PRIM_DIMS, 2, m->g32a, m->b2, nullptr, 0, st))) return rc;
        if ((rc = conv_wgrad(m->b1, hs(Lp[1].cin), Lp[1].cin, m->g32a, hs(Lp[1].cout), Lp[1].cout, PRIM_DIMS, 1,
                             dW + Lp[1].fw_off, dW + Lp[1].fb_off, wacc(m, Lp[1]), m->status, st))) return rc;
        if ((rc = conv_dx(m, Lp[1], m->g32a, hs(Lp[1].cout), PRIM_DIMS, 2, m->g32b, m->b1, nullptr, 0, st))) return rc;
        gin = m->g32b;
        gcp = hs(Lp[0].cout);
    } else {
        const long long nvh = (long long)B * m->nvox / 8;
        auto wg = [&](const LayerSpec &L, const __nv_bfloat16 *x, int cpx, const __nv_bfloat16 *dy, int cpy, int half) {
            return half ? conv_wgrad(x, cpx, L.cin, dy, cpy, L.cout, UNET_HALF, 1, dW + L.fw_off, dW + L.fb_off, 0,
                                     m->status, st)
                        : conv_wgrad(x, cpx, L.cin, dy, cpy, L.cout, PRIM_DIMS, 1, dW + L.fw_off, dW + L.fb_off, 0,
                                     m->status, st);
        };
        // out = avg6(t): dt (masked by t) in u_ga
        if ((rc = wg(Lp[5], m->u_t, 32, m->gsmall, 8, 0))) return rc;
        if ((rc = conv_dx(m, Lp[5], m->gsmall, 8, PRIM_DIMS, 2, m->u_ga, m->u_t, nullptr, 0, st, 32))) return rc;
        // t = g5(C): dC (masked by C) in g32b, 48 channels in 64 slots
        if ((rc = wg(Lp[4], m->u_C, 64, m->u_ga, 32, 0))) return rc;
        if ((rc = conv_dx(m, Lp[4], m->u_ga, 32, PRIM_DIMS, 2, m->g32b, m->u_C, nullptr, 0, st, 64))) return rc;
        // C[0..8F) = up(r): dr = block sums of dC's first 4 groups (half resolution, u_h1)
        k_pool2_rb<<<rb_grid(nvh * 4), 256, 0, st>>>(Rb{m->g32b, 64, 0}, Rb{m->u_h1, 32, 0}, 4, UNET_FULL_N, 1.f);
        if ((rc = wg(Lp[3], m->u_q, 32, m->u_h1, 32, 1))) return rc;
        if ((rc = conv_dx(m, Lp[3], m->u_h1, 32, UNET_HALF, 2, m->u_h2, m->u_q, nullptr, 0, st, 32))) return rc;
        if ((rc = wg(Lp[2], m->u_p, 32, m->u_h2, 32, 1))) return rc;
        // d pool(s): no activation after the pooling (slope 1 leaves the sum as it is), 16 slots
        if ((rc = conv_dx(m, Lp[2], m->u_h2, 32, UNET_HALF, 0, m->u_h1, nullptr, nullptr, 0, st, 16, 1.f))) return rc;
        // ds = dC's groups 4, 5 (masked) + mask(s) x pool adjoint, into u_ga
        k_skip_grad_rb<<<rb_grid(nvh * 8 * 2), 256, 0, st>>>(Rb{m->g32b, 64, 4}, Rb{m->u_C, 64, 4}, Rb{m->u_h1, 16, 0},
                                                              Rb{m->u_ga, 32, 0}, 2, UNET_FULL_N, m->d.slope);
        if ((rc = wg(Lp[1], m->u_a, 32, m->u_ga, 32, 0))) return rc;
        if ((rc = conv_dx(m, Lp[1], m->u_ga, 32, PRIM_DIMS, 2, m->u_gb, m->u_a, nullptr, 0, st, 32))) return rc;
        gin = m->u_gb;
        gcp = 32;
    }
    if ((rc = conv_wgrad(m->pin, 8, Lp[0].cin, gin, gcp, Lp[0].cout, PRIM_DIMS, 1, dW + Lp[0].fw_off, dW + Lp[0].fb_off,
                         wacc(m, Lp[0]), m->status, st))) return rc;
    return conv_apply(gin, PRIM_DIMS, gcp, 1, m->params + Lp[0].fw_off, nullptr, Lp[0].cin, Lp[0].cout, 1, 1,
                      m->d.slope, nullptr, 32, nullptr, gdst, gdst, sstride, m->status, st, nullptr, 0, map, 0);
}

static int lpd_iter_fwd(cbct_lpd *m, int n, const float *f_in, const float *h_in, float *f_out, float *h_out,
                        float *pf, float *bp, cudaStream_t st, bool h_zero = false) {
    const int B = m->batch;
    const long long NV = m->nvox * B, NP = m->nproj * B;  // one channel of the batch
    const int M = m->d.n_mem;
    const LayerSpec *Ld = &m->layers[m->dual_at[n]], *Lp = &m->layers[m->prim_at[n]];
    void *sv = (void *)st;
    // dual block input [h (M), mu_ref P f_1, y (, mu_ref P f_1 - y)]
    int rc = forward_project(m->g, f_in + 1 * NV, pf, B, 0, sv);
    if (rc) return rc;
    const Planes pl = dual_planes(m, h_zero ? nullptr : h_in, pf, m->y);
    k_pack8<<<grid_n(NP), 256, 0, st>>>(pl, NP, m->din);
    if ((rc = conv_fwd(m, Ld[0], m->din, 8, DUAL_DIMS, 0, m->a1, nullptr, 0, st))) return rc;
    if ((rc = conv_fwd(m, Ld[1], m->a1, hs(Ld[1].cin), DUAL_DIMS, 0, m->a2, nullptr, 0, st))) return rc;
    if ((rc = conv_fwd(m, Ld[2], m->a2, hs(Ld[2].cin), DUAL_DIMS, 1, nullptr, h_out, NP, st, h_in, h_zero))) return rc;
    // primal block input [f (M), bp_scale P^T (w h_1)]
    rc = back_project_colw(m->g, h_out + 1 * NP, m->wred, bp, B, 0, st);
    if (rc) return rc;
    Planes pp{};
    for (int c = 0; c < M; ++c) { pp.p[c] = f_in + c * NV; pp.s[c] = 1.f; }
    pp.p[M] = bp; pp.s[M] = m->bp_scale;
    k_pack8<<<grid_n(NV), 256, 0, st>>>(pp, NV, m->pin);
    if ((rc = prim_hidden(m, Lp, B, st))) return rc;
    if ((rc = conv_fwd(m, prim_out(m, Lp), prim_out_in(m, Lp), prim_out_cp(m, Lp), PRIM_DIMS, 1, nullptr, f_out, NV, st,
                       f_in))) return rc;
    CBCT_LAUNCH_CHECK("lpd iteration");
    return 0;
}

extern "C" int lpd_create(const cbct_geom *g, const cbct_lpd_desc *desc, cbct_lpd **out) {
    if (!g || !desc || !out) return fail(CBCT_EINVAL, "lpd_create: NULL argument");
    *out = nullptr;
    const cbct_lpd_desc &d = *desc;
    const int maxb = d.max_batch < 1 ? 1 : d.max_batch;
    const bool rev = d.reversible != 0;
    const bool mem_ok = rev ? (d.n_mem >= 2 && d.n_mem <= 8 && d.n_mem % 2 == 0)
                            : (d.n_mem >= 2 && d.n_mem <= 6 && (!d.residual_input || d.n_mem <= 5));
    if (d.n_iter < 1 || d.n_iter > 64 || !mem_ok || (d.width != 32 && d.width != 64) || !(d.mu_ref > 0) ||
        !(d.slope >= 0.f && d.slope <= 1.f) || (d.residual_input != 0 && d.residual_input != 1) ||
        (d.reversible != 0 && d.reversible != 1) || (d.lire != 0 && d.lire != 1) || (d.lire && !rev) ||
        (d.lire && d.residual_input) || maxb > 64 || (long long)maxb * g->dev.na * (d.lire ? 2 : 1) > 65535)
        return fail(CBCT_EINVAL, "lpd_create: need 1 <= n_iter <= 64, width 32 or 64, mu_ref > 0, 0 <= slope <= 1, "
                                 "residual_input and reversible 0 or 1, max_batch <= 64, max_batch * n_angles <= "
                                 "65535 (half that with lire), and 2 <= n_mem <= 6 (<= 5 with the residual channel) or, reversible, "
                                 "n_mem even in [2, 8]; lire needs reversible and no residual_input");
    if ((d.unet != 0 && d.unet != 1) || (d.weight_norm != 0 && d.weight_norm != 1) ||
        (d.unet && (!d.p4 || g->dev.n[0] % 2 || g->dev.n[1] % 2 || g->dev.n[2] % 2)))
        return fail(CBCT_EINVAL, "lpd_create: unet and weight_norm are 0 or 1; unet needs p4 and even volume sizes "
                                 "(2 x 2 x 2 pooling)");
    cbct_lpd *m = new (std::nothrow) cbct_lpd();
    if (!m) return fail(CBCT_ENOMEM, "lpd_create: host allocation");
    m->g = g;
    m->d = d;
    m->maxb = maxb;
    m->unet = d.unet;
    const int K = rev ? d.n_mem / 2 : d.n_mem;  // channels a block reads from / writes to each state
    m->nd = K + 2 + d.residual_input;
    m->nvox = (long long)g->dev.n[0] * g->dev.n[1] * g->dev.n[2];
    m->nproj = (long long)g->dev.na * g->dev.nv * g->dev.nu;
    const int M = d.n_mem, W = d.width;
    long long off = 0;
    auto add = [&](int cin, int cout, int t3, int H, int cpin, int last) {
        LayerSpec L;
        L.cin = cin; L.cout = cout; L.taps3d = t3; L.H = H; L.cpin = cpin; L.last = last;
        L.w_off = off; off += (long long)cout * (t3 ? 27 : 9) * cin;
        L.b_off = off; off += cout;
        if (d.weight_norm) { L.g_off = off; off += 1; }
        L.fw_off = L.w_off; L.fb_off = L.b_off;
        m->layers.push_back(L);
    };
    // P4 primal layers (3x3x3, width = 4 x 8 group channels): base filters [cb][27][cin]
    // (lifting) or [cb][4][27][cib] (group, averaged), biases [cb]; the full weights they
    // expand to are placed after all learnable parameters (below)
    constexpr int kP4Base = 8;
    auto add_p4 = [&](int kind, int cin_full, int cout_full, int H, int cpin, int last) {
        LayerSpec L;
        L.kind = kind; L.taps3d = 1; L.H = H; L.cin = cin_full; L.cout = cout_full; L.cpin = cpin; L.last = last;
        L.cb = kind == 3 ? cout_full : cout_full / 4;
        L.cib = kind == 1 ? cin_full : cin_full / 4;
        L.w_off = off; off += (long long)L.cb * (kind == 1 ? 1 : 4) * 27 * L.cib;
        L.b_off = off; off += L.cb;
        if (d.weight_norm) { L.g_off = off; off += 1; }
        m->layers.push_back(L);
    };
    // U-Net: 4F group channels (16) at full resolution in 32 slots (the upper 16 stay zero, so
    // the weight gradients run on the tensor cores), 8F at half resolution (32), the
    // concatenation [up(r), s] of 12F channels in 64 slots
    constexpr int kUF = 4;
    auto add_primal = [&](int cin, int H) {
        if (d.unet) {
            add_p4(1, cin, 4 * kUF, H, 8, 0);                  // a = lift(x)
            add_p4(2, 4 * kUF, 4 * kUF, H, 32, 0);             // s = g2(a)
            add_p4(2, 4 * kUF, 8 * kUF, H / 2, 32, 0);         // q = g3(pool(s))
            add_p4(2, 8 * kUF, 8 * kUF, H / 2, 32, 0);         // r = g4(q)
            add_p4(2, 12 * kUF, 4 * kUF, H, 64, 0);            // t = g5([up(r), s])
            add_p4(3, 4 * kUF, K, H, 32, 1);                   // group average
        } else if (d.p4) {
            add_p4(1, cin, 4 * kP4Base, H, 8, 0); add_p4(2, 4 * kP4Base, 4 * kP4Base, H, 32, 0);
            add_p4(3, 4 * kP4Base, K, H, 32, 1);
        } else {
            add(cin, W, 1, H, 8, 0); add(W, W, 1, H, hs(W), 0); add(W, K, 1, H, hs(W), 1);
        }
    };
    for (int n = 0; n < d.n_iter; ++n) {
        const int nv = g->dev.nv, ny = g->dev.n[1];
        m->dual_at.push_back((int)m->layers.size());
        if (d.lire) {
            // Algorithm 1 blocks: 3x3x3 over (angle, v, u) and over the volume, K + 4 inputs each,
            // then the output convolution's omega [n_mem] and beta
            add(K + 4, W, 1, nv, 8, 0); add(W, W, 1, nv, hs(W), 0); add(W, K, 1, nv, hs(W), 1);   // dual
            m->prim_at.push_back((int)m->layers.size());
            add_primal(K + 4, ny);                                                                // primal
            m->out_off.push_back(off);
            off += M + 1;
        } else {
            add(m->nd, W, 0, nv, 8, 0); add(W, W, 0, nv, hs(W), 0); add(W, K, 0, nv, hs(W), 1);   // dual
            m->prim_at.push_back((int)m->layers.size());
            add_primal(K + 1, ny);                                                                // primal
        }
    }
    m->nparams = off;
    // weight normalisation: the normalised filters of every layer (a plain layer's convolution
    // weights, with a copy of its biases; a P4 layer's base filters, expanded below)
    std::vector<WnJob> wnjobs;
    if (d.weight_norm) {
        m->wn = 1;
        m->wn_lo = off;
        for (LayerSpec &L : m->layers) {
            const int rows = L.kind ? L.cb : L.cout;
            const int len = (int)((L.b_off - L.w_off) / rows);
            L.nw_off = off; off += (long long)rows * len;
            WnJob j{L.w_off, L.nw_off, L.g_off, rows, len, 0, 0, 0};
            if (!L.kind) {
                L.fw_off = L.nw_off;
                L.fb_off = off; off += L.cout;
                j.b_raw = L.b_off; j.b_dst = L.fb_off; j.nb = L.cout;
            }
            wnjobs.push_back(j);
        }
        m->wn_hi = off;
        m->n_wn = (int)wnjobs.size();
    }
    // expansion area of the P4 layers: full weights [cout][27][cin] and biases, after the
    // learnable parameters (the same offsets in the gradient buffer hold full gradients)
    std::vector<P4Job> p4jobs;
    for (LayerSpec &L : m->layers) {
        if (!L.kind) continue;
        L.fw_off = off; off += (long long)L.cout * 27 * L.cin;
        L.fb_off = off; off += L.cout;
        p4jobs.push_back(P4Job{L.kind, L.cb, L.cib, L.cout, L.cin, m->wn ? L.nw_off : L.w_off, L.b_off, L.fw_off,
                               L.fb_off, m->wn});
        m->p4_max = std::max(m->p4_max, (long long)L.cout * 27 * L.cin);
    }
    m->n_p4 = (int)p4jobs.size();
    m->nexp = off - m->nparams;
    // initial weights: He normal for hidden layers, 0.1 x that for the last layer of each block
    std::vector<float> hp(off, 0.f);
    InitRng rng{d.seed};
    for (size_t i = 0; i < m->layers.size(); ++i) {
        const LayerSpec &L = m->layers[i];
        const int taps = L.taps3d ? 27 : 9;
        const double sd = sqrt(2.0 / (L.cin * taps)) * (L.last ? 0.1 : 1.0);  // fan-in of the full layer
        const long long nw = L.b_off - L.w_off;
        for (long long k = 0; k < nw; ++k) hp[L.w_off + k] = (float)(sd * rng.normal());
        // gain = the expected norm of the He-initialised filter (sqrt 2, 10x smaller for the last layer)
        if (L.g_off >= 0) hp[L.g_off] = (float)(sqrt(2.0) * (L.last ? 0.1 : 1.0));
    }
    for (long long o : m->out_off)
        for (int c = 0; c < M; ++c) hp[o + c] = (float)(0.01 * rng.normal());  // omega; beta = 0
    if (rev) {
        // per iteration a primal and a dual permutation that mix the halves (Fisher-Yates on
        // the same SplitMix64 stream, redrawn until the new first half takes a channel of the
        // old second half)
        auto draw = [&](std::vector<int> &p) {
            p.resize(M);
            do {
                for (int c = 0; c < M; ++c) p[c] = c;
                for (int c = M - 1; c > 0; --c) std::swap(p[c], p[(int)(rng.next() % (uint64_t)(c + 1))]);
            } while (!perm_mixes(p.data(), M));
        };
        m->perm_f.resize(d.n_iter);
        m->perm_h.resize(d.n_iter);
        for (int n = 0; n < d.n_iter; ++n) { draw(m->perm_f[n]); draw(m->perm_h[n]); }
    }
    const long long NV = m->nvox * maxb, NP = m->nproj * maxb;  // one channel of a full batch
    const int S = rev ? 1 : d.n_iter + 1;  // stored state slots: every iterate, or the last one
    const int NI = rev ? 0 : d.n_iter;     // stored projector outputs
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    al((void **)&m->params, sizeof(float) * off);
    al((void **)&m->grads, sizeof(float) * off);
    al((void **)&m->adam_m, sizeof(float) * m->nparams);
    al((void **)&m->adam_v, sizeof(float) * m->nparams);
    if (m->n_p4) al((void **)&m->p4_jobs, sizeof(P4Job) * m->n_p4);
    if (m->n_wn) al((void **)&m->wn_jobs, sizeof(WnJob) * m->n_wn);
    al((void **)&m->wred, sizeof(float) * g->dev.nu);
    al((void **)&m->f, sizeof(float) * S * M * NV);
    al((void **)&m->h, sizeof(float) * S * M * NP);
    al((void **)&m->y, sizeof(float) * NP);
    al((void **)&m->tproj, sizeof(float) * NP);
    al((void **)&m->tproj2, sizeof(float) * NP);
    al((void **)&m->tvol, sizeof(float) * NV);
    al((void **)&m->pf_saved, sizeof(float) * std::max(1, NI) * NP);
    al((void **)&m->clip, sizeof(double) * (608 + 2));
    al((void **)&m->bp_saved, sizeof(float) * std::max(1, NI) * NV);
    al((void **)&m->din, sizeof(__nv_bfloat16) * NP * 8);
    // hidden activations: dual layers at the model width, primal layers at it too (P4: 4 x 8)
    const int sd = hs(W), sp = d.unet ? 64 : (d.p4 ? 32 : hs(W));
    al((void **)&m->a1, sizeof(__nv_bfloat16) * NP * sd);
    al((void **)&m->a2, sizeof(__nv_bfloat16) * NP * sd);
    al((void **)&m->pin, sizeof(__nv_bfloat16) * NV * 8);
    al((void **)&m->b1, sizeof(__nv_bfloat16) * NV * (d.unet ? 8 : sp));
    al((void **)&m->b2, sizeof(__nv_bfloat16) * NV * (d.unet ? 8 : sp));
    if (d.unet) {
        al((void **)&m->u_a, sizeof(__nv_bfloat16) * NV * 32);
        al((void **)&m->u_C, sizeof(__nv_bfloat16) * NV * 64);
        al((void **)&m->u_t, sizeof(__nv_bfloat16) * NV * 32);
        al((void **)&m->u_p, sizeof(__nv_bfloat16) * (NV / 8) * 32);
        al((void **)&m->u_q, sizeof(__nv_bfloat16) * (NV / 8) * 32);
        al((void **)&m->u_r, sizeof(__nv_bfloat16) * (NV / 8) * 32);
        al((void **)&m->u_h1, sizeof(__nv_bfloat16) * (NV / 8) * 32);
        al((void **)&m->u_h2, sizeof(__nv_bfloat16) * (NV / 8) * 32);
        al((void **)&m->u_ga, sizeof(__nv_bfloat16) * NV * 32);
        al((void **)&m->u_gb, sizeof(__nv_bfloat16) * NV * 32);
        // 16-channel tensors in 32 slots: the upper slots are never written and stay zero
        for (__nv_bfloat16 *z : {m->u_a, m->u_t, m->u_p, m->u_ga, m->u_gb})
            if (e == cudaSuccess && z) e = cudaMemset(z, 0, sizeof(__nv_bfloat16) * (z == m->u_p ? NV / 8 : NV) * 32);
    }
    al((void **)&m->g32a, sizeof(__nv_bfloat16) * std::max(NP * sd, NV * sp));
    al((void **)&m->g32b, sizeof(__nv_bfloat16) * std::max(NP * sd, NV * sp));
    al((void **)&m->gsmall, sizeof(__nv_bfloat16) * std::max(NP, NV) * 8);
    al((void **)&m->gf, sizeof(float) * (M + 4) * NV);
    al((void **)&m->gh, sizeof(float) * (M + 5) * NP);
    if (d.lire) {
        al((void **)&m->x, sizeof(float) * NV);
        al((void **)&m->gx, sizeof(float) * NV);
        al((void **)&m->Vb, sizeof(float) * NV);
        al((void **)&m->t2v, sizeof(float) * 2 * NV);
        al((void **)&m->t2p, sizeof(float) * 2 * NP);
        al((void **)&m->opart, sizeof(float) * kOutBlocks * (M + 1));
    }
    al((void **)&m->status, sizeof(int));
    // forward convolutions: packing plan of every layer (first layer of a block reads 8
    // channel slots, the others the hidden width; 2-D blocks run over the nv rows, 3-D
    // over ny), one job per launch of at most 32 outputs
    std::vector<ConvPackJob> jobs;
    long long pk_bytes = 0;
    for (size_t i = 0; i < m->layers.size(); ++i) {
        LayerSpec &L = m->layers[i];
        ConvPackJob lj[kConvMaxOut / 32];
        const long long b = conv_plan(L.taps3d, L.H, L.cpin, L.cin, L.cout, 0, lj);
        if (b < 0) {
            lpd_destroy(m);
            return fail(CBCT_EINVAL, "lpd_create: no convolution plan for layer " + std::to_string(i));
        }
        L.pk_off = pk_bytes;
        for (int h = 0; h < conv_halves(L.cout); ++h) {
            lj[h].w_off = L.fw_off;
            lj[h].out_off += pk_bytes;
            jobs.push_back(lj[h]);
            m->pack_max_nelem = std::max(m->pack_max_nelem, lj[h].nelem);
        }
        pk_bytes += b;
    }
    m->n_pack_jobs = (int)jobs.size();
    al((void **)&m->wpk, (size_t)pk_bytes);
    al((void **)&m->pack_jobs, sizeof(ConvPackJob) * jobs.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(m->pack_jobs, jobs.data(), sizeof(ConvPackJob) * jobs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->params, hp.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->grads, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(m->adam_m, 0, sizeof(float) * m->nparams);
    if (e == cudaSuccess) e = cudaMemset(m->adam_v, 0, sizeof(float) * m->nparams);
    if (e == cudaSuccess && m->n_p4)
        e = cudaMemcpy(m->p4_jobs, p4jobs.data(), sizeof(P4Job) * m->n_p4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m->n_wn)
        e = cudaMemcpy(m->wn_jobs, wnjobs.data(), sizeof(WnJob) * m->n_wn, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->status, 0, sizeof(int));
    if (e != cudaSuccess) {
        lpd_destroy(m);
        return cuda_fail(e, "lpd_create: allocation");
    }
    int rc = cbct_redundancy_weight(g, m->wred, nullptr);
    if (rc == 0 && d.lire) {
        // the FoV tensor V (a primal input of Algorithm 1), once per batch item
        rc = cbct_fov(g, m->Vb, nullptr);
        for (int b = 1; b < maxb && rc == 0; ++b) {
            e = cudaMemcpy(m->Vb + b * m->nvox, m->Vb, sizeof(float) * m->nvox, cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess) rc = cuda_fail(e, "lpd_create: FoV copies");
        }
    }
    // backprojection scale: 1 / max_voxel P^T(w 1)
    if (rc == 0) {
        if (d.bp_scale > 0) {
            m->bp_scale = d.bp_scale;
        } else {
            k_fill_f<<<grid_n(m->nproj), 256>>>(m->tproj2, m->nproj, 1.f);
            rc = back_project_colw(g, m->tproj2, m->wred, m->tvol, 1, 0, nullptr);
            float mx = 0.f;
            if (rc == 0) {
                cudaMemset(m->tproj2, 0, sizeof(float));
                k_max_reduce<<<grid_n(m->nvox), 256>>>(m->tvol, m->nvox, m->tproj2);
                e = cudaMemcpy(&mx, m->tproj2, sizeof(float), cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) rc = cuda_fail(e, "lpd_create: bp scale");
            }
            m->bp_scale = mx > 0.f ? 1.f / mx : 1.f;
        }
    }
    if (rc == 0) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_fail(e, "lpd_create");
    }
    if (rc) {
        lpd_destroy(m);
        return rc;
    }
    *out = m;
    return 0;
}

extern "C" void lpd_destroy(cbct_lpd *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    void *ptrs[] = {m->p4_jobs, m->wn_jobs, m->x, m->gx, m->Vb, m->t2v, m->t2p, m->opart, m->wpk, m->pack_jobs, m->clip, m->pf_saved, m->bp_saved, m->params, m->grads, m->adam_m, m->adam_v, m->wred, m->f, m->h,
                    m->y, m->tproj, m->tproj2, m->tvol, m->din, m->a1, m->a2, m->pin, m->b1, m->b2, m->g32a, m->g32b, m->gsmall, m->gf, m->gh,
                    m->u_a, m->u_C, m->u_t, m->u_p, m->u_q, m->u_r, m->u_h1, m->u_h2, m->u_ga, m->u_gb,
                    m->status};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

extern "C" int lpd_get_perms(const cbct_lpd *m, int *host) {
    if (!m || !host || !m->d.reversible) return fail(CBCT_EINVAL, "lpd_get_perms: need a reversible model");
    const int M = m->d.n_mem;
    for (int n = 0; n < m->d.n_iter; ++n)
        for (int c = 0; c < M; ++c) {
            host[(2 * n) * M + c] = m->perm_f[n][c];
            host[(2 * n + 1) * M + c] = m->perm_h[n][c];
        }
    return 0;
}

extern "C" int lpd_set_perms(cbct_lpd *m, const int *host) {
    if (!m || !host || !m->d.reversible) return fail(CBCT_EINVAL, "lpd_set_perms: need a reversible model");
    const int M = m->d.n_mem;
    for (int r = 0; r < 2 * m->d.n_iter; ++r) {
        const int *p = host + r * M;
        int seen = 0;
        for (int c = 0; c < M; ++c) {
            if (p[c] < 0 || p[c] >= M || (seen >> p[c]) & 1) return fail(CBCT_EINVAL, "lpd_set_perms: not a permutation");
            seen |= 1 << p[c];
        }
        if (!perm_mixes(p, M)) return fail(CBCT_EINVAL, "lpd_set_perms: a permutation does not mix the halves");
    }
    for (int n = 0; n < m->d.n_iter; ++n) {
        m->perm_f[n].assign(host + (2 * n) * M, host + (2 * n) * M + M);
        m->perm_h[n].assign(host + (2 * n + 1) * M, host + (2 * n + 1) * M + M);
    }
    return 0;
}

extern "C" int lpd_info(const cbct_lpd *m, long long *nparams, float **params, float **grads, float *bp_scale) {
    if (!m) return fail(CBCT_EINVAL, "lpd_info: NULL model");
    if (nparams) *nparams = m->nparams;
    if (params) *params = m->params;
    if (grads) *grads = m->grads;
    if (bp_scale) *bp_scale = m->bp_scale;
    return 0;
}

// Forward pass of a batch of B volumes from the initial states f_0 (f0, or x0 / mu_ref in
// every channel) and h_0 (h0, or zero); x_out = mu_ref f_N[0] when given. The final states
// stay in the model (slot N with save_for_backward, else slot 0) for lpd_get_state.
static int lpd_forward_impl(cbct_lpd *m, const float *y, const float *x0, const float *f0, const float *h0,
                            float *x_out, int save_for_backward, int B, cudaStream_t st) {
    m->batch = B;
    const long long NV = m->nvox * B, NP = m->nproj * B;
    const int M = m->d.n_mem, N = m->d.n_iter;
    weights_expand(m, st);
    int prc = conv_pack_jobs(m->pack_jobs, m->n_pack_jobs, m->pack_max_nelem, m->params, m->wpk, st);
    if (prc) return prc;
    CBCT_CUDA_TRY(cudaMemcpyAsync(m->y, y, sizeof(float) * NP, cudaMemcpyDeviceToDevice, st));
    if (f0) {
        CBCT_CUDA_TRY(cudaMemcpyAsync(m->f, f0, sizeof(float) * M * NV, cudaMemcpyDeviceToDevice, st));
    } else {
        k_init_f<<<grid_n(NV), 256, 0, st>>>(x0, m->f, NV, M, 1.f / m->d.mu_ref);
    }
    // h_0 = 0: an inference pass does not store it (the first dual block reads no h);
    // a training pass keeps it for the backward
    const bool h_zero = !h0 && !save_for_backward;
    if (h0) {
        CBCT_CUDA_TRY(cudaMemcpyAsync(m->h, h0, sizeof(float) * M * NP, cudaMemcpyDeviceToDevice, st));
    } else if (!h_zero) {
        CBCT_CUDA_TRY(cudaMemsetAsync(m->h, 0, sizeof(float) * M * NP, st));
    }
    for (int n = 0; n < N; ++n) {
        const int si = save_for_backward ? n : 0, so = save_for_backward ? n + 1 : 0;
        float *pf = save_for_backward ? m->pf_saved + (long long)n * NP : m->tproj;
        float *bp = save_for_backward ? m->bp_saved + (long long)n * NV : m->tvol;
        int rc = lpd_iter_fwd(m, n, m->f + (long long)si * M * NV, m->h + (long long)si * M * NP,
                              m->f + (long long)so * M * NV, m->h + (long long)so * M * NP, pf, bp, st,
                              h_zero && n == 0);
        if (rc) return rc;
    }
    const long long last = save_for_backward ? N : 0;
    if (x_out) k_sum_channels<<<grid_n(NV), 256, 0, st>>>(m->f + last * M * NV, 1, NV, m->d.mu_ref, x_out, 0);
    m->saved = save_for_backward;
    m->last = (int)last;
    CBCT_LAUNCH_CHECK("lpd_forward");
    return 0;
}

// ---- reversible mode: additive coupling and channel permutations (Algorithm 1) ----------
//
// The states f = [p1, p2], h = [d1, d2] (halves of K = n_mem / 2 channels) live in
// n_mem planes each; which plane holds logical channel c is tracked on the host
// (pf[c], ph[c]), so a permutation moves no data. Per iteration n:
//   d2 <- d2 + Gamma_n([d1, mu_ref P p2[0], y (, mu_ref P p2[0] - y)])
//   p2 <- p2 + Lambda_n([p1, bp_scale P^T (w d2[0])])
//   f <- f[perm_f[n]], h <- h[perm_h[n]]
// Each update reads only the half it leaves unchanged, so the backward pass recovers
// every iterate from the final states by undoing the permutations and subtracting the
// same block outputs in reverse order (the kernels are deterministic, so a recomputed
// block output equals the forward one bit for bit): no iterate is stored.

// plane map after applying permutation p: new[c] = old[p[c]]
static void map_permute(int *map, const std::vector<int> &p, int M) {
    int t[8];
    for (int c = 0; c < M; ++c) t[c] = map[p[c]];
    for (int c = 0; c < M; ++c) map[c] = t[c];
}
// inverse: old[p[c]] = new[c]
static void map_unpermute(int *map, const std::vector<int> &p, int M) {
    int t[8];
    for (int c = 0; c < M; ++c) t[p[c]] = map[c];
    for (int c = 0; c < M; ++c) map[c] = t[c];
}

static Planes rev_dual_planes(const cbct_lpd *m, const float *h, const int *ph, long long NP, const float *pf,
                              const float *y) {
    const int K = m->d.n_mem / 2;
    Planes pl{};
    for (int c = 0; c < K; ++c) { pl.p[c] = h + ph[c] * NP; pl.s[c] = 1.f; }
    pl.p[K] = pf; pl.s[K] = m->d.mu_ref;
    pl.p[K + 1] = y; pl.s[K + 1] = 1.f;
    if (m->d.residual_input) { pl.p[K + 2] = pf; pl.s[K + 2] = m->d.mu_ref; pl.q[K + 2] = y; }
    return pl;
}

static Planes rev_primal_planes(const cbct_lpd *m, const float *f, const int *pfm, long long NV, const float *bp) {
    const int K = m->d.n_mem / 2;
    Planes pp{};
    for (int c = 0; c < K; ++c) { pp.p[c] = f + pfm[c] * NV; pp.s[c] = 1.f; }
    pp.p[K] = bp; pp.s[K] = m->bp_scale;
    return pp;
}

// block output conv (layer 3) as a residual update of the mapped second-half planes
// (ssub = 1 subtracts it again)
static int rev_update(cbct_lpd *m, const LayerSpec &L, const __nv_bfloat16 *act, int nimg, int D, int H, int W,
                      float *state, const int *map2, long long sstride, int ssub, cudaStream_t st) {
    return conv_apply(act, nimg, D, H, W, L.cpin, L.taps3d, m->params + L.fw_off, m->params + L.fb_off, L.cin, L.cout,
                      0, 1, m->d.slope, nullptr, 32, nullptr, state, state, sstride, m->status, st, m->wpk + L.pk_off, 0,
                      map2, ssub);
}

static int lpd_rev_forward(cbct_lpd *m, const float *y, const float *x0, float *x_out, int save_for_backward, int B,
                           cudaStream_t st) {
    m->batch = B;
    void *sv = (void *)st;
    const long long NV = m->nvox * B, NP = m->nproj * B;
    const int M = m->d.n_mem, K = M / 2, N = m->d.n_iter;
    weights_expand(m, st);
    int rc = conv_pack_jobs(m->pack_jobs, m->n_pack_jobs, m->pack_max_nelem, m->params, m->wpk, st);
    if (rc) return rc;
    CBCT_CUDA_TRY(cudaMemcpyAsync(m->y, y, sizeof(float) * NP, cudaMemcpyDeviceToDevice, st));
    k_init_f<<<grid_n(NV), 256, 0, st>>>(x0, m->f, NV, M, 1.f / m->d.mu_ref);
    CBCT_CUDA_TRY(cudaMemsetAsync(m->h, 0, sizeof(float) * M * NP, st));
    int pfm[8], phm[8];
    for (int c = 0; c < M; ++c) pfm[c] = phm[c] = c;
    for (int n = 0; n < N && rc == 0; ++n) {
        const LayerSpec *Ld = &m->layers[m->dual_at[n]], *Lp = &m->layers[m->prim_at[n]];
        // dual: d2 += Gamma([d1, mu_ref P p2[0], y (, residual)])
        if ((rc = forward_project(m->g, m->f + pfm[K] * NV, m->tproj, B, 0, sv))) break;
        const Planes pl = rev_dual_planes(m, m->h, phm, NP, m->tproj, m->y);
        k_pack8<<<grid_n(NP), 256, 0, st>>>(pl, NP, m->din);
        if ((rc = conv_fwd(m, Ld[0], m->din, 8, DUAL_DIMS, 0, m->a1, nullptr, 0, st))) break;
        if ((rc = conv_fwd(m, Ld[1], m->a1, hs(Ld[1].cin), DUAL_DIMS, 0, m->a2, nullptr, 0, st))) break;
        if ((rc = rev_update(m, Ld[2], m->a2, DUAL_DIMS, m->h, phm + K, NP, 0, st))) break;
        // primal: p2 += Lambda([p1, bp_scale P^T (w d2[0])])
        if ((rc = back_project_colw(m->g, m->h + phm[K] * NP, m->wred, m->tvol, B, 0, st))) break;
        const Planes pp = rev_primal_planes(m, m->f, pfm, NV, m->tvol);
        k_pack8<<<grid_n(NV), 256, 0, st>>>(pp, NV, m->pin);
        if ((rc = prim_hidden(m, Lp, B, st))) break;
        if ((rc = rev_update(m, prim_out(m, Lp), prim_out_in(m, Lp), PRIM_DIMS, m->f, pfm + K, NV, 0, st))) break;
        map_permute(pfm, m->perm_f[n], M);
        map_permute(phm, m->perm_h[n], M);
    }
    if (rc) return rc;
    if (x_out) k_sum_channels<<<grid_n(NV), 256, 0, st>>>(m->f + pfm[0] * NV, 1, NV, m->d.mu_ref, x_out, 0);
    for (int c = 0; c < M; ++c) { m->fin_f[c] = m->cur_f[c] = pfm[c]; m->fin_h[c] = m->cur_h[c] = phm[c]; }
    m->saved = save_for_backward;
    m->last = 0;
    CBCT_LAUNCH_CHECK("lpd_forward (reversible)");
    return 0;
}

// Backward by inversion: from the final states, each iteration (last first) is undone —
// permutations reversed, p2 -= Lambda(...), d2 -= Gamma(...) — while the gradients run
// through the same blocks. The states end at the recovered initial states.
static int lpd_rev_backward(cbct_lpd *m, const float *grad_x, float *grad_y, float *grad_x0, cudaStream_t st) {
    void *sv = (void *)st;
    const int B = m->batch;
    const long long NV = m->nvox * B, NP = m->nproj * B;
    const int M = m->d.n_mem, K = M / 2, N = m->d.n_iter;
    float *gf = m->gf, *gh = m->gh, *dW = m->grads;  // gf: M planes + plane M (scratch); gh: M + 3 planes
    weights_expand(m, st);
    int rc = conv_pack_jobs(m->pack_jobs, m->n_pack_jobs, m->pack_max_nelem, m->params, m->wpk, st);
    if (rc) return rc;
    int pfm[8], phm[8];
    for (int c = 0; c < M; ++c) { pfm[c] = m->fin_f[c]; phm[c] = m->fin_h[c]; }
    cudaMemsetAsync(gf, 0, sizeof(float) * (M + 1) * NV, st);
    cudaMemsetAsync(gh, 0, sizeof(float) * (M + 3) * NP, st);
    k_axpy<<<grid_n(NV), 256, 0, st>>>(gf + pfm[0] * NV, grad_x, NV, m->d.mu_ref);
    if (grad_y) cudaMemsetAsync(grad_y, 0, sizeof(float) * NP, st);
    for (int n = N - 1; n >= 0 && rc == 0; --n) {
        const LayerSpec *Ld = &m->layers[m->dual_at[n]], *Lp = &m->layers[m->prim_at[n]];
        map_unpermute(pfm, m->perm_f[n], M);
        map_unpermute(phm, m->perm_h[n], M);
        // ---- primal update undone: recompute its input from p1 and the final d2[0]
        if ((rc = back_project_colw(m->g, m->h + phm[K] * NP, m->wred, m->tvol, B, 0, st))) break;
        const Planes pp = rev_primal_planes(m, m->f, pfm, NV, m->tvol);
        k_pack8<<<grid_n(NV), 256, 0, st>>>(pp, NV, m->pin);
        if ((rc = prim_hidden(m, Lp, B, st))) break;
        if ((rc = rev_update(m, prim_out(m, Lp), prim_out_in(m, Lp), PRIM_DIMS, m->f, pfm + K, NV, 1, st))) break;
        // gradients through Lambda: upstream dL/dp2 (identity through the residual)
        Planes gp{};
        for (int c = 0; c < K; ++c) { gp.p[c] = gf + pfm[K + c] * NV; gp.s[c] = 1.f; }
        k_pack8<<<grid_n(NV), 256, 0, st>>>(gp, NV, m->gsmall);
        // dL/d[p1, bp]: p1's planes accumulate, the bp channel goes to scratch plane M
        int mp[8];
        for (int c = 0; c < K; ++c) mp[c] = pfm[c];
        mp[K] = M;
        cudaMemsetAsync(gf + (long long)M * NV, 0, sizeof(float) * NV, st);
        if ((rc = prim_bwd(m, Lp, B, gf, NV, mp, dW, st))) break;
        // bp = bp_scale P^T (w d2[0])  =>  dL/dd2[0] += w bp_scale P (dL/dbp)
        if ((rc = forward_project(m->g, gf + (long long)M * NV, m->tproj, B, 0, sv))) break;
        k_scale_cols<<<grid_n(NP), 256, 0, st>>>(m->tproj, m->wred, NP, m->g->dev.nu, m->bp_scale, m->tproj2);
        k_axpy<<<grid_n(NP), 256, 0, st>>>(gh + phm[K] * NP, m->tproj2, NP, 1.f);
        // ---- dual update undone: recompute its input from d1 and the recovered p2[0]
        if ((rc = forward_project(m->g, m->f + pfm[K] * NV, m->tproj, B, 0, sv))) break;
        const Planes pl = rev_dual_planes(m, m->h, phm, NP, m->tproj, m->y);
        k_pack8<<<grid_n(NP), 256, 0, st>>>(pl, NP, m->din);
        if ((rc = conv_fwd(m, Ld[0], m->din, 8, DUAL_DIMS, 0, m->a1, nullptr, 0, st))) break;
        if ((rc = conv_fwd(m, Ld[1], m->a1, hs(Ld[1].cin), DUAL_DIMS, 0, m->a2, nullptr, 0, st))) break;
        if ((rc = rev_update(m, Ld[2], m->a2, DUAL_DIMS, m->h, phm + K, NP, 1, st))) break;
        // gradients through Gamma: upstream dL/dd2
        Planes gd{};
        for (int c = 0; c < K; ++c) { gd.p[c] = gh + phm[K + c] * NP; gd.s[c] = 1.f; }
        k_pack8<<<grid_n(NP), 256, 0, st>>>(gd, NP, m->gsmall);
        if ((rc = conv_wgrad(m->a2, hs(Ld[2].cin), Ld[2].cin, m->gsmall, 8, Ld[2].cout, DUAL_DIMS, 0, dW + Ld[2].fw_off,
                             dW + Ld[2].fb_off, wacc(m, Ld[2]), m->status, st))) break;
        if ((rc = conv_dx(m, Ld[2], m->gsmall, 8, DUAL_DIMS, 2, m->g32a, m->a2, nullptr, 0, st))) break;
        if ((rc = conv_wgrad(m->a1, hs(Ld[1].cin), Ld[1].cin, m->g32a, hs(Ld[1].cout), Ld[1].cout, DUAL_DIMS, 0, dW + Ld[1].fw_off,
                             dW + Ld[1].fb_off, wacc(m, Ld[1]), m->status, st))) break;
        if ((rc = conv_dx(m, Ld[1], m->g32a, hs(Ld[1].cout), DUAL_DIMS, 2, m->g32b, m->a1, nullptr, 0, st))) break;
        if ((rc = conv_wgrad(m->din, 8, Ld[0].cin, m->g32b, hs(Ld[0].cout), Ld[0].cout, DUAL_DIMS, 0, dW + Ld[0].fw_off,
                             dW + Ld[0].fb_off, wacc(m, Ld[0]), m->status, st))) break;
        // dL/d[d1, pf, y (, residual)]: d1's planes accumulate, the others go to scratch planes M..
        const int nin = Ld[0].cin;
        for (int c = 0; c < K; ++c) mp[c] = phm[c];
        for (int c = K; c < nin; ++c) mp[c] = M + (c - K);
        cudaMemsetAsync(gh + (long long)M * NP, 0, sizeof(float) * 3 * NP, st);
        if ((rc = conv_apply(m->g32b, DUAL_DIMS, hs(Ld[0].cout), Ld[0].taps3d, m->params + Ld[0].fw_off, nullptr, Ld[0].cin,
                             Ld[0].cout, 1, 1, m->d.slope, nullptr, 32, nullptr, gh, gh, NP, m->status, st, nullptr,
                             0, mp, 0))) break;
        float *g_pf = gh + (long long)M * NP, *g_y = gh + (long long)(M + 1) * NP;
        if (m->d.residual_input) {
            const float *g_res = gh + (long long)(M + 2) * NP;
            if (grad_y) k_add_diff<<<grid_n(NP), 256, 0, st>>>(grad_y, g_y, g_res, NP);
            k_axpy<<<grid_n(NP), 256, 0, st>>>(g_pf, g_res, NP, 1.f);
        } else if (grad_y) {
            k_axpy<<<grid_n(NP), 256, 0, st>>>(grad_y, g_y, NP, 1.f);
        }
        // pf channel = mu_ref P p2[0]  =>  dL/dp2[0] += mu_ref P^T (dL/dpf)
        if ((rc = back_project(m->g, g_pf, m->tvol, B, 0, sv))) break;
        k_axpy<<<grid_n(NV), 256, 0, st>>>(gf + pfm[K] * NV, m->tvol, NV, m->d.mu_ref);
    }
    if (rc) return rc;
    // back at the initial states (every plane map is the identity again): f_0 = x0 / mu_ref
    // in every channel  =>  dL/dx0 = sum_c gf[c] / mu_ref
    if (grad_x0) k_sum_channels<<<grid_n(NV), 256, 0, st>>>(gf, M, NV, 1.f / m->d.mu_ref, grad_x0, 0);
    for (int c = 0; c < M; ++c) { m->cur_f[c] = pfm[c]; m->cur_h[c] = phm[c]; }
    m->saved = 0;  // the states now hold the recovered initial iterate
    weights_contract(m, st);
    CBCT_LAUNCH_CHECK("lpd_backward (reversible)");
    return 0;
}

// ---- LIRE mode: Algorithm 1 at one resolution ----------------------------------------------
//
// Reversible latents as above (halves of K channels, permutations by bookkeeping) plus a
// separate FP32 reconstruction x, per iteration n:
//   p_op = [mu_ref P p2[0], P x]                        one batched forward projection
//   d2 += Gamma_n([d1, p_op, y, P x - y])               3x3x3 convs over (angle, v, u)
//   b_op = s P^T(w d2[0]), LW = s P^T(P x - y)          one batched backprojection
//   p2 += Lambda_n([p1, b_op, x / mu_ref, LW, V])       3x3x3 convs over the volume
//   x += mu_ref (beta_n + sum_c omega_n[c] f[c])        1x1x1 output convolution
//   permute f, h
// from x = x0, f = [x0 / mu_ref, s P^T(w y), ...], h = y in every channel. The backward
// undoes the iterations (x first, then p2, then d2) while the gradients run through them.

static Planes lire_f_planes(const cbct_lpd *m, const int *pfm, long long NV) {
    Planes fp{};
    for (int c = 0; c < m->d.n_mem; ++c) { fp.p[c] = m->f + pfm[c] * NV; fp.s[c] = 1.f; }
    return fp;
}

// dual input [d1 (K), mu_ref P p2[0], P x, y, P x - y] from the projections in t2p
static Planes lire_dual_planes(const cbct_lpd *m, const int *phm, long long NP) {
    const int K = m->d.n_mem / 2;
    Planes pl{};
    for (int c = 0; c < K; ++c) { pl.p[c] = m->h + phm[c] * NP; pl.s[c] = 1.f; }
    pl.p[K] = m->t2p; pl.s[K] = m->d.mu_ref;
    pl.p[K + 1] = m->t2p + NP; pl.s[K + 1] = 1.f;
    pl.p[K + 2] = m->y; pl.s[K + 2] = 1.f;
    pl.p[K + 3] = m->t2p + NP; pl.s[K + 3] = 1.f; pl.q[K + 3] = m->y;
    return pl;
}

// primal input [p1 (K), s P^T(w d2[0]), x / mu_ref, s LW, V] from the backprojections in t2v
static Planes lire_primal_planes(const cbct_lpd *m, const int *pfm, long long NV) {
    const int K = m->d.n_mem / 2;
    Planes pp{};
    for (int c = 0; c < K; ++c) { pp.p[c] = m->f + pfm[c] * NV; pp.s[c] = 1.f; }
    pp.p[K] = m->t2v; pp.s[K] = m->bp_scale;
    pp.p[K + 1] = m->x; pp.s[K + 1] = 1.f / m->d.mu_ref;
    pp.p[K + 2] = m->t2v + NV; pp.s[K + 2] = m->bp_scale;
    pp.p[K + 3] = m->Vb; pp.s[K + 3] = 1.f;
    return pp;
}

#define LIRE_DUAL_DIMS B, m->g->dev.na, m->g->dev.nv, m->g->dev.nu

// t2p = [P p2[0], P x] (one forward projection of 2B volumes)
static int lire_project(cbct_lpd *m, const int *pfm, int B, cudaStream_t st) {
    const long long NV = m->nvox * B;
    const int K = m->d.n_mem / 2;
    CBCT_CUDA_TRY(cudaMemcpyAsync(m->t2v, m->f + pfm[K] * NV, sizeof(float) * NV, cudaMemcpyDeviceToDevice, st));
    CBCT_CUDA_TRY(cudaMemcpyAsync(m->t2v + NV, m->x, sizeof(float) * NV, cudaMemcpyDeviceToDevice, st));
    return forward_project(m->g, m->t2v, m->t2p, 2 * B, 0, (void *)st);
}

// t2v = [P^T(w d2[0]), P^T(P x - y)] (one backprojection of 2B items; t2p[1] must hold P x)
static int lire_backproject(cbct_lpd *m, const int *phm, int B, cudaStream_t st) {
    const long long NP = m->nproj * B;
    const int K = m->d.n_mem / 2;
    k_scale_cols<<<grid_n(NP), 256, 0, st>>>(m->h + phm[K] * NP, m->wred, NP, m->g->dev.nu, 1.f, m->t2p);
    k_diff<<<grid_n(NP), 256, 0, st>>>(m->t2p + NP, m->t2p + NP, m->y, NP);
    return back_project(m->g, m->t2p, m->t2v, 2 * B, 0, (void *)st);
}

static int lire_forward(cbct_lpd *m, const float *y, const float *x0, float *x_out, int save_for_backward, int B,
                        cudaStream_t st) {
    m->batch = B;
    const long long NV = m->nvox * B, NP = m->nproj * B;
    const int M = m->d.n_mem, K = M / 2, N = m->d.n_iter;
    weights_expand(m, st);
    int rc = conv_pack_jobs(m->pack_jobs, m->n_pack_jobs, m->pack_max_nelem, m->params, m->wpk, st);
    if (rc) return rc;
    CBCT_CUDA_TRY(cudaMemcpyAsync(m->y, y, sizeof(float) * NP, cudaMemcpyDeviceToDevice, st));
    CBCT_CUDA_TRY(cudaMemcpyAsync(m->x, x0, sizeof(float) * NV, cudaMemcpyDeviceToDevice, st));
    // f = [x0 / mu, s P^T(w y), ...], h = y in every channel
    if ((rc = back_project_colw(m->g, m->y, m->wred, m->tvol, B, 0, st))) return rc;
    k_lire_init_f<<<grid_n(NV), 256, 0, st>>>(x0, m->tvol, m->f, NV, M, 1.f / m->d.mu_ref, m->bp_scale);
    for (int c = 0; c < M; ++c)
        CBCT_CUDA_TRY(cudaMemcpyAsync(m->h + c * NP, m->y, sizeof(float) * NP, cudaMemcpyDeviceToDevice, st));
    int pfm[8], phm[8];
    for (int c = 0; c < M; ++c) pfm[c] = phm[c] = c;
    for (int n = 0; n < N && rc == 0; ++n) {
        const LayerSpec *Ld = &m->layers[m->dual_at[n]], *Lp = &m->layers[m->prim_at[n]];
        if ((rc = lire_project(m, pfm, B, st))) break;
        const Planes pl = lire_dual_planes(m, phm, NP);
        k_pack8<<<grid_n(NP), 256, 0, st>>>(pl, NP, m->din);
        if ((rc = conv_fwd(m, Ld[0], m->din, 8, LIRE_DUAL_DIMS, 0, m->a1, nullptr, 0, st))) break;
        if ((rc = conv_fwd(m, Ld[1], m->a1, hs(Ld[1].cin), LIRE_DUAL_DIMS, 0, m->a2, nullptr, 0, st))) break;
        if ((rc = rev_update(m, Ld[2], m->a2, LIRE_DUAL_DIMS, m->h, phm + K, NP, 0, st))) break;
        if ((rc = lire_backproject(m, phm, B, st))) break;
        const Planes pp = lire_primal_planes(m, pfm, NV);
        k_pack8<<<grid_n(NV), 256, 0, st>>>(pp, NV, m->pin);
        if ((rc = prim_hidden(m, Lp, B, st))) break;
        if ((rc = rev_update(m, prim_out(m, Lp), prim_out_in(m, Lp), PRIM_DIMS, m->f, pfm + K, NV, 0, st))) break;
        k_outconv<<<grid_n(NV), 256, 0, st>>>(m->x, lire_f_planes(m, pfm, NV), m->params + m->out_off[n],
                                              m->d.mu_ref, NV, M, 1.f);
        map_permute(pfm, m->perm_f[n], M);
        map_permute(phm, m->perm_h[n], M);
    }
    if (rc) return rc;
    if (x_out) CBCT_CUDA_TRY(cudaMemcpyAsync(x_out, m->x, sizeof(float) * NV, cudaMemcpyDeviceToDevice, st));
    for (int c = 0; c < M; ++c) { m->fin_f[c] = m->cur_f[c] = pfm[c]; m->fin_h[c] = m->cur_h[c] = phm[c]; }
    m->saved = save_for_backward;
    m->last = 0;
    CBCT_LAUNCH_CHECK("lpd_forward (lire)");
    return 0;
}

static int lire_backward(cbct_lpd *m, const float *grad_x, float *grad_y, float *grad_x0, cudaStream_t st) {
    void *sv = (void *)st;
    const int B = m->batch;
    const long long NV = m->nvox * B, NP = m->nproj * B;
    const int M = m->d.n_mem, K = M / 2, N = m->d.n_iter;
    const float mu = m->d.mu_ref, s = m->bp_scale;
    // gf: M planes + scratch M .. M+3 (dL/d b_op, dL/d LW, dL/d(x / mu), dL/dV);
    // gh: M planes + scratch M .. M+3 (dL/d of mu P p2[0], P x, y, P x - y) + M+4 (dL/d(P x) via LW)
    float *gf = m->gf, *gh = m->gh, *gx = m->gx, *dW = m->grads;
    float *gy = grad_y ? grad_y : m->tproj2;  // dL/dy is accumulated even when not returned
    float *g_plw = gh + (long long)(M + 4) * NP;
    weights_expand(m, st);
    int rc = conv_pack_jobs(m->pack_jobs, m->n_pack_jobs, m->pack_max_nelem, m->params, m->wpk, st);
    if (rc) return rc;
    int pfm[8], phm[8];
    for (int c = 0; c < M; ++c) { pfm[c] = m->fin_f[c]; phm[c] = m->fin_h[c]; }
    cudaMemsetAsync(gf, 0, sizeof(float) * (M + 4) * NV, st);
    cudaMemsetAsync(gh, 0, sizeof(float) * (M + 5) * NP, st);
    CBCT_CUDA_TRY(cudaMemcpyAsync(gx, grad_x, sizeof(float) * NV, cudaMemcpyDeviceToDevice, st));
    cudaMemsetAsync(gy, 0, sizeof(float) * NP, st);
    for (int n = N - 1; n >= 0 && rc == 0; --n) {
        const LayerSpec *Ld = &m->layers[m->dual_at[n]], *Lp = &m->layers[m->prim_at[n]];
        map_unpermute(pfm, m->perm_f[n], M);
        map_unpermute(phm, m->perm_h[n], M);
        // ---- output convolution: its gradients (with the states after the update), then undone
        PlanesW gp{};
        for (int c = 0; c < M; ++c) gp.p[c] = gf + pfm[c] * NV;
        k_outconv_grad<<<kOutBlocks, 256, 0, st>>>(gx, lire_f_planes(m, pfm, NV), gp, m->params + m->out_off[n], mu,
                                                   NV, M, m->opart);
        k_sum_partials<<<1, 32, 0, st>>>(m->opart, kOutBlocks, M + 1, dW + m->out_off[n]);
        k_outconv<<<grid_n(NV), 256, 0, st>>>(m->x, lire_f_planes(m, pfm, NV), m->params + m->out_off[n], mu, NV, M,
                                              -1.f);
        // ---- primal update undone: inputs from p1, d2[0] and the recovered x
        if ((rc = forward_project(m->g, m->x, m->t2p + NP, B, 0, sv))) break;
        if ((rc = lire_backproject(m, phm, B, st))) break;
        const Planes pp = lire_primal_planes(m, pfm, NV);
        k_pack8<<<grid_n(NV), 256, 0, st>>>(pp, NV, m->pin);
        if ((rc = prim_hidden(m, Lp, B, st))) break;
        if ((rc = rev_update(m, prim_out(m, Lp), prim_out_in(m, Lp), PRIM_DIMS, m->f, pfm + K, NV, 1, st))) break;
        // gradients through Lambda (upstream dL/dp2)
        Planes gpl{};
        for (int c = 0; c < K; ++c) { gpl.p[c] = gf + pfm[K + c] * NV; gpl.s[c] = 1.f; }
        k_pack8<<<grid_n(NV), 256, 0, st>>>(gpl, NV, m->gsmall);
        // input channels [p1 (K), b_op, x / mu, LW, V] -> p1's planes, scratch M, M+2, M+1, M+3
        int mp[8];
        for (int c = 0; c < K; ++c) mp[c] = pfm[c];
        mp[K] = M; mp[K + 1] = M + 2; mp[K + 2] = M + 1; mp[K + 3] = M + 3;
        cudaMemsetAsync(gf + (long long)M * NV, 0, sizeof(float) * 4 * NV, st);
        if ((rc = prim_bwd(m, Lp, B, gf, NV, mp, dW, st))) break;
        // [P dL/db_op, P dL/dLW] in one forward projection of the adjacent scratch planes M, M+1
        if ((rc = forward_project(m->g, gf + (long long)M * NV, m->t2p, 2 * B, 0, sv))) break;
        // b_op = s P^T(w d2[0])  =>  dL/dd2[0] += s w P(dL/db_op)
        k_scale_cols<<<grid_n(NP), 256, 0, st>>>(m->t2p, m->wred, NP, m->g->dev.nu, s, m->tproj);
        k_axpy<<<grid_n(NP), 256, 0, st>>>(gh + phm[K] * NP, m->tproj, NP, 1.f);
        // LW = s P^T(P x - y)  =>  dL/d(P x) += s P(dL/dLW), dL/dy -= s P(dL/dLW)
        cudaMemsetAsync(g_plw, 0, sizeof(float) * NP, st);
        k_axpy<<<grid_n(NP), 256, 0, st>>>(g_plw, m->t2p + NP, NP, s);
        k_axpy<<<grid_n(NP), 256, 0, st>>>(gy, m->t2p + NP, NP, -s);
        // x / mu channel
        k_axpy<<<grid_n(NV), 256, 0, st>>>(gx, gf + (long long)(M + 2) * NV, NV, 1.f / mu);
        // ---- dual update undone: inputs from d1 and the recovered p2[0] and x
        if ((rc = lire_project(m, pfm, B, st))) break;
        const Planes pl = lire_dual_planes(m, phm, NP);
        k_pack8<<<grid_n(NP), 256, 0, st>>>(pl, NP, m->din);
        if ((rc = conv_fwd(m, Ld[0], m->din, 8, LIRE_DUAL_DIMS, 0, m->a1, nullptr, 0, st))) break;
        if ((rc = conv_fwd(m, Ld[1], m->a1, hs(Ld[1].cin), LIRE_DUAL_DIMS, 0, m->a2, nullptr, 0, st))) break;
        if ((rc = rev_update(m, Ld[2], m->a2, LIRE_DUAL_DIMS, m->h, phm + K, NP, 1, st))) break;
        // gradients through Gamma (upstream dL/dd2)
        Planes gdl{};
        for (int c = 0; c < K; ++c) { gdl.p[c] = gh + phm[K + c] * NP; gdl.s[c] = 1.f; }
        k_pack8<<<grid_n(NP), 256, 0, st>>>(gdl, NP, m->gsmall);
        if ((rc = conv_wgrad(m->a2, hs(Ld[2].cin), Ld[2].cin, m->gsmall, 8, Ld[2].cout, LIRE_DUAL_DIMS, 1, dW + Ld[2].fw_off,
                             dW + Ld[2].fb_off, wacc(m, Ld[2]), m->status, st))) break;
        if ((rc = conv_dx(m, Ld[2], m->gsmall, 8, LIRE_DUAL_DIMS, 2, m->g32a, m->a2, nullptr, 0, st))) break;
        if ((rc = conv_wgrad(m->a1, hs(Ld[1].cin), Ld[1].cin, m->g32a, hs(Ld[1].cout), Ld[1].cout, LIRE_DUAL_DIMS, 1, dW + Ld[1].fw_off,
                             dW + Ld[1].fb_off, wacc(m, Ld[1]), m->status, st))) break;
        if ((rc = conv_dx(m, Ld[1], m->g32a, hs(Ld[1].cout), LIRE_DUAL_DIMS, 2, m->g32b, m->a1, nullptr, 0, st))) break;
        if ((rc = conv_wgrad(m->din, 8, Ld[0].cin, m->g32b, hs(Ld[0].cout), Ld[0].cout, LIRE_DUAL_DIMS, 1, dW + Ld[0].fw_off,
                             dW + Ld[0].fb_off, wacc(m, Ld[0]), m->status, st))) break;
        // input channels [d1 (K), mu P p2[0], P x, y, P x - y] -> d1's planes, scratch M .. M+3
        for (int c = 0; c < K; ++c) mp[c] = phm[c];
        for (int c = 0; c < 4; ++c) mp[K + c] = M + c;
        cudaMemsetAsync(gh + (long long)M * NP, 0, sizeof(float) * 4 * NP, st);
        if ((rc = conv_apply(m->g32b, LIRE_DUAL_DIMS, hs(Ld[0].cout), 1, m->params + Ld[0].fw_off, nullptr, Ld[0].cin, Ld[0].cout,
                             1, 1, m->d.slope, nullptr, 32, nullptr, gh, gh, NP, m->status, st, nullptr, 0, mp,
                             0))) break;
        float *g_pp2 = gh + (long long)M * NP, *g_px = gh + (long long)(M + 1) * NP;
        const float *g_ych = gh + (long long)(M + 2) * NP, *g_res = gh + (long long)(M + 3) * NP;
        k_add_diff<<<grid_n(NP), 256, 0, st>>>(gy, g_ych, g_res, NP);
        k_axpy<<<grid_n(NP), 256, 0, st>>>(g_px, g_res, NP, 1.f);
        k_axpy<<<grid_n(NP), 256, 0, st>>>(g_px, g_plw, NP, 1.f);
        // [P^T dL/d(mu P p2[0]), P^T dL/d(P x)] in one backprojection of the adjacent planes M, M+1
        if ((rc = back_project(m->g, g_pp2, m->t2v, 2 * B, 0, sv))) break;
        k_axpy<<<grid_n(NV), 256, 0, st>>>(gf + pfm[K] * NV, m->t2v, NV, mu);
        k_axpy<<<grid_n(NV), 256, 0, st>>>(gx, m->t2v + NV, NV, 1.f);
    }
    if (rc) return rc;
    for (int c = 0; c < M; ++c)
        if (pfm[c] != c || phm[c] != c) return fail(CBCT_ECUDA, "lpd_backward (lire): plane maps not restored");
    // initial states: x = x0, f = [x0 / mu, s P^T(w y), ...], h = y in every channel
    if (grad_x0) {
        CBCT_CUDA_TRY(cudaMemcpyAsync(grad_x0, gx, sizeof(float) * NV, cudaMemcpyDeviceToDevice, st));
        for (int c = 0; c < M; c += 2) k_axpy<<<grid_n(NV), 256, 0, st>>>(grad_x0, gf + c * NV, NV, 1.f / mu);
    }
    if (grad_y) {
        cudaMemsetAsync(m->tvol, 0, sizeof(float) * NV, st);
        for (int c = 1; c < M; c += 2) k_axpy<<<grid_n(NV), 256, 0, st>>>(m->tvol, gf + c * NV, NV, s);
        if ((rc = forward_project(m->g, m->tvol, m->tproj, B, 0, sv))) return rc;
        k_scale_cols<<<grid_n(NP), 256, 0, st>>>(m->tproj, m->wred, NP, m->g->dev.nu, 1.f, m->t2p);
        k_axpy<<<grid_n(NP), 256, 0, st>>>(grad_y, m->t2p, NP, 1.f);
        for (int c = 0; c < M; ++c) k_axpy<<<grid_n(NP), 256, 0, st>>>(grad_y, gh + c * NP, NP, 1.f);
    }
    for (int c = 0; c < M; ++c) { m->cur_f[c] = c; m->cur_h[c] = c; }
    m->saved = 0;
    weights_contract(m, st);
    CBCT_LAUNCH_CHECK("lpd_backward (lire)");
    return 0;
}

extern "C" int lpd_forward(cbct_lpd *m, const float *y, const float *x0, float *x_out, int batch, int save_for_backward,
                           void *stream) {
    if (!m || !y || !x0 || !x_out) return fail(CBCT_EINVAL, "lpd_forward: NULL argument");
    if (batch < 1 || batch > m->maxb)
        return fail(CBCT_EINVAL, "lpd_forward: batch must lie in [1, max_batch = " + std::to_string(m->maxb) + "]");
    if (m->d.lire) return lire_forward(m, y, x0, x_out, save_for_backward, batch, (cudaStream_t)stream);
    if (m->d.reversible) return lpd_rev_forward(m, y, x0, x_out, save_for_backward, batch, (cudaStream_t)stream);
    return lpd_forward_impl(m, y, x0, nullptr, nullptr, x_out, save_for_backward, batch, (cudaStream_t)stream);
}

extern "C" int lpd_forward_latent(cbct_lpd *m, const float *y, const float *x0, const float *f0, const float *h0,
                                  float *x_out, int save_for_backward, void *stream) {
    if (!m || !y || (!x0 && !f0)) return fail(CBCT_EINVAL, "lpd_forward_latent: need y and x0 or f0");
    if (m->d.reversible) return fail(CBCT_EINVAL, "lpd_forward_latent: not available for a reversible model");
    return lpd_forward_impl(m, y, x0, f0, h0, x_out, save_for_backward, 1, (cudaStream_t)stream);
}

extern "C" int lpd_get_state(const cbct_lpd *m, float *f_out, float *h_out, void *stream) {
    if (!m || m->last < 0) return fail(CBCT_EINVAL, "lpd_get_state: no forward pass yet");
    cudaStream_t st = (cudaStream_t)stream;
    const long long NV = m->nvox * m->batch, NP = m->nproj * m->batch, M = m->d.n_mem;
    if (m->d.reversible) {
        // logical channel order (the planes are permuted by bookkeeping only)
        for (int c = 0; c < M; ++c) {
            if (f_out)
                CBCT_CUDA_TRY(cudaMemcpyAsync(f_out + c * NV, m->f + m->cur_f[c] * NV, sizeof(float) * NV,
                                              cudaMemcpyDeviceToDevice, st));
            if (h_out)
                CBCT_CUDA_TRY(cudaMemcpyAsync(h_out + c * NP, m->h + m->cur_h[c] * NP, sizeof(float) * NP,
                                              cudaMemcpyDeviceToDevice, st));
        }
        return 0;
    }
    if (f_out)
        CBCT_CUDA_TRY(cudaMemcpyAsync(f_out, m->f + (long long)m->last * M * NV, sizeof(float) * M * NV,
                                      cudaMemcpyDeviceToDevice, st));
    if (h_out)
        CBCT_CUDA_TRY(cudaMemcpyAsync(h_out, m->h + (long long)m->last * M * NP, sizeof(float) * M * NP,
                                      cudaMemcpyDeviceToDevice, st));
    return 0;
}

// Backward pass of the last forward's batch: upstream dL/dx_out (grad_x) and/or dL/df_N,
// dL/dh_N (the final states, e.g. from a finer level); accumulates the parameter gradients
// (summed over the batch) and returns dL/dy, dL/dx0 and dL/df_0, dL/dh_0 where asked.
static int lpd_backward_impl(cbct_lpd *m, const float *grad_x, const float *grad_fN, const float *grad_hN,
                             float *grad_y, float *grad_x0, float *grad_f0, float *grad_h0, cudaStream_t st) {
    void *sv = (void *)st;
    const int B = m->batch;
    const long long NV = m->nvox * B, NP = m->nproj * B;
    const int M = m->d.n_mem, N = m->d.n_iter, ND = m->nd;
    // gf: [M + 1][B][nvox] (last = grad of the bp channel); gh: [ND][B][nproj] (h, pf, y, residual)
    float *gf = m->gf, *gh = m->gh;
    // the recomputed forward convolutions read the packed weights: refresh them (the
    // parameters may have changed since the forward pass)
    weights_expand(m, st);
    int prc = conv_pack_jobs(m->pack_jobs, m->n_pack_jobs, m->pack_max_nelem, m->params, m->wpk, st);
    if (prc) return prc;
    // dL/df_N: channel 0 gets mu_ref dL/dx; plus the given state gradients
    cudaMemsetAsync(gf, 0, sizeof(float) * (M + 1) * NV, st);
    cudaMemsetAsync(gh, 0, sizeof(float) * ND * NP, st);
    if (grad_x) k_axpy<<<grid_n(NV), 256, 0, st>>>(gf, grad_x, NV, m->d.mu_ref);
    if (grad_fN) k_axpy<<<grid_n((long long)M * NV), 256, 0, st>>>(gf, grad_fN, (long long)M * NV, 1.f);
    if (grad_hN) k_axpy<<<grid_n((long long)M * NP), 256, 0, st>>>(gh, grad_hN, (long long)M * NP, 1.f);
    if (grad_y) cudaMemsetAsync(grad_y, 0, sizeof(float) * NP, st);
    int rc = 0;
    for (int n = N - 1; n >= 0 && rc == 0; --n) {
        const float *f_n = m->f + (long long)n * M * NV, *h_n = m->h + (long long)n * M * NP;
        const LayerSpec *Ld = &m->layers[m->dual_at[n]], *Lp = &m->layers[m->prim_at[n]];
        float *dW = m->grads;
        const float *pf_n = m->pf_saved + (long long)n * NP;
        // recompute the dual block input and activations of iteration n (P f_1 kept)
        const Planes pl = dual_planes(m, h_n, pf_n, m->y);
        k_pack8<<<grid_n(NP), 256, 0, st>>>(pl, NP, m->din);
        if ((rc = conv_fwd(m, Ld[0], m->din, 8, DUAL_DIMS, 0, m->a1, nullptr, 0, st))) break;
        if ((rc = conv_fwd(m, Ld[1], m->a1, hs(Ld[1].cin), DUAL_DIMS, 0, m->a2, nullptr, 0, st))) break;
        // recompute the primal block input and activations (P^T (w h_{n+1}) kept)
        Planes pp{};
        for (int c = 0; c < M; ++c) { pp.p[c] = f_n + c * NV; pp.s[c] = 1.f; }
        pp.p[M] = m->bp_saved + (long long)n * NV; pp.s[M] = m->bp_scale;
        k_pack8<<<grid_n(NV), 256, 0, st>>>(pp, NV, m->pin);
        if ((rc = prim_hidden(m, Lp, B, st))) break;

        // ---- primal block backward: upstream gf[0..M) = dL/df_{n+1}
        Planes gp{};
        for (int c = 0; c < M; ++c) { gp.p[c] = gf + c * NV; gp.s[c] = 1.f; }
        k_pack8<<<grid_n(NV), 256, 0, st>>>(gp, NV, m->gsmall);
        // dL/d(primal input) -> gf[0..M) += (residual path kept), gf[M] = dL/d(bp channel)
        cudaMemsetAsync(gf + (long long)M * NV, 0, sizeof(float) * NV, st);
        if ((rc = prim_bwd(m, Lp, B, gf, NV, nullptr, dW, st))) break;
        // bp = bp_scale P^T (w h_1)  =>  dL/dh_{n+1}[1] += w * bp_scale * P (dL/dbp)
        if ((rc = forward_project(m->g, gf + (long long)M * NV, m->tproj, B, 0, sv))) break;
        k_scale_cols<<<grid_n(NP), 256, 0, st>>>(m->tproj, m->wred, NP, m->g->dev.nu, m->bp_scale, m->tproj2);
        k_axpy<<<grid_n(NP), 256, 0, st>>>(gh + NP, m->tproj2, NP, 1.f);

        // ---- dual block backward: upstream gh[0..M) = dL/dh_{n+1}
        Planes gd{};
        for (int c = 0; c < M; ++c) { gd.p[c] = gh + c * NP; gd.s[c] = 1.f; }
        k_pack8<<<grid_n(NP), 256, 0, st>>>(gd, NP, m->gsmall);
        if ((rc = conv_wgrad(m->a2, hs(Ld[2].cin), Ld[2].cin, m->gsmall, 8, Ld[2].cout, DUAL_DIMS, 0, dW + Ld[2].fw_off,
                             dW + Ld[2].fb_off, wacc(m, Ld[2]), m->status, st))) break;
        if ((rc = conv_dx(m, Ld[2], m->gsmall, 8, DUAL_DIMS, 2, m->g32a, m->a2, nullptr, 0, st))) break;
        if ((rc = conv_wgrad(m->a1, hs(Ld[1].cin), Ld[1].cin, m->g32a, hs(Ld[1].cout), Ld[1].cout, DUAL_DIMS, 0, dW + Ld[1].fw_off,
                             dW + Ld[1].fb_off, wacc(m, Ld[1]), m->status, st))) break;
        if ((rc = conv_dx(m, Ld[1], m->g32a, hs(Ld[1].cout), DUAL_DIMS, 2, m->g32b, m->a1, nullptr, 0, st))) break;
        if ((rc = conv_wgrad(m->din, 8, Ld[0].cin, m->g32b, hs(Ld[0].cout), Ld[0].cout, DUAL_DIMS, 0, dW + Ld[0].fw_off,
                             dW + Ld[0].fb_off, wacc(m, Ld[0]), m->status, st))) break;
        // dL/d(dual input): gh[0..M) += (residual), gh[M] = dL/d(pf channel), gh[M+1] = dL/d(y channel),
        // gh[M+2] = dL/d(residual channel mu_ref pf - y)
        cudaMemsetAsync(gh + (long long)M * NP, 0, sizeof(float) * (ND - M) * NP, st);
        if ((rc = conv_dx(m, Ld[0], m->g32b, hs(Ld[0].cout), DUAL_DIMS, 1, nullptr, nullptr, gh, NP, st))) break;
        float *g_pf = gh + (long long)M * NP, *g_y = gh + (long long)(M + 1) * NP;
        if (m->d.residual_input) {
            // residual channel = pf channel - y: its gradient adds to the pf channel's and
            // subtracts from y's
            const float *g_res = gh + (long long)(M + 2) * NP;
            if (grad_y) k_add_diff<<<grid_n(NP), 256, 0, st>>>(grad_y, g_y, g_res, NP);
            k_axpy<<<grid_n(NP), 256, 0, st>>>(g_pf, g_res, NP, 1.f);
        } else if (grad_y) {
            k_axpy<<<grid_n(NP), 256, 0, st>>>(grad_y, g_y, NP, 1.f);
        }
        // pf channel = mu_ref P f_1  =>  dL/df_n[1] += mu_ref P^T (dL/dpf channel)
        if ((rc = back_project(m->g, g_pf, m->tvol, B, 0, sv))) break;
        k_axpy<<<grid_n(NV), 256, 0, st>>>(gf + NV, m->tvol, NV, m->d.mu_ref);
    }
    if (rc) return rc;
    // f_0 = x0 / mu_ref repeated  =>  dL/dx0 = sum_c gf[c] / mu_ref
    if (grad_x0) k_sum_channels<<<grid_n(NV), 256, 0, st>>>(gf, M, NV, 1.f / m->d.mu_ref, grad_x0, 0);
    if (grad_f0) CBCT_CUDA_TRY(cudaMemcpyAsync(grad_f0, gf, sizeof(float) * M * NV, cudaMemcpyDeviceToDevice, st));
    if (grad_h0) CBCT_CUDA_TRY(cudaMemcpyAsync(grad_h0, gh, sizeof(float) * M * NP, cudaMemcpyDeviceToDevice, st));
    weights_contract(m, st);
    CBCT_LAUNCH_CHECK("lpd_backward");
    return 0;
}

extern "C" int lpd_backward(cbct_lpd *m, const float *grad_x, float *grad_y, float *grad_x0, void *stream) {
    if (!m || !grad_x) return fail(CBCT_EINVAL, "lpd_backward: NULL argument");
    if (!m->saved) return fail(CBCT_EINVAL, "lpd_backward: call lpd_forward with save_for_backward = 1 first");
    if (m->d.lire) return lire_backward(m, grad_x, grad_y, grad_x0, (cudaStream_t)stream);
    if (m->d.reversible) return lpd_rev_backward(m, grad_x, grad_y, grad_x0, (cudaStream_t)stream);
    return lpd_backward_impl(m, grad_x, nullptr, nullptr, grad_y, grad_x0, nullptr, nullptr, (cudaStream_t)stream);
}

extern "C" int lpd_backward_latent(cbct_lpd *m, const float *grad_x, const float *grad_fN, const float *grad_hN,
                                   float *grad_y, float *grad_x0, float *grad_f0, float *grad_h0, void *stream) {
    if (!m || (!grad_x && !grad_fN && !grad_hN)) return fail(CBCT_EINVAL, "lpd_backward_latent: no upstream gradient");
    if (!m->saved) return fail(CBCT_EINVAL, "lpd_backward_latent: call the forward with save_for_backward = 1 first");
    if (m->d.reversible) return fail(CBCT_EINVAL, "lpd_backward_latent: not available for a reversible model");
    return lpd_backward_impl(m, grad_x, grad_fN, grad_hN, grad_y, grad_x0, grad_f0, grad_h0, (cudaStream_t)stream);
}

extern "C" int lpd_zero_grad(cbct_lpd *m, void *stream) {
    if (!m) return fail(CBCT_EINVAL, "lpd_zero_grad: NULL model");
    CBCT_CUDA_TRY(cudaMemsetAsync(m->grads, 0, sizeof(float) * m->nparams, (cudaStream_t)stream));
    return 0;
}

namespace {

constexpr int kNormBlocks = 608;

// partial[blk] = sum of g^2 over the block's grid-stride share (FP64, tree in shared
// memory: a fixed order)
__global__ void __launch_bounds__(256) k_sumsq_blocks(const float *__restrict__ g, long long n,
                                                      double *__restrict__ partial) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        s += (double)g[i] * g[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// out[0] = ||grad_scale g||, out[1] = clip factor min(1, max_norm / out[0]) (0 if not finite)
__global__ void k_clip_factor(const double *__restrict__ partial, int nblk, double grad_scale, double max_norm,
                              double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[b];
    const double nrm = sqrt(s) * fabs(grad_scale);
    out[0] = nrm;
    out[1] = isfinite(nrm) ? (nrm > max_norm ? max_norm / nrm : 1.0) : 0.0;
}

__global__ void k_scale_by_factor(float *__restrict__ g, long long n, const double *__restrict__ f) {
    const float k = (float)f[1];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        g[i] = k == 0.f ? 0.f : g[i] * k;
}

}  // namespace

extern "C" int lpd_clip_grads(cbct_lpd *m, float max_norm, float grad_scale, double *norm_out, void *stream) {
    if (!m || !(max_norm > 0.f)) return fail(CBCT_EINVAL, "lpd_clip_grads: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    k_sumsq_blocks<<<kNormBlocks, 256, 0, st>>>(m->grads, m->nparams, m->clip);
    k_clip_factor<<<1, 32, 0, st>>>(m->clip, kNormBlocks, grad_scale, max_norm, m->clip + kNormBlocks);
    k_scale_by_factor<<<grid_n(m->nparams), 256, 0, st>>>(m->grads, m->nparams, m->clip + kNormBlocks);
    CBCT_LAUNCH_CHECK("lpd_clip_grads");
    if (norm_out) {
        CBCT_CUDA_TRY(cudaMemcpyAsync(norm_out, m->clip + kNormBlocks, sizeof(double), cudaMemcpyDeviceToHost, st));
        CBCT_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return 0;
}

extern "C" int lpd_adam_step(cbct_lpd *m, float lr, float beta1, float beta2, float eps, int step, float grad_scale,
                             void *stream) {
    if (!m || step < 1) return fail(CBCT_EINVAL, "lpd_adam_step: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_adam<<<grid_n(m->nparams), 256, 0, st>>>(m->params, m->grads, m->adam_m, m->adam_v, m->nparams, lr, beta1, beta2,
                                               eps, c1, c2, grad_scale);
    // forced weight normalisation: each raw filter back to zero mean and norm sqrt(len)
    if (m->n_wn) k_wn_force<<<m->n_wn, 256, 0, st>>>(m->wn_jobs, m->params);
    CBCT_LAUNCH_CHECK("lpd_adam_step");
    return 0;
}

extern "C" int lpd_device_status(const cbct_lpd *m, int *out, int clear) {
    if (!m || !out) return fail(CBCT_EINVAL, "lpd_device_status: NULL argument");
    int v = 0;
    CBCT_CUDA_TRY(cudaMemcpy(&v, m->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (clear && v) CBCT_CUDA_TRY(cudaMemset(m->status, 0, sizeof(int)));
    *out = v;
    return 0;
}

extern "C" int lpd_set_params(cbct_lpd *m, const float *host, long long n) {
    if (!m || !host || n != m->nparams) return fail(CBCT_EINVAL, "lpd_set_params: size mismatch");
    CBCT_CUDA_TRY(cudaMemcpy(m->params, host, sizeof(float) * n, cudaMemcpyHostToDevice));
    return 0;
}

extern "C" int lpd_get_params(const cbct_lpd *m, float *host, long long n) {
    if (!m || !host || n != m->nparams) return fail(CBCT_EINVAL, "lpd_get_params: size mismatch");
    CBCT_CUDA_TRY(cudaMemcpy(host, m->params, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return 0;
}

extern "C" int lpd_get_grads(const cbct_lpd *m, float *host, long long n) {
    if (!m || !host || n != m->nparams) return fail(CBCT_EINVAL, "lpd_get_grads: size mismatch");
    CBCT_CUDA_TRY(cudaMemcpy(host, m->grads, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return 0;
}

extern "C" int cbct_masked_mse(const float *x, const float *ref, const float *V, float thr, long long n, float *loss,
                               float *grad, void *stream) {
    if (!x || !ref || !loss || n < 1) return fail(CBCT_EINVAL, "cbct_masked_mse: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = 256;
    double *part = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&part, sizeof(double) * 2 * nb + 16, st));
    float *cnt = reinterpret_cast<float *>(part + 2 * nb);
    k_mse_partial<<<nb, 256, 0, st>>>(x, ref, V, thr, n, part, part + nb);
    k_mse_final<<<1, 1, 0, st>>>(part, part + nb, nb, loss, cnt);
    if (grad) k_mse_grad<<<grid_n(n), 256, 0, st>>>(x, ref, V, thr, n, cnt, grad);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, st);
    if (e != cudaSuccess) return cuda_fail(e, "cbct_masked_mse");
    return 0;
}
