// 3x3 (2D, dual block) and 3x3x3 (3D, primal block) convolutions of the learned
// primal-dual network (paper Sec. 2.4, Algorithm 1 blocks Gamma and Lambda; here
// the 3-layer width-32 blocks of the learned primal-dual workload), stride 1, zero
// "same" padding. BF16 operands, FP32 accumulation.
//
// Forward (and input-gradient) convolution = implicit GEMM on the fifth-generation
// tensor cores: D[128 pixels][N out channels] = sum_K A[pixel][K] B[n][K], K = (tap,
// input channel). A CTA walks a contiguous range of tiles of 128 consecutive
// output pixels along W; for every K chunk of 64 it loads the shifted input
// pixels with TMA: one box of [128 output pixels][8 channels] per (tap, channel
// group) is exactly one K-major core-matrix column, zero-filled outside the image.
// A producer warp fills a 4-stage ring, one thread issues 128 x N x 16 tcgen05.mma
// into double-buffered TMEM accumulators, four epilogue warps drain them. The
// packed weights (B) stay in shared memory for the CTA's lifetime. The epilogue
// reads TMEM with tcgen05.ld and applies bias + LeakyReLU (BF16 channels-last
// out), a residual update of an FP32 channel-first state, or an activation mask.
//
// Weight gradients run on the CUDA cores (register-blocked FP32 accumulation over
// pixel chunks, partial sums reduced in a fixed order).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "geom_impl.h"
#include "tcgen05.cuh"

namespace cbct {

constexpr int kConvThreads = 128;
constexpr int kChunkGroups = 8;  // K groups (of 8 channels) per A chunk = 64 K elements
constexpr int kAStageBytes = kChunkGroups * 16 * 128;  // 8 K-groups x 16 row groups x 128 B

enum ConvEpi { EPI_ACT_BF16 = 0, EPI_RESIDUAL_F32 = 1, EPI_MASK_BF16 = 2 };

struct ConvArgs {
    const __nv_bfloat16 *x;  // [nimg][D][H][W][cpin], channels-last
    const uint8_t *wpk;      // packed B operand: kgroups x (NPAD/8) core matrices
    const float *bias;       // [cout] or null
    int nimg, D, H, W;
    int cpin, cin_groups;    // channel stride (multiple of 8), cpin / 8
    int taps3d;              // 1: 3x3x3, 0: 3x3 over (H, W)
    int kgroups;             // padded K / 8 (even)
    int cout;
    float slope;
    __nv_bfloat16 *y;        // EPI_ACT_BF16 / EPI_MASK_BF16 output, channel stride cpout
    int cpout;
    const __nv_bfloat16 *mask;  // EPI_MASK_BF16: forward activation (same layout as y); out *= (mask > 0 ? 1 : slope)
    float *state;            // EPI_RESIDUAL_F32: state[c * sstride + pixel] += v
    long long sstride;
    int *status;
};

__device__ __forceinline__ void tap_offset(int tap, int taps3d, int &dd, int &dh, int &dw) {
    if (taps3d) {
        dd = tap / 9 - 1;
        dh = (tap / 3) % 3 - 1;
        dw = tap % 3 - 1;
    } else {
        dd = 0;
        dh = tap / 3 - 1;
        dw = tap % 3 - 1;
    }
}

constexpr int kStages = 4;          // A ring: kStages x 16 KiB
constexpr int kWsThreads = 192;     // warps 0-3 epilogue, 4 producer, 5 MMA

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}

// Tile t = ((img * D + d) * H + h) * ntw + wt covers output pixels (img, d, h, 128 wt + r).
struct TileCoord {
    int img, d, h, w0;
};
__device__ __forceinline__ TileCoord tile_coord(long long t, int D, int H, int ntw) {
    TileCoord c;
    c.w0 = (int)(t % ntw) * 128; t /= ntw;
    c.h = (int)(t % H); t /= H;
    c.d = (int)(t % D);
    c.img = (int)(t / D);
    return c;
}

// Epilogue of one tile row: TMEM accumulators -> bias / activation / residual.
template <int NPAD, int EPI>
__device__ __forceinline__ void conv_epilogue(const ConvArgs &a, const float *acc, long long p) {
    if constexpr (EPI == EPI_RESIDUAL_F32) {
#pragma unroll
        for (int c = 0; c < NPAD; ++c) {
            if (c < a.cout) {
                const float v = acc[c] + (a.bias ? __ldg(a.bias + c) : 0.f);
                float *o = a.state + c * a.sstride + p;
                *o += v;
            }
        }
    } else {
        __nv_bfloat16 *o = a.y + p * a.cpout;
        const __nv_bfloat16 *mk = EPI == EPI_MASK_BF16 ? a.mask + p * a.cpout : nullptr;
#pragma unroll
        for (int c0 = 0; c0 < NPAD; c0 += 8) {
            if (c0 >= a.cpout) break;
            __align__(16) __nv_bfloat16 out8[8];
            uint4 mv = make_uint4(0u, 0u, 0u, 0u);
            if constexpr (EPI == EPI_MASK_BF16) mv = *reinterpret_cast<const uint4 *>(mk + c0);
            const __nv_bfloat16 *m8 = reinterpret_cast<const __nv_bfloat16 *>(&mv);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + j;
                float v = 0.f;
                if (c < a.cout) {
                    v = acc[c];
                    if constexpr (EPI == EPI_ACT_BF16) {
                        if (a.bias) v += __ldg(a.bias + c);
                        v = v > 0.f ? v : v * a.slope;
                    } else {
                        v = __bfloat162float(m8[j]) > 0.f ? v : v * a.slope;
                    }
                }
                out8[j] = __float2bfloat16_rn(v);
            }
            *reinterpret_cast<uint4 *>(o + c0) = *reinterpret_cast<const uint4 *>(out8);
        }
    }
}

// Warp-specialized convolution tile loop. Item i of a CTA = (tile t_begin + i / nch,
// K chunk i % nch) on ring stage i % kStages.
//  producer (warp 4, one lane): waits until the stage is free (empty[s]), then TMA-loads
//    the chunk's K groups, each a [128 pixels][8 channels] box = one K-major core-matrix
//    column (16 B rows, 128 B between 8-row groups); taps outside the image and K padding
//    come back as zeros.
//  MMA (warp 5, one lane): per tile picks TMEM accumulator j & 1 once the epilogue has
//    drained it (acce), waits for each chunk (full[s]), issues 128 x N x 16 MMAs, commits
//    the stage to empty[s] and, after the tile's last chunk, the accumulator to accf.
//  epilogue (warps 0-3): waits for accf, reads its 32 TMEM lanes, releases the
//    accumulator, applies the epilogue and stores.
template <int NPAD, int EPI>
__global__ void __launch_bounds__(kWsThreads) k_conv_tc(const __grid_constant__ CUtensorMap xmap, ConvArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int bbytes = a.kgroups * NPAD * 16;
    unsigned char *sA = sm;                                         // kStages x 16 KiB
    unsigned char *sB = sm + kStages * kAStageBytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + ((bbytes + 127) & ~127));
    uint64_t *empty = full + kStages;
    uint64_t *accf = empty + kStages;
    uint64_t *acce = accf + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acce + 2);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr uint32_t kCols = 2 * NPAD < 32 ? 32 : 2 * NPAD;
    constexpr uint32_t kIdesc = idesc_bf16_f32(128, NPAD);

    if (warp == 0) tmem_alloc(tmem_slot, kCols);
    if (tid == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int j = 0; j < 2; ++j) {
            mbar_init(&accf[j], 1);
            mbar_init(&acce[j], 4);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    for (int i = tid; i < bbytes / 16; i += kWsThreads)
        reinterpret_cast<uint4 *>(sB)[i] = __ldg(reinterpret_cast<const uint4 *>(a.wpk) + i);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int ntw = (a.W + 127) / 128;
    const long long ntiles = (long long)a.nimg * a.D * a.H * ntw;
    const int ntaps = a.taps3d ? 27 : 9;
    const int nch = (a.kgroups + kChunkGroups - 1) / kChunkGroups;
    const long long per_cta = (ntiles + gridDim.x - 1) / gridDim.x;
    const long long t_begin = (long long)blockIdx.x * per_cta;
    const long long my_tiles = t_begin < ntiles ? min(per_cta, ntiles - t_begin) : 0;
    const long long total = my_tiles * nch;

    if (warp == 4) {
        if (lane == 0) {
            prefetch_tmap(&xmap);
            for (long long i = 0; i < total; ++i) {
                const int s = (int)(i % kStages), c = (int)(i % nch);
                const long long u = i / kStages;
                if (u > 0 && !mbar_wait(&empty[s], (uint32_t)((u - 1) & 1), a.status)) {
                    *abort_flag = 1;
                    break;
                }
                const TileCoord tc = tile_coord(t_begin + i / nch, a.D, a.H, ntw);
                const int gn = min(kChunkGroups, a.kgroups - c * kChunkGroups);
                mbar_arrive_expect_tx(&full[s], (uint32_t)gn * 2048u);
                for (int kj = 0; kj < gn; ++kj) {
                    const int G = c * kChunkGroups + kj;
                    const int tap = G / a.cin_groups, cg = G - tap * a.cin_groups;
                    int dd = 0, dh = 0, dw = 0;
                    int x1 = a.W + 256;  // K padding: a box entirely outside the image (zeros)
                    if (tap < ntaps) {
                        tap_offset(tap, a.taps3d, dd, dh, dw);
                        x1 = tc.w0 + dw;
                    }
                    tma_load_5d(sA + s * kAStageBytes + kj * 2048, &xmap, cg * 8, x1, tc.h + dh, tc.d + dd, tc.img,
                                &full[s]);
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            const uint32_t sA_u = smem_u32(sA), sB_u = smem_u32(sB);
            long long i = 0;
            for (long long j = 0; j < my_tiles && !*abort_flag; ++j) {
                const int ab = (int)(j & 1);
                if (j >= 2 && !mbar_wait(&acce[ab], (uint32_t)(((j >> 1) - 1) & 1), a.status)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(ab * NPAD);
                for (int c = 0; c < nch; ++c, ++i) {
                    const int s = (int)(i % kStages);
                    if (!mbar_wait(&full[s], (uint32_t)((i / kStages) & 1), a.status)) {
                        *abort_flag = 1;
                        break;
                    }
                    tc_fence_after();
                    const int ksteps = min(kChunkGroups, a.kgroups - c * kChunkGroups) / 2;
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint64_t ad = smem_desc_kmajor(sA_u + s * kAStageBytes + ks * 2 * 2048, 2048, 128);
                        const uint64_t bd = smem_desc_kmajor(sB_u + (c * kChunkGroups + ks * 2) * (NPAD / 8) * 128,
                                                             (NPAD / 8) * 128, 128);
                        mma_bf16(dt, ad, bd, kIdesc, (c > 0 || ks > 0) ? 1u : 0u);
                    }
                    mma_commit(&empty[s]);
                }
                if (*abort_flag) break;
                mma_commit(&accf[ab]);
            }
        }
    } else {
        // epilogue warps 0-3: TMEM lanes 32 warp .. + 31 = tile rows
        for (long long j = 0; j < my_tiles; ++j) {
            const int ab = (int)(j & 1);
            if (!mbar_wait(&accf[ab], (uint32_t)((j >> 1) & 1), a.status)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            float acc[NPAD];
#pragma unroll
            for (int c0 = 0; c0 < NPAD; c0 += 16)
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ab * NPAD + c0), acc + c0);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[ab]);
            const TileCoord tc = tile_coord(t_begin + j, a.D, a.H, ntw);
            const int w = tc.w0 + tid;
            if (w < a.W) {
                const long long p = (((long long)tc.img * a.D + tc.d) * a.H + tc.h) * a.W + w;
                conv_epilogue<NPAD, EPI>(a, acc, p);
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// ---- weight packing ---------------------------------------------------------------------

// B operand of the forward convolution: row n = output channel, K = (tap, input
// channel) with the input channels padded to cpin. w: FP32 [cout][taps][cin].
// flip = 1 packs the input-gradient convolution instead: row n = input channel, K =
// (tap, output channel) with the mirrored tap (cpin = padded output channels).
__global__ void k_pack_weights(const float *__restrict__ w, int cout, int ntaps, int cin, int cpin, int npad,
                               int kgroups, int flip, uint8_t *__restrict__ out) {
    const long long total = (long long)npad * kgroups * 8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(e / (kgroups * 8));
        const int k = (int)(e - (long long)n * kgroups * 8);
        const int tap = k / cpin, ch = k - tap * cpin;
        float v = 0.f;
        if (tap < ntaps) {
            if (!flip) {
                if (n < cout && ch < cin) v = w[((long long)n * ntaps + tap) * cin + ch];
            } else {
                // input-gradient conv: out channel n = ci, in channel ch = co, tap mirrored
                if (n < cin && ch < cout) v = w[((long long)ch * ntaps + (ntaps - 1 - tap)) * cin + n];
            }
        }
        const int kg = k >> 3, kin = k & 7;
        const long long off = ((long long)kg * (npad / 8) + (n >> 3)) * 128 + (n & 7) * 16 + kin * 2;
        *reinterpret_cast<__nv_bfloat16 *>(out + off) = __float2bfloat16_rn(v);
    }
}

// ---- weight gradient (CUDA cores) ---------------------------------------------------------

// partial[blk][co][tap][ci] = sum over this block's pixels of dY[p][co] * X[p + tap][ci]
// and partial_b[blk][co] = sum dY[p][co]. Each thread owns 4 output channels x 4
// input channels of one tap.
__global__ void k_conv_wgrad(const __nv_bfloat16 *__restrict__ x, int cpin, int cin, const __nv_bfloat16 *__restrict__ dy,
                             int cpout, int cout, int nimg, int D, int H, int W, int taps3d, int pix_per_block,
                             float *__restrict__ partial, float *__restrict__ partial_b) {
    const int ntaps = taps3d ? 27 : 9;
    const int cog = (cout + 3) / 4, cig = (cin + 3) / 4;
    const int nwork = ntaps * cog * cig;
    const long long npix = (long long)nimg * D * H * W;
    const long long p0 = (long long)blockIdx.x * pix_per_block;
    const long long p1 = min(npix, p0 + pix_per_block);
    for (int wi = threadIdx.x; wi < nwork; wi += blockDim.x) {
        const int tap = wi / (cog * cig), r = wi - tap * cog * cig;
        const int co0 = (r / cig) * 4, ci0 = (r % cig) * 4;
        int dd, dh, dw;
        tap_offset(tap, taps3d, dd, dh, dw);
        float acc[4][4] = {};
        long long t0 = p0;
        int w_ = (int)(t0 % W); t0 /= W;
        int h_ = (int)(t0 % H); t0 /= H;
        int d_ = (int)(t0 % D);
        long long img = t0 / D;
        for (long long p = p0; p < p1; ++p) {
            const int d2 = d_ + dd, h2 = h_ + dh, w2 = w_ + dw;
            const bool inside = d2 >= 0 && d2 < D && h2 >= 0 && h2 < H && w2 >= 0 && w2 < W;
            // advance the pixel counter (w fastest)
            const int wc = w_, hc = h_, dc = d_;
            const long long ic = img;
            if (++w_ == W) { w_ = 0; if (++h_ == H) { h_ = 0; if (++d_ == D) { d_ = 0; ++img; } } }
            if (!inside) continue;
            (void)wc; (void)hc; (void)dc; (void)ic;
            const __nv_bfloat16 *xs = x + (((ic * D + d2) * H + h2) * W + w2) * cpin + ci0;
            const __nv_bfloat16 *ds = dy + p * cpout + co0;
            float xv[4], dv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                xv[j] = ci0 + j < cin ? __bfloat162float(xs[j]) : 0.f;
                dv[j] = co0 + j < cout ? __bfloat162float(ds[j]) : 0.f;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(dv[i], xv[j], acc[i][j]);
        }
        float *pb = partial + (long long)blockIdx.x * cout * ntaps * cin;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (co0 + i < cout && ci0 + j < cin) pb[((co0 + i) * ntaps + tap) * cin + ci0 + j] = acc[i][j];
    }
    // bias gradient
    for (int co = threadIdx.x; co < cout; co += blockDim.x) {
        float s = 0.f;
        for (long long p = p0; p < p1; ++p) s += __bfloat162float(dy[p * cpout + co]);
        partial_b[(long long)blockIdx.x * cout + co] = s;
    }
}

// out[i] (+)= sum_b partial[b][i], fixed order
__global__ void k_reduce_rows(const float *__restrict__ partial, int nblk, int n, float *__restrict__ out,
                              int accumulate) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float s = accumulate ? out[i] : 0.f;
        for (int b = 0; b < nblk; ++b) s += partial[(long long)b * n + i];
        out[i] = s;
    }
}

// ---- host launchers -------------------------------------------------------------------------

static int pad_npad(int cout) { return cout <= 16 ? 16 : 32; }

int conv_packed_bytes(int n_out, int ntaps, int cp_in) {
    const int npad = pad_npad(n_out);
    const int k = ntaps * cp_in, kpad = (k + 15) & ~15;
    return npad * kpad * 2;
}

int conv_pack(const float *w, int cout, int ntaps, int cin, int cp_in, int flip, uint8_t *out, cudaStream_t st) {
    const int n_out = flip ? cin : cout;
    const int npad = pad_npad(n_out);
    const int k = ntaps * cp_in, kpad = (k + 15) & ~15;
    const long long total = (long long)npad * kpad;
    k_pack_weights<<<(int)std::min<long long>(4096, (total + 255) / 256), 256, 0, st>>>(w, cout, ntaps, cin, cp_in,
                                                                                       npad, kpad / 8, flip, out);
    CBCT_LAUNCH_CHECK("conv weight pack");
    return 0;
}

template <int NPAD, int EPI>
static int launch_conv(const ConvArgs &a, cudaStream_t st) {
    const int bbytes = a.kgroups * NPAD * 16;
    const size_t smem = 1024 + kStages * kAStageBytes + ((bbytes + 127) & ~127) + 8 * (2 * kStages + 4) + 64;
    if (smem > 220 * 1024) return fail(CBCT_EINVAL, "conv: weights do not fit in shared memory");
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<NPAD, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "conv smem attribute");
    // x as a 5-D tensor (channels, W, H, D, images); one box = 8 channels x 128 pixels
    CUtensorMap xmap;
    const uint64_t cp = (uint64_t)a.cpin;
    const uint64_t dims[5] = {cp, (uint64_t)a.W, (uint64_t)a.H, (uint64_t)a.D, (uint64_t)a.nimg};
    const uint64_t strides[4] = {cp * 2, cp * 2 * a.W, cp * 2 * a.W * a.H, cp * 2 * a.W * a.H * a.D};
    const uint32_t box[5] = {8, 128, 1, 1, 1};
    int rc = encode_tmap(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, a.x, dims, strides, box);
    if (rc) return rc;
    int dev = 0, nsm = 152, smem_sm = 228 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int per_sm = std::max(1, std::min(8, smem_sm / (int)(smem + 1024)));
    const long long ntiles = (long long)a.nimg * a.D * a.H * ((a.W + 127) / 128);
    const int grid = (int)std::min<long long>(ntiles, (long long)nsm * per_sm);
    k_conv_tc<NPAD, EPI><<<grid, kWsThreads, smem, st>>>(xmap, a);
    CBCT_LAUNCH_CHECK("conv launch");
    return 0;
}

// Runs one convolution with packed weights (see conv_pack). n_out = number of GEMM
// output channels (cout, or cin for the input-gradient convolution).
int conv_run(const ConvArgs &a0, int n_out, int epi, cudaStream_t st) {
    ConvArgs a = a0;
    const int npad = pad_npad(n_out);
    if (a.cpin % 8 || (epi != EPI_RESIDUAL_F32 && a.cpout % 8)) return fail(CBCT_EINVAL, "conv: channel strides must be multiples of 8");
    a.cin_groups = a.cpin / 8;
    const int k = (a.taps3d ? 27 : 9) * a.cpin;
    a.kgroups = ((k + 15) & ~15) / 8;
    if (npad == 16) {
        if (epi == EPI_ACT_BF16) return launch_conv<16, EPI_ACT_BF16>(a, st);
        if (epi == EPI_RESIDUAL_F32) return launch_conv<16, EPI_RESIDUAL_F32>(a, st);
        return launch_conv<16, EPI_MASK_BF16>(a, st);
    }
    if (epi == EPI_ACT_BF16) return launch_conv<32, EPI_ACT_BF16>(a, st);
    if (epi == EPI_RESIDUAL_F32) return launch_conv<32, EPI_RESIDUAL_F32>(a, st);
    return launch_conv<32, EPI_MASK_BF16>(a, st);
}

// dW (+)= sum_p dY[p] x X[p + tap], db (+)= sum_p dY[p]; partial sums in scratch.
int conv_wgrad(const __nv_bfloat16 *x, int cpin, int cin, const __nv_bfloat16 *dy, int cpout, int cout, int nimg, int D,
               int H, int W, int taps3d, float *dw, float *db, int accumulate, cudaStream_t st) {
    const int ntaps = taps3d ? 27 : 9;
    const long long npix = (long long)nimg * D * H * W;
    const int nblk = (int)std::min<long long>(152LL * 4, std::max<long long>(1, (npix + 1023) / 1024));
    const int ppb = (int)((npix + nblk - 1) / nblk);
    const int nw = cout * ntaps * cin;
    float *part = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&part, sizeof(float) * (long long)nblk * (nw + cout), st));
    float *partb = part + (long long)nblk * nw;
    k_conv_wgrad<<<nblk, 256, 0, st>>>(x, cpin, cin, dy, cpout, cout, nimg, D, H, W, taps3d, ppb, part, partb);
    k_reduce_rows<<<(nw + 255) / 256, 256, 0, st>>>(part, nblk, nw, dw, accumulate);
    k_reduce_rows<<<1, 256, 0, st>>>(partb, nblk, cout, db, accumulate);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, st);
    if (e != cudaSuccess) return cuda_fail(e, "conv wgrad");
    return 0;
}

}  // namespace cbct

using namespace cbct;

extern "C" int cbct_conv(const void *x, int nimg, int D, int H, int W, int cpin, int taps3d, const float *w,
                         const float *bias, int cin, int cout, int flip, int epi, float slope, void *y, int cpout,
                         const void *mask, float *state, long long sstride, int *status, void *stream) {
    if (!x || !w || nimg < 1 || D < 1 || H < 1 || W < 1 || cin < 1 || cout < 1 || cpin % 8 ||
        cpin < (flip ? cout : cin))
        return fail(CBCT_EINVAL, "cbct_conv: invalid argument (sizes, or cpin below the input channels)");
    const int n_out = flip ? cin : cout;
    if (n_out > 32) return fail(CBCT_EINVAL, "cbct_conv: at most 32 output channels");
    if (epi < 0 || epi > 2) return fail(CBCT_EINVAL, "cbct_conv: bad epilogue");
    if ((epi == EPI_RESIDUAL_F32 && !state) || (epi != EPI_RESIDUAL_F32 && (!y || cpout < n_out)) ||
        (epi == EPI_MASK_BF16 && !mask) || !status)
        return fail(CBCT_EINVAL, "cbct_conv: missing output");
    cudaStream_t st = (cudaStream_t)stream;
    const int ntaps = taps3d ? 27 : 9;
    const int bytes = conv_packed_bytes(n_out, ntaps, cpin);
    uint8_t *pk = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&pk, bytes, st));
    int rc = conv_pack(w, cout, ntaps, cin, cpin, flip, pk, st);
    if (rc == 0) {
        ConvArgs a{};
        a.x = static_cast<const __nv_bfloat16 *>(x);
        a.wpk = pk;
        a.bias = bias;
        a.nimg = nimg; a.D = D; a.H = H; a.W = W;
        a.cpin = cpin;
        a.taps3d = taps3d;
        a.cout = n_out;
        a.slope = slope;
        a.y = static_cast<__nv_bfloat16 *>(y);
        a.cpout = cpout;
        a.mask = static_cast<const __nv_bfloat16 *>(mask);
        a.state = state;
        a.sstride = sstride;
        a.status = status;
        rc = conv_run(a, n_out, epi, st);
    }
    cudaFreeAsync(pk, st);
    return rc;
}

extern "C" int cbct_conv_wgrad(const void *x, int cpin, int cin, const void *dy, int cpout, int cout, int nimg, int D,
                               int H, int W, int taps3d, float *dw, float *db, int accumulate, void *stream) {
    if (!x || !dy || !dw || !db || cin < 1 || cout < 1) return fail(CBCT_EINVAL, "cbct_conv_wgrad: invalid argument");
    return conv_wgrad(static_cast<const __nv_bfloat16 *>(x), cpin, cin, static_cast<const __nv_bfloat16 *>(dy), cpout,
                      cout, nimg, D, H, W, taps3d, dw, db, accumulate, (cudaStream_t)stream);
}
