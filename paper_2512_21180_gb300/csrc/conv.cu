// 3x3 (2D, dual block) and 3x3x3 (3D, primal block) convolutions of the learned
// primal-dual network (paper Sec. 2.6, Algorithm 1 blocks Gamma and Lambda; here
// the 3-layer width-32 blocks of the learned primal-dual workload), stride 1, zero
// "same" padding. BF16 operands, FP32 accumulation.
//
// Forward (and input-gradient) convolution = implicit GEMM on the fifth-generation
// tensor cores: D[128 pixels][N] = sum_K A[pixel][K] B[n][K], K = (tap, input
// channel). A CTA walks a contiguous range of tiles of 128 consecutive output pixels
// along W and RPT output rows. One TMA producer warp loads, per tile and input
// plane, the RPT + 2 input rows the 3x3 taps touch (130 pixels with the halo, zero
// outside the image) as one box into a ring of stages; since a K-major core matrix
// is 8 pixels x 16 B contiguous, every column tap is the same row region addressed
// 16 B per pixel later, so each input row is read once per tile rather than once
// per tap. One thread issues 128 x N x 16 tcgen05.mma, N = RPT x NPAD (the RPT
// output rows' weights stacked), into several TMEM accumulators; sixteen epilogue
// warps drain them with tcgen05.ld. The packed weights (B) stay in shared memory
// for the CTA's lifetime. The epilogue applies bias + LeakyReLU (BF16 row-blocked
// out), a residual update of an FP32 channel-first state, or an activation mask.
//
// Weight gradients run on the tensor cores as well (the pixels are the K dimension,
// operands MN-major straight from the same row-halo stages), one partial per CTA
// reduced in a fixed order; a CUDA-core kernel covers 16-channel inputs.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "geom_impl.h"
#include "tcgen05.cuh"

namespace cbct {

enum ConvEpi { EPI_ACT_BF16 = 0, EPI_RESIDUAL_F32 = 1, EPI_MASK_BF16 = 2 };

struct ConvArgs {
    const __nv_bfloat16 *x;  // [nimg][D][H][cpin / 8][W][8]: rows of channel groups
    const uint8_t *wpk;      // packed B operand (k_pack_weights)
    const float *bias;       // [cout] or null
    int nimg, D, H, W;
    int cpin, cin_groups;    // channels per pixel (8, 16, 32 or 64), cpin / 8
    int G;                   // pixels per TMA box row (4, 2 or 1: the largest dividing W)
    int taps3d;              // 1: 3x3x3, 0: 3x3 over (H, W)
    int bbytes;              // packed B operand bytes (conv_packed_bytes)
    int cout;
    int cin;                 // weight gradient: input channels
    float slope;
    __nv_bfloat16 *y;        // EPI_ACT_BF16 / EPI_MASK_BF16 output [nimg][D][H][cpout / 8][W][8]
    int cpout;
    const __nv_bfloat16 *mask;  // EPI_MASK_BF16: forward activation (same layout as y); out *= (mask > 0 ? 1 : slope)
    float *state;            // EPI_RESIDUAL_F32: state[c * sstride + pixel] = state_in[..] + v
    const float *state_in;   // (may equal state)
    int state_in_zero;       // the old state is zero: state = v without reading state_in
    long long sstride;
    int smap_on;             // EPI_RESIDUAL_F32: channel c lives in plane smap[c] (c < 8) instead of c
    int smap[8];
    int ssub;                // EPI_RESIDUAL_F32: state = state_in - v (undoes an additive update)
    int qoff;                // first output channel group of this launch (outputs 8 qoff on): a
                             // layer with more than 32 outputs runs as launches of 32
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

// Epilogue of one output pixel: TMEM accumulators -> bias / activation / residual.
// `row` = (img * D + d) * H + h, `w` the column; `bias` is held in registers (zeros
// when the layer has none). The mask is read through the read-only path so that no
// load waits behind the stores of earlier rows. Every global load is issued before the first
// store so that one memory latency covers the row.
template <int NPAD, int EPI>
__device__ __forceinline__ void conv_epilogue(const ConvArgs &a, const float *acc, const float *bias, long long row,
                                              int w) {
    const long long p = row * a.W + w;
    if constexpr (EPI == EPI_RESIDUAL_F32) {
#pragma unroll
        for (int c0 = 0; c0 < NPAD; c0 += 8) {  // 8 channels per batch of loads
            if (c0 >= a.cout) break;
            float old[8];
            long long off[8];
#pragma unroll
            for (int c = 0; c < 8; ++c)
                off[c] = (long long)(a.smap_on && c0 == 0 ? a.smap[c] : 8 * a.qoff + c0 + c) * a.sstride + p;
#pragma unroll
            for (int c = 0; c < 8; ++c) old[c] = (c0 + c < a.cout && !a.state_in_zero) ? a.state_in[off[c]] : 0.f;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c0 + c < a.cout) {
                    const float v = acc[c0 + c] + bias[c0 + c];
                    a.state[off[c]] = a.ssub ? old[c] - v : old[c] + v;
                }
        }
    } else {
        // channel group qoff + q of this pixel: (row * (cpout / 8) + qoff + q) * W * 8 + w * 8
        const long long gstride = (long long)a.W * 8, o0 = (row * (a.cpout / 8) * a.W + w) * 8 + a.qoff * gstride;
        __nv_bfloat16 *o = a.y + o0;
        constexpr int kG = NPAD / 8;
        uint4 mv[kG];
#pragma unroll
        for (int q = 0; q < kG; ++q) {
            mv[q] = make_uint4(0u, 0u, 0u, 0u);
            if constexpr (EPI == EPI_MASK_BF16)
                if ((a.qoff + q) * 8 < a.cpout) mv[q] = __ldg(reinterpret_cast<const uint4 *>(a.mask + o0 + q * gstride));
        }
#pragma unroll
        for (int q = 0; q < kG; ++q) {
            if ((a.qoff + q) * 8 >= a.cpout) break;
            // padded channels (c >= cout) hold exact zeros: zero weights and zero bias
            const __nv_bfloat162 *m2 = reinterpret_cast<const __nv_bfloat162 *>(&mv[q]);
            uint32_t packed[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = q * 8 + 2 * j;
                float v0 = acc[c], v1 = acc[c + 1];
                if constexpr (EPI == EPI_ACT_BF16) {
                    // LeakyReLU as max(v, slope v): 0 <= slope <= 1 (checked on the host)
                    v0 += bias[c];
                    v1 += bias[c + 1];
                    v0 = fmaxf(v0, v0 * a.slope);
                    v1 = fmaxf(v1, v1 * a.slope);
                } else {
                    const float2 m = __bfloat1622float2(m2[j]);
                    v0 = m.x > 0.f ? v0 : v0 * a.slope;
                    v1 = m.y > 0.f ? v1 : v1 * a.slope;
                }
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(v0, v1);
                packed[j] = *reinterpret_cast<const uint32_t *>(&h2);
            }
            *reinterpret_cast<uint4 *>(o + q * gstride) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        }
    }
}

// Row-halo layout. A tile is 128 consecutive output pixels along W of RPT output
// rows h0 .. h0 + RPT - 1 (RPT from 1 to 4, the most whose weights fit in shared
// memory next to two input stages, see conv_rpt); an A stage holds
// the NR = RPT + 2 input rows h0 - 1 .. h0 + RPT of one input plane as NR * CGP
// regions (CGP = CG rounded up to even) of RS = 16 G R bytes (2176, 2112 or 2080;
// at most kRowStride). Region r * CG + g holds channel group g of input row h0 - 1 + r
// as 8-channel pixels 16 B apart from column w0 - G on, where G (4, 2 or 1) is the
// TMA box row width in pixels. In
// the row-blocked input layout a row's channel group is W x 16 contiguous bytes, so
// one TMA box {G pixels x 8 channels, R = ceil((129 + G) / G), CG groups, NR image
// rows} fills a stage (zero outside the image); stages start on 128-byte boundaries
// as a tiled TMA destination must. A K-major core matrix is 8 rows x 16 B = 128
// contiguous bytes, so with the 8-row group stride SBO = 128 the A operand for input
// row r and column tap dw is region r started (G - 1 + dw) pixels in, and the
// K-adjacent core matrix (next channel group) lies LBO = RS further. The B operand of
// input row r stacks the weights of tap (dh = r - 1 - o, dw) for the output rows o it
// feeds (the row units below), so one MMA serves up to three output rows (four for a
// row pair). With a single channel group (CG = 1) the two K halves of an MMA are
// instead two consecutive input rows (LBO = RS) and only region NR, the partner of the
// last row when NR is odd, stays zero. Every input row is loaded once per tile.
constexpr int kRowStride = 2176;         // 17 x 128 >= RS = 16 R G for G = 1, 2, 4
__host__ __device__ constexpr int conv_box_rows(int G) { return (129 + G + G - 1) / G; }
constexpr int kMaxStages = 8;            // A ring depth (chosen per launch, <= 8)
constexpr int kMaxAcc = 8;               // TMEM accumulators (tiles in flight past the MMA), at most
__host__ __device__ constexpr int conv_nacc(int n) { return 512 / n < kMaxAcc ? 512 / n : kMaxAcc; }
__host__ __device__ constexpr int conv_pow2(int n) { return n <= 32 ? 32 : 2 * conv_pow2((n + 1) / 2); }
constexpr int kEpiGroups = 4;            // epilogue warpgroups; group q drains the tiles j = q mod 4
constexpr int kWsThreads = 32 * (4 * kEpiGroups + 2);  // epilogue warps, then the TMA producer and the MMA warp
constexpr int kProdWarp = 4 * kEpiGroups, kMmaWarp = 4 * kEpiGroups + 1;

__host__ __device__ constexpr int conv_cgp(int cg) { return (cg + 1) & ~1; }
__host__ __device__ constexpr int conv_stage_bytes(int cg, int rpt) { return (rpt + 2) * conv_cgp(cg) * kRowStride; }

// Row units of the B operand. Unit j is input row j of the NR = RPT + 2 rows of a box
// or, with one channel group (pair), the row pair (2j, 2j + 1), row NR being the zero
// partner when NR is odd. Input row r feeds output rows o = r - 2 .. r (tap
// dh = r - 1 - o), so unit j stacks the weights of output rows lo .. hi only:
// N = (hi - lo + 1) NPAD, accumulated into TMEM columns lo NPAD onwards. The
// "initialising" units — rows 2, 5, 8, ... (output rows 3t .. 3t + 2), or pairs
// 1, 3, 5, ... (output rows 4t .. 4t + 3) — cover the RPT output rows exactly once, so
// issuing them first, each starting with an overwriting MMA, writes the whole
// accumulator before any other unit adds to it.
__host__ __device__ constexpr int conv_imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int conv_units(int rpt, int pair) { return pair ? (rpt + 3) / 2 : rpt + 2; }
__host__ __device__ constexpr bool conv_unit_init(int j, int pair) { return pair ? (j & 1) == 1 : j % 3 == 2; }
__host__ __device__ constexpr int conv_unit_lo(int j, int pair) {
    return (pair ? 2 * j : j) >= 2 ? (pair ? 2 * j : j) - 2 : 0;
}
__host__ __device__ constexpr int conv_unit_hi(int j, int rpt, int pair) {
    return conv_imin(pair ? conv_imin(2 * j + 1, rpt + 1) : j, rpt - 1);
}
// j-th unit in issue order: the initialising units, then the others, each in row order
__host__ __device__ constexpr int conv_unit_order(int jj, int rpt, int pair) {
    int k = 0;
    for (int j = 0; j < conv_units(rpt, pair); ++j)
        if (conv_unit_init(j, pair) && k++ == jj) return j;
    for (int j = 0; j < conv_units(rpt, pair); ++j)
        if (!conv_unit_init(j, pair) && k++ == jj) return j;
    return 0;
}
__host__ __device__ constexpr int conv_unit_rows(int j, int rpt, int pair) {
    return conv_unit_hi(j, rpt, pair) - conv_unit_lo(j, pair) + 1;
}
// K groups (8 channels each) of a unit, ordered (column tap, channel group) or (column tap, half)
__host__ __device__ constexpr int conv_unit_groups(int cgp, int pair) { return pair ? 6 : 3 * cgp; }
__host__ __device__ constexpr int conv_unit_off(int j, int rpt, int pair, int cgp, int npad) {
    int o = 0;
    for (int i = 0; i < j; ++i) o += conv_unit_groups(cgp, pair) * conv_unit_rows(i, rpt, pair) * npad * 16;
    return o;
}
__host__ __device__ constexpr int conv_plane_bytes(int rpt, int pair, int cgp, int npad) {
    return conv_unit_off(conv_units(rpt, pair), rpt, pair, cgp, npad);
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}

// Tile t = ((img * D + d) * nh + th) * ntw + wt: output rows th * RPT .. + RPT - 1 of
// plane (img, d), columns w0 = 128 wt .. w0 + 127. Consecutive tiles are stepped
// without divisions.
struct TileCoord {
    int img, d, th, w0;
};
__device__ __forceinline__ TileCoord tile_coord(long long t, int D, int nh, int ntw) {
    TileCoord c;
    c.w0 = (int)(t % ntw) * 128; t /= ntw;
    c.th = (int)(t % nh); t /= nh;
    c.d = (int)(t % D);
    c.img = (int)(t / D);
    return c;
}
__device__ __forceinline__ void tile_next(TileCoord &c, int D, int nh, int W) {
    c.w0 += 128;
    if (c.w0 < W) return;
    c.w0 = 0;
    if (++c.th < nh) return;
    c.th = 0;
    if (++c.d < D) return;
    c.d = 0;
    ++c.img;
}

// Warp-specialized convolution over row-halo stages. Item i of a CTA = (tile
// t_begin + i / nch, input plane dd = i % nch - 1 for 3-D, the tile's own plane for
// 2-D) on ring stage i % nst.
//  producer (warp 16, one lane): waits until the stage is free (empty[s]) and loads
//    the item's NR input rows with one TMA box, completion counted on full[s]; an
//    input plane outside the volume only arrives (its MMAs are skipped).
//  MMA (warp 17, one lane): per tile picks TMEM accumulator j % nacc once the epilogue
//    has drained it (acce), waits for each item (full[s]), issues one 128 x N x 16
//    MMA per (input row, column tap, pair of channel groups) or, for CG = 1, per
//    (pair of input rows, column tap), commits the stage to
//    empty[s] and, after the tile's last item, the accumulator to accf.
//  epilogue (warps 0-15): warpgroup q takes the tiles j = q mod 4; each warp waits
//    for accf, reads its 32 TMEM lanes (= pixels), releases the accumulator, applies
//    the epilogue to each of the RPT output rows and stores.
template <int NPAD, int EPI, int CG, int RPT>
__global__ void __launch_bounds__(kWsThreads) k_conv_tc(const __grid_constant__ CUtensorMap xmap, ConvArgs a, int nst) {
    constexpr int kCGP = conv_cgp(CG);
    constexpr int kNR = RPT + 2;
    constexpr int kN = RPT * NPAD;
    constexpr bool kPair = CG == 1;               // K halves = consecutive input rows
    constexpr int kStageBytes = conv_stage_bytes(CG, RPT);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int bbytes = a.bbytes;
    unsigned char *sA = sm;
    unsigned char *sB = sm + nst * kStageBytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + ((bbytes + 127) & ~127));
    uint64_t *empty = full + kMaxStages;
    uint64_t *accf = empty + kMaxStages;
    uint64_t *acce = accf + kMaxAcc;
    float *sbias = reinterpret_cast<float *>(acce + kMaxAcc);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sbias + NPAD);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kAcc = conv_nacc(kN);
    // warpgroup q's first tile is tile q: with fewer accumulators than warpgroups it would
    // wait on a barrier phase that has not started yet (a parity wait that passes at once)
    static_assert(kAcc >= kEpiGroups, "need one TMEM accumulator per epilogue warpgroup");
    constexpr uint32_t kCols = conv_pow2(kAcc * kN);  // TMEM allocation: a power of two >= 32
    constexpr uint32_t kIdesc = idesc_bf16_f32(128, kN);
    const int rs = 16 * a.G * conv_box_rows(a.G);  // region stride (bytes)

    if (warp == 0) tmem_alloc(tmem_slot, kCols);
    if (tid == 32) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int j = 0; j < kAcc; ++j) {
            mbar_init(&accf[j], 1);
            mbar_init(&acce[j], 4);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (tid < NPAD) sbias[tid] = (a.bias && tid < a.cout) ? a.bias[tid] : 0.f;
    for (int i = tid; i < bbytes / 16; i += kWsThreads)
        reinterpret_cast<uint4 *>(sB)[i] = __ldg(reinterpret_cast<const uint4 *>(a.wpk) + i);
    if constexpr (kPair && (kNR & 1)) {
        // CG = 1, odd NR: region NR is the zero partner of the last row (its weights
        // are zero too)
        constexpr int kQ = kRowStride / 16;
        for (int i = tid; i < nst * kQ; i += kWsThreads) {
            const int s = i / kQ, q = i - s * kQ;
            reinterpret_cast<uint4 *>(sA + s * kStageBytes + kNR * rs)[q] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int ntw = (a.W + 127) / 128, nh = (a.H + RPT - 1) / RPT;
    const long long ntiles = (long long)a.nimg * a.D * nh * ntw;
    const int nch = a.taps3d ? 3 : 1;
    const long long per_cta = (ntiles + gridDim.x - 1) / gridDim.x;
    const long long t_begin = (long long)blockIdx.x * per_cta;
    const long long my_tiles = t_begin < ntiles ? min(per_cta, ntiles - t_begin) : 0;
    const long long total = my_tiles * nch;
    const uint32_t sA_u = smem_u32(sA), sB_u = smem_u32(sB);

    if (warp == kProdWarp) {
        if (lane == 0) {
            prefetch_tmap(&xmap);
            TileCoord tc = tile_coord(t_begin, a.D, nh, ntw);
            const uint32_t box_bytes = (uint32_t)(kNR * CG * rs);
            int c = 0, s = 0;
            uint32_t ph = 0;
            for (long long i = 0; i < total; ++i) {
                if (i >= nst && !mbar_wait(&empty[s], ph ^ 1u, a.status)) {
                    *abort_flag = 1;
                    break;
                }
                const int d2 = tc.d + (nch == 3 ? c - 1 : 0);
                if (d2 < 0 || d2 >= a.D) {
                    mbar_arrive_expect_tx(&full[s], 0u);  // plane outside the volume: no MMAs either
                } else {
                    mbar_arrive_expect_tx(&full[s], box_bytes);
                    tma_load_5d(sA_u + (uint32_t)(s * kStageBytes), &xmap, 0, tc.w0 / a.G - 1, 0, tc.th * RPT - 1,
                                tc.img * a.D + d2, &full[s]);
                }
                if (++c == nch) {
                    c = 0;
                    tile_next(tc, a.D, nh, a.W);
                }
                if (++s == nst) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            // column tap dw of input row r reads region r from pixel G - 1 + dw on
            const uint32_t rs16 = (uint32_t)(rs / 16);
            const uint64_t adesc0 = smem_desc_kmajor(sA_u + (uint32_t)((a.G - 1) * 16), rs, 128);
            constexpr int kNU = conv_units(RPT, kPair);
            constexpr int kPlaneB = conv_plane_bytes(RPT, kPair, kCGP, NPAD);
            TileCoord tc = tile_coord(t_begin, a.D, nh, ntw);
            int s = 0;
            uint32_t ph = 0;
            for (long long j = 0; j < my_tiles && !*abort_flag; ++j) {
                const int ab = (int)(j % kAcc);
                if (j >= kAcc && !mbar_wait(&acce[ab], (uint32_t)(((j / kAcc) - 1) & 1), a.status)) {
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(ab * kN);
                uint32_t acc_flag = 0;  // the tile's first MMA overwrites the accumulator
                for (int c = 0; c < nch; ++c) {
                    if (!mbar_wait(&full[s], ph, a.status)) {
                        *abort_flag = 1;
                        break;
                    }
                    const int d2 = tc.d + (nch == 3 ? c - 1 : 0);
                    if (d2 >= 0 && d2 < a.D) {
                        tc_fence_after();
                        // descriptor start-address fields are address >> 4: offsets add directly
                        const uint64_t ad = adesc0 + (uint64_t)((s * kStageBytes) >> 4);
                        // the initialising units first (their first MMA overwrites its columns in
                        // the tile's first plane), then the others
#pragma unroll
                        for (int jj = 0; jj < kNU; ++jj) {
                            const int j = conv_unit_order(jj, RPT, kPair);
                            const int nj = conv_unit_rows(j, RPT, kPair) * NPAD;
                            const uint32_t idesc = idesc_bf16_f32(128, nj);
                            const uint32_t dtj = dt + (uint32_t)(conv_unit_lo(j, kPair) * NPAD);
                            const uint64_t bd = smem_desc_kmajor(
                                sB_u + (uint32_t)(c * kPlaneB + conv_unit_off(j, RPT, kPair, kCGP, NPAD)),
                                (uint32_t)(nj * 16), 128);
                            uint32_t acc = conv_unit_init(j, kPair) ? acc_flag : 1u;
                            if constexpr (kPair) {
#pragma unroll
                                for (int dw = 0; dw < 3; ++dw) {
                                    const uint32_t ao = (uint32_t)(2 * j) * rs16 + (uint32_t)dw;
                                    const uint32_t bo = (uint32_t)((dw * 2 * nj * 16) >> 4);
                                    mma_bf16(dtj, ad + ao, bd + bo, idesc, acc);
                                    acc = 1u;
                                }
                            } else {
#pragma unroll
                                for (int dw = 0; dw < 3; ++dw)
#pragma unroll
                                    for (int kp = 0; kp < kCGP; kp += 2) {
                                        const uint32_t ao = (uint32_t)(j * CG + kp) * rs16 + (uint32_t)dw;
                                        const uint32_t bo = (uint32_t)(((dw * kCGP + kp) * nj * 16) >> 4);
                                        mma_bf16(dtj, ad + ao, bd + bo, idesc, acc);
                                        acc = 1u;
                                    }
                            }
                        }
                        acc_flag = 1u;
                    }
                    mma_commit(&empty[s]);
                    if (++s == nst) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (*abort_flag) break;
                mma_commit(&accf[ab]);
                tile_next(tc, a.D, nh, a.W);
            }
        }
    } else {
        // epilogue: warpgroup q = warp / 4 takes tiles q, q + 4, ...; warp w reads TMEM
        // lanes 32 (w % 4) .. + 31 = tile pixels
        const int q = warp >> 2, wq = warp & 3;
        float bias[NPAD];
#pragma unroll
        for (int c = 0; c < NPAD; ++c) bias[c] = sbias[c];
        TileCoord tc = tile_coord(t_begin + q, a.D, nh, ntw);
        for (long long j = q; j < my_tiles; j += kEpiGroups) {
            const int ab = (int)(j % kAcc);
            if (!mbar_wait(&accf[ab], (uint32_t)((j / kAcc) & 1), a.status)) {
                *abort_flag = 1;
                break;
            }
            tc_fence_after();
            const int w = tc.w0 + wq * 32 + lane;
            // one output row at a time (NPAD accumulator columns each); the accumulator is
            // released after the last row's columns are in registers
#pragma unroll
            for (int o = 0; o < RPT; ++o) {
                uint32_t raw[NPAD];
#pragma unroll
                for (int c0 = 0; c0 < NPAD; c0 += 16)
                    tmem_ld16_issue(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)(ab * kN + o * NPAD + c0), raw + c0);
                tmem_wait_ld();
                if (o == RPT - 1) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acce[ab]);
                }
                const int h = tc.th * RPT + o;
                float acc[NPAD];
#pragma unroll
                for (int c = 0; c < NPAD; ++c) acc[c] = __uint_as_float(raw[c]);
                if (w < a.W && h < a.H)
                    conv_epilogue<NPAD, EPI>(a, acc, bias, ((long long)tc.img * a.D + tc.d) * a.H + h, w);
            }
#pragma unroll
            for (int k = 0; k < kEpiGroups; ++k) tile_next(tc, a.D, nh, a.W);
        }
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// ---- weight packing ---------------------------------------------------------------------

// B operand in row units (see conv_unit_lo): per input plane c of nch, unit j,
// group g = dw * cgp + cg (or dw * 2 + half with pair_rows), rows n = (o - lo) * npad +
// co for output rows o = lo .. hi and output channels co, 8 K-channels each, as
// K-major core matrices (8 rows x 16 B) — element e of the buffer is
// ((plane, unit, g, n) x 8 + k) in that order. The weight is that of tap
// (dd = c - 1, dh = r - 1 - o, dw - 1) with r = j (or 2 j + half), zero when |dh| > 1
// or r = NR. w: FP32 [cout][taps][cin]. flip = 1 packs the input-gradient
// convolution instead: output channel co = ci, input channel = co of w, mirrored tap.
// o0 = first output channel of the launch (0, or 32 for the second half of a layer
// with more than 32 outputs): slot co holds output o0 + co.
// Value of element e of the packed B operand (layout above).
__device__ __forceinline__ float pack_weight_value(const float *__restrict__ w, long long e, int cout, int taps3d,
                                                   int cin, int cgp, int npad, int rpt, int pair_rows, int flip,
                                                   int o0) {
    const int ntaps = taps3d ? 27 : 9, nr = rpt + 2;
    const int nu = conv_units(rpt, pair_rows), ng = conv_unit_groups(cgp, pair_rows);
    const long long plane = conv_plane_bytes(rpt, pair_rows, cgp, npad) / 2;  // elements
    const int c = (int)(e / plane);
    long long rem = e - c * plane;
    int j = 0;
    for (; j < nu - 1; ++j) {
        const long long ub = (long long)ng * conv_unit_rows(j, rpt, pair_rows) * npad * 8;
        if (rem < ub) break;
        rem -= ub;
    }
    const int nj = conv_unit_rows(j, rpt, pair_rows) * npad;
    const int kin = (int)(rem & 7);
    const int n = (int)((rem >> 3) % nj);
    const int g = (int)((rem >> 3) / nj);
    int r, dw, cg;
    if (pair_rows) {
        dw = g >> 1;
        r = 2 * j + (g & 1);
        cg = 0;
    } else {
        dw = g / cgp;
        cg = g - dw * cgp;
        r = j;
    }
    const int o = conv_unit_lo(j, pair_rows) + n / npad, co = o0 + n % npad, ch = cg * 8 + kin, dh = r - 1 - o;
    float v = 0.f;
    if (r < nr && dh >= -1 && dh <= 1) {
        const int tap = taps3d ? (c * 3 + dh + 1) * 3 + dw : (dh + 1) * 3 + dw;
        if (!flip) {
            if (co < cout && ch < cin) v = w[((long long)co * ntaps + tap) * cin + ch];
        } else {
            if (co < cin && ch < cout) v = w[((long long)ch * ntaps + (ntaps - 1 - tap)) * cin + co];
        }
    }
    return v;
}

__global__ void k_pack_weights(const float *__restrict__ w, int cout, int taps3d, int cin, int cgp, int npad, int rpt,
                               int pair_rows, int flip, int o0, uint8_t *__restrict__ out) {
    const long long total = (taps3d ? 3 : 1) * (long long)conv_plane_bytes(rpt, pair_rows, cgp, npad) / 2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
        reinterpret_cast<__nv_bfloat16 *>(out)[e] =
            __float2bfloat16_rn(pack_weight_value(w, e, cout, taps3d, cin, cgp, npad, rpt, pair_rows, flip, o0));
}

// Several layers in one launch: job blockIdx.y packs params + w_off into out + out_off.
__global__ void k_pack_jobs(const ConvPackJob *__restrict__ jobs, const float *__restrict__ params,
                            uint8_t *__restrict__ out) {
    const ConvPackJob J = jobs[blockIdx.y];
    __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(out + J.out_off);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < J.nelem; e += (long long)gridDim.x * blockDim.x)
        o[e] = __float2bfloat16_rn(pack_weight_value(params + J.w_off, e, J.cout, J.taps3d, J.cin, J.cgp, J.npad,
                                                     J.rpt, J.pair, J.flip, J.o0));
}

// ---- weight gradient on the tensor cores ------------------------------------------------
//
// dW[co][tap][ci] = sum over output pixels p of dY[p][co] X[p + tap][ci]: a GEMM whose K
// dimension is the pixels. In the row-blocked layout a row's channel group is pixels
// 16 B apart with 8 channels contiguous, which is exactly the MN-major canonical core
// matrix (8 M/N elements contiguous x 8 K rows 16 B apart) — so the same row-halo TMA
// stages feed it, with the operands marked transposed in the instruction descriptor
// (for this layout the descriptor's leading byte offset steps along K, the stride
// byte offset along M / N).
// A tile is 128 output pixels of two output rows h0, h0 + 1 of one image plane d; a CTA
// handles one depth tap dd (3-D: input plane d + dd - 1; the grid's y index) for all its
// tiles. Its stage holds the input rows h0 - 1 .. h0 + 2 (4 rows x 4 channel groups, the
// region layout of the forward) and the tile's two dY rows (row o at NCG o groups of 2048
// B, groups beyond the data zero). Per column tap dw and 16-pixel K step, one MMA with
// A = 4 input rows x 32 input channels (M = 128: core matrix j = region j, M stride RS,
// K stride 128 B) and B = both dY rows (N = 2 x 8 NCG: core matrix (o, g) at (o NCG + g)
// 2048 B) accumulates D_dw[(r, ci)][(o, co)] in TMEM over every tile of the CTA. Entry
// (r, o) belongs to tap dh = r - 1 - o: six of the eight (r, o) pairs are taps, and two
// pairs give each tap, so each CTA writes both (o = 0, 1) partials of its 9 taps and a
// fixed-order reduction adds everything (deterministic). Two dY rows per MMA halve the
// MMA count per output row, and the three taps dd in separate CTAs keep the accumulators
// at 3 x N <= 192 TMEM columns, so two CTAs (two MMA issuers) share an SM.
constexpr int kWgThreads = 192;  // warps 0-3 epilogue, 4 TMA producer, 5 MMA
constexpr int kWgStages = 2;
constexpr int kWgXBytes = 4 * 4 * kRowStride;  // 4 input rows x 4 channel groups

__host__ __device__ constexpr uint32_t idesc_bf16_f32_mn(int M, int N) {
    return idesc_bf16_f32(M, N) | (1u << 15) | (1u << 16);  // A and B MN-major
}

// XCG = input channel groups (4, or 1 for 8-channel inputs: each input row is then
// loaded to region 4 r and the regions of groups 1..3 stay zero); NCG = output-channel
// groups per dY row: 2 (16 outputs, the second group zero when cout <= 8) or 4.
// partial: [ndd][gridDim.x][2][cout][9][cin].
template <int XCG, int NCG>
__global__ void __launch_bounds__(kWgThreads) k_conv_wgrad_tc(const __grid_constant__ CUtensorMap xmap,
                                                              const __grid_constant__ CUtensorMap ymap, ConvArgs a,
                                                              int cgo, float *__restrict__ partial) {
    constexpr int kN = 2 * NCG * 8;
    constexpr int kYBytes = 2 * NCG * 2048;
    constexpr int kStage = kWgXBytes + kYBytes;
    constexpr uint32_t kCols = 3 * kN <= 128 ? 128u : 256u;  // 3 accumulators (dw) of kN columns
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + kWgStages * kStage);
    uint64_t *empty = full + kWgStages;
    uint64_t *done = empty + kWgStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);
    int *used = abort_flag + 1;  // [3]: accumulator dw received an MMA
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int dd = blockIdx.y;   // depth tap (3-D: input plane d + dd - 1)
    constexpr uint32_t kIdesc = idesc_bf16_f32_mn(128, kN);
    const int rs = 16 * a.G * conv_box_rows(a.G);

    if (warp == 0) tmem_alloc(tmem_slot, kCols);
    if (tid == 32) {
        for (int s = 0; s < kWgStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 2);  // the MMAs' commit + the MMA thread's release of used[]
        *abort_flag = 0;
        for (int i = 0; i < 3; ++i) used[i] = 0;
        fence_mbar_init();
    }
    if (cgo < NCG) {
        // output-channel groups beyond the data stay zero in both dY rows of every stage
        const int per = 2 * (NCG - cgo) * 128;  // uint4 per stage
        for (int i = tid; i < kWgStages * per; i += kWgThreads) {
            const int s = i / per, q = i - s * per, o = q / ((NCG - cgo) * 128), r = q - o * (NCG - cgo) * 128;
            reinterpret_cast<uint4 *>(sm + s * kStage + kWgXBytes + (o * NCG + cgo) * 2048)[r] =
                make_uint4(0u, 0u, 0u, 0u);
        }
    }
    if constexpr (XCG == 1) {
        // regions 4 r + g, g = 1..3: zero input channels 8..31
        const int q16 = rs / 16;
        for (int i = tid; i < kWgStages * 12 * q16; i += kWgThreads) {
            const int s = i / (12 * q16), rem = i - s * 12 * q16, k = rem / q16, q = rem - k * q16;
            const int region = (k / 3) * 4 + 1 + k % 3;
            reinterpret_cast<uint4 *>(sm + s * kStage + region * rs)[q] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int ntw = (a.W + 127) / 128, nh = (a.H + 1) / 2;
    const long long ntiles = (long long)a.nimg * a.D * nh * ntw;
    const long long per_cta = (ntiles + gridDim.x - 1) / gridDim.x;
    const long long t_begin = (long long)blockIdx.x * per_cta;
    const long long my_tiles = t_begin < ntiles ? min(per_cta, ntiles - t_begin) : 0;
    const uint32_t sm_u = smem_u32(sm);

    if (warp == 4) {
        if (lane == 0) {
            prefetch_tmap(&xmap);
            prefetch_tmap(&ymap);
            TileCoord tc = tile_coord(t_begin, a.D, nh, ntw);
            const uint32_t xbytes = (uint32_t)(4 * XCG * rs), ybytes = (uint32_t)(2 * cgo * 2048);
            int s = 0;
            uint32_t ph = 0;
            for (long long i = 0; i < my_tiles; ++i) {
                if (i >= kWgStages && !mbar_wait(&empty[s], ph ^ 1u, a.status)) {
                    *abort_flag = 1;
                    break;
                }
                const int d2 = tc.d + (a.taps3d ? dd - 1 : 0);
                if (d2 < 0 || d2 >= a.D) {
                    mbar_arrive_expect_tx(&full[s], 0u);  // input plane outside the volume: no MMAs
                } else {
                    const uint32_t st = sm_u + (uint32_t)(s * kStage);
                    mbar_arrive_expect_tx(&full[s], xbytes + ybytes);
                    if constexpr (XCG == 4) {
                        tma_load_5d(st, &xmap, 0, tc.w0 / a.G - 1, 0, 2 * tc.th - 1, tc.img * a.D + d2, &full[s]);
                    } else {
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            tma_load_5d(st + (uint32_t)(4 * r * rs), &xmap, 0, tc.w0 / a.G - 1, 0, 2 * tc.th - 1 + r,
                                        tc.img * a.D + d2, &full[s]);
                    }
#pragma unroll
                    for (int o = 0; o < 2; ++o)
                        tma_load_5d(st + (uint32_t)(kWgXBytes + o * NCG * 2048), &ymap, 0, tc.w0 / a.G, 0,
                                    2 * tc.th + o, tc.img * a.D + tc.d, &full[s]);
                }
                tile_next(tc, a.D, nh, a.W);
                if (++s == kWgStages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            TileCoord tc = tile_coord(t_begin, a.D, nh, ntw);
            int s = 0;
            uint32_t ph = 0;
            uint32_t usedm = 0;  // bit dw: accumulator initialised
            for (long long i = 0; i < my_tiles && !*abort_flag; ++i) {
                if (!mbar_wait(&full[s], ph, a.status)) {
                    *abort_flag = 1;
                    break;
                }
                const int d2 = tc.d + (a.taps3d ? dd - 1 : 0);
                if (d2 >= 0 && d2 < a.D) {
                    tc_fence_after();
                    const uint32_t st = sm_u + (uint32_t)(s * kStage);
#pragma unroll
                    for (int dw = 0; dw < 3; ++dw) {
                        const uint32_t dt = tmem + (uint32_t)(dw * kN);
#pragma unroll
                        for (int ks = 0; ks < 8; ++ks) {
                            // MN-major, no swizzle: the leading byte offset steps along K (8
                            // pixels = 128 B), the stride byte offset along M / N
                            const uint64_t ad = smem_desc_kmajor(st + (uint32_t)((a.G - 1 + dw) * 16 + ks * 256), 128, rs);
                            const uint64_t bd = smem_desc_kmajor(st + kWgXBytes + (uint32_t)(ks * 256), 128, 2048);
                            mma_bf16(dt, ad, bd, kIdesc, (usedm >> dw) & 1u);
                            usedm |= 1u << dw;
                        }
                    }
                }
                mma_commit(&empty[s]);
                tile_next(tc, a.D, nh, a.W);
                if (++s == kWgStages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            for (int k = 0; k < 3; ++k) used[k] = (usedm >> k) & 1u;
            // a CTA without tiles (the last ones when the tiles do not divide evenly) issued
            // no MMA: it arrives directly instead of committing
            if (usedm) mma_commit(done);
            else mbar_arrive(done);
            mbar_arrive(done);
        }
    } else {
        // epilogue (warps 0-3, once): warp w holds accumulator rows 32 w .. 32 w + 31 = input
        // row r = w, input channel = lane; columns (o, co). Pair (r, o) is tap dh = r - 1 - o.
        const bool ok = mbar_wait(done, 0u, a.status);
        tc_fence_after();
        const int r = warp, ci = lane;
        const long long slot = ((long long)dd * gridDim.x + blockIdx.x) * 2;
        const long long per_o = (long long)a.cout * 9 * a.cin;
        for (int dw = 0; dw < 3; ++dw) {
            float v[kN];
#pragma unroll
            for (int c0 = 0; c0 < kN; c0 += 16)
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(dw * kN + c0), v + c0);
            const bool valid = ok && !*abort_flag && used[dw];
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int dh = r - 1 - o;
                if (dh < -1 || dh > 1 || ci >= a.cin) continue;
                float *pb = partial + (slot + o) * per_o;
                const int t9 = (dh + 1) * 3 + dw;
#pragma unroll
                for (int co = 0; co < NCG * 8; ++co)
                    if (co < a.cout) pb[((long long)co * 9 + t9) * a.cin + ci] = valid ? v[o * NCG * 8 + co] : 0.f;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
}

// out[co0 + co][tap][ci0 + ci] (+)= sum over the CTAs of their tap's partials (both
// output-row halves), fixed order: partial [ndd][gpd][2][cout][9][cin], tap = dd * 9 + t9;
// out has cin_full input channels per tap.
__global__ void k_reduce_wgrad(const float *__restrict__ partial, int gpd, int ndd, int cout, int cin,
                               float *__restrict__ out, int accumulate, int co0, int ci0, int cin_full) {
    const int n = cout * 9 * ndd * cin;
    const long long per_o = (long long)cout * 9 * cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % cin, tap = (i / cin) % (9 * ndd), co = i / (cin * 9 * ndd);
        const int d = tap / 9, t9 = tap % 9;
        const long long e = ((long long)co * 9 + t9) * cin + ci;
        const long long o = ((long long)(co0 + co) * 9 * ndd + tap) * cin_full + ci0 + ci;
        float s = accumulate ? out[o] : 0.f;
        for (int b = 0; b < gpd; ++b) {
            const float *p = partial + ((long long)d * gpd + b) * 2 * per_o;
            s += p[e] + p[per_o + e];
        }
        out[o] = s;
    }
}

// partial_b[blk][co] = sum over the block's image rows of dY[row][co] (row-blocked dY,
// cgo channel groups read, rows cgs groups apart): thread (group q, column lane) reads
// 16-byte pixels along the row, then the lanes of each channel are summed in a fixed order.
__global__ void __launch_bounds__(256) k_bias_grad(const __nv_bfloat16 *__restrict__ dy, int cgo, int cgs, int cout,
                                                   long long nrows, int W, int rows_per_block,
                                                   float *__restrict__ partial_b) {
    __shared__ float red[256][9];
    const int tpq = 256 / cgo, q = threadIdx.x / tpq, l = threadIdx.x - q * tpq;
    const long long r0 = (long long)blockIdx.x * rows_per_block, r1 = min(nrows, r0 + rows_per_block);
    float acc[8] = {};
    for (long long row = r0; row < r1; ++row) {
        const uint4 *src = reinterpret_cast<const uint4 *>(dy + (row * cgs + q) * (long long)W * 8);
        for (int w = l; w < W; w += tpq) {
            const uint4 v = __ldg(src + w);
            const __nv_bfloat16 *b = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(b[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) red[threadIdx.x][j] = acc[j];
    __syncthreads();
    const int c = threadIdx.x;
    if (c < cout) {
        const int qc = c / 8, j = c % 8;
        float t = 0.f;
        for (int k = 0; k < tpq; ++k) t += red[qc * tpq + k][j];
        partial_b[(long long)blockIdx.x * cout + c] = t;
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
            // row-blocked layouts: (row * (cp / 8) + c / 8) * W * 8 + w * 8 + c % 8
            const __nv_bfloat16 *xs =
                x + ((((ic * D + d2) * H + h2) * (cpin / 8) + ci0 / 8) * W + w2) * 8 + (ci0 & 7);
            const __nv_bfloat16 *ds = dy + ((((ic * D + dc) * H + hc) * (cpout / 8) + co0 / 8) * W + wc) * 8 + (co0 & 7);
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
        for (long long p = p0; p < p1; ++p) {
            const long long row = p / W;
            const int w = (int)(p - row * W);
            s += __bfloat162float(dy[((row * (cpout / 8) + co / 8) * W + w) * 8 + (co & 7)]);
        }
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

// Bytes of the packed B operand (row units, see conv_unit_lo).
static long long conv_packed_bytes(int n_out, int taps3d, int cpin, int rpt) {
    const int cg = cpin / 8;
    return (long long)(taps3d ? 3 : 1) * conv_plane_bytes(rpt, cg == 1, conv_cgp(cg), pad_npad(n_out));
}
// Output rows per tile: the most of 4 .. 2 with RPT x NPAD <= kMaxTileN (at least one
// TMEM accumulator per epilogue warpgroup) whose weights fit in shared memory next to two
// input stages; 1 otherwise. Channel strides of 16 and 64 take at most 2; row pairs (8-channel
// inputs) take an even count (an odd one leaves a zero partner row). More rows per tile
// mean fewer MMAs per output row, (RPT + 2) / RPT input rows each, but fewer input stages
// in flight; four rows balance the two (192 x 256 images, 200 of them): on the 32 -> 32
// layer 4 rows with two stages took 270 us against 290 with 3 rows (three stages) and 355
// with 2 (five); on the 32 -> 5 residual layer 4 rows (three stages) took 262 us against
// 342 with 6 (two stages), 291 with 3 and 349 with 2.
constexpr int kMaxRpt = 4, kMaxTileN = 128;
// Dynamic shared memory a CTA may opt into (227 KB on sm_100-family GPUs).
constexpr long long kConvSmemLimit = 227 * 1024;
static int conv_rpt(int taps3d, int H, int cpin, int n_out) {
    const int npad = pad_npad(n_out);
    for (int rpt = kMaxRpt; rpt >= 2; --rpt) {
        if (rpt > H || rpt * npad > kMaxTileN || ((cpin == 16 || cpin == 64) && rpt > 2) || (cpin == 8 && (rpt & 1)))
            continue;
        const long long fixed = 1024 + ((conv_packed_bytes(n_out, taps3d, cpin, rpt) + 127) & ~127LL) +
                                8 * (2 * kMaxStages + 2 * kMaxAcc) + 4 * npad + 64;
        if (fixed + 2LL * conv_stage_bytes(cpin / 8, rpt) <= kConvSmemLimit) return rpt;
    }
    return 1;
}

// Packs the weights of one launch: outputs o0 .. o0 + n_out - 1 of the layer.
static int conv_pack(const float *w, int cout, int taps3d, int cin, int cpin, int flip, int rpt, int o0, int n_out,
                     uint8_t *out, cudaStream_t st) {
    const long long total = conv_packed_bytes(n_out, taps3d, cpin, rpt) / 2;
    k_pack_weights<<<(int)std::min<long long>(4096, (total + 255) / 256), 256, 0, st>>>(
        w, cout, taps3d, cin, ((cpin / 8) + 1) & ~1, pad_npad(n_out), rpt, cpin == 8, flip, o0, out);
    CBCT_LAUNCH_CHECK("conv weight pack");
    return 0;
}

template <int NPAD, int EPI, int CG, int RPT>
static int launch_conv(const ConvArgs &a, cudaStream_t st) {
    constexpr int kN = RPT * NPAD;
    const int bbytes = a.bbytes;
    const size_t fixed = 1024 + ((bbytes + 127) & ~127) + 8 * (2 * kMaxStages + 2 * kMaxAcc) + 4 * NPAD + 64;
    const size_t limit = (size_t)kConvSmemLimit, stage = conv_stage_bytes(CG, RPT);
    if (fixed + 2 * stage > limit) return fail(CBCT_EINVAL, "conv: input rows and weights do not fit in shared memory");
    const int nst = (int)std::min<size_t>(6, (limit - fixed) / stage);
    const size_t smem = fixed + (size_t)nst * stage;
    cudaError_t e =
        cudaFuncSetAttribute(k_conv_tc<NPAD, EPI, CG, RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "conv smem attribute");
    // x as a 5-D tensor (G pixels x 8 channels, W / G, channel groups, H, D * images);
    // one box = R rows of G pixels, all channel groups, RPT + 2 image rows
    CUtensorMap xmap;
    const uint64_t G = (uint64_t)a.G, W = (uint64_t)a.W, cg = (uint64_t)a.cin_groups;
    const uint64_t dims[5] = {8 * G, W / G, cg, (uint64_t)a.H, (uint64_t)a.D * a.nimg};
    const uint64_t strides[4] = {16 * G, 16 * W, 16 * W * cg, 16 * W * cg * a.H};
    const uint32_t box[5] = {(uint32_t)(8 * G), (uint32_t)conv_box_rows(a.G), (uint32_t)cg, (uint32_t)(RPT + 2), 1};
    int rc = encode_tmap(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, a.x, dims, strides, box);
    if (rc) return rc;
    int dev = 0, nsm = 152, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_conv_tc<NPAD, EPI, CG, RPT>, kWsThreads, smem);
    // TMEM: conv_nacc(kN) x kN columns per CTA, 512 per SM
    const int per_sm = std::max(1, std::min({4, occ, 512 / conv_pow2(conv_nacc(kN) * kN)}));
    const long long ntiles = (long long)a.nimg * a.D * ((a.H + RPT - 1) / RPT) * ((a.W + 127) / 128);
    const int grid = (int)std::min<long long>(ntiles, (long long)nsm * per_sm);
    k_conv_tc<NPAD, EPI, CG, RPT><<<grid, kWsThreads, smem, st>>>(xmap, a, nst);
    CBCT_LAUNCH_CHECK("conv launch");
    return 0;
}

template <int NPAD, int EPI, int RPT>
static int launch_conv_cg(const ConvArgs &a, cudaStream_t st) {
    if constexpr (RPT * NPAD > kMaxTileN) {
        return fail(CBCT_EINVAL, "conv: tile too tall for this channel count");
    } else {
        switch (a.cin_groups) {
            case 1:
                if constexpr (RPT % 2 == 0 || RPT == 1) return launch_conv<NPAD, EPI, 1, RPT>(a, st);
                return fail(CBCT_EINVAL, "conv: no tile shape for this channel stride");
            case 2:
                if constexpr (RPT <= 2) return launch_conv<NPAD, EPI, 2, RPT>(a, st);
                return fail(CBCT_EINVAL, "conv: no tile shape for this channel stride");
            case 4: return launch_conv<NPAD, EPI, 4, RPT>(a, st);
            case 8:
                if constexpr (RPT <= 2) return launch_conv<NPAD, EPI, 8, RPT>(a, st);
                return fail(CBCT_EINVAL, "conv: no tile shape for this channel stride");
            default: return fail(CBCT_EINVAL, "conv: channel stride must be 8, 16, 32 or 64");
        }
    }
}

template <int NPAD, int EPI>
static int launch_conv_rpt(const ConvArgs &a, int rpt, cudaStream_t st) {
    switch (rpt) {
        case 4: return launch_conv_cg<NPAD, EPI, 4>(a, st);
        case 3: return launch_conv_cg<NPAD, EPI, 3>(a, st);
        case 2: return launch_conv_cg<NPAD, EPI, 2>(a, st);
        default: return launch_conv_cg<NPAD, EPI, 1>(a, st);
    }
}

// Runs one convolution with weights packed by conv_pack for the same rpt. n_out =
// number of GEMM output channels (cout, or cin for the input-gradient convolution).
static int conv_run(const ConvArgs &a0, int n_out, int epi, int rpt, cudaStream_t st) {
    ConvArgs a = a0;
    const int npad = pad_npad(n_out);
    if (a.cpin % 8 || (epi != EPI_RESIDUAL_F32 && a.cpout % 8)) return fail(CBCT_EINVAL, "conv: channel strides must be multiples of 8");
    a.cin_groups = a.cpin / 8;
    a.bbytes = (int)conv_packed_bytes(n_out, a.taps3d, a.cpin, rpt);
    a.G = a.W % 4 == 0 ? 4 : (a.W % 2 == 0 ? 2 : 1);
    if (npad == 16) {
        if (epi == EPI_ACT_BF16) return launch_conv_rpt<16, EPI_ACT_BF16>(a, rpt, st);
        if (epi == EPI_RESIDUAL_F32) return launch_conv_rpt<16, EPI_RESIDUAL_F32>(a, rpt, st);
        return launch_conv_rpt<16, EPI_MASK_BF16>(a, rpt, st);
    }
    if (epi == EPI_ACT_BF16) return launch_conv_rpt<32, EPI_ACT_BF16>(a, rpt, st);
    if (epi == EPI_RESIDUAL_F32) return launch_conv_rpt<32, EPI_RESIDUAL_F32>(a, rpt, st);
    return launch_conv_rpt<32, EPI_MASK_BF16>(a, rpt, st);
}

// Tensor-core weight gradient of one block of at most 32 x 32 channels: x holds 8 XCG
// input slots of rows xgs channel groups apart (a view into a wider input), dy cgo output
// groups of rows ygs groups apart. dw[co0 + co][tap][ci0 + ci] (cin_full channels per tap)
// (+)= the block's per-CTA partials, reduced in a fixed order; db[co0 + co] (+)= the bias
// gradient when db is not null (CUDA cores).
template <int XCG, int NCG>
static int conv_wgrad_tc(const __nv_bfloat16 *x, int xgs, int cin, const __nv_bfloat16 *dy, int cgo, int ygs,
                         int cout, int nimg, int D, int H, int W, int taps3d, float *dw, int co0, int ci0,
                         int cin_full, float *db, int accumulate, int *status, cudaStream_t st) {
    ConvArgs a{};
    a.x = x;
    a.nimg = nimg; a.D = D; a.H = H; a.W = W;
    a.cpin = 8 * XCG; a.cin_groups = XCG;
    a.taps3d = taps3d;
    a.cout = cout; a.cin = cin;
    a.G = W % 4 == 0 ? 4 : (W % 2 == 0 ? 2 : 1);
    a.status = status;
    const uint64_t G = (uint64_t)a.G, Wl = (uint64_t)W;
    CUtensorMap xmap, ymap;
    {
        const uint64_t dims[5] = {8 * G, Wl / G, (uint64_t)XCG, (uint64_t)H, (uint64_t)D * nimg};
        const uint64_t strides[4] = {16 * G, 16 * Wl, 16 * (uint64_t)xgs * Wl, 16 * (uint64_t)xgs * Wl * H};
        const uint32_t box[5] = {(uint32_t)(8 * G), (uint32_t)conv_box_rows(a.G), (uint32_t)XCG, XCG == 4 ? 4u : 1u, 1};
        int rc = encode_tmap(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, x, dims, strides, box);
        if (rc) return rc;
    }
    {
        const uint64_t dims[5] = {8 * G, Wl / G, (uint64_t)cgo, (uint64_t)H, (uint64_t)D * nimg};
        const uint64_t strides[4] = {16 * G, 16 * Wl, 16 * Wl * (uint64_t)ygs, 16 * Wl * (uint64_t)ygs * H};
        const uint32_t box[5] = {(uint32_t)(8 * G), (uint32_t)(128 / a.G), (uint32_t)cgo, 1, 1};
        int rc = encode_tmap(&ymap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, dy, dims, strides, box);
        if (rc) return rc;
    }
    constexpr size_t kStage = kWgXBytes + 2 * NCG * 2048;
    const size_t smem = 1024 + kWgStages * kStage + 8 * (2 * kWgStages + 1) + 4 * 5 + 64;
    CBCT_CUDA_TRY(cudaFuncSetAttribute(k_conv_wgrad_tc<XCG, NCG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nsm = sm_count();
    const int ndd = taps3d ? 3 : 1;
    const long long ntiles = (long long)nimg * D * ((H + 1) / 2) * ((W + 127) / 128);
    const int gpd = (int)std::max<long long>(1, std::min<long long>(ntiles, 2LL * nsm));  // CTAs per depth tap
    const long long per_cta = 2LL * cout * 9 * cin;
    const int nw = cout * 9 * ndd * cin;
    const long long nrows = (long long)nimg * D * H;
    const int nbb = (int)std::min<long long>(4LL * nsm, nrows);
    const int rpb = (int)((nrows + nbb - 1) / nbb);
    float *part = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&part, sizeof(float) * ((long long)ndd * gpd * per_cta + (long long)nbb * cout),
                                  st));
    float *partb = part + (long long)ndd * gpd * per_cta;
    k_conv_wgrad_tc<XCG, NCG><<<dim3(gpd, ndd), kWgThreads, smem, st>>>(xmap, ymap, a, cgo, part);
    k_reduce_wgrad<<<(nw + 255) / 256, 256, 0, st>>>(part, gpd, ndd, cout, cin, dw, accumulate, co0, ci0, cin_full);
    if (db) {
        k_bias_grad<<<nbb, 256, 0, st>>>(dy, cgo, ygs, cout, nrows, W, rpb, partb);
        k_reduce_rows<<<1, 256, 0, st>>>(partb, nbb, cout, db + co0, accumulate);
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, st);
    if (e != cudaSuccess) return cuda_fail(e, "conv wgrad (tensor cores)");
    return 0;
}

// dW (+)= sum_p dY[p] x X[p + tap], db (+)= sum_p dY[p]; partial sums in scratch.
// Inputs and outputs of 64 channel slots run as 32 x 32 blocks: views of 4 channel groups
// (32 W elements apart within a row) of the wider operand.
int conv_wgrad(const __nv_bfloat16 *x, int cpin, int cin, const __nv_bfloat16 *dy, int cpout, int cout, int nimg, int D,
               int H, int W, int taps3d, float *dw, float *db, int accumulate, int *status, cudaStream_t st) {
    if ((cpin == 64 || cpin == 32 || cpin == 8) && cin <= cpin && cout <= cpout &&
        (cpout == 8 || cpout == 16 || cpout == 32 || cpout == 64)) {
        if (!status) return fail(CBCT_EINVAL, "conv wgrad: NULL status word");
        const int xgs = cpin / 8, ygs = cpout / 8;
        for (int xh = 0; 32 * xh < cin; ++xh) {
            const __nv_bfloat16 *xv = x + 32LL * xh * W;
            const int cin_s = std::min(32, cin - 32 * xh);
            for (int yh = 0; 32 * yh < cout; ++yh) {
                const __nv_bfloat16 *yv = dy + 32LL * yh * W;
                const int cout_s = std::min(32, cout - 32 * yh), cgo = std::min(4, ygs);
                float *dbv = xh == 0 ? db : nullptr;
                int rc;
                if (cpin == 8)
                    rc = cgo <= 2 ? conv_wgrad_tc<1, 2>(xv, xgs, cin_s, yv, cgo, ygs, cout_s, nimg, D, H, W, taps3d, dw,
                                                        32 * yh, 32 * xh, cin, dbv, accumulate, status, st)
                                  : conv_wgrad_tc<1, 4>(xv, xgs, cin_s, yv, cgo, ygs, cout_s, nimg, D, H, W, taps3d, dw,
                                                        32 * yh, 32 * xh, cin, dbv, accumulate, status, st);
                else
                    rc = cgo <= 2 ? conv_wgrad_tc<4, 2>(xv, xgs, cin_s, yv, cgo, ygs, cout_s, nimg, D, H, W, taps3d, dw,
                                                        32 * yh, 32 * xh, cin, dbv, accumulate, status, st)
                                  : conv_wgrad_tc<4, 4>(xv, xgs, cin_s, yv, cgo, ygs, cout_s, nimg, D, H, W, taps3d, dw,
                                                        32 * yh, 32 * xh, cin, dbv, accumulate, status, st);
                if (rc) return rc;
            }
        }
        return 0;
    }
    const int ntaps = taps3d ? 27 : 9;
    const long long npix = (long long)nimg * D * H * W;
    const int nblk = (int)std::min<long long>(4LL * sm_count(), std::max<long long>(1, (npix + 1023) / 1024));
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

static bool conv_cpin_ok(int cpin) { return cpin == 8 || cpin == 16 || cpin == 32 || cpin == 64; }

long long cbct::conv_plan(int taps3d, int H, int cpin, int cin, int cout, int flip, ConvPackJob *jobs) {
    const int n_out = flip ? cin : cout;
    if (!conv_cpin_ok(cpin) || n_out < 1 || n_out > kConvMaxOut || !jobs) return -1;
    long long off = 0;
    for (int h = 0; h < conv_halves(n_out); ++h) {
        const int nh = conv_half_nout(n_out, h);
        const int rpt = conv_rpt(taps3d, H, cpin, nh);
        const long long bytes = conv_packed_bytes(nh, taps3d, cpin, rpt);
        ConvPackJob &job = jobs[h];
        job.nelem = bytes / 2;
        job.cout = cout;
        job.taps3d = taps3d;
        job.cin = cin;
        job.cgp = ((cpin / 8) + 1) & ~1;
        job.npad = pad_npad(nh);
        job.rpt = rpt;
        job.pair = cpin == 8;
        job.flip = flip;
        job.o0 = 32 * h;
        job.out_off = off;
        off += (bytes + 255) & ~255LL;
    }
    return off;
}

int cbct::conv_pack_jobs(const ConvPackJob *jobs, int njobs, long long max_nelem, const float *params, uint8_t *out,
                         cudaStream_t st) {
    if (njobs < 1 || njobs > 65535 || max_nelem < 1) return fail(CBCT_EINVAL, "conv_pack_jobs: bad job count");
    dim3 grd((unsigned)std::min<long long>(1024, (max_nelem + 255) / 256), (unsigned)njobs);
    k_pack_jobs<<<grd, 256, 0, st>>>(jobs, params, out);
    CBCT_LAUNCH_CHECK("conv weight pack (jobs)");
    return 0;
}

int cbct::conv_apply(const void *x, int nimg, int D, int H, int W, int cpin, int taps3d, const float *w, const float *bias,
                     int cin, int cout, int flip, int epi, float slope, void *y, int cpout, const void *mask,
                     const float *state_in, float *state, long long sstride, int *status, cudaStream_t st,
                     const uint8_t *packed, int zero_state_in, const int *smap, int ssub) {
    if (!x || !w || nimg < 1 || D < 1 || H < 1 || W < 1 || cin < 1 || cout < 1 || !conv_cpin_ok(cpin) ||
        cpin < (flip ? cout : cin))
        return fail(CBCT_EINVAL, "conv: invalid argument (sizes, or cpin below the input channels)");
    const int n_out = flip ? cin : cout;
    if (n_out > kConvMaxOut) return fail(CBCT_EINVAL, "conv: at most 64 output channels");
    if (epi < 0 || epi > 2) return fail(CBCT_EINVAL, "conv: bad epilogue");
    if (!(slope >= 0.f && slope <= 1.f)) return fail(CBCT_EINVAL, "conv: LeakyReLU slope must lie in [0, 1]");
    if ((epi == EPI_RESIDUAL_F32 && !state) || (epi != EPI_RESIDUAL_F32 && (!y || cpout < n_out)) ||
        (epi == EPI_MASK_BF16 && !mask) || !status)
        return fail(CBCT_EINVAL, "conv: missing output");
    if (smap && (epi != EPI_RESIDUAL_F32 || n_out > 8))
        return fail(CBCT_EINVAL, "conv: a plane map needs the residual epilogue and at most 8 outputs");
    ConvPackJob jobs[kConvMaxOut / 32];
    const long long bytes = conv_plan(taps3d, H, cpin, cin, cout, flip, jobs);
    uint8_t *pk = nullptr;
    int rc = 0;
    if (!packed) {
        CBCT_CUDA_TRY(cudaMallocAsync((void **)&pk, bytes, st));
        for (int h = 0; h < conv_halves(n_out) && rc == 0; ++h)
            rc = conv_pack(w, cout, taps3d, cin, cpin, flip, jobs[h].rpt, jobs[h].o0, conv_half_nout(n_out, h),
                           pk + jobs[h].out_off, st);
    }
    for (int h = 0; h < conv_halves(n_out) && rc == 0; ++h) {
        const int nh = conv_half_nout(n_out, h);
        ConvArgs a{};
        a.x = static_cast<const __nv_bfloat16 *>(x);
        a.wpk = (packed ? packed : pk) + jobs[h].out_off;
        a.bias = bias ? bias + 32 * h : nullptr;
        a.nimg = nimg; a.D = D; a.H = H; a.W = W;
        a.cpin = cpin;
        a.taps3d = taps3d;
        a.cout = nh;
        a.slope = slope;
        a.y = static_cast<__nv_bfloat16 *>(y);
        a.cpout = cpout;
        a.mask = static_cast<const __nv_bfloat16 *>(mask);
        a.state = state;
        a.state_in = state_in ? state_in : state;
        a.state_in_zero = zero_state_in;
        a.sstride = sstride;
        a.smap_on = smap ? 1 : 0;
        for (int c = 0; c < 8; ++c) a.smap[c] = smap ? smap[c < n_out ? c : 0] : c;
        a.ssub = ssub ? 1 : 0;
        a.qoff = 4 * h;
        a.status = status;
        rc = conv_run(a, nh, epi, jobs[h].rpt, st);
    }
    if (pk) cudaFreeAsync(pk, st);
    return rc;
}

extern "C" int cbct_conv(const void *x, int nimg, int D, int H, int W, int cpin, int taps3d, const float *w,
                         const float *bias, int cin, int cout, int flip, int epi, float slope, void *y, int cpout,
                         const void *mask, float *state, long long sstride, int *status, void *stream) {
    return conv_apply(x, nimg, D, H, W, cpin, taps3d, w, bias, cin, cout, flip, epi, slope, y, cpout, mask, state,
                      state, sstride, status, (cudaStream_t)stream);
}

extern "C" int cbct_conv_plan(int taps3d, int H, int cpin, int cin, int cout, int flip, int *rpt,
                              long long *packed_bytes, int *stages, int *accumulators) {
    const int n_out = flip ? cin : cout;
    if (H < 1 || cin < 1 || cout < 1 || n_out > kConvMaxOut || !conv_cpin_ok(cpin) || cpin < (flip ? cout : cin))
        return fail(CBCT_EINVAL, "cbct_conv_plan: invalid shape");
    const int n0 = conv_half_nout(n_out, 0);  // the first launch (32 outputs when there are more)
    const int r = conv_rpt(taps3d ? 1 : 0, H, cpin, n0), npad = pad_npad(n0);
    const long long bytes = conv_packed_bytes(n0, taps3d ? 1 : 0, cpin, r);
    const long long fixed = 1024 + ((bytes + 127) & ~127LL) + 8 * (2 * kMaxStages + 2 * kMaxAcc) + 4 * npad + 64;
    const long long st = std::min<long long>(6, (kConvSmemLimit - fixed) / conv_stage_bytes(cpin / 8, r));
    if (rpt) *rpt = r;
    if (packed_bytes) *packed_bytes = bytes;
    if (stages) *stages = (int)st;
    if (accumulators) *accumulators = conv_nacc(r * npad);
    return 0;
}

extern "C" int cbct_conv_wgrad(const void *x, int cpin, int cin, const void *dy, int cpout, int cout, int nimg, int D,
                               int H, int W, int taps3d, float *dw, float *db, int accumulate, int *status,
                               void *stream) {
    if (!x || !dy || !dw || !db || !status || cin < 1 || cout < 1)
        return fail(CBCT_EINVAL, "cbct_conv_wgrad: invalid argument");
    return conv_wgrad(static_cast<const __nv_bfloat16 *>(x), cpin, cin, static_cast<const __nv_bfloat16 *>(dy), cpout,
                      cout, nimg, D, H, W, taps3d, dw, db, accumulate, status, (cudaStream_t)stream);
}
