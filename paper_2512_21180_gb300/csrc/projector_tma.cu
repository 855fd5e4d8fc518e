// Forward projector with TMA-staged volume tiles (a2, paper Sec. 2.2 projection
// operator; Joseph-style ray sums as in projector.cu).
//
// Layout: the volume is first copied plane-major for each principal axis,
// T_x[x][z][y] (planes of constant x, y fastest) and T_y[y][z][x], rows padded to a
// multiple of 4 floats. For both axes a plane is then a contiguous [z][b] slab
// whose fastest index is the in-plane coordinate b that varies along a detector
// row, so a warp's bilinear reads hit distinct shared-memory banks.
//
// CTA = one angle x a 32 (u) x 8 (v) ray tile: 4 consumer warps and one producer
// warp. A consumer thread carries the two rays of its column in rows v and v + 4:
// both share the column's in-plane coordinate q_b, principal axis and source-to-
// pixel parameter on every plane, and their z-dependent arithmetic runs as packed
// FP32 pairs (fma/add.rn.f32x2, each half rounded like the scalar operation). The planes are
// processed in chunks of 8; for each chunk the producer computes the box of
// voxels the tile's rays can touch (from the four corner rays at the chunk's end
// planes: the sample position is monotone in column, row and plane) and TMA-loads
// it (box BW x ZH x 8) into a 2-stage shared-memory ring. TMA fills voxels outside
// the volume with zeros, so the consumers sample without bounds checks. A chunk
// whose footprint exceeds the box falls back to bounds-checked global loads; a
// chunk whose box misses the volume is skipped (all its samples are zero). Tiles
// that contain rays of both principal axes (near 45 degrees) make one pass per
// axis. Every mbarrier wait is bounded in time (tma.cuh).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "geom_impl.h"
#include "tma.cuh"

namespace cbct {

// Two stages of 8 planes (32 KB with the 32 x 16 box) let six CTAs share an SM: measured
// at the clinical size, 15.1 ms against 18.0 ms with three stages (four CTAs per SM) and
// 21.9 ms with four (three CTAs per SM); four planes per stage took 16.9 ms.
constexpr int kTU = 32, kTV = 8, kP = 8, kStages = 2;
constexpr int kRowsPerThread = 2;
constexpr int kConsumerWarps = kTV / kRowsPerThread;  // warp w: rows w and w + kConsumerWarps
constexpr int kThreads = 32 * (kConsumerWarps + 1);

struct ChunkInfo {
    int b0, z0, flag;  // flag: 0 skip (box outside the volume), 1 TMA box, 2 global fallback
};

// ---- tensor maps -------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

int encode_tmap(CUtensorMap *map, CUtensorMapDataType dt, int rank, const void *base, const uint64_t *dims,
                const uint64_t *strides, const uint32_t *box) {
    auto fn = encode_fn();
    if (!fn) return fail(CBCT_ECUDA, "cuTensorMapEncodeTiled unavailable");
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(map, dt, (cuuint32_t)rank, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CBCT_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return 0;
}

static int encode_4d(CUtensorMap *map, const float *base, const uint64_t dims[4], const uint64_t strides[3],
                     const uint32_t box[4]) {
    auto fn = encode_fn();
    if (!fn) return fail(CBCT_ECUDA, "cuTensorMapEncodeTiled unavailable");
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CBCT_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return 0;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// ---- plane-major copies ----------------------------------------------------------------

// T_y[b][y][z][x] = V[b][z][y][x]   (row pitch py >= nx)
__global__ void k_planes_y(const float *__restrict__ V, float *__restrict__ T, int nx, int ny, int nz, int py) {
    const int y = blockIdx.x, z = blockIdx.y, b = blockIdx.z;
    const float *src = V + (((long long)b * nz + z) * ny + y) * nx;
    float *dst = T + (((long long)b * ny + y) * nz + z) * py;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) dst[x] = src[x];
}

// T_x[b][x][z][y] = V[b][z][y][x]   (row pitch px >= ny), 32x32 tiles through smem
__global__ void k_planes_x(const float *__restrict__ V, float *__restrict__ T, int nx, int ny, int nz, int px) {
    __shared__ float tile[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int z = blockIdx.z % nz, b = blockIdx.z / nz;
    const float *src = V + ((long long)b * nz + z) * ny * (long long)nx;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int y = y0 + j, x = x0 + threadIdx.x;
        tile[j][threadIdx.x] = (y < ny && x < nx) ? src[(long long)y * nx + x] : 0.0f;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int x = x0 + j, y = y0 + threadIdx.x;
        if (x < nx && y < ny) T[(((long long)b * nx + x) * nz + z) * px + y] = tile[threadIdx.x][j];
    }
}

// ---- the staged forward kernel -----------------------------------------------------------

__device__ __forceinline__ int floor_i(float v) { return (int)floorf(fminf(fmaxf(v, -1.0e8f), 1.0e8f)); }

template <int BW, int ZH>
__global__ void __launch_bounds__(kThreads) k_forward_tma(const __grid_constant__ CUtensorMap map_x,
                                                          const __grid_constant__ CUtensorMap map_y, GeomDev g,
                                                          const float *__restrict__ tx, const float *__restrict__ ty,
                                                          int px, int py, float *__restrict__ proj, int accumulate,
                                                          int *status) {
    constexpr int SE = kP * ZH * BW;  // floats per stage
    constexpr uint32_t kBytes = SE * 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations: 128-byte aligned (the launch reserves 128 bytes of slack)
    float *stages = reinterpret_cast<float *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    uint64_t *full = reinterpret_cast<uint64_t *>(stages + kStages * SE);
    uint64_t *empty = full + kStages;
    ChunkInfo *info = reinterpret_cast<ChunkInfo *>(empty + kStages);
    int &abort_flag = *reinterpret_cast<int *>(info + (max(g.n[0], g.n[1]) + kP - 1) / kP);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.z % g.na, b = blockIdx.z / g.na;
    const int u0 = blockIdx.x * kTU, v0 = blockIdx.y * kTV;
    const Frame32 &F = g.f32[k];

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&map_x);
        prefetch_tmap(&map_y);
    }
    __syncthreads();

    // consumer ray set-up (the canonical per-ray quantities of common.cuh): column
    // terms once, row terms for both rows (a row past the panel reads the last row's
    // table entry and is dropped at the store)
    const bool consumer = warp < kConsumerWarps;
    const int iu = u0 + lane, iv0 = v0 + warp, iv1 = iv0 + kConsumerWarps;
    const bool col_ok = consumer && iu < g.nu;
    const int my_a = col_ok ? principal_axis(F, iu) : -1;
    ColT<float> c{0.f, 0.f, 0.f, 0.f};
    float2 dqz = make_float2(0.f, 0.f), qcz = make_float2(0.f, 0.f), step = make_float2(0.f, 0.f);
    bool t_all = true;
    if (col_ok) {
        c = col_of<float>(g, k, iu);
        ray_row(g, c, rz_of<float>(g, min(iv0, g.nv - 1)), dqz.x, qcz.x);
        ray_row(g, c, rz_of<float>(g, min(iv1, g.nv - 1)), dqz.y, qcz.y);
        step.x = ray_step<float>(g, my_a, c.dqb, dqz.x);
        step.y = ray_step<float>(g, my_a, c.dqb, dqz.y);
        const float ca = 0.5f * (float)(g.n[my_a] - 1);
        const float t0 = fma_rn(-ca, c.inv, c.tc), t1 = fma_rn(ca, c.inv, c.tc);
        t_all = t0 > 0.f && t0 < 1.f && t1 > 0.f && t1 < 1.f;
    }
    float2 acc = make_float2(0.f, 0.f);
    int gc = 0;  // chunks issued so far (both passes): stage = gc % kStages, use = gc / kStages

    for (int a = 0; a < 2; ++a) {
        const int lo = a == 0 ? F.ux_lo : F.uy_lo, hi = a == 0 ? F.ux_hi : F.uy_hi;
        const int ua = max(u0, lo), ub = min(min(u0 + kTU, g.nu) - 1, hi);
        if (ua > ub) continue;  // block-uniform
        const int na = g.n[a], nb = g.n[1 - a], nz = g.n[2];
        const int nch = (na + kP - 1) / kP;
        const float ca = 0.5f * (float)(na - 1);

        if (warp == kConsumerWarps) {
            // chunk boxes from the tile's corner rays at the chunk's end planes
            const ColT<float> cA = col_of<float>(g, k, ua), cB = col_of<float>(g, k, ub);
            const float rzA = rz_of<float>(g, v0), rzB = rz_of<float>(g, min(v0 + kTV, g.nv) - 1);
            for (int ch = lane; ch < nch; ch += 32) {
                const int i0 = ch * kP, i1 = min(i0 + kP, na) - 1;
                const float d0 = (float)i0 - ca, d1 = (float)i1 - ca;
                float bmin = INFINITY, bmax = -INFINITY, zmin = INFINITY, zmax = -INFINITY;
                const ColT<float> cc[2] = {cA, cB};
                const float rr[2] = {rzA, rzB};
                const float dd[2] = {d0, d1};
#pragma unroll
                for (int iu2 = 0; iu2 < 2; ++iu2)
#pragma unroll
                    for (int id = 0; id < 2; ++id) {
                        const float qb = fma_rn(dd[id], cc[iu2].dqb, cc[iu2].qcb);
                        bmin = fminf(bmin, qb);
                        bmax = fmaxf(bmax, qb);
#pragma unroll
                        for (int ir = 0; ir < 2; ++ir) {
                            float dz, qz0;
                            ray_row(g, cc[iu2], rr[ir], dz, qz0);
                            const float qz = fma_rn(dd[id], dz, qz0);
                            zmin = fminf(zmin, qz);
                            zmax = fmaxf(zmax, qz);
                        }
                    }
                ChunkInfo ci;
                const bool finite = isfinite(bmin) && isfinite(bmax) && isfinite(zmin) && isfinite(zmax);
                const int jb0 = floor_i(bmin) - 1, jb1 = floor_i(bmax) + 2;
                const int jz0 = floor_i(zmin) - 1, jz1 = floor_i(zmax) + 2;
                ci.b0 = jb0 & ~3;
                ci.z0 = jz0;
                if (!finite || jb1 > ci.b0 + BW - 1 || jz1 > ci.z0 + ZH - 1) ci.flag = 2;
                else if (ci.b0 + BW <= 0 || ci.b0 >= nb || ci.z0 + ZH <= 0 || ci.z0 >= nz) ci.flag = 0;
                else ci.flag = 1;
                info[ch] = ci;
            }
        }
        __syncthreads();
        if (abort_flag) break;

        if (warp == kConsumerWarps) {
            if (lane == 0) {
                const CUtensorMap *map = a == 0 ? &map_x : &map_y;
                for (int ch = 0; ch < nch; ++ch) {
                    const int q = gc + ch, s = q % kStages, use = q / kStages;
                    if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, status)) {
                        abort_flag = 1;
                        // let the copies already issued land before leaving
                        for (int r = 1; r <= kStages && q - r >= 0; ++r) {
                            const int qq = q - r;
                            mbar_wait(&full[qq % kStages], (qq / kStages) & 1, status);
                        }
                        break;
                    }
                    const ChunkInfo ci = info[ch];
                    if (ci.flag == 1) {
                        mbar_arrive_expect_tx(&full[s], kBytes);
                        tma_load_4d(stages + s * SE, map, ci.b0, ci.z0, ch * kP, b, &full[s]);
                    } else {
                        mbar_arrive(&full[s]);
                    }
                }
            }
        } else {
            const bool mine = my_a == a;
            const float *T = a == 0 ? tx : ty;
            const int pitch = a == 0 ? px : py;
            const long long tbase = (long long)b * na * nz * pitch;
            for (int ch = 0; ch < nch; ++ch) {
                const int q = gc + ch, s = q % kStages, use = q / kStages;
                if (!mbar_wait(&full[s], use & 1, status)) {
                    abort_flag = 1;
                    break;
                }
                const ChunkInfo ci = info[ch];
                if (mine && ci.flag != 0) {
                    const int i0 = ch * kP;
                    const float d0 = (float)i0 - ca;
                    if (ci.flag == 1) {
                        const float *st = stages + s * SE;
                        const int base = -(ci.z0 * BW + ci.b0);
#pragma unroll
                        for (int p = 0; p < kP; ++p) {
                            if (i0 + p < na) {
                                const float di = d0 + (float)p;
                                const float qb = fma_rn(di, c.dqb, c.qcb);
                                const float fb0 = floorf(qb), fb = qb - fb0;
                                const float2 qz = __ffma2_rn(make_float2(di, di), dqz, qcz);
                                const float2 fz0 = make_float2(floorf(qz.x), floorf(qz.y));
                                const float2 fz = __fadd2_rn(qz, make_float2(-fz0.x, -fz0.y));
                                // fz0 BW + fb0 is an exact small integer in FP32: one conversion
                                const float2 offf = __ffma2_rn(fz0, make_float2((float)BW, (float)BW),
                                                               make_float2(fb0, fb0));
                                const int o0 = (int)min((unsigned)((int)offf.x + base), (unsigned)(ZH * BW - BW - 2));
                                const int o1 = (int)min((unsigned)((int)offf.y + base), (unsigned)(ZH * BW - BW - 2));
                                const float *r0 = st + p * ZH * BW + o0, *r1 = st + p * ZH * BW + o1;
                                const float2 v00 = make_float2(r0[0], r1[0]), v10 = make_float2(r0[1], r1[1]);
                                const float2 v01 = make_float2(r0[BW], r1[BW]), v11 = make_float2(r0[BW + 1], r1[BW + 1]);
                                const float2 fbb = make_float2(fb, fb);
                                const float2 a0 = __ffma2_rn(fbb, __fadd2_rn(v10, make_float2(-v00.x, -v00.y)), v00);
                                const float2 a1 = __ffma2_rn(fbb, __fadd2_rn(v11, make_float2(-v01.x, -v01.y)), v01);
                                const float2 val = __ffma2_rn(fz, __fadd2_rn(a1, make_float2(-a0.x, -a0.y)), a0);
                                if (t_all) acc = __fadd2_rn(acc, val);
                                else {
                                    const float t = fma_rn(di, c.inv, c.tc);
                                    if (t > 0.f && t < 1.f) acc = __fadd2_rn(acc, val);
                                }
                            }
                        }
                    } else {
                        for (int p = 0; p < kP && i0 + p < na; ++p) {
                            const int i = i0 + p;
                            const float di = d0 + (float)p;
                            const float t = fma_rn(di, c.inv, c.tc);
                            if (!(t > 0.f && t < 1.f)) continue;
                            const float qb = fma_rn(di, c.dqb, c.qcb);
                            if (!(qb > -1.f && qb < (float)nb)) continue;
                            const float fb0 = floorf(qb), fb = qb - fb0;
                            const int jb = (int)fb0;
                            const bool b0k = jb >= 0, b1k = jb + 1 < nb;
                            const float *P = T + tbase + (long long)i * nz * pitch;
#pragma unroll
                            for (int rr = 0; rr < kRowsPerThread; ++rr) {
                                const float qz = fma_rn(di, rr ? dqz.y : dqz.x, rr ? qcz.y : qcz.x);
                                if (!(qz > -1.f && qz < (float)nz)) continue;
                                const float fz0 = floorf(qz), fz = qz - fz0;
                                const int jz = (int)fz0;
                                const bool z0k = jz >= 0, z1k = jz + 1 < nz;
                                const float v00 = (b0k && z0k) ? __ldg(P + (long long)jz * pitch + jb) : 0.f;
                                const float v10 = (b1k && z0k) ? __ldg(P + (long long)jz * pitch + jb + 1) : 0.f;
                                const float v01 = (b0k && z1k) ? __ldg(P + (long long)(jz + 1) * pitch + jb) : 0.f;
                                const float v11 = (b1k && z1k) ? __ldg(P + (long long)(jz + 1) * pitch + jb + 1) : 0.f;
                                const float a0 = fmaf(fb, v10 - v00, v00);
                                const float a1 = fmaf(fb, v11 - v01, v01);
                                const float val = fmaf(fz, a1 - a0, a0);
                                if (rr) acc.y += val;
                                else acc.x += val;
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
        }
        gc += nch;
        __syncthreads();
        if (abort_flag) break;
    }
    if (consumer && !abort_flag) {
        // per row: when the row's 32 columns lie inside the panel and start on a 16-byte
        // boundary, every fourth lane stores its own and its three neighbours' rays as one
        // float4 (eight vector stores per warp and row); otherwise one float per ray
#pragma unroll
        for (int rr = 0; rr < kRowsPerThread; ++rr) {
            const int iv = rr ? iv1 : iv0;
            const bool ray_ok = col_ok && iv < g.nv;
            const float r = ray_ok ? (rr ? acc.y * step.y : acc.x * step.x) * g.scale : 0.f;
            float *out = proj + (((long long)b * g.na + k) * g.nv + iv) * g.nu + iu;
            if ((g.nu & 3) == 0 && u0 + kTU <= g.nu && iv < g.nv) {  // uniform over the warp
                const float r1 = __shfl_down_sync(0xffffffffu, r, 1);
                const float r2 = __shfl_down_sync(0xffffffffu, r, 2);
                const float r3 = __shfl_down_sync(0xffffffffu, r, 3);
                if ((lane & 3) == 0) {
                    float4 v = make_float4(r, r1, r2, r3);
                    if (accumulate) {
                        const float4 q = *reinterpret_cast<const float4 *>(out);
                        v.x += q.x; v.y += q.y; v.z += q.z; v.w += q.w;
                    }
                    *reinterpret_cast<float4 *>(out) = v;
                }
            } else if (ray_ok) {
                *out = accumulate ? *out + r : r;
            }
        }
    }
}

// ---- launcher ----------------------------------------------------------------------

struct FwdCfg {
    int bw, zh;
};
static const FwdCfg kCfgs[] = {{20, 8}, {24, 12}, {32, 16}, {44, 20}};

template <int BW, int ZH>
static int launch_cfg(const cbct_geom *g, const CUtensorMap &mx, const CUtensorMap &my, const float *tx,
                      const float *ty, int px, int py, float *proj, int batch, int accumulate, cudaStream_t st) {
    const GeomDev &d = g->dev;
    const int maxch = (std::max(d.n[0], d.n[1]) + kP - 1) / kP;
    const size_t smem =
        128 + (size_t)kStages * kP * ZH * BW * 4 + 2 * kStages * 8 + (size_t)maxch * sizeof(ChunkInfo) + sizeof(int);
    cudaError_t e = cudaFuncSetAttribute(k_forward_tma<BW, ZH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "forward_project: smem attribute");
    dim3 grd((d.nu + kTU - 1) / kTU, (d.nv + kTV - 1) / kTV, d.na * batch);
    k_forward_tma<BW, ZH><<<grd, kThreads, smem, st>>>(mx, my, d, tx, ty, px, py, proj, accumulate, g->status);
    CBCT_LAUNCH_CHECK("forward_project (staged) launch");
    return 0;
}

// Returns 1 if the staged kernel handled the call, 0 if the caller should use the
// direct kernel, negative on error.
int forward_staged(const cbct_geom *g, const float *vol, float *proj, int batch, int accumulate, cudaStream_t st) {
    if (g->fwd_cfg < 0) return 0;
    const GeomDev &d = g->dev;
    const int nx = d.n[0], ny = d.n[1], nz = d.n[2];
    const int px = (ny + 3) & ~3, py = (nx + 3) & ~3;
    const long long ex = (long long)batch * nx * nz * px, ey = (long long)batch * ny * nz * py;
    float *buf = nullptr;
    CBCT_CUDA_TRY(cudaMallocAsync((void **)&buf, sizeof(float) * (ex + ey), st));
    float *tx = buf, *ty = buf + ex;
    int rc = 0;
    {
        dim3 gx((nx + 31) / 32, (ny + 31) / 32, nz * batch);
        k_planes_x<<<gx, dim3(32, 8), 0, st>>>(vol, tx, nx, ny, nz, px);
        dim3 gy(ny, nz, batch);
        k_planes_y<<<gy, 128, 0, st>>>(vol, ty, nx, ny, nz, py);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "forward_project: plane copies");
    }
    const FwdCfg cf = kCfgs[g->fwd_cfg];
    CUtensorMap mx, my;
    if (rc == 0) {
        const uint64_t dx[4] = {(uint64_t)ny, (uint64_t)nz, (uint64_t)nx, (uint64_t)batch};
        const uint64_t sx[3] = {(uint64_t)px * 4, (uint64_t)px * nz * 4, (uint64_t)px * nz * nx * 4};
        const uint64_t dy[4] = {(uint64_t)nx, (uint64_t)nz, (uint64_t)ny, (uint64_t)batch};
        const uint64_t sy[3] = {(uint64_t)py * 4, (uint64_t)py * nz * 4, (uint64_t)py * nz * ny * 4};
        const uint32_t box[4] = {(uint32_t)cf.bw, (uint32_t)cf.zh, (uint32_t)kP, 1};
        rc = encode_4d(&mx, tx, dx, sx, box);
        if (rc == 0) rc = encode_4d(&my, ty, dy, sy, box);
    }
    if (rc == 0) {
        switch (g->fwd_cfg) {
            case 0: rc = launch_cfg<20, 8>(g, mx, my, tx, ty, px, py, proj, batch, accumulate, st); break;
            case 1: rc = launch_cfg<24, 12>(g, mx, my, tx, ty, px, py, proj, batch, accumulate, st); break;
            case 2: rc = launch_cfg<32, 16>(g, mx, my, tx, ty, px, py, proj, batch, accumulate, st); break;
            default: rc = launch_cfg<44, 20>(g, mx, my, tx, ty, px, py, proj, batch, accumulate, st); break;
        }
    }
    cudaFreeAsync(buf, st);
    return rc == 0 ? 1 : rc;
}

// Pick the smallest box that holds a tile's footprint over one chunk (from the
// host bounds of geometry_create), or -1 for the direct kernel.
int choose_forward_cfg(double need_b, double need_z) {
    for (int i = 0; i < (int)(sizeof(kCfgs) / sizeof(kCfgs[0])); ++i)
        if (need_b <= kCfgs[i].bw && need_z <= kCfgs[i].zh) return i;
    return -1;
}

}  // namespace cbct
