// Host-side layout of the opaque geometry handle (internal to the library).
#pragma once
#include <stdint.h>

#include <vector>

#include "common.cuh"

struct cbct_geom {
    cbct_geom_desc desc{};                 // copy of the descriptor (angles pointer cleared)
    std::vector<double> angles;            // explicit angles, empty for uniform 2 pi k / n
    std::vector<cbct::Frame32> h32;        // host copy of the FP32 ray tables
    int device = 0;
    cbct::Frame32 *f32 = nullptr;          // device tables
    cbct::Frame64 *f64 = nullptr;
    cbct::Col32 *col32 = nullptr;          // [na][nu]
    cbct::Col64 *col64 = nullptr;
    float *rz32 = nullptr;                 // [nv]
    double *rz64 = nullptr;
    double2 *cs = nullptr;                 // [na] (cos, sin) of each angle, for FDK
    cbct::GeomDev dev{};                   // kernel view
    int *status = nullptr;                 // device status word of this geometry's kernels
    int fwd_cfg = -1;                      // staged forward box configuration, -1: direct kernel
    double fwd_need_b = 0.0, fwd_need_z = 0.0;  // host bounds of a tile's chunk footprint
    bool axis_contiguous = true;           // x- and y-principal columns form intervals at every angle
};

namespace cbct {
// ||P|| by power iteration on P^T P (FP32 operators, FP64 norms), used for the
// normalised operators. Synchronises the current device.
int operator_norm(cbct_geom *g, int iters, double *out);
// P^T (colw[u] * proj): adjoint of a column-weighted projection (colw: [nu] device).
int back_project_colw(const cbct_geom *g, const float *proj, const float *colw, float *vol, int batch, int accumulate,
                      cudaStream_t st);
// cbct_conv with the residual epilogue reading its old state from state_in (which may
// equal state) and writing state = state_in + conv (state = conv without reading
// state_in when zero_state_in; state_in - conv with ssub). packed: the layer's B operand
// already packed by conv_pack_jobs for the same (taps3d, H, cpin, cin, cout, flip), or
// null to pack it here. smap (host, up to 8 entries, residual epilogue only): output
// channel c lives in plane smap[c] of state / state_in (stride sstride), or plane c
// when null.
int conv_apply(const void *x, int nimg, int D, int H, int W, int cpin, int taps3d, const float *w, const float *bias,
               int cin, int cout, int flip, int epi, float slope, void *y, int cpout, const void *mask,
               const float *state_in, float *state, long long sstride, int *status, cudaStream_t st,
               const uint8_t *packed = nullptr, int zero_state_in = 0, const int *smap = nullptr, int ssub = 0);
// Packing of one layer's weights: the shape part is filled by conv_plan, the offsets
// (weights within the parameter array, bytes within the packed buffer) by the caller.
struct ConvPackJob {
    long long w_off, out_off, nelem;
    int cout, taps3d, cin, cgp, npad, rpt, pair, flip, o0;
};
// A convolution with more than 32 outputs runs as launches of 32 outputs ("halves"),
// each with its own packed weights; half h starts conv_half_offset(.., h) bytes into
// the layer's packed buffer.
constexpr int kConvMaxOut = 64;
inline int conv_halves(int n_out) { return (n_out + 31) / 32; }
inline int conv_half_nout(int n_out, int h) { return n_out - 32 * h < 32 ? n_out - 32 * h : 32; }
// Fills jobs[0 .. conv_halves(n_out) - 1] (shape fields, o0, and out_off relative to the
// layer's packed buffer) for a convolution of the given shape; returns the packed bytes
// of all halves (each rounded up to 256), or a negative value for an unsupported shape.
long long conv_plan(int taps3d, int H, int cpin, int cin, int cout, int flip, ConvPackJob *jobs);
// Packs njobs layers (jobs: device array) from params into out in one launch.
int conv_pack_jobs(const ConvPackJob *jobs, int njobs, long long max_nelem, const float *params, uint8_t *out,
                   cudaStream_t st);
// Looks up (once per device) the device address of back_project_noalloc's fixed
// scratch array on `dev`, the current device. geometry_create calls it so that the
// module holding the array is loaded, and the array placed, when the geometry is made.
int noalloc_prime(int dev);
// Staged (TMA) forward: returns 1 if it ran, 0 if the direct kernel must be used.
int forward_staged(const cbct_geom *g, const float *vol, float *proj, int batch, int accumulate, cudaStream_t st);
int choose_forward_cfg(double need_b, double need_z);
}  // namespace cbct
