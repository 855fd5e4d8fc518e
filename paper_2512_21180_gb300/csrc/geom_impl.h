// Host-side layout of the opaque geometry handle (internal to the library).
#pragma once

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
    cbct::GeomDev dev{};                   // kernel view
};

namespace cbct {
// ||P|| by power iteration on P^T P (FP32 operators, FP64 norms), used for the
// normalised operators. Synchronises the current device.
int operator_norm(cbct_geom *g, int iters, double *out);
}  // namespace cbct
