// Mixed-precision A*X path of libxs (tc.cu): split (hi + lo) float operands on
// the tensor cores with float32 accumulation, float32 G build.
#pragma once

#include "common.cuh"

namespace xs {

void products_mixed(Ctx& c, DevMol& m, int method, int nvec, const double* X, double* Y1, double* Y2,
                    bool triplet = false);

}  // namespace xs
