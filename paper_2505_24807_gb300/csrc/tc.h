// Mixed-precision A*X path of libxs (tc.cu): split (hi + lo) float operands on
// the tensor cores with float32 accumulation, float32 G build.
#pragma once

#include "common.cuh"

namespace xs {

// mx1, mx2: optional per-vector abs_hi maxima of Y1 / Y2 (see products.h)
void products_mixed(Ctx& c, DevMol& m, int method, int nvec, const double* X, double* Y1, double* Y2,
                    bool triplet = false, unsigned int* mx1 = nullptr, unsigned int* mx2 = nullptr);

}  // namespace xs
