// A*X products of libxs (products.cu, tc.cu).
#pragma once

#include "common.cuh"

namespace xs {

// internal precision code: float32 SIMT products (polish step of mixed solves)
constexpr int kPrecF32 = 2;

// Y1 = A X (CIS) or Y1 = (A+B) X, Y2 = (A-B) X (TDHF) for nvec vectors
// X (nvec x nocc x nvir, float64, device).  precision: XS_FP64 or XS_MIXED.
// triplet: the spin-adapted triplet matrices (no Coulomb terms in G).
// mx1, mx2 (XS_MIXED only, else ignored): per output vector abs_hi of its
// largest |y| (common.cuh), formed by the epilogue that writes Y1 / Y2 (the
// digit split of the Davidson subspace needs it).
void products(Ctx& c, DevMol& m, int method, int precision, int nvec, const double* X, double* Y1, double* Y2,
              bool triplet = false, unsigned int* mx1 = nullptr, unsigned int* mx2 = nullptr);
void products_fp64(Ctx& c, const DevMol& m, int method, int nvec, const double* X, double* Y1, double* Y2,
                   bool triplet = false);
// G_CIS(R) of nvec AO matrices (float64 device arrays)
void gmatrix(Ctx& c, const DevMol& m, int precision, int nvec, const double* R, double* G);
// vectors per pass of the AO work arrays
int product_batch(const DevMol& m);

}  // namespace xs
