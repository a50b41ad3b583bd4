// Small dense float64 eigensolver and Cholesky of libxs (syev.cu).
#pragma once

#include "common.cuh"

namespace xs {

// k lowest eigenpairs of the symmetric S x S matrix A (lda; not modified):
// eigenvalues ascending in w[0..k), eigenvectors in the columns of Z (S x k, ldz).
void syevk(cudaStream_t s, int S, int k, const double* A, int lda, double* w, double* Z, int ldz,
           DevBuf<double>& scratch, int* info);
// In-place lower Cholesky factor of the symmetric positive definite A; flag
// (device int) becomes 1 when a pivot is not positive.
void cholesky(cudaStream_t s, int S, double* A, int lda, int* flag);

}  // namespace xs
