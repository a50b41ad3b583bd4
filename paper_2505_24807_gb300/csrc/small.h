// Launchers of the small dense subspace kernels (small.cu).
#pragma once

#include <cuda_runtime.h>

namespace xs {

void sym_upper(cudaStream_t s, int S, const double* a, int lda, double* E, int lde);
// A[:, j] *= d[j]^(1/2) (mode 0), d[j]^(-1/2) (mode 1) or 1/d[j] (mode 2)
void scale_cols(cudaStream_t s, int rows, int ncols, double* A, int lda, const double* d, int mode);
void lowdin(cudaStream_t s, int n, const double* lam, const double* Q, int ldq, double thresh, double* Bm, int ldb,
            int* nkeep);
void sqrt_roots(cudaStream_t s, int k, const double* w2, double* omega, int* flag);
void unit_vectors(cudaStream_t s, int k, long long ld, const long long* idx, double* V);
void set_diag(cudaStream_t s, int S, const double* vals, double* a, int lda);

}  // namespace xs
