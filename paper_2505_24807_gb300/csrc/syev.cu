// Lowest eigenpairs of the small symmetric Davidson matrices, float64, one CTA
// (paper, Section "GPU Implementation", batched step 3: diagonalise the
// projected matrix and keep the lowest K states).
//
// This part's float64 pipe issues one warp instruction per 64 cycles per
// sub-partition whatever the number of active lanes, and a float64 divide
// costs ~640 cycles, so the kernel keeps float64 work in as few warps as hold
// data and moves what can be approximate to float32:
//   1. Householder tridiagonalisation Q^T A Q = T in float64 on the packed
//      lower triangle (half the rank-2 update's float64 instructions; shared
//      memory up to S = kSmemMax = 224, else global scratch, which runs ~3x
//      slower per step); the reflectors go to
//      global scratch, the matrix-vector product of each step is split over
//      row segments, reductions run only in the warps that hold data;
//   2. the k lowest eigenvalues of T by Sturm-count multisection in float32,
//      one warp per eigenvalue and 32 counts per round, to ~2e-7 |T|;
//   3. float64 inverse iteration on T (pivoted tridiagonal LU, one thread per
//      eigenvector, vector and LU in the freed shared memory when they fit):
//      two solves with the float32 shift, then a third shifted by the
//      Rayleigh quotient; the Rayleigh quotient of the result is the float64
//      eigenvalue (its error is quadratic in the vector's).  Shifts closer
//      than 2e-6 |T| form clusters: spread apart, solved three times with
//      their own shift, re-orthogonalised (Gram-Schmidt) and, up to four
//      members, rotated by a Rayleigh-Ritz step inside the cluster;
//   4. back-transformation z = H_0 H_1 ... H_{S-3} y, one warp per vector.
//
// Also: Cholesky factorisation a = L L^T of the TDHF matrix a- (positive
// definite unless the reference is unstable).
#include <cfloat>

#include "kernels.h"
#include "prof.h"
#include "syev.h"
#include "syev_body.cuh"

namespace xs {

namespace {

template <bool SMEM>
__global__ void __launch_bounds__(1024) syevk_kernel(int S, int k, const double* __restrict__ Ain, int lda,
                                                     double* __restrict__ wout, double* __restrict__ Z, int ldz,
                                                     double* __restrict__ gscratch, int* info) {
  syevk_body<SMEM>(S, k, Ain, lda, wout, Z, ldz, gscratch, info);
}

template <bool SMEM>
__global__ void __launch_bounds__(1024) cholesky_kernel(int S, double* A, int lda, int* flag) {
  cholesky_body<SMEM>(S, A, lda, flag);
}

}  // namespace


void syevk(cudaStream_t s, int S, int k, const double* A, int lda, double* w, double* Z, int ldz,
           DevBuf<double>& scratch, int* info) {
  if (S <= 0 || k <= 0) return;
  if (k > S) k = S;
  if (S > 1024) throw Error(XS_EINVAL, "syevk: matrix larger than 1024");
  // working set (matrix, tridiagonal, reflector, products, eigenvalues,
  // float32 copy, cluster indices) in doubles
  const size_t wd = syevk_work_doubles(S);
  scratch.ensure(syevk_scratch_doubles(S, k));
  ProfScope ps(s, "syevk_f64", 0.0, (4.0 / 3.0) * S * (double)S * S);
  if (S <= kSmemMax) {
    const size_t smem = sizeof(double) * wd;
    static const bool attr = [&] {   // once per process (thread-safe initialisation)
      XS_CUDA(cudaFuncSetAttribute(syevk_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(sizeof(double) * syevk_work_doubles(kSmemMax))));
      return true;
    }();
    (void)attr;
    syevk_kernel<true><<<1, 1024, smem, s>>>(S, k, A, lda, w, Z, ldz, scratch.get(), info);
  } else {
    syevk_kernel<false><<<1, 1024, 0, s>>>(S, k, A, lda, w, Z, ldz, scratch.get(), info);
  }
  XS_CHECK_LAUNCH();
}

void cholesky(cudaStream_t s, int S, double* A, int lda, int* flag) {
  if (S <= 0) return;
  ProfScope ps(s, "cholesky_f64", 0.0, S * (double)S * S / 3.0);
  if (S <= kCholSmemMax) {
    const size_t smem = sizeof(double) * (size_t)S * (S + 1) / 2;
    static const bool attr = [] {   // once per process (thread-safe initialisation)
      XS_CUDA(cudaFuncSetAttribute(cholesky_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(sizeof(double) * kCholSmemMax * (kCholSmemMax + 1) / 2)));
      return true;
    }();
    (void)attr;
    cholesky_kernel<true><<<1, 1024, smem, s>>>(S, A, lda, flag);
  } else {
    cholesky_kernel<false><<<1, 1024, 0, s>>>(S, A, lda, flag);
  }
  XS_CHECK_LAUNCH();
}

}  // namespace xs
