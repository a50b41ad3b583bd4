// Float64-accurate tall-skinny products of the Davidson subspace on the BF16
// tensor cores (ozaki.cu).
//
// Every float64 vector x (one row of V, (A+B)V, (A-B)V, ...) is stored as
// eight balanced base-128 digit planes: with a per-row exponent e,
//   x[l] = 2^e * sum_{i=1..8} d_i[l] 2^(-7 i) + O(2^(e-57)),  |d_i| <= 64,
// the error-free splitting of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms
// 59, 95-118 (2012)).  The digits are small integers, exact in bfloat16; a
// product of two digits is at most 2^12 in magnitude, so up to 4096 of them
// sum exactly in the tensor cores' float32 accumulators.  Products of digit
// planes are therefore exact, and the float64 result is assembled from them
// with the digit weights -- the same accuracy as a float64 GEMM, at tensor-core
// rather than float64-pipe speed.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace xs {

using oz_t = uint16_t;           // bfloat16 bit pattern of one digit
constexpr int kOzDigits = 8;     // digit planes per float64 row
constexpr int kOzChunk = 4096;   // digit products summed exactly per float32 accumulator

struct OzWork {
  DevBuf<double> part;              // split partial sums of oz_gram
  DevBuf<oz_t> bmat;                // digit matrix of the oz_combine coefficients
  DevBuf<double> scale;             // their per-output weights (two per output)
  DevBuf<unsigned int> mx;          // per-row abs_hi of max |x|
};

// e[r] such that max_l |X[r][l]| < 2^(e[r]-1), rows r < nvec (row stride ldx).
// A non-finite entry raises the error word (code 10).
void oz_exponents(cudaStream_t s, int nvec, long long L, const double* X, long long ldx, int* e, OzWork& w,
                  int* err);

// The same exponents from per-row maxima already formed by the kernel that
// wrote the rows (abs_hi of max |x|, common.cuh; see oz_combine's rowmax).
void oz_exponents_from_max(cudaStream_t s, int nvec, const unsigned int* mx, int* e, int* err);

// Digit planes of rows r < nvec of X (exponents e[r]), written as
//   tn: plane p = (tn_r0 + r) * 8 + i (i = 0 the most significant digit) in
//       blocks of 64 amplitudes: element (p, l) at ((l / 64) * P + p) * 64 +
//       l % 64, P the array's plane capacity (each block holds all its planes'
//       64 digits contiguously, so a tile of consecutive planes is one
//       contiguous read); amplitudes L..oz_lp(L)-1 are set to 0;
//   nn: column k = (nn_r0 + r) * 8 + i of amplitude row l, in blocks of 64
//       columns: element (l, k) at ((k / 64) * L + l) * 64 + k % 64 (each
//       block holds its 64 columns of every amplitude contiguously; ldk, a
//       multiple of 64, is the column capacity).
// Either output may be null.
void oz_slice(cudaStream_t s, int nvec, long long L, const double* X, long long ldx, const int* e, oz_t* tn,
              long long P, int tn_r0, oz_t* nn, int ldk, int nn_r0);

// C (M x N, row stride ldc) = alpha * A B^T + beta * C, where A holds M rows and
// B holds N rows of length L as tn digit planes (plane capacities AP, BP) with
// exponents eA, eB.  Split over L into float32-exact chunks of 4096.
void oz_gram(cudaStream_t s, int M, int N, long long L, const oz_t* Atn, long long AP, const int* eA,
             const oz_t* Btn, long long BP, const int* eB, double alpha, double beta, double* C, int ldc,
             OzWork& w, int* err);

// One block of a combination: the first S rows of a stored set (nn digit
// layout with column capacity ldk, exponents e) and its coefficients
// coef[m][k] (row stride ldc).
struct OzBlock {
  const oz_t* nn;
  int ldk;
  const int* e;
  const double* coef;
  int ldc;
};

// Y[k][l] (row stride ldy) = alpha * sum_b sum_{m<S} coef_b[m][k] X_b[m][l] + beta * Y[k][l]
// for k < nout, l < L, over nb <= 3 blocks.  rowmax (optional, nout entries):
// per output row abs_hi (common.cuh) of the largest |Y[k][l]|, formed in the
// epilogue (input of oz_exponents_from_max).
void oz_combine(cudaStream_t s, int nb, const OzBlock* blk, int S, int nout, long long L, double alpha, double beta,
                double* Y, long long ldy, OzWork& w, int* err, unsigned int* rowmax = nullptr);

// Column capacity of the nn layout for up to S rows (whole 64-column blocks).
inline int oz_ldk(int S) { return ((S * kOzDigits + 63) / 64) * 64; }
// Amplitudes of the tn layout for vectors of length L (whole 64-amplitude blocks).
inline long long oz_lp(long long L) { return ((L + 63) / 64) * 64; }

}  // namespace xs
