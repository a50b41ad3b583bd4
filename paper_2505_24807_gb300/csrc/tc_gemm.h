// Split-precision (TF32 hi + lo) tensor-core GEMM of libxs (tc_gemm.cu).
#pragma once

#include <cuda_runtime.h>

namespace xs {

// One K-major operand: rows x Kpad float32 pairs (hi, lo), row stride ld
// (a multiple of 4 floats, 16-byte aligned base), batch entries bstride apart
// when batched.  Kpad is a multiple of 32 and the padding columns are zero.
struct TcOperand {
  const float* hi;
  const float* lo;
  int ld;
  long long bstride;
  bool batched;
};

// Epilogue: mode 0 stores float D; mode 1 stores the TF32 pair (D, Dlo) of the
// result; mode 2 stores double Y = D + (eps[o + col] - eps[row]) X and, when
// rowmax is set, raises rowmax[b] to abs_hi of the largest |Y| of batch entry
// b (common.cuh; the caller zeroes it first).
struct TcEpilogue {
  int mode = 0;
  float* D = nullptr;
  float* Dlo = nullptr;
  double* Y = nullptr;
  const double* X = nullptr;
  const double* eps = nullptr;
  int ld = 0;
  long long bstride = 0;
  int o = 0;
  unsigned int* rowmax = nullptr;
};

// D[b] (M x N) = A[b] B[b]^T from TF32 pairs: hi*hi + hi*lo + lo*hi, float32
// accumulation.  d_err: device int set to a nonzero code when a bounded
// device-side wait timed out.  The first call of a new problem class runs the
// product several times (tile-width timing), so the output must not alias an
// input.
void tc_gemm(cudaStream_t s, const TcOperand& A, const TcOperand& B, int M, int N, int Kpad, int batch,
             const TcEpilogue& e, int* d_err);

// Zero-padded TF32 pair of a row-major matrix (rows x cols, source row stride
// ld_src), optionally transposed (dst[r][c] = src[c][r]); batched over
// grid.z with the given strides.
template <typename S>
void split_pad(cudaStream_t s, int rows, int cols, int ld_dst, const S* src, int ld_src, long long sstride,
               long long dstride, int batch, bool transpose, float* hi, float* lo);

// Transposed split of float64 matrices through shared-memory tiles:
// dst[r][c] (rows x ld_dst) = TF32 pair of src[c][r] for c < cols, zero up to
// ld_dst; src holds cols rows of row stride ld_src; batched over grid.z.
void split_pad_t(cudaStream_t s, int rows, int cols, int ld_dst, const double* src, int ld_src, long long sstride,
                 long long dstride, int batch, float* hi, float* lo);

int pad32(int k);

}  // namespace xs
