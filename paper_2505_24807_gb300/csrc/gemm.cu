// Register-tiled SIMT GEMM (float64 / float32) of libxs.
//
// Used for the float64 transforms of the A*X product (Eq. cis_matrix_vector:
// R = C_occ X C_vir^T and C_occ^T G C_vir), the Coulomb supermatrix product
// J = W r, the Davidson subspace projections and Ritz vectors, and the SCF.
// A BM x BN output tile per 256-thread CTA, K staged 16 at a time through
// shared memory; thread (tx, ty) owns rows ty + (BM/TM) i and columns
// tx + (BN/TN) j so that shared-memory reads are conflict free.  Three
// shapes: 64x64 (4x4 per thread) for square problems, 32x128 (2x8) when M
// is small (Ritz vectors and Gram-Schmidt updates: M = roots), 128x32 (8x2)
// when N is small (split-K Gram products of the subspace).
#include "kernels.h"
#include "prof.h"

namespace xs {

namespace {

constexpr int BK = 16;

template <typename T, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, T alpha, const T* __restrict__ A,
                                                   int lda, long long sA, bool transA, const T* __restrict__ B,
                                                   int ldb, long long sB, bool transB, T beta, T* __restrict__ C,
                                                   int ldc, long long sC, int kSplit, long long sSplit) {
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads per CTA");
  constexpr int RY = BM / TM, RX = BN / TN;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % RX, ty = tid / RX;
  const int z = blockIdx.z;
  const int b = z / kSplit, ks = z % kSplit;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  A += b * sA;
  B += b * sB;
  C += b * sC + ks * sSplit;
  int kc = (K + kSplit - 1) / kSplit;
  kc = ((kc + BK - 1) / BK) * BK;
  const int kbeg = ks * kc;
  const int kend = min(K, kbeg + kc);

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / 256; ++r) {
      const int idx = tid + 256 * r;
      int m, k;
      if (!transA) { m = idx / BK; k = idx % BK; } else { k = idx / BM; m = idx % BM; }
      const int gm = m0 + m, gk = k0 + k;
      T val = T(0);
      if (gm < M && gk < kend) val = transA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[k][m] = val;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / 256; ++r) {
      const int idx = tid + 256 * r;
      int n, k;
      if (!transB) { k = idx / BN; n = idx % BN; } else { n = idx / BK; k = idx % BK; }
      const int gn = n0 + n, gk = k0 + k;
      T val = T(0);
      if (gn < N && gk < kend) val = transB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[k][n] = val;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + RY * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + RX * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + RY * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + RX * j;
      if (gn >= N) continue;
      T* c = C + (long long)gm * ldc + gn;
      T r = alpha * acc[i][j];
      if (beta != T(0)) r = fma(beta, *c, r);
      *c = r;
    }
  }
}

// C = alpha * sum_s P[s] + beta * C over the split partials.
template <typename T>
__global__ void reduce_split(int M, int N, int kSplit, const T* __restrict__ P, T alpha, T beta, T* __restrict__ C,
                             int ldc) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  int m = idx / N, n = idx % N;
  T s = T(0);
  for (int k = 0; k < kSplit; ++k) s += P[(long long)k * M * N + idx];
  T* c = C + (long long)m * ldc + n;
  T r = alpha * s;
  if (beta != T(0)) r = fma(beta, *c, r);
  *c = r;
}

enum class Shape { Square, SmallM, SmallN };

Shape pick_shape(int M, int N) {
  if (M <= 32 && N > 64) return Shape::SmallM;
  if (N <= 32 && M > 64) return Shape::SmallN;
  return Shape::Square;
}

int tiles_of(Shape sh, int M, int N) {
  if (sh == Shape::SmallM) return ((N + 127) / 128) * ((M + 31) / 32);
  if (sh == Shape::SmallN) return ((N + 31) / 32) * ((M + 127) / 128);
  return ((N + 63) / 64) * ((M + 63) / 64);
}

template <typename T>
void launch_gemm(cudaStream_t s, Shape sh, int M, int N, int K, T alpha, const T* A, int lda, long long sA, bool tA,
                 const T* B, int ldb, long long sB, bool tB, T beta, T* C, int ldc, long long sC, int zdim, int kSplit,
                 long long sSplit) {
  if (sh == Shape::SmallM) {
    dim3 grid((N + 127) / 128, (M + 31) / 32, zdim);
    gemm_kernel<T, 32, 128, 2, 8><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, tA, B, ldb, sB, tB, beta, C, ldc,
                                                       sC, kSplit, sSplit);
  } else if (sh == Shape::SmallN) {
    dim3 grid((N + 31) / 32, (M + 127) / 128, zdim);
    gemm_kernel<T, 128, 32, 8, 2><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, tA, B, ldb, sB, tB, beta, C, ldc,
                                                       sC, kSplit, sSplit);
  } else {
    dim3 grid((N + 63) / 64, (M + 63) / 64, zdim);
    gemm_kernel<T, 64, 64, 4, 4><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, tA, B, ldb, sB, tB, beta, C, ldc,
                                                      sC, kSplit, sSplit);
  }
}

}  // namespace

template <typename T>
void gemm(cudaStream_t s, bool transA, bool transB, int M, int N, int K, T alpha, const T* A, int lda, long long sA,
          const T* B, int ldb, long long sB, T beta, T* C, int ldc, long long sC, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K < 0) K = 0;
  ProfScope ps(s, sizeof(T) == 8 ? "gemm_f64" : "gemm_f32", 0.0, 2.0 * M * N * (double)K * batch);
  launch_gemm<T>(s, pick_shape(M, N), M, N, K, alpha, A, lda, sA, transA, B, ldb, sB, transB, beta, C, ldc, sC, batch,
                 1, 0);
  XS_CHECK_LAUNCH();
}

template <typename T>
void gram(cudaStream_t s, int M, int N, int L, const T* A, int lda, const T* B, int ldb, T* C, int ldc, T alpha,
          T beta, DevBuf<T>& ws) {
  if (M <= 0 || N <= 0) return;
  const Shape sh = pick_shape(M, N);
  const int tiles = tiles_of(sh, M, N);
  int kSplit = (2 * 152 + tiles - 1) / tiles;
  const int maxSplit = (L + 4 * BK - 1) / (4 * BK);
  if (kSplit > maxSplit) kSplit = maxSplit;
  if (kSplit < 1) kSplit = 1;
  ws.ensure((size_t)kSplit * M * N);
  {
    ProfScope ps(s, sizeof(T) == 8 ? "gram_f64" : "gram_f32", sizeof(T) * (double)L * (M + N),
                 2.0 * M * N * (double)L);
    launch_gemm<T>(s, sh, M, N, L, T(1), A, lda, 0, false, B, ldb, 0, true, T(0), ws.get(), N, 0, kSplit, kSplit,
                   (long long)M * N);
    XS_CHECK_LAUNCH();
  }
  reduce_split<T><<<grid1((long long)M * N, 256), 256, 0, s>>>(M, N, kSplit, ws.get(), alpha, beta, C, ldc);
  XS_CHECK_LAUNCH();
}

template void gemm<double>(cudaStream_t, bool, bool, int, int, int, double, const double*, int, long long,
                           const double*, int, long long, double, double*, int, long long, int);
template void gemm<float>(cudaStream_t, bool, bool, int, int, int, float, const float*, int, long long, const float*,
                          int, long long, float, float*, int, long long, int);
template void gram<double>(cudaStream_t, int, int, int, const double*, int, const double*, int, double*, int, double,
                           double, DevBuf<double>&);
template void gram<float>(cudaStream_t, int, int, int, const float*, int, const float*, int, float*, int, float, float,
                          DevBuf<float>&);

}  // namespace xs
