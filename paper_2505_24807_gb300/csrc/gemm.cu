// Register-tiled SIMT GEMM (float64 / float32) of libxs.
//
// Used for the float64 transforms of the A*X product (Eq. cis_matrix_vector:
// R = C_occ X C_vir^T and C_occ^T G C_vir), the Coulomb supermatrix product
// J = W r, the Davidson subspace projections and the SCF.  64 x 64 output
// tile per 256-thread CTA, 4 x 4 outputs per thread strided by 16 so that
// shared-memory reads are conflict free; K staged 16 at a time.
#include "kernels.h"
#include "prof.h"

namespace xs {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <typename T>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, T alpha, const T* __restrict__ A,
                                                   int lda, long long sA, bool transA, const T* __restrict__ B,
                                                   int ldb, long long sB, bool transB, T beta, T* __restrict__ C,
                                                   int ldc, long long sC, int kSplit, long long sSplit) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
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

  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = tid + 256 * r;
      int m, k;
      if (!transA) { m = idx / BK; k = idx % BK; } else { k = idx / BM; m = idx % BM; }
      int gm = m0 + m, gk = k0 + k;
      T val = T(0);
      if (gm < M && gk < kend) val = transA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[k][m] = val;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int idx = tid + 256 * r;
      int n, k;
      if (!transB) { k = idx / BN; n = idx % BN; } else { n = idx / BK; k = idx % BK; }
      int gn = n0 + n, gk = k0 + k;
      T val = T(0);
      if (gn < N && gk < kend) val = transB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
      Bs[k][n] = val;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
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

}  // namespace

template <typename T>
void gemm(cudaStream_t s, bool transA, bool transB, int M, int N, int K, T alpha, const T* A, int lda,
          long long sA, const T* B, int ldb, long long sB, T beta, T* C, int ldc, long long sC, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    // C = beta C: use the kernel with an empty K loop
    K = 0;
  }
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  ProfScope ps(s, sizeof(T) == 8 ? "gemm_f64" : "gemm_f32", 0.0, 2.0 * M * N * (double)K * batch);
  gemm_kernel<T><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, transA, B, ldb, sB, transB, beta, C, ldc,
                                      sC, 1, 0);
  XS_CHECK_LAUNCH();
}

template <typename T>
void gram(cudaStream_t s, int M, int N, int L, const T* A, int lda, const T* B, int ldb, T* C, int ldc,
          T alpha, T beta, DevBuf<T>& ws) {
  if (M <= 0 || N <= 0) return;
  int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int kSplit = (2 * 152 + tiles - 1) / tiles;
  int maxSplit = (L + 4 * BK - 1) / (4 * BK);
  if (kSplit > maxSplit) kSplit = maxSplit;
  if (kSplit < 1) kSplit = 1;
  ws.ensure((size_t)kSplit * M * N);
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, kSplit);
  ProfScope ps(s, sizeof(T) == 8 ? "gram_f64" : "gram_f32", sizeof(T) * (double)L * (M + N), 2.0 * M * N * (double)L);
  gemm_kernel<T><<<grid, 256, 0, s>>>(M, N, L, T(1), A, lda, 0, false, B, ldb, 0, true, T(0), ws.get(), N, 0,
                                      kSplit, (long long)M * N);
  XS_CHECK_LAUNCH();
  reduce_split<T><<<grid1((long long)M * N, 256), 256, 0, s>>>(M, N, kSplit, ws.get(), alpha, beta, C, ldc);
  XS_CHECK_LAUNCH();
}

template void gemm<double>(cudaStream_t, bool, bool, int, int, int, double, const double*, int, long long,
                           const double*, int, long long, double, double*, int, long long, int);
template void gemm<float>(cudaStream_t, bool, bool, int, int, int, float, const float*, int, long long,
                          const float*, int, long long, float, float*, int, long long, int);
template void gram<double>(cudaStream_t, int, int, int, const double*, int, const double*, int, double*, int,
                           double, double, DevBuf<double>&);
template void gram<float>(cudaStream_t, int, int, int, const float*, int, const float*, int, float*, int, float,
                          float, DevBuf<float>&);

}  // namespace xs
