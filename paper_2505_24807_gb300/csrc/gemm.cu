// Register-tiled SIMT GEMM (float64 / float32) of libxs.
//
// Used for the float64 transforms of the A*X product (Eq. cis_matrix_vector:
// R = C_occ X C_vir^T and C_occ^T G C_vir), the Coulomb supermatrix product
// J = W r, the Davidson subspace projections and Ritz vectors, and the SCF.
// A BM x BN output tile per 256-thread CTA, K staged 16 at a time through
// shared memory; thread (tx, ty) owns rows ty + (BM/TM) i and columns
// tx + (BN/TN) j so that shared-memory reads are conflict free.  Eleven tile
// shapes, from 64x64 for square problems to 8x512 (Ritz vectors and
// Gram-Schmidt updates: M = roots) and 256x8 (split-K Gram products: N = new
// vectors); the one that pads the problem least is launched.
#include <cstring>
#include <mutex>
#include <unordered_map>

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
    for (int r = 0; r < (BM * BK + 255) / 256; ++r) {
      const int idx = tid + 256 * r;
      if (idx >= BM * BK) break;
      int m, k;
      if (!transA) { m = idx / BK; k = idx % BK; } else { k = idx / BM; m = idx % BM; }
      const int gm = m0 + m, gk = k0 + k;
      T val = T(0);
      if (gm < M && gk < kend) val = transA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[k][m] = val;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK + 255) / 256; ++r) {
      const int idx = tid + 256 * r;
      if (idx >= BN * BK) break;
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

// float32 C = alpha op(A) op(B) + beta C for large M and N: 128 x 128 tiles,
// 8 x 8 outputs per thread (as 2 x 2 blocks of 4 x 4 for conflict-free
// float4 shared-memory reads), K staged 8 at a time through a double-buffered
// shared-memory ring with the next tile prefetched into registers.  vecA /
// vecB: the operand allows aligned float4 global loads along its contiguous
// dimension.
constexpr int FB = 128, FK = 8;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_big_kernel(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                        int lda, long long sA, const float* __restrict__ B, int ldb,
                                                        long long sB, float beta, float* __restrict__ C, int ldc,
                                                        long long sC, int vecA, int vecB) {
  __shared__ __align__(16) float As[2][FK][FB + 4];
  __shared__ __align__(16) float Bs[2][FK][FB + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * FB, n0 = blockIdx.x * FB;
  A += blockIdx.z * sA;
  B += blockIdx.z * sB;
  C += blockIdx.z * sC;

  float ra[4], rb[4];
  // global -> registers for the K tile starting at k0
  auto load_tiles = [&](int k0) {
    if (!TA) {
      const int m = tid / 2, kk = (tid % 2) * 4;
      const int gm = m0 + m, gk = k0 + kk;
      if (vecA && gm < M && gk + 3 < K) {
        const float4 t = *reinterpret_cast<const float4*>(A + (long long)gm * lda + gk);
        ra[0] = t.x; ra[1] = t.y; ra[2] = t.z; ra[3] = t.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) ra[q] = (gm < M && gk + q < K) ? A[(long long)gm * lda + gk + q] : 0.0f;
      }
    } else {
      const int kk = tid / 32, m = (tid % 32) * 4;
      const int gk = k0 + kk, gm = m0 + m;
      if (vecA && gk < K && gm + 3 < M) {
        const float4 t = *reinterpret_cast<const float4*>(A + (long long)gk * lda + gm);
        ra[0] = t.x; ra[1] = t.y; ra[2] = t.z; ra[3] = t.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) ra[q] = (gk < K && gm + q < M) ? A[(long long)gk * lda + gm + q] : 0.0f;
      }
    }
    if (!TB) {
      const int kk = tid / 32, n = (tid % 32) * 4;
      const int gk = k0 + kk, gn = n0 + n;
      if (vecB && gk < K && gn + 3 < N) {
        const float4 t = *reinterpret_cast<const float4*>(B + (long long)gk * ldb + gn);
        rb[0] = t.x; rb[1] = t.y; rb[2] = t.z; rb[3] = t.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) rb[q] = (gk < K && gn + q < N) ? B[(long long)gk * ldb + gn + q] : 0.0f;
      }
    } else {
      const int n = tid / 2, kk = (tid % 2) * 4;
      const int gn = n0 + n, gk = k0 + kk;
      if (vecB && gn < N && gk + 3 < K) {
        const float4 t = *reinterpret_cast<const float4*>(B + (long long)gn * ldb + gk);
        rb[0] = t.x; rb[1] = t.y; rb[2] = t.z; rb[3] = t.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) rb[q] = (gn < N && gk + q < K) ? B[(long long)gn * ldb + gk + q] : 0.0f;
      }
    }
  };
  auto store_tiles = [&](int buf) {
    if (!TA) {
      const int m = tid / 2, kk = (tid % 2) * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q) As[buf][kk + q][m] = ra[q];
    } else {
      const int kk = tid / 32, m = (tid % 32) * 4;
      *reinterpret_cast<float4*>(&As[buf][kk][m]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
    }
    if (!TB) {
      const int kk = tid / 32, n = (tid % 32) * 4;
      *reinterpret_cast<float4*>(&Bs[buf][kk][n]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    } else {
      const int n = tid / 2, kk = (tid % 2) * 4;
#pragma unroll
      for (int q = 0; q < 4; ++q) Bs[buf][kk + q][n] = rb[q];
    }
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  load_tiles(0);
  store_tiles(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += FK) {
    const bool more = k0 + FK < K;
    if (more) load_tiles(k0 + FK);
#pragma unroll
    for (int kk = 0; kk < FK; ++kk) {
      float a[8], b[8];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w; a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w; b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store_tiles(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
      if (gn >= N) continue;
      float* c = C + (long long)gm * ldc + gn;
      float r = alpha * acc[i][j];
      if (beta != 0.0f) r = fmaf(beta, *c, r);
      *c = r;
    }
  }
}

void sgemm_big(cudaStream_t s, bool tA, bool tB, int M, int N, int K, float alpha, const float* A, int lda,
               long long sA, const float* B, int ldb, long long sB, float beta, float* C, int ldc, long long sC,
               int batch) {
  auto al = [](const float* p, int ld, long long st) {
    return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && (ld % 4 == 0) && (st % 4 == 0) ? 1 : 0;
  };
  const int vA = al(A, lda, sA), vB = al(B, ldb, sB);
  dim3 grid((N + FB - 1) / FB, (M + FB - 1) / FB, batch);
  if (!tA && !tB) sgemm_big_kernel<false, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, vA, vB);
  else if (!tA && tB) sgemm_big_kernel<false, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, vA, vB);
  else if (tA && !tB) sgemm_big_kernel<true, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, vA, vB);
  else sgemm_big_kernel<true, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, vA, vB);
}

// Tile shapes (BM, BN, TM, TN), all 256 threads.  The float64 pipe of this
// part is narrow enough that the Davidson GEMMs run pipe-bound, so every
// padded row or column of a tile is lost time: the shape that pads M x N
// least is taken (ties: earlier entries, which block more registers).
struct TileShape {
  int bm, bn;
};
constexpr TileShape kShapes[] = {{64, 64}, {32, 128}, {16, 256}, {8, 512}, {128, 32}, {256, 16},
                                 {256, 8}, {64, 32},  {32, 32},  {64, 16}, {32, 16}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

int pick_shape(int M, int N) {
  int best = 0;
  long long best_area = -1;
  for (int s = 0; s < kNumShapes; ++s) {
    const int bm = kShapes[s].bm, bn = kShapes[s].bn;
    const long long area = (long long)((M + bm - 1) / bm) * bm * (long long)((N + bn - 1) / bn) * bn;
    if (best_area < 0 || area < best_area) {
      best = s;
      best_area = area;
    }
  }
  return best;
}

int tiles_of(int sh, int M, int N) {
  const int bm = kShapes[sh].bm, bn = kShapes[sh].bn;
  return ((N + bn - 1) / bn) * ((M + bm - 1) / bm);
}

template <typename T, int BM, int BN, int TM, int TN>
void launch_one(cudaStream_t s, int M, int N, int K, T alpha, const T* A, int lda, long long sA, bool tA, const T* B,
                int ldb, long long sB, bool tB, T beta, T* C, int ldc, long long sC, int zdim, int kSplit,
                long long sSplit) {
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, zdim);
  gemm_kernel<T, BM, BN, TM, TN><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, tA, B, ldb, sB, tB, beta, C, ldc,
                                                      sC, kSplit, sSplit);
}

template <typename T>
void launch_gemm(cudaStream_t s, int sh, int M, int N, int K, T alpha, const T* A, int lda, long long sA, bool tA,
                 const T* B, int ldb, long long sB, bool tB, T beta, T* C, int ldc, long long sC, int zdim, int kSplit,
                 long long sSplit) {
#define XS_GEMM_CASE(I, BM_, BN_, TM_, TN_)                                                                       \
  case I:                                                                                                         \
    launch_one<T, BM_, BN_, TM_, TN_>(s, M, N, K, alpha, A, lda, sA, tA, B, ldb, sB, tB, beta, C, ldc, sC, zdim, \
                                      kSplit, sSplit);                                                            \
    break;
  switch (sh) {
    XS_GEMM_CASE(1, 32, 128, 2, 8)
    XS_GEMM_CASE(2, 16, 256, 2, 8)
    XS_GEMM_CASE(3, 8, 512, 1, 16)
    XS_GEMM_CASE(4, 128, 32, 8, 2)
    XS_GEMM_CASE(5, 256, 16, 8, 2)
    XS_GEMM_CASE(6, 256, 8, 8, 1)
    XS_GEMM_CASE(7, 64, 32, 4, 2)
    XS_GEMM_CASE(8, 32, 32, 2, 2)
    XS_GEMM_CASE(9, 64, 16, 4, 1)
    XS_GEMM_CASE(10, 32, 16, 2, 1)
    default:
      launch_one<T, 64, 64, 4, 4>(s, M, N, K, alpha, A, lda, sA, tA, B, ldb, sB, tB, beta, C, ldc, sC, zdim, kSplit,
                                  sSplit);
  }
#undef XS_GEMM_CASE
}

// ---- tile-shape autotuner ----------------------------------------------------
// The first time a problem class is met -- element type, transposes, batch > 1
// and M, N, K rounded up to powers of two -- every tile shape whose padded
// area is within 1.5x of the least is timed on a scratch output (one warm-up
// launch, then two timed with CUDA events on the caller's stream) and the
// fastest is kept for the process.  Classes whose output exceeds 8M elements,
// calls inside stream capture and calls from allocation-free entry points use
// the least-padding rule directly.
thread_local int g_no_tune = 0;

int ceil_log2(long long x) {
  int l = 0;
  while ((1LL << l) < x) ++l;
  return l;
}

std::mutex g_tune_mutex;
std::unordered_map<unsigned long long, int> g_tuned;

template <typename T>
int tuned_shape(cudaStream_t s, bool tA, bool tB, int M, int N, int K, const T* A, int lda, long long sA,
                const T* B, int ldb, long long sB, int batch) {
  const int heuristic = pick_shape(M, N);
  if (g_no_tune || (long long)M * N * batch > (8LL << 20)) return heuristic;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return heuristic;
  const unsigned long long key = (unsigned long long)(sizeof(T) == 8) | ((unsigned long long)tA << 1) |
                                 ((unsigned long long)tB << 2) | ((unsigned long long)(batch > 1) << 3) |
                                 ((unsigned long long)ceil_log2(M) << 8) | ((unsigned long long)ceil_log2(N) << 16) |
                                 ((unsigned long long)ceil_log2(K) << 24);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
  }
  const auto area = [&](int sh) {
    return (double)((M + kShapes[sh].bm - 1) / kShapes[sh].bm) * kShapes[sh].bm *
           (double)((N + kShapes[sh].bn - 1) / kShapes[sh].bn) * kShapes[sh].bn;
  };
  const double amin = area(heuristic);
  T* Cs = nullptr;
  if (cudaMalloc(&Cs, sizeof(T) * (size_t)M * N * batch) != cudaSuccess) {
    cudaGetLastError();
    return heuristic;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = heuristic;
  float best_ms = 1e30f;
  for (int sh = 0; sh < kNumShapes; ++sh) {
    if (area(sh) > 1.5 * amin) continue;
    launch_gemm<T>(s, sh, M, N, K, T(1), A, lda, sA, tA, B, ldb, sB, tB, T(0), Cs, N, (long long)M * N, batch, 1, 0);
    cudaEventRecord(e0, s);
    for (int r = 0; r < 2; ++r)
      launch_gemm<T>(s, sh, M, N, K, T(1), A, lda, sA, tA, B, ldb, sB, tB, T(0), Cs, N, (long long)M * N, batch, 1,
                     0);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = sh;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(Cs);
  XS_CHECK_LAUNCH();
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tuned[key] = best;
  return best;
}

}  // namespace

NoTuneScope::NoTuneScope() { ++g_no_tune; }
NoTuneScope::~NoTuneScope() { --g_no_tune; }
bool tuning_disabled() { return g_no_tune > 0; }

template <typename T>
void gemm(cudaStream_t s, bool transA, bool transB, int M, int N, int K, T alpha, const T* A, int lda, long long sA,
          const T* B, int ldb, long long sB, T beta, T* C, int ldc, long long sC, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K < 0) K = 0;
  ProfScope ps(s, sizeof(T) == 8 ? "gemm_f64" : "gemm_f32", 0.0, 2.0 * M * N * (double)K * batch);
  if (sizeof(T) == 4 && M >= 64 && N >= 64 && K >= 32) {
    sgemm_big(s, transA, transB, M, N, K, static_cast<float>(alpha), reinterpret_cast<const float*>(A), lda, sA,
              reinterpret_cast<const float*>(B), ldb, sB, static_cast<float>(beta), reinterpret_cast<float*>(C), ldc,
              sC, batch);
    XS_CHECK_LAUNCH();
    return;
  }
  const int sh = tuned_shape<T>(s, transA, transB, M, N, K, A, lda, sA, B, ldb, sB, batch);
  launch_gemm<T>(s, sh, M, N, K, alpha, A, lda, sA, transA, B, ldb, sB, transB, beta, C, ldc, sC, batch, 1, 0);
  XS_CHECK_LAUNCH();
}

template <typename T>
void gram(cudaStream_t s, int M, int N, int L, const T* A, int lda, const T* B, int ldb, T* C, int ldc, T alpha,
          T beta, DevBuf<T>& ws) {
  if (M <= 0 || N <= 0) return;
  const int sh = pick_shape(M, N);
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
