// Small dense float64 kernels of libxs's Davidson subspace step (paper,
// Section "GPU Implementation", batched steps 3-6: diagonalise the projected
// matrix, orthonormalise the new directions).
//
// jacobi_eig: cyclic two-sided Jacobi with the round-robin (tournament)
// ordering, so the n/2 rotations of one round touch disjoint rows and columns
// and run in parallel within one CTA; float64 throughout.
#include <cfloat>

#include "kernels.h"
#include "small.h"
#include "prof.h"
#include "jacobi.cuh"

namespace xs {

namespace {

__global__ void __launch_bounds__(1024) jacobi_kernel(int n, double* A, int lda, double* V, int ldv, double* w,
                                                      int* info, int max_sweeps) {
  extern __shared__ double sh[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int sweep = jacobi_sweeps(n, A, lda, V, ldv, sh, max_sweeps);
  // eigenvalues ascending (rank by value, ties by index); V columns permuted
  // through A as scratch
  double* wv = sh;                                   // reuse: n values
  int* rk = reinterpret_cast<int*>(sh + n);          // n ranks
  __syncthreads();
  for (int j = tid; j < n; j += nt) wv[j] = A[(long long)j * lda + j];
  __syncthreads();
  for (int j = tid; j < n; j += nt) {
    int r = 0;
    for (int i = 0; i < n; ++i) r += (wv[i] < wv[j]) || (wv[i] == wv[j] && i < j);
    rk[j] = r;
  }
  __syncthreads();
  for (int j = tid; j < n; j += nt) w[rk[j]] = wv[j];
  for (int idx = tid; idx < n * n; idx += nt) {
    int i = idx / n, j = idx % n;
    A[(long long)i * lda + j] = V[(long long)i * ldv + j];
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nt) {
    int i = idx / n, j = idx % n;
    V[(long long)i * ldv + rk[j]] = A[(long long)i * lda + j];
  }
  if (tid == 0 && info) *info = (sweep >= max_sweeps) ? 1 : 0;
}

// Small matrices (n <= kJacobiSmemMax): A and V staged in shared memory (odd
// row stride n + 1 against bank conflicts), a 256-thread CTA; the same
// rotations in the same order as the global-memory form.  The input A is left
// unchanged.
constexpr int kJacobiSmemMax = 64;

__global__ void __launch_bounds__(256) jacobi_smem_kernel(int n, const double* __restrict__ A, int lda,
                                                          double* __restrict__ V, int ldv, double* __restrict__ w,
                                                          int* info, int max_sweeps) {
  extern __shared__ double sh[];
  const int ld = n + 1;
  const int m = n + (n & 1);
  double* As = sh;
  double* Vs = As + (size_t)n * ld;
  double* scratch = Vs + (size_t)n * ld;   // 2 (m / 2) doubles + 2 (m / 2) ints
  int* rk = reinterpret_cast<int*>(scratch + 2 * m);
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    As[i * ld + j] = A[(long long)i * lda + j];
  }
  __syncthreads();
  const int sweep = jacobi_sweeps(n, As, ld, Vs, ld, scratch, max_sweeps);
  __syncthreads();
  // eigenvalues ascending (rank by value, ties by index), V columns permuted
  for (int j = tid; j < n; j += nt) {
    const double x = As[j * ld + j];
    int r = 0;
    for (int i = 0; i < n; ++i) {
      const double y = As[i * ld + i];
      r += (y < x) || (y == x && i < j);
    }
    rk[j] = r;
    w[r] = x;
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nt) {
    const int i = idx / n, j = idx % n;
    V[(long long)i * ldv + rk[j]] = Vs[i * ld + j];
  }
  if (tid == 0 && info) *info = (sweep >= max_sweeps) ? 1 : 0;
}

// E[i][j] = a[min(i,j)][max(i,j)]: full symmetric copy from the valid upper part
__global__ void sym_upper_kernel(int S, const double* __restrict__ a, int lda, double* __restrict__ E, int lde) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * S) return;
  int i = idx / S, j = idx % S;
  int lo = i < j ? i : j, hi = i < j ? j : i;
  E[(long long)i * lde + j] = a[(long long)lo * lda + hi];
}

// A[:, j] *= f(d[j]) with f = d^power (power in {0.5, -0.5, -1}) for j < ncols
__global__ void scale_cols_kernel(int rows, int ncols, double* A, int lda, const double* __restrict__ d, int mode) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * ncols) return;
  int i = idx / ncols, j = idx % ncols;
  double x = d[j];
  double f = (mode == 0) ? sqrt(x) : (mode == 1) ? 1.0 / sqrt(x) : 1.0 / x;
  A[(long long)i * lda + j] *= f;
}

// Loewdin canonical orthonormalisation coefficients: eigenpairs (lam, Q) of a
// Gram matrix (ascending); keep lam > thresh * max(lam, 1) and write
// B[k][:] = Q[:, j]^T / sqrt(lam_j) for the kept j (largest first).
__global__ void lowdin_kernel(int n, const double* __restrict__ lam, const double* __restrict__ Q, int ldq,
                              double thresh, double* __restrict__ Bm, int ldb, int* nkeep) {
  __shared__ int first;
  if (threadIdx.x == 0) {
    double lmax = lam[n - 1] > 1.0 ? lam[n - 1] : 1.0;
    int f = n;
    for (int j = n - 1; j >= 0; --j) {
      if (lam[j] > thresh * lmax) f = j; else break;
    }
    first = f;
    *nkeep = n - f;
  }
  __syncthreads();
  int keep = n - first;
  for (int idx = threadIdx.x; idx < keep * n; idx += blockDim.x) {
    int k = idx / n, i = idx % n;
    int j = n - 1 - k;
    Bm[(long long)k * ldb + i] = Q[(long long)i * ldq + j] / sqrt(lam[j]);
  }
}

// omega[j] = sqrt(w2[j]) for j < k; flag[0] = 1 if any w2 <= 0
__global__ void sqrt_roots_kernel(int k, const double* __restrict__ w2, double* __restrict__ omega, int* flag) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double x = w2[j];
  if (!(x > 0.0)) { atomicExch(flag, 1); x = 0.0; }
  omega[j] = sqrt(x);
}

// V[j][idx[j]] = 1 for the guess unit vectors (V zeroed beforehand)
__global__ void unit_vectors_kernel(int k, long long ld, const long long* __restrict__ idx, double* V) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) V[(long long)j * ld + idx[j]] = 1.0;
}

// diag(vals) into an S x S matrix with leading dimension lda
__global__ void set_diag_kernel(int S, const double* __restrict__ vals, double* a, int lda) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= S * S) return;
  int i = idx / S, j = idx % S;
  a[(long long)i * lda + j] = (i == j) ? vals[i] : 0.0;
}

}  // namespace
}  // namespace xs

namespace xs {

void jacobi_eig(cudaStream_t s, int n, double* A, int lda, double* V, int ldv, double* w, int* info) {
  if (n <= 0) return;
  if (n > 1024) throw Error(XS_EINVAL, "jacobi_eig: matrix larger than 1024");
  int m = n + (n & 1);
  ProfScope ps(s, "jacobi_f64", 0.0, 0.0);
  if (n <= kJacobiSmemMax) {
    // A, V (n x (n + 1)), scratch 2m doubles (c, s, and the pair indices), n ranks
    const size_t smem = sizeof(double) * (2 * (size_t)n * (n + 1) + 2 * m) + sizeof(int) * n;
    static const bool attr = [] {   // once per process (thread-safe initialisation)
      const size_t most = sizeof(double) * (2 * (size_t)kJacobiSmemMax * (kJacobiSmemMax + 1) + 2 * kJacobiSmemMax) +
                          sizeof(int) * kJacobiSmemMax;
      XS_CUDA(cudaFuncSetAttribute(jacobi_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(most)));
      return true;
    }();
    (void)attr;
    jacobi_smem_kernel<<<1, 256, smem, s>>>(n, A, lda, V, ldv, w, info, 60);
    XS_CHECK_LAUNCH();
    return;
  }
  size_t smem = sizeof(double) * (2 * (m / 2)) + sizeof(int) * 2 * (m / 2);
  size_t smem2 = sizeof(double) * n + sizeof(int) * n;
  if (smem2 > smem) smem = smem2;
  jacobi_kernel<<<1, 1024, smem, s>>>(n, A, lda, V, ldv, w, info, 60);
  XS_CHECK_LAUNCH();
}

void sym_upper(cudaStream_t s, int S, const double* a, int lda, double* E, int lde) {
  if (S <= 0) return;
  sym_upper_kernel<<<grid1((long long)S * S, 256), 256, 0, s>>>(S, a, lda, E, lde);
  XS_CHECK_LAUNCH();
}
void scale_cols(cudaStream_t s, int rows, int ncols, double* A, int lda, const double* d, int mode) {
  if (rows <= 0 || ncols <= 0) return;
  scale_cols_kernel<<<grid1((long long)rows * ncols, 256), 256, 0, s>>>(rows, ncols, A, lda, d, mode);
  XS_CHECK_LAUNCH();
}
void lowdin(cudaStream_t s, int n, const double* lam, const double* Q, int ldq, double thresh, double* Bm, int ldb,
            int* nkeep) {
  lowdin_kernel<<<1, 256, 0, s>>>(n, lam, Q, ldq, thresh, Bm, ldb, nkeep);
  XS_CHECK_LAUNCH();
}
void sqrt_roots(cudaStream_t s, int k, const double* w2, double* omega, int* flag) {
  sqrt_roots_kernel<<<grid1(k, 64), 64, 0, s>>>(k, w2, omega, flag);
  XS_CHECK_LAUNCH();
}
void unit_vectors(cudaStream_t s, int k, long long ld, const long long* idx, double* V) {
  unit_vectors_kernel<<<grid1(k, 64), 64, 0, s>>>(k, ld, idx, V);
  XS_CHECK_LAUNCH();
}
void set_diag(cudaStream_t s, int S, const double* vals, double* a, int lda) {
  set_diag_kernel<<<grid1((long long)S * S, 256), 256, 0, s>>>(S, vals, a, lda);
  XS_CHECK_LAUNCH();
}

}  // namespace xs
