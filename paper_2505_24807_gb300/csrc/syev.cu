// Lowest eigenpairs of the small symmetric Davidson matrices, float64, one CTA
// (paper, Section "GPU Implementation", batched step 3: diagonalise the
// projected matrix and keep the lowest K states).
//
//   1. Householder tridiagonalisation Q^T A Q = T, the reflectors stored in
//      place below the diagonal (shared memory when S <= kSmemMax, else a
//      global scratch copy);
//   2. the k lowest eigenvalues of T by Sturm-count bisection, one thread each;
//   3. their eigenvectors by inverse iteration on T (pivoted tridiagonal
//      elimination, one thread each), re-orthogonalised inside clusters of
//      close eigenvalues;
//   4. back-transformation z = H_0 H_1 ... H_{S-3} y, one warp per vector.
// About (4/3) S^3 float64 operations instead of the ~10 S^3 per sweep-set of
// two-sided Jacobi -- on a part whose float64 pipe is narrow this decides the
// cost of the subspace step.
//
// Also: Cholesky factorisation a = L L^T of the TDHF matrix a- (positive
// definite unless the reference is unstable).
#include "kernels.h"
#include "prof.h"
#include "syev.h"

namespace xs {

namespace {

constexpr int kSmemMax = 150;

__device__ __forceinline__ double block_sum(double x, double* red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  double s = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// number of eigenvalues of the tridiagonal (d, e) below x
__device__ int sturm_count(int n, const double* d, const double* e, double x, double tiny) {
  int c = 0;
  double q = d[0] - x;
  if (q < 0.0) ++c;
  for (int i = 1; i < n; ++i) {
    if (fabs(q) < tiny) q = (q < 0.0) ? -tiny : tiny;
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    if (q < 0.0) ++c;
  }
  return c;
}

template <bool SMEM>
__global__ void __launch_bounds__(1024) syevk_kernel(int S, int k, const double* __restrict__ Ain, int lda,
                                                     double* __restrict__ wout, double* __restrict__ Z, int ldz,
                                                     double* __restrict__ gscratch, int* info) {
  extern __shared__ double sh[];
  __shared__ double red[32];
  const int ld = S + 1;
  double* a = SMEM ? sh : gscratch;            // S x ld working copy
  double* d = SMEM ? sh + (size_t)S * ld : gscratch + (size_t)S * ld;
  double* e = d + S;
  double* v = e + S;                           // current reflector
  double* p = v + S;                           // A v, then w
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;

  for (int idx = tid; idx < S * S; idx += nt) {
    const int i = idx / S, j = idx % S;
    a[i * ld + j] = Ain[(long long)i * lda + j];
  }
  __syncthreads();

  // 1. tridiagonalisation
  for (int j = 0; j + 2 < S; ++j) {
    const int r0 = j + 1, m = S - r0;
    double part = 0.0;
    for (int i = tid; i < m; i += nt) {
      const double x = a[(r0 + i) * ld + j];
      part += x * x;
    }
    const double sigma = block_sum(part, red);
    const double x0 = a[r0 * ld + j];
    const double nx = sqrt(sigma);
    const double scale_ref = fabs(a[j * ld + j]) + nx;
    double alpha = 0.0;
    bool skip = !(nx > 1e-300) || nx <= 1e-300 * scale_ref;
    if (!skip) {
      alpha = (x0 > 0.0) ? -nx : nx;
      // v = x - alpha e_0, normalised
      const double vn2 = sigma - x0 * x0 + (x0 - alpha) * (x0 - alpha);
      const double inv = 1.0 / sqrt(vn2);
      for (int i = tid; i < m; i += nt) {
        const double x = a[(r0 + i) * ld + j];
        v[i] = ((i == 0) ? (x - alpha) : x) * inv;
      }
    } else {
      alpha = x0;
      for (int i = tid; i < m; i += nt) v[i] = 0.0;
    }
    __syncthreads();
    if (!skip) {
      // p = B v  (B = trailing block, symmetric, full storage)
      for (int i = warp; i < m; i += nwarp) {
        double s = 0.0;
        const double* row = a + (r0 + i) * ld + r0;
        for (int l = lane; l < m; l += 32) s += row[l] * v[l];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) p[i] = s;
      }
      __syncthreads();
      double kp = 0.0;
      for (int i = tid; i < m; i += nt) kp += v[i] * p[i];
      const double K = block_sum(kp, red);
      for (int i = tid; i < m; i += nt) p[i] = 2.0 * p[i] - 2.0 * K * v[i];   // w
      __syncthreads();
      for (int idx = tid; idx < m * m; idx += nt) {
        const int i = idx / m, l = idx % m;
        a[(r0 + i) * ld + r0 + l] -= v[i] * p[l] + p[i] * v[l];
      }
    }
    if (tid == 0) {
      d[j] = a[j * ld + j];
      e[j] = alpha;
    }
    __syncthreads();
    // keep the reflector in column j below the diagonal
    for (int i = tid; i < m; i += nt) a[(r0 + i) * ld + j] = v[i];
    __syncthreads();
  }
  if (tid == 0) {
    if (S >= 2) {
      d[S - 2] = a[(S - 2) * ld + S - 2];
      e[S - 2] = a[(S - 1) * ld + S - 2];
    }
    d[S - 1] = a[(S - 1) * ld + S - 1];
    if (S >= 2) a[(S - 1) * ld + S - 2] = 0.0;   // no reflector for the last two columns
  }
  __syncthreads();

  // 2. k lowest eigenvalues by bisection (Gershgorin bracket)
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < S; ++i) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < S ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
  }
  const double tnorm = fmax(fabs(lo), fabs(hi));
  const double tiny = 1e-300 + 1e-30 * tnorm;
  double* wl = p;  // eigenvalues, reuse p (k <= S)
  for (int t = tid; t < k; t += nt) {
    double a0 = lo - 1e-12 * tnorm - 1e-300, b0 = hi + 1e-12 * tnorm + 1e-300;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (a0 + b0);
      if (mid <= a0 || mid >= b0 || (b0 - a0) <= 2.2e-16 * fmax(fabs(a0), fabs(b0)) + 1e-300) break;
      if (sturm_count(S, d, e, mid, tiny) > t) b0 = mid; else a0 = mid;
    }
    wl[t] = 0.5 * (a0 + b0);
  }
  __syncthreads();

  // 3. inverse iteration for the tridiagonal eigenvectors (thread t -> Z column t)
  for (int t = tid; t < k; t += nt) {
    const double lam = wl[t];
    // pivoted Gaussian elimination of (T - lam I): rows hold (u0, u1, u2) = diag, super, super-super
    // stored transiently in Z's column t region is not possible (needs 3 S), so factor on the fly
    double* y = Z + t;  // stride ldz
    for (int i = 0; i < S; ++i) y[(long long)i * ldz] = 1.0 / sqrt((double)S) * (1.0 + 0.01 * ((i * 7 + t * 3) % 11));
    for (int iter = 0; iter < 3; ++iter) {
      // forward elimination with partial pivoting on a 3-band system, right-hand side y
      // band rows: row i has entries (c0, c1, c2) at columns i, i+1, i+2 after pivoting
      double c0 = d[0] - lam, c1 = (S > 1) ? e[0] : 0.0, c2 = 0.0;
      double rhs = y[0];
      // store the upper factor and multipliers compactly in registers is impossible for all i,
      // so do elimination and keep U rows in the global workspace region of this thread
      double* U = gscratch + (size_t)(SMEM ? 0 : (size_t)S * ld + 4 * S) + (size_t)t * 3 * S;
      double* yv = U + 0;  // reuse: U[3*i .. 3*i+2]
      (void)yv;
      for (int i = 0; i < S - 1; ++i) {
        // next row: (e[i], d[i+1]-lam, e[i+1])
        double n0 = e[i], n1 = d[i + 1] - lam, n2 = (i + 2 < S) ? e[i + 1] : 0.0;
        double nr = y[(long long)(i + 1) * ldz];
        if (fabs(n0) > fabs(c0)) {
          // swap current and next row
          double t0 = c0, t1 = c1, t2 = c2, tr = rhs;
          c0 = n0; c1 = n1; c2 = n2; rhs = nr;
          n0 = t0; n1 = t1; n2 = t2; nr = tr;
        }
        if (fabs(c0) < tiny) c0 = tiny;
        const double f = n0 / c0;
        U[3 * i] = c0;
        U[3 * i + 1] = c1;
        U[3 * i + 2] = c2;
        y[(long long)i * ldz] = rhs;
        // eliminate: next row becomes (n1 - f c1, n2 - f c2, 0) for columns i+1, i+2
        c0 = n1 - f * c1;
        c1 = n2 - f * c2;
        c2 = 0.0;
        rhs = nr - f * rhs;
      }
      if (fabs(c0) < tiny) c0 = tiny;
      U[3 * (S - 1)] = c0;
      U[3 * (S - 1) + 1] = 0.0;
      U[3 * (S - 1) + 2] = 0.0;
      y[(long long)(S - 1) * ldz] = rhs;
      // back substitution
      double nrm = 0.0;
      for (int i = S - 1; i >= 0; --i) {
        double s = y[(long long)i * ldz];
        if (i + 1 < S) s -= U[3 * i + 1] * y[(long long)(i + 1) * ldz];
        if (i + 2 < S) s -= U[3 * i + 2] * y[(long long)(i + 2) * ldz];
        s /= U[3 * i];
        y[(long long)i * ldz] = s;
        nrm += s * s;
      }
      const double inv = 1.0 / sqrt(nrm);
      for (int i = 0; i < S; ++i) y[(long long)i * ldz] *= inv;
    }
  }
  __syncthreads();
  // re-orthogonalise inside clusters of close eigenvalues (modified Gram-Schmidt, one thread)
  if (tid == 0) {
    const double gap = 1e-7 * (tnorm + 1e-300);
    int c0 = 0;
    while (c0 < k) {
      int c1 = c0 + 1;
      while (c1 < k && wl[c1] - wl[c1 - 1] < gap) ++c1;
      for (int t = c0 + 1; t < c1; ++t) {
        for (int u = c0; u < t; ++u) {
          double dot = 0.0;
          for (int i = 0; i < S; ++i) dot += Z[(long long)i * ldz + t] * Z[(long long)i * ldz + u];
          for (int i = 0; i < S; ++i) Z[(long long)i * ldz + t] -= dot * Z[(long long)i * ldz + u];
        }
        double nrm = 0.0;
        for (int i = 0; i < S; ++i) nrm += Z[(long long)i * ldz + t] * Z[(long long)i * ldz + t];
        nrm = 1.0 / sqrt(nrm);
        for (int i = 0; i < S; ++i) Z[(long long)i * ldz + t] *= nrm;
      }
      c0 = c1;
    }
  }
  __syncthreads();
  // 4. back-transformation, one warp per eigenvector
  for (int t = warp; t < k; t += nwarp) {
    for (int j = S - 3; j >= 0; --j) {
      const int r0 = j + 1, m = S - r0;
      double s = 0.0;
      for (int l = lane; l < m; l += 32) s += a[(r0 + l) * ld + j] * Z[(long long)(r0 + l) * ldz + t];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      for (int l = lane; l < m; l += 32) Z[(long long)(r0 + l) * ldz + t] -= 2.0 * s * a[(r0 + l) * ld + j];
      __syncwarp();
    }
  }
  for (int t = tid; t < k; t += nt) wout[t] = wl[t];
  if (tid == 0 && info) *info = 0;
}

// a = L L^T (lower L, in place, lda), flag[0] = 1 when a pivot is not positive
__global__ void __launch_bounds__(1024) cholesky_kernel(int S, double* A, int lda, int* flag) {
  __shared__ double piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < S; ++j) {
    if (tid == 0) {
      double x = A[(long long)j * lda + j];
      if (!(x > 0.0)) { *flag = 1; x = 1e-300; }
      piv = sqrt(x);
      A[(long long)j * lda + j] = piv;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < S; i += nt) A[(long long)i * lda + j] /= piv;
    __syncthreads();
    // trailing update of the lower triangle
    const int m = S - j - 1;
    for (int idx = tid; idx < m * m; idx += nt) {
      const int i = j + 1 + idx / m, l = j + 1 + idx % m;
      if (l <= i) A[(long long)i * lda + l] -= A[(long long)i * lda + j] * A[(long long)l * lda + j];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < S * S; idx += nt) {
    const int i = idx / S, l = idx % S;
    if (l > i) A[(long long)i * lda + l] = 0.0;
  }
}

}  // namespace

void syevk(cudaStream_t s, int S, int k, const double* A, int lda, double* w, double* Z, int ldz,
           DevBuf<double>& scratch, int* info) {
  if (S <= 0 || k <= 0) return;
  if (k > S) k = S;
  const int ld = S + 1;
  // global scratch: inverse-iteration U rows (3 S per vector) and, past kSmemMax, the matrix
  const size_t gm = (size_t)S * ld + 4 * (size_t)S;
  scratch.ensure(gm + (size_t)k * 3 * S + 64);
  ProfScope ps(s, "syevk_f64", 0.0, (4.0 / 3.0) * S * (double)S * S);
  if (S <= kSmemMax) {
    const size_t smem = sizeof(double) * ((size_t)S * ld + 4 * (size_t)S);
    static bool attr = false;
    if (!attr) {
      XS_CUDA(cudaFuncSetAttribute(syevk_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(sizeof(double) * ((size_t)kSmemMax * (kSmemMax + 1) +
                                                                      4 * (size_t)kSmemMax))));
      attr = true;
    }
    syevk_kernel<true><<<1, 1024, smem, s>>>(S, k, A, lda, w, Z, ldz, scratch.get(), info);
  } else {
    syevk_kernel<false><<<1, 1024, 0, s>>>(S, k, A, lda, w, Z, ldz, scratch.get(), info);
  }
  XS_CHECK_LAUNCH();
}

void cholesky(cudaStream_t s, int S, double* A, int lda, int* flag) {
  if (S <= 0) return;
  ProfScope ps(s, "cholesky_f64", 0.0, S * (double)S * S / 3.0);
  cholesky_kernel<<<1, 1024, 0, s>>>(S, A, lda, flag);
  XS_CHECK_LAUNCH();
}

}  // namespace xs
