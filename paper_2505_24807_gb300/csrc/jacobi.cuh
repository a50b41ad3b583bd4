// Cyclic two-sided Jacobi eigensolver body of libxs (float64, one CTA):
// the round-robin (tournament) ordering lets the n/2 rotations of one round
// touch disjoint rows and columns and run in parallel.  Included by small.cu
// (one matrix per launch) and batch.cu (one matrix per CTA, one CTA per
// molecule).
#pragma once

#include <cuda_runtime.h>

namespace xs {
namespace {

// reciprocal to ~1e-14 relative (float32 estimate, one float64 Newton step);
// exact division outside the float32 range
__device__ __forceinline__ double rcp_approx(double x) {
  const float ax = fabsf(static_cast<float>(x));
  if (!(ax > 1e-36f && ax < 1e36f)) return 1.0 / x;
  const double r = static_cast<double>(__frcp_rn(static_cast<float>(x)));
  return r * fma(-x, r, 2.0);
}

__device__ __forceinline__ int tour(int i, int r, int m) {
  // player at seat i in round r of an m-player round robin (seat 0 fixed)
  return (i == 0) ? 0 : ((i - 1 + r) % (m - 1)) + 1;
}

// Sweeps of cyclic two-sided Jacobi on A (n x n, row stride lda) accumulating
// the rotations into V (row stride ldv, initialised here to the identity),
// run by the whole CTA; A and V may live in global or shared memory.
// scratch: 2 * (m / 2) doubles + 2 * (m / 2) ints (m = n rounded up to even).
// Returns the number of sweeps taken (max_sweeps when not converged).
__device__ int jacobi_sweeps(int n, double* A, int lda, double* V, int ldv, double* scratch, int max_sweeps) {
  const int m = n + (n & 1);
  const int half = m / 2;
  double* cs = scratch;            // c of each pair
  double* sn = scratch + half;     // s of each pair
  int* pp = reinterpret_cast<int*>(scratch + 2 * half);
  int* qq = pp + half;
  __shared__ double red[2][32];
  __shared__ int done;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int idx = tid; idx < n * n; idx += nt) {
    int i = idx / n, j = idx % n;
    V[(long long)i * ldv + j] = (i == j) ? 1.0 : 0.0;
  }
  if (tid == 0) done = 0;
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // convergence test: off-diagonal vs diagonal mass
    double off = 0.0, dia = 0.0;
    for (int idx = tid; idx < n * n; idx += nt) {
      int i = idx / n, j = idx % n;
      double x = A[(long long)i * lda + j];
      if (i == j) dia += x * x; else off += x * x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if ((tid & 31) == 0) { red[0][tid >> 5] = off; red[1][tid >> 5] = dia; }
    __syncthreads();
    if (tid == 0) {
      double so = 0.0, sd = 0.0;
      for (int k = 0; k < (nt + 31) / 32; ++k) { so += red[0][k]; sd += red[1][k]; }
      done = (so <= 1e-30 * (sd + so) || so == 0.0) ? 1 : 0;
    }
    __syncthreads();
    if (done) break;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = tid; k < half; k += nt) {
        int p = tour(k, r, m), q = tour(m - 1 - k, r, m);
        if (p > q) { int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < n) {
          double apq = A[(long long)p * lda + q];
          double app = A[(long long)p * lda + p], aqq = A[(long long)q * lda + q];
          if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
            // the float64 pipe's divide and square root are slow: approximate
            // reciprocals for the angle (any angle near the exact one keeps
            // the quadratic convergence), c = rsqrt(1 + t^2), s = t c keeps
            // the rotation orthogonal to rounding
            double theta = (aqq - app) * rcp_approx(2.0 * apq);
            double t = (fabs(theta) > 1e150) ? 0.5 * rcp_approx(theta)
                                             : copysign(rcp_approx(fabs(theta) + sqrt(fma(theta, theta, 1.0))), theta);
            c = rsqrt(fma(t, t, 1.0));
            s = t * c;
          }
        }
        pp[k] = p; qq[k] = (q < n) ? q : -1; cs[k] = c; sn[k] = s;
      }
      __syncthreads();
      // rows p, q of A  <-  P^T A
      for (int idx = tid; idx < half * n; idx += nt) {
        int k = idx / n, j = idx % n;
        int q = qq[k];
        if (q < 0 || sn[k] == 0.0) continue;
        int p = pp[k];
        double c = cs[k], s = sn[k];
        double apj = A[(long long)p * lda + j], aqj = A[(long long)q * lda + j];
        A[(long long)p * lda + j] = c * apj - s * aqj;
        A[(long long)q * lda + j] = s * apj + c * aqj;
      }
      __syncthreads();
      // columns p, q of A and V  <-  (.) P
      for (int idx = tid; idx < half * n; idx += nt) {
        int k = idx % half, i = idx / half;
        int q = qq[k];
        if (q < 0 || sn[k] == 0.0) continue;
        int p = pp[k];
        double c = cs[k], s = sn[k];
        double aip = A[(long long)i * lda + p], aiq = A[(long long)i * lda + q];
        A[(long long)i * lda + p] = c * aip - s * aiq;
        A[(long long)i * lda + q] = s * aip + c * aiq;
        double vip = V[(long long)i * ldv + p], viq = V[(long long)i * ldv + q];
        V[(long long)i * ldv + p] = c * vip - s * viq;
        V[(long long)i * ldv + q] = s * vip + c * viq;
      }
      __syncthreads();
    }
  }
  return sweep;
}

}  // namespace
}  // namespace xs
