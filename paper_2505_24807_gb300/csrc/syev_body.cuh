// Device bodies of libxs's small float64 eigensolver and Cholesky factor:
// one CTA (up to 1024 threads) per matrix.  Included by syev.cu (one matrix
// per launch) and batch.cu (one matrix per CTA, one CTA per molecule).  The
// algorithm is described at the top of syev.cu.
#pragma once

#include <cfloat>

#include "common.cuh"

namespace xs {
namespace {


constexpr int kSmemMax = 224;   // largest S whose working set fits in shared memory
constexpr int kSeg = 8;         // row segments of the tridiagonalisation's matrix-vector product
constexpr int kMaxRR = 4;       // clusters up to this size get a Rayleigh-Ritz rotation

// packed lower triangle: element (i, j), j <= i
__host__ __device__ __forceinline__ size_t tri(int i, int j) { return (size_t)i * (i + 1) / 2 + j; }

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// block-wide sum (red: 33 doubles); every thread gets the result
__device__ double block_sum(double x, double* red) {
  x = warp_sum(x);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = x;
  __syncthreads();
  if (w == 0) {
    double y = l < nw ? red[l] : 0.0;
    y = warp_sum(y);
    if (l == 0) red[32] = y;
  }
  __syncthreads();
  return red[32];
}

// reciprocal to ~1e-14 relative: a float32 estimate refined by one Newton
// step (inverse iteration needs directions, not correctly rounded quotients)
__device__ __forceinline__ double rcp_fast(double x) {
  const float xf = static_cast<float>(x);
  const float ax = fabsf(xf);
  if (!(ax > 1e-36f && ax < 1e36f)) return 1.0 / x;
  const double r = static_cast<double>(__frcp_rn(xf));
  return r * fma(-x, r, 2.0);
}

// number of eigenvalues of the float32 tridiagonal (d, e^2) below x
__device__ int sturm_count_f(int n, const float* d, const float* e2, float x, float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (q < 0.0f) ++c;
  for (int i = 1; i < n; ++i) {
    if (fabsf(q) < pivmin) q = -pivmin;
    q = d[i] - x - __fdividef(e2[i - 1], q);
    if (q < 0.0f) ++c;
  }
  return c;
}

// y^T T y for the float64 tridiagonal (d, e), y with stride ldy
__device__ double rayleigh(int n, const double* d, const double* e, const double* y, int ldy) {
  double s = 0.0, yp = 0.0;
  for (int i = 0; i < n; ++i) {
    const double yi = y[(long long)i * ldy];
    s = fma(d[i] * yi, yi, s);
    if (i > 0) s = fma(2.0 * e[i - 1] * yp, yi, s);
    yp = yi;
  }
  return s;
}

// Solve (T - shift I) x = y in place (y: stride ldy), factoring the pivoted
// LU into lu (5 n doubles: 1/pivot, the two super-diagonals of U, the
// multiplier, the row-swap flag) when factor is set, else reusing it; then
// normalise y.  Pivots below tiny are raised to tiny.
__device__ void inverse_step(int n, const double* d, const double* e, double shift, double tiny, bool factor,
                             double* lu, double* y, int ldy) {
  double* rc = lu;
  double* u1 = lu + n;
  double* u2 = lu + 2 * n;
  double* fm = lu + 3 * n;
  double* sw = lu + 4 * n;
  double cur = y[0];
  if (factor) {
    double c0 = d[0] - shift, c1 = n > 1 ? e[0] : 0.0, c2 = 0.0;
    for (int i = 0; i + 1 < n; ++i) {
      double n0 = e[i], n1 = d[i + 1] - shift, n2 = (i + 2 < n) ? e[i + 1] : 0.0;
      double nr = y[(long long)(i + 1) * ldy];
      const bool swp = fabs(n0) > fabs(c0);
      if (swp) {
        double t0 = c0, t1 = c1, t2 = c2, tr = cur;
        c0 = n0; c1 = n1; c2 = n2; cur = nr;
        n0 = t0; n1 = t1; n2 = t2; nr = tr;
      }
      if (fabs(c0) < tiny) c0 = c0 < 0.0 ? -tiny : tiny;
      const double r = rcp_fast(c0);
      const double f = n0 * r;
      rc[i] = r; u1[i] = c1; u2[i] = c2; fm[i] = f; sw[i] = swp ? 1.0 : 0.0;
      y[(long long)i * ldy] = cur;
      c0 = fma(-f, c1, n1);
      c1 = fma(-f, c2, n2);
      c2 = 0.0;
      cur = fma(-f, cur, nr);
    }
    if (fabs(c0) < tiny) c0 = c0 < 0.0 ? -tiny : tiny;
    rc[n - 1] = rcp_fast(c0); u1[n - 1] = 0.0; u2[n - 1] = 0.0;
    y[(long long)(n - 1) * ldy] = cur;
  } else {
    for (int i = 0; i + 1 < n; ++i) {
      double nr = y[(long long)(i + 1) * ldy];
      if (sw[i] != 0.0) { const double t = cur; cur = nr; nr = t; }
      y[(long long)i * ldy] = cur;
      cur = fma(-fm[i], cur, nr);
    }
    y[(long long)(n - 1) * ldy] = cur;
  }
  // back substitution, then normalisation
  double y1 = 0.0, y2 = 0.0, nrm = 0.0;
  for (int i = n - 1; i >= 0; --i) {
    const double yi = (y[(long long)i * ldy] - u1[i] * y1 - u2[i] * y2) * rc[i];
    y[(long long)i * ldy] = yi;
    nrm = fma(yi, yi, nrm);
    y2 = y1;
    y1 = yi;
  }
  const double inv = 1.0 / sqrt(nrm);
  for (int i = 0; i < n; ++i) y[(long long)i * ldy] *= inv;
}

// Jacobi eigen-decomposition of a c x c symmetric matrix (c <= kMaxRR), one
// thread: H is overwritten by its eigenvalues on the diagonal, R holds the
// eigenvectors in columns; then sorted ascending.
__device__ void jacobi_small(int c, double (*H)[kMaxRR], double (*R)[kMaxRR]) {
  for (int i = 0; i < c; ++i)
    for (int j = 0; j < c; ++j) R[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 12; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = 0; i < c; ++i)
      for (int j = 0; j < c; ++j) (i == j ? dia : off) += H[i][j] * H[i][j];
    if (off <= 1e-32 * dia || off == 0.0) break;
    for (int p = 0; p < c; ++p)
      for (int q = p + 1; q < c; ++q) {
        if (H[p][q] == 0.0) continue;
        const double th = (H[q][q] - H[p][p]) / (2.0 * H[p][q]);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < c; ++k) {
          const double hp = H[k][p], hq = H[k][q];
          H[k][p] = cs * hp - sn * hq;
          H[k][q] = sn * hp + cs * hq;
        }
        for (int k = 0; k < c; ++k) {
          const double hp = H[p][k], hq = H[q][k];
          H[p][k] = cs * hp - sn * hq;
          H[q][k] = sn * hp + cs * hq;
        }
        for (int k = 0; k < c; ++k) {
          const double rp = R[k][p], rq = R[k][q];
          R[k][p] = cs * rp - sn * rq;
          R[k][q] = sn * rp + cs * rq;
        }
      }
  }
  for (int i = 0; i < c; ++i)
    for (int j = i + 1; j < c; ++j)
      if (H[j][j] < H[i][i]) {
        const double t = H[i][i]; H[i][i] = H[j][j]; H[j][j] = t;
        for (int k = 0; k < c; ++k) { const double r = R[k][i]; R[k][i] = R[k][j]; R[k][j] = r; }
      }
}

// sum over the first nact threads' x (red: 33 doubles); only the warps that
// hold data spend float64 instructions (each costs 64 cycles of its
// sub-partition's float64 pipe, whether or not its lanes are active)
__device__ double active_sum(double x, double* red, int nact) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nw = (nact + 31) >> 5;
  if (w < nw) {
    x = warp_sum(x);
    if (l == 0) red[w] = x;
  }
  __syncthreads();
  if (w == 0) {
    double y = l < nw ? red[l] : 0.0;
    if (nw > 1) y = warp_sum(y);
    if (l == 0) red[32] = y;
  }
  __syncthreads();
  return red[32];
}

template <bool SMEM>
__device__ void syevk_body(int S, int k, const double* __restrict__ Ain, int lda, double* __restrict__ wout,
                           double* __restrict__ Z, int ldz, double* __restrict__ gscratch, int* info) {
  extern __shared__ double sh[];
  __shared__ double red[33];
  __shared__ double scal[8];
  double* base = SMEM ? sh : gscratch;
  double* a = base;                          // packed lower triangle; later Z and LU scratch
  double* d = a + tri(S, 0);
  double* e = d + S;
  double* v = e + S;                         // current reflector
  double* p = v + S;                         // B v, then w
  double* ps = p + S;                        // kSeg x S matrix-vector partials
  double* lam = ps + (size_t)kSeg * S;       // eigenvalues
  float* df = reinterpret_cast<float*>(lam + S);
  float* e2f = df + S;
  int* cl = reinterpret_cast<int*>(e2f + S); // first index of each eigenvalue's cluster
  double* gfree = gscratch + (SMEM ? 0 : (tri(S, 0) + (size_t)(5 + kSeg) * S + 2 * S));
  double* R = gfree;                         // reflectors: row j holds v_j (S - j - 1 entries)
  // eigenvectors and inverse-iteration LU rows: in the freed matrix area of
  // shared memory when they fit, else in global scratch
  const bool zsm = SMEM && 12 * k <= S + 1;   // 6 S k doubles in the S (S + 1) / 2 of the matrix
  double* Zw = zsm ? a : gfree + (size_t)S * S;      // S x k, row stride k
  double* lu = Zw + (size_t)S * k;                    // 5 S per vector
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;

  for (int idx = tid; idx < S * S; idx += nt) {
    const int i = idx / S, j = idx % S;
    if (j <= i) a[tri(i, j)] = Ain[(long long)i * lda + j];
  }
  __syncthreads();

  // 1. tridiagonalisation
  for (int j = 0; j + 2 < S; ++j) {
    const int r0 = j + 1, m = S - r0;
    double part = 0.0;
    if (tid < m) {
      const double x = a[tri(r0 + tid, j)];
      part = x * x;
    }
    // column norm; the final reduction's lane forms the step's scalars (in
    // one thread: float64 instructions in every warp would cost 32 times as
    // much) and broadcasts them through shared memory
    {
      const int nw = (m + 31) >> 5;
      if (warp < nw) {
        part = warp_sum(part);
        if (lane == 0) red[warp] = part;
      }
      __syncthreads();
      if (warp == 0) {
        double y = lane < nw ? red[lane] : 0.0;
        if (nw > 1) y = warp_sum(y);
        if (lane == 0) {
          const double sigma = y;
          const double x0 = a[tri(r0, j)];
          const double nx = sqrt(sigma);
          const double scale_ref = fabs(a[tri(j, j)]) + nx;
          const bool sk = !(nx > 1e-300) || nx <= 1e-300 * scale_ref;
          const double al = sk ? x0 : ((x0 > 0.0) ? -nx : nx);
          scal[0] = al;
          scal[1] = sk ? 0.0 : rsqrt(2.0 * (sigma - x0 * al));
          scal[2] = sk ? 1.0 : 0.0;
        }
      }
      __syncthreads();
    }
    const bool skip = scal[2] != 0.0;
    const double alpha = scal[0];
    double* Rj = R + (size_t)j * S;
    if (!skip) {
      const double inv = scal[1];
      if (tid < m) {
        const double x = a[tri(r0 + tid, j)];
        const double vi = ((tid == 0) ? (x - alpha) : x) * inv;
        v[tid] = vi;
        Rj[tid] = vi;
      }
      __syncthreads();
      // p = B v, B symmetric and held as its lower triangle (B[i][l] read
      // from row max(i, l)), split over nseg row segments summed in order
      const int nseg = min(kSeg, nt / m);
      const int len = (m + nseg - 1) / nseg;
      if (tid < nseg * m) {
        const int i = tid % m, g = tid / m;
        const int l1 = min(m, (g + 1) * len);
        double acc = 0.0;
        for (int l = g * len; l < l1; ++l) {
          const size_t at = (l >= i) ? tri(r0 + l, r0 + i) : tri(r0 + i, r0 + l);
          acc = fma(a[at], v[l], acc);
        }
        ps[g * m + i] = acc;
      }
      __syncthreads();
      double kp = 0.0, pi = 0.0;
      if (tid < m) {
        for (int g = 0; g < nseg; ++g) pi += ps[g * m + tid];
        kp = v[tid] * pi;
      }
      const double K = active_sum(kp, red, m);
      if (tid < m) p[tid] = 2.0 * pi - 2.0 * K * v[tid];   // w
      __syncthreads();
      // rank-2 update of the lower triangle only: B -= v w^T + w v^T
      for (int i = warp; i < m; i += nwarp) {
        const double vi = v[i], wi = p[i];
        double* row = a + tri(r0 + i, r0);
        for (int l = lane; l <= i; l += 32) row[l] = fma(-vi, p[l], fma(-wi, v[l], row[l]));
      }
    } else if (tid < m) {
      v[tid] = 0.0;
      Rj[tid] = 0.0;
    }
    if (tid == 0) {
      d[j] = a[tri(j, j)];
      e[j] = alpha;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (S >= 2) {
      d[S - 2] = a[tri(S - 2, S - 2)];
      e[S - 2] = a[tri(S - 1, S - 2)];
    }
    d[S - 1] = a[tri(S - 1, S - 1)];
  }
  __syncthreads();
  for (int i = tid; i < S; i += nt) {
    df[i] = static_cast<float>(d[i]);
    e2f[i] = (i + 1 < S) ? static_cast<float>(e[i] * e[i]) : 0.0f;
  }
  __syncthreads();

  // 2. float32 multisection: one warp per eigenvalue, 32 Sturm counts per
  //    round, to about 2e-7 of |T| (inverse iteration refines it)
  // Gershgorin bracket and scale, warp 0
  if (warp == 0) {
    double lo = 1e300, hi = -1e300, emax2 = 0.0;
    for (int i = lane; i < S; i += 32) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < S ? fabs(e[i]) : 0.0);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
      if (i + 1 < S) emax2 = fmax(emax2, e[i] * e[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
    }
    if (lane == 0) {
      scal[3] = lo;
      scal[4] = hi;
      scal[5] = fmax(fmax(fabs(lo), fabs(hi)), 1e-300);
      scal[6] = fmax(1e-30 * fmax(emax2, 1.0), 1e-30 * scal[5]);
    }
  }
  __syncthreads();
  const double lo = scal[3], hi = scal[4], tnorm = scal[5];
  const float pivmin = static_cast<float>(scal[6]);
  for (int t = warp; t < k; t += nwarp) {
    const float span = static_cast<float>(hi - lo);
    float a0 = static_cast<float>(lo) - 1e-6f * span - 1e-30f, b0 = static_cast<float>(hi) + 1e-6f * span + 1e-30f;
    const float tolf = 2e-7f * static_cast<float>(tnorm);
    for (int round = 0; round < 16 && (b0 - a0) > tolf; ++round) {
      const float x = a0 + (b0 - a0) * (static_cast<float>(lane + 1) / 33.0f);
      const bool above = sturm_count_f(S, df, e2f, x, pivmin) > t;
      const unsigned mask = __ballot_sync(0xffffffffu, above);
      const int f = mask ? __ffs(mask) - 1 : 32;
      const float xf = __shfl_sync(0xffffffffu, x, f < 32 ? f : 31);
      const float xl = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
      const float na = f > 0 ? xl : a0;
      const float nb = f < 32 ? xf : b0;
      if (!(nb > na) || (na == a0 && nb == b0)) break;
      a0 = na;
      b0 = nb;
    }
    if (lane == 0) lam[t] = 0.5 * (static_cast<double>(a0) + static_cast<double>(b0));
  }
  __syncthreads();
  // clusters: shifts closer than sep are spread apart by sep
  const double sep = 2e-6 * tnorm;
  if (tid == 0) {
    cl[0] = 0;
    for (int t = 1; t < k; ++t) {
      if (lam[t] - lam[t - 1] < sep) {
        lam[t] = lam[t - 1] + sep;
        cl[t] = cl[t - 1];
      } else {
        cl[t] = t;
      }
    }
  }
  __syncthreads();

  // 3. float64 inverse iteration, one thread per cluster (an isolated
  //    eigenvalue is a cluster of one) -> columns of Zw.  Inside a cluster the
  //    members are found in order, each solve followed by Gram-Schmidt against
  //    the members already found: independent iterations of a nearly
  //    degenerate pair converge to nearly the same vector, and orthogonalising
  //    them afterwards would magnify their error outside the cluster by the
  //    inverse of the angle between them.
  const double tiny = 1e-30 * tnorm;
  auto orth_against = [&](double* y, int c0, int u) {   // y -= sum_{c0 <= v < u} (z_v . y) z_v, then normalise
    for (int v = c0; v < u; ++v) {
      const double* z = Zw + v;
      double dot = 0.0;
      for (int i = 0; i < S; ++i) dot = fma(z[(long long)i * k], y[(long long)i * k], dot);
      for (int i = 0; i < S; ++i) y[(long long)i * k] = fma(-dot, z[(long long)i * k], y[(long long)i * k]);
    }
    double nrm = 0.0;
    for (int i = 0; i < S; ++i) nrm = fma(y[(long long)i * k], y[(long long)i * k], nrm);
    const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
    for (int i = 0; i < S; ++i) y[(long long)i * k] *= inv;
  };
  for (int c0 = tid; c0 < k; c0 += nt) {
    if (cl[c0] != c0) continue;   // not the first member of its cluster
    int c1 = c0 + 1;
    while (c1 < k && cl[c1] == c0) ++c1;
    for (int t = c0; t < c1; ++t) {
      double* y = Zw + t;
      double* lut = lu + (size_t)t * 5 * S;
      for (int i = 0; i < S; ++i) y[(long long)i * k] = 1.0 + 0.01 * ((i * 7 + t * 3) % 11);
      inverse_step(S, d, e, lam[t], tiny, true, lut, y, k);
      orth_against(y, c0, t);
      inverse_step(S, d, e, lam[t], tiny, false, lut, y, k);
      orth_against(y, c0, t);
      // one more solve shifted by the Rayleigh quotient: the spread shift of
      // a cluster member sits up to (members) x sep from the cluster, which
      // leaves neighbouring eigenvectors in y at (sep / gap)^2; shifted by the
      // Rayleigh quotient they fall by a further (spread inside / gap)
      const double rq = rayleigh(S, d, e, y, k);
      inverse_step(S, d, e, rq, tiny, true, lut, y, k);
      if (c1 - c0 > 1) orth_against(y, c0, t);
    }
    for (int t = c0; t < c1; ++t) lam[t] = rayleigh(S, d, e, Zw + t, k);
  }
  __syncthreads();
  // clusters: Gram-Schmidt inside each, then (up to kMaxRR members) a
  // Rayleigh-Ritz rotation; warp 0, lanes over rows
  if (warp == 0) {
    int c0 = 0;
    while (c0 < k) {
      int c1 = c0 + 1;
      while (c1 < k && cl[c1] == c0) ++c1;
      if (c1 - c0 > 1) {
        for (int t = c0; t < c1; ++t) {
          for (int u = c0; u < t; ++u) {
            double dot = 0.0;
            for (int i = lane; i < S; i += 32) dot = fma(Zw[i * k + t], Zw[i * k + u], dot);
            dot = warp_sum(dot);
            for (int i = lane; i < S; i += 32) Zw[i * k + t] -= dot * Zw[i * k + u];
          }
          double nn = 0.0;
          for (int i = lane; i < S; i += 32) nn = fma(Zw[i * k + t], Zw[i * k + t], nn);
          nn = warp_sum(nn);
          const double inv = 1.0 / sqrt(nn);
          for (int i = lane; i < S; i += 32) Zw[i * k + t] *= inv;
          __syncwarp();
        }
        const int c = c1 - c0;
        if (c <= kMaxRR) {
          // H = Yc^T T Yc, (T y)_i = e_{i-1} y_{i-1} + d_i y_i + e_i y_{i+1}
          double H[kMaxRR][kMaxRR], Rr[kMaxRR][kMaxRR];
          for (int aa = 0; aa < c; ++aa)
            for (int bb = aa; bb < c; ++bb) {
              double h = 0.0;
              for (int i = lane; i < S; i += 32) {
                const double* yb = Zw + c0 + bb;
                double ty = d[i] * yb[i * k];
                if (i > 0) ty = fma(e[i - 1], yb[(i - 1) * k], ty);
                if (i + 1 < S) ty = fma(e[i], yb[(i + 1) * k], ty);
                h = fma(Zw[i * k + c0 + aa], ty, h);
              }
              h = warp_sum(h);
              H[aa][bb] = h;
              H[bb][aa] = h;
            }
          jacobi_small(c, H, Rr);   // every lane, same result
          __syncwarp();
          for (int i = lane; i < S; i += 32) {
            double yrow[kMaxRR];
            for (int aa = 0; aa < c; ++aa) yrow[aa] = Zw[i * k + c0 + aa];
            for (int bb = 0; bb < c; ++bb) {
              double z = 0.0;
              for (int aa = 0; aa < c; ++aa) z = fma(yrow[aa], Rr[aa][bb], z);
              Zw[i * k + c0 + bb] = z;
            }
          }
          if (lane == 0)
            for (int aa = 0; aa < c; ++aa) lam[c0 + aa] = H[aa][aa];
        } else {
          __syncwarp();
          for (int t = c0; t < c1; ++t) {
            const double r = rayleigh(S, d, e, Zw + t, k);   // identical in every lane
            if (lane == 0) lam[t] = r;
          }
        }
        __syncwarp();
      }
      c0 = c1;
    }
  }
  __syncthreads();
  // 4. back-transformation z = H_0 ... H_{S-3} y, one warp per eigenvector,
  //    then the result into Z
  for (int t = warp; t < k; t += nwarp) {
    for (int j = S - 3; j >= 0; --j) {
      const int r0 = j + 1, m = S - r0;
      const double* Rj = R + (size_t)j * S;
      double sacc = 0.0;
      for (int l = lane; l < m; l += 32) sacc = fma(Rj[l], Zw[(r0 + l) * k + t], sacc);
      sacc = warp_sum(sacc);
      for (int l = lane; l < m; l += 32) Zw[(r0 + l) * k + t] -= 2.0 * sacc * Rj[l];
      __syncwarp();
    }
    for (int i = lane; i < S; i += 32) Z[(long long)i * ldz + t] = Zw[i * k + t];
  }
  for (int t = tid; t < k; t += nt) wout[t] = lam[t];
  if (tid == 0 && info) *info = 0;
}

// a = L L^T (lower L, in place, lda), flag[0] = 1 when a pivot is not positive
// Right-looking Cholesky on the lower triangle, one CTA: the triangle staged
// packed in shared memory when it fits, the column scaled by one reciprocal
// per step, the trailing update one warp per row.
constexpr int kCholSmemMax = 224;

template <bool SMEM>
__device__ void cholesky_body(int S, double* A, int lda, int* flag) {
  extern __shared__ double sh[];
  __shared__ double inv;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  // element (i, l), l <= i: packed in shared memory, else in place in A
  auto at = [&](int i, int l) -> double& { return SMEM ? sh[tri(i, l)] : A[(long long)i * lda + l]; };
  if (SMEM) {
    for (int idx = tid; idx < S * S; idx += nt) {
      const int i = idx / S, l = idx % S;
      if (l <= i) sh[tri(i, l)] = A[(long long)i * lda + l];
    }
    __syncthreads();
  }
  for (int j = 0; j < S; ++j) {
    if (tid == 0) {
      double x = at(j, j);
      if (!(x > 0.0)) { *flag = 1; x = 1e-300; }
      const double piv = sqrt(x);
      at(j, j) = piv;
      inv = 1.0 / piv;
    }
    __syncthreads();
    const double r = inv;
    for (int i = j + 1 + tid; i < S; i += nt) at(i, j) *= r;
    __syncthreads();
    // trailing update of the lower triangle
    for (int i = j + 1 + warp; i < S; i += nwarp) {
      const double lij = at(i, j);
      for (int l = j + 1 + lane; l <= i; l += 32) at(i, l) = fma(-lij, at(l, j), at(i, l));
    }
    __syncthreads();
  }
  for (int idx = tid; idx < S * S; idx += nt) {
    const int i = idx / S, l = idx % S;
    if (l > i) A[(long long)i * lda + l] = 0.0;
    else if (SMEM) A[(long long)i * lda + l] = sh[tri(i, l)];
  }
}


// working set of syevk_body in doubles (matrix, tridiagonal, reflector,
// products, eigenvalues, float32 copy, cluster indices); shared memory when
// S <= kSmemMax
__host__ __device__ constexpr size_t syevk_work_doubles(int n) {
  return (size_t)n * (n + 1) / 2 + (size_t)(5 + kSeg) * n + 2 * (size_t)n;
}
// global scratch of syevk_body: the working set past kSmemMax, the
// reflectors (S x S), then eigenvectors and inverse-iteration LU rows (6 S per
// vector) when they do not fit in the freed shared-memory matrix area
__host__ __device__ constexpr size_t syevk_scratch_doubles(int S, int k) {
  return (S <= kSmemMax ? 0 : syevk_work_doubles(S)) + (size_t)S * S + (size_t)k * 6 * S + 64;
}

}  // namespace
}  // namespace xs
