// Elementwise and reduction kernels of libxs (Davidson steps 4-6 of the
// paper's Section "GPU Implementation": residuals, norms, diagonal
// preconditioner; and the orbital-energy term of Eq. cis_matrix_vector).
#include <algorithm>
#include <cfloat>

#include "kernels.h"

namespace xs {

namespace {

template <typename T>
__global__ void diag_term_kernel(int nvec, int o, int v, const double* __restrict__ eps, const T* __restrict__ X,
                                 T* __restrict__ Y) {
  long long ov = (long long)o * v;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ov * nvec) return;
  long long e = idx % ov;
  int i = static_cast<int>(e / v), a = static_cast<int>(e % v);
  double de = eps[o + a] - eps[i];
  Y[idx] = static_cast<T>(static_cast<double>(Y[idx]) + de * static_cast<double>(X[idx]));
}

// t = r / (omega - d eps - shift), denominator magnitude clamped to >= 1e-4 eV.
// The preconditioned residual is only a search direction (it is
// re-orthogonalised in float64 afterwards), so the denominator and its
// reciprocal are formed in float32: the float64 divide costs ~640 cycles on
// this part.  Orbital energies and the nvec Ritz values are staged as float32
// in shared memory once per CTA; each thread forms its amplitude's gap and
// shift once and serves every vector (a few CTAs per SM, grid-stride).
__global__ void precond_kernel(int n, int o, int v, int nvec, const double* __restrict__ eps,
                               const double* __restrict__ omega, const double* __restrict__ R,
                               double* __restrict__ Tt, const double* __restrict__ shift) {
  extern __shared__ float epsf[];   // n orbital energies, then nvec Ritz values
  float* omf = epsf + n;
  for (int p = threadIdx.x; p < n; p += blockDim.x) epsf[p] = static_cast<float>(eps[p]);
  for (int k = threadIdx.x; k < nvec; k += blockDim.x) omf[k] = static_cast<float>(omega[k]);
  __syncthreads();
  const long long ov = (long long)o * v;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < ov; e += (long long)gridDim.x * blockDim.x) {
    const int i = static_cast<int>(e / v), a = static_cast<int>(e - (long long)i * v);
    const float gap = epsf[o + a] - epsf[i];
    const float sh = shift ? static_cast<float>(shift[e]) : 0.0f;
    // the residuals of 8 vectors loaded before any store (R and Tt may be the
    // same array: each thread reads its own elements before writing them)
    for (int k0 = 0; k0 < nvec; k0 += 8) {
      double rv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) rv[q] = (k0 + q < nvec) ? R[(long long)(k0 + q) * ov + e] : 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + q;
        if (k >= nvec) break;
        float d = omf[k] - gap;
        if (shift) d -= sh;
        if (fabsf(d) < 1e-4f) d = (d < 0.0f) ? -1e-4f : 1e-4f;
        Tt[(long long)k * ov + e] = rv[q] * static_cast<double>(__frcp_rn(d));
      }
    }
  }
}

__device__ __forceinline__ double warp_sum(double x) {
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

// per row k: R = A - omega_k B (if R != nullptr); per-block partial sums of
// |A - omega_k B|^2 into part[k * gridDim.x + block] (summed in a fixed order
// afterwards, so the norms do not depend on scheduling)
__global__ void resid_kernel(long long len, const double* __restrict__ A, const double* __restrict__ B,
                             const double* __restrict__ omega, double* __restrict__ part, double* __restrict__ R) {
  int k = blockIdx.y;
  const double* a = A + (long long)k * len;
  const double* b = B ? B + (long long)k * len : nullptr;
  double w = omega ? omega[k] : 0.0;
  // four independent elements per step (loads in flight, fixed order)
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double* Rk = R ? R + (long long)k * len : nullptr;
  for (; i + 3 * stride < len; i += 4 * stride) {
    double r0 = a[i], r1 = a[i + stride], r2 = a[i + 2 * stride], r3 = a[i + 3 * stride];
    if (b) {
      r0 -= w * b[i];
      r1 -= w * b[i + stride];
      r2 -= w * b[i + 2 * stride];
      r3 -= w * b[i + 3 * stride];
    }
    if (Rk) {
      Rk[i] = r0;
      Rk[i + stride] = r1;
      Rk[i + 2 * stride] = r2;
      Rk[i + 3 * stride] = r3;
    }
    s0 = fma(r0, r0, s0);
    s1 = fma(r1, r1, s1);
    s2 = fma(r2, r2, s2);
    s3 = fma(r3, r3, s3);
  }
  for (; i < len; i += stride) {
    const double r = b ? (a[i] - w * b[i]) : a[i];
    if (Rk) Rk[i] = r;
    s0 = fma(r, r, s0);
  }
  double s = (s0 + s1) + (s2 + s3);
  __shared__ double sh[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[(long long)k * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void sum_sqrt_kernel(int nvec, int nblocks, const double* __restrict__ part, double* out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nvec) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += part[(long long)k * nblocks + b];
  out[k] = sqrt(s);
}

__global__ void sqrt_kernel(int n, double* x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = sqrt(x[i]);
}

// row r of X scaled by scale[r]; with rowmax, abs_hi of the largest |scaled
// x| of the row (one atomic max per warp)
__global__ void scale_rows_kernel(long long len, double* X, const double* __restrict__ scale,
                                  unsigned int* __restrict__ rowmax) {
  const int r = blockIdx.y;
  double* x = X + (long long)r * len;
  const double f = scale[r];
  unsigned int m = 0;
  for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < len; l += (long long)gridDim.x * blockDim.x) {
    const double y = x[l] * f;
    x[l] = y;
    m = max(m, abs_hi(y));
  }
  if (rowmax) {
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&rowmax[r], m);
  }
}

__global__ void d2f_kernel(long long n, const double* __restrict__ a, float* __restrict__ b) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = static_cast<float>(a[i]);
}
__global__ void f2d_kernel(long long n, const float* __restrict__ a, double* __restrict__ b) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = static_cast<double>(a[i]);
}
__global__ void split_kernel(long long n, const double* __restrict__ a, float* __restrict__ hi, float* __restrict__ lo) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float h = static_cast<float>(a[i]);
    hi[i] = h;
    lo[i] = static_cast<float>(a[i] - static_cast<double>(h));
  }
}
__global__ void fill_kernel(long long n, double* a, double v) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}
__global__ void scal_kernel(long long n, double alpha, double* __restrict__ x) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= alpha;
}
__global__ void axpy_kernel(long long n, double alpha, const double* __restrict__ x, double* __restrict__ y) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += alpha * x[i];
}
__global__ void maxabs_kernel(long long n, const double* __restrict__ a, unsigned long long* out) {
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  // non-negative doubles order like their bit patterns
  if ((threadIdx.x & 31) == 0) atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(m)));
}
__global__ void scatter_kernel(int n, const long long* __restrict__ idx, const double* __restrict__ val,
                               double* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[idx[k]] = val[k];
}
__global__ void transpose_kernel(int rows, int cols, const double* __restrict__ a, double* __restrict__ b) {
  __shared__ double tile[32][33];
  int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 32 + threadIdx.y;
  for (int j = 0; j < 32; j += 8)
    if (x < cols && y + j < rows) tile[threadIdx.y + j][threadIdx.x] = a[(long long)(y + j) * cols + x];
  __syncthreads();
  x = blockIdx.y * 32 + threadIdx.x;
  y = blockIdx.x * 32 + threadIdx.y;
  for (int j = 0; j < 32; j += 8)
    if (x < rows && y + j < cols) b[(long long)(y + j) * rows + x] = tile[threadIdx.x][threadIdx.y + j];
}

}  // namespace

template <typename T>
void add_diag_term(cudaStream_t s, int nvec, int o, int v, const double* eps, const T* X, T* Y) {
  long long n = (long long)nvec * o * v;
  if (n == 0) return;
  diag_term_kernel<T><<<grid1(n, 256), 256, 0, s>>>(nvec, o, v, eps, X, Y);
  XS_CHECK_LAUNCH();
}
template void add_diag_term<double>(cudaStream_t, int, int, int, const double*, const double*, double*);
template void add_diag_term<float>(cudaStream_t, int, int, int, const double*, const float*, float*);

void precondition(cudaStream_t s, int nvec, int o, int v, const double* eps, const double* omega, const double* R,
                  double* T, const double* shift) {
  long long n = (long long)nvec * o * v;
  if (n == 0) return;
  const int nao = o + v;
  if (nao + nvec > 12000) throw Error(XS_EINVAL, "precondition: more than 12000 orbitals and vectors");
  static const int nsm = [] {
    int dev = 0, count = 0;
    XS_CUDA(cudaGetDevice(&dev));
    XS_CUDA(cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev));
    return count;
  }();
  const int bx = static_cast<int>(std::min<long long>(4LL * nsm, ((long long)o * v + 255) / 256));
  ProfScope ps(s, "precond", 16.0 * n, 0.0);
  precond_kernel<<<bx, 256, sizeof(float) * (nao + nvec), s>>>(nao, o, v, nvec, eps, omega, R, T, shift);
  XS_CHECK_LAUNCH();
}

void residual_norms(cudaStream_t s, int nvec, long long len, const double* A, const double* B, const double* omega,
                    double* out_norm, double* R) {
  if (nvec == 0) return;
  const int blocks = static_cast<int>(std::min<long long>(256, (len + 255) / 256));
  static thread_local DevBuf<double> part;
  part.ensure((size_t)nvec * blocks);
  ProfScope ps(s, "resid_norms", 8.0 * nvec * len * (B ? 2.0 : 1.0) + (R ? 8.0 * nvec * len : 0.0), 0.0);
  resid_kernel<<<dim3(blocks, nvec), 256, 0, s>>>(len, A, B, omega, part.get(), R);
  XS_CHECK_LAUNCH();
  sum_sqrt_kernel<<<grid1(nvec, 64), 64, 0, s>>>(nvec, blocks, part.get(), out_norm);
  XS_CHECK_LAUNCH();
}

void row_norms(cudaStream_t s, int nvec, long long len, const double* X, double* out_norm) {
  residual_norms(s, nvec, len, X, nullptr, nullptr, out_norm, nullptr);
}

void scale_rows(cudaStream_t s, int nvec, long long len, double* X, const double* scale,
                unsigned int* rowmax) {
  long long n = (long long)nvec * len;
  if (n == 0) return;
  ProfScope ps(s, "scale_rows", 16.0 * n, 0.0);
  if (rowmax) XS_CUDA(cudaMemsetAsync(rowmax, 0, sizeof(unsigned int) * nvec, s));
  // about 8 CTAs per SM over all rows, at least 1024 elements per CTA
  const long long per_row = std::max<long long>(1, std::min<long long>((8LL * 152 + nvec - 1) / nvec, (len + 1023) / 1024));
  scale_rows_kernel<<<dim3(static_cast<unsigned>(per_row), nvec), 256, 0, s>>>(len, X, scale, rowmax);
  XS_CHECK_LAUNCH();
}

void convert_d2f(cudaStream_t s, long long n, const double* a, float* b) {
  if (n == 0) return;
  d2f_kernel<<<grid1(n, 256), 256, 0, s>>>(n, a, b);
  XS_CHECK_LAUNCH();
}
void convert_f2d(cudaStream_t s, long long n, const float* a, double* b) {
  if (n == 0) return;
  f2d_kernel<<<grid1(n, 256), 256, 0, s>>>(n, a, b);
  XS_CHECK_LAUNCH();
}
void split_d2f(cudaStream_t s, long long n, const double* a, float* hi, float* lo) {
  if (n == 0) return;
  split_kernel<<<grid1(n, 256), 256, 0, s>>>(n, a, hi, lo);
  XS_CHECK_LAUNCH();
}
void fill(cudaStream_t s, long long n, double* a, double v) {
  if (n == 0) return;
  fill_kernel<<<grid1(n, 256), 256, 0, s>>>(n, a, v);
  XS_CHECK_LAUNCH();
}
void axpy(cudaStream_t s, long long n, double alpha, const double* x, double* y) {
  if (n == 0) return;
  axpy_kernel<<<grid1(n, 256), 256, 0, s>>>(n, alpha, x, y);
  XS_CHECK_LAUNCH();
}
void scal(cudaStream_t s, long long n, double alpha, double* x) {
  if (n == 0) return;
  scal_kernel<<<grid1(n, 256), 256, 0, s>>>(n, alpha, x);
  XS_CHECK_LAUNCH();
}
void max_abs(cudaStream_t s, long long n, const double* a, double* out) {
  XS_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  if (n == 0) return;
  int blocks = static_cast<int>(std::min<long long>(1024, (n + 255) / 256));
  maxabs_kernel<<<blocks, 256, 0, s>>>(n, a, reinterpret_cast<unsigned long long*>(out));
  XS_CHECK_LAUNCH();
}
void scatter(cudaStream_t s, int n, const long long* idx, const double* val, double* out) {
  if (n == 0) return;
  scatter_kernel<<<grid1(n, 256), 256, 0, s>>>(n, idx, val, out);
  XS_CHECK_LAUNCH();
}
void transpose(cudaStream_t s, int rows, int cols, const double* a, double* b) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(rows, cols, a, b);
  XS_CHECK_LAUNCH();
}

void check_device_error(Ctx& c) {
  if (!c.tc_err.get()) return;
  int h = 0;
  XS_CUDA(cudaMemcpyAsync(&h, c.tc_err.get(), sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  XS_CUDA(cudaStreamSynchronize(c.stream));
  if (h) {
    XS_CUDA(cudaMemsetAsync(c.tc_err.get(), 0, sizeof(int), c.stream));
    throw Error(h >= 10 ? XS_ECUDA : XS_ETIMEOUT,
                h >= 10 ? "non-finite value in a float64 digit split (code " + std::to_string(h) + ")"
                        : "tensor-core kernel: a bounded device wait timed out (code " + std::to_string(h) + ")");
  }
}

}  // namespace xs
