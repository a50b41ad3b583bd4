// Mixed-precision A*X path of libxs (see tc.h).
#include "kernels.h"
#include "products.h"
#include "tc.h"

namespace xs {

namespace {

template <typename T>
void pbuild_f(cudaStream_t s, int n, int o, int v, int nvec, const T* CT, const T* X, T* R, T* tmp) {
  const T* CTocc = CT;
  const T* CTvir = CT + (size_t)o * n;
  if (v <= o) {
    gemm<T>(s, true, false, n, v, o, T(1), CTocc, n, 0, X, v, (long long)o * v, T(0), tmp, v, (long long)n * v, nvec);
    gemm<T>(s, false, false, nvec * n, n, v, T(1), tmp, v, 0, CTvir, n, 0, T(0), R, n, 0, 1);
  } else {
    gemm<T>(s, false, false, nvec * o, n, v, T(1), X, v, 0, CTvir, n, 0, T(0), tmp, n, 0, 1);
    gemm<T>(s, true, false, n, n, o, T(1), CTocc, n, 0, tmp, n, (long long)o * n, T(0), R, n, (long long)n * n, nvec);
  }
}

template <typename T>
void backtransform_f(cudaStream_t s, int n, int o, int v, int nvec, const T* CT, const T* G, T* Y, T* tmp) {
  const T* CTocc = CT;
  const T* CTvir = CT + (size_t)o * n;
  if (v <= o) {
    gemm<T>(s, false, true, nvec * n, v, n, T(1), G, n, 0, CTvir, n, 0, T(0), tmp, v, 0, 1);
    gemm<T>(s, false, false, o, v, n, T(1), CTocc, n, 0, tmp, v, (long long)n * v, T(0), Y, v, (long long)o * v, nvec);
  } else {
    gemm<T>(s, false, false, o, n, n, T(1), CTocc, n, 0, G, n, (long long)n * n, T(0), tmp, n, (long long)o * n, nvec);
    gemm<T>(s, false, true, nvec * o, v, n, T(1), tmp, n, 0, CTvir, n, 0, T(0), Y, v, 0, 1);
  }
}

}  // namespace

void products_mixed(Ctx& c, DevMol& m, int method, int nvec, const double* X, double* Y1, double* Y2) {
  cudaStream_t s = c.stream;
  const int n = m.n, o = m.o, v = m.v;
  const long long ov = (long long)o * v, nn = (long long)n * n;
  if (!m.Wf.get()) {
    m.Wf.alloc((size_t)m.np * m.np);
    convert_d2f(s, (long long)m.np * m.np, m.W.get(), m.Wf.get());
  }
  if (!m.CTf_hi.get()) {
    m.CTf_hi.alloc(nn);
    m.CTf_lo.alloc(nn);
    split_d2f(s, nn, m.CT.get(), m.CTf_hi.get(), m.CTf_lo.get());
  }
  const int nb = product_batch(m);
  const int chunk = nvec < nb ? nvec : nb;
  c.fs0.ensure((size_t)chunk * nn * 3 + (size_t)chunk * n * (o > v ? o : v) + (size_t)chunk * ov * 2);
  float* R = c.fs0.get();
  float* G = R + (size_t)chunk * nn;
  float* Gm = G + (size_t)chunk * nn;
  float* tmp = Gm + (size_t)chunk * nn;
  float* Xf = tmp + (size_t)chunk * n * (o > v ? o : v);
  float* Yf = Xf + (size_t)chunk * ov;
  for (int k0 = 0; k0 < nvec; k0 += chunk) {
    const int k = (nvec - k0) < chunk ? (nvec - k0) : chunk;
    const double* Xk = X + k0 * ov;
    convert_d2f(s, k * ov, Xk, Xf);
    pbuild_f<float>(s, n, o, v, k, m.CTf_hi.get(), Xf, R, tmp);
    if (method == XS_CIS) {
      gbuild<float>(s, m, c.d_par.get(), G_CIS, k, R, G, nullptr, c.fs1);
      backtransform_f<float>(s, n, o, v, k, m.CTf_hi.get(), G, Yf, tmp);
      convert_f2d(s, k * ov, Yf, Y1 + k0 * ov);
      add_diag_term<double>(s, k, o, v, m.eps.get(), Xk, Y1 + k0 * ov);
    } else {
      gbuild<float>(s, m, c.d_par.get(), G_RPA, k, R, G, Gm, c.fs1);
      backtransform_f<float>(s, n, o, v, k, m.CTf_hi.get(), G, Yf, tmp);
      convert_f2d(s, k * ov, Yf, Y1 + k0 * ov);
      add_diag_term<double>(s, k, o, v, m.eps.get(), Xk, Y1 + k0 * ov);
      backtransform_f<float>(s, n, o, v, k, m.CTf_hi.get(), Gm, Yf, tmp);
      convert_f2d(s, k * ov, Yf, Y2 + k0 * ov);
      add_diag_term<double>(s, k, o, v, m.eps.get(), Xk, Y2 + k0 * ov);
    }
  }
}

}  // namespace xs
