// The Davidson matrix-vector product of libxs (paper, Section "GPU
// Implementation", Eqs. cis_matrix_vector and ftilde):
//   (1) R_k = C_occ X_k C_vir^T                    (transition densities)
//   (2) G_k = G(R_k) over the atom-pair blocks      (gbuild.cu)
//   (3) Y_k = C_occ^T G_k C_vir + (eps_a - eps_i) X_k
// For TDHF one G build gives G+ and G- and two back-transforms give (A+B)X and
// (A-B)X.  The two transforms contract the smaller of nocc and nvir against
// n^2 last.  Batches of vectors share each GEMM (the vectors are stacked into
// one tall operand where the shared factor is on the right).
#include "kernels.h"
#include "products.h"
#include "tc.h"

namespace xs {

namespace {

// R (nvec x n x n) from X (nvec x o x v); CT is the MO-major coefficient matrix.
template <typename T>
void pbuild(cudaStream_t s, int n, int o, int v, int nvec, const T* CT, const T* X, T* R, T* tmp) {
  const T* CTocc = CT;
  const T* CTvir = CT + (size_t)o * n;
  if (v <= o) {
    // T_k = C_occ X_k (n x v), then R = [T_1; ..; T_k] C_vir^T
    gemm<T>(s, true, false, n, v, o, T(1), CTocc, n, 0, X, v, (long long)o * v, T(0), tmp, v, (long long)n * v, nvec);
    gemm<T>(s, false, false, nvec * n, n, v, T(1), tmp, v, 0, CTvir, n, 0, T(0), R, n, 0, 1);
  } else {
    // U = [X_1; ..; X_k] C_vir^T (o x n each), then R_k = C_occ U_k
    gemm<T>(s, false, false, nvec * o, n, v, T(1), X, v, 0, CTvir, n, 0, T(0), tmp, n, 0, 1);
    gemm<T>(s, true, false, n, n, o, T(1), CTocc, n, 0, tmp, n, (long long)o * n, T(0), R, n, (long long)n * n, nvec);
  }
}

// Y (nvec x o x v) = C_occ^T G_k C_vir
template <typename T>
void backtransform(cudaStream_t s, int n, int o, int v, int nvec, const T* CT, const T* G, T* Y, T* tmp) {
  const T* CTocc = CT;
  const T* CTvir = CT + (size_t)o * n;
  if (v <= o) {
    // S = [G_1; ..; G_k] C_vir (n x v each), Y_k = C_occ^T S_k
    gemm<T>(s, false, true, nvec * n, v, n, T(1), G, n, 0, CTvir, n, 0, T(0), tmp, v, 0, 1);
    gemm<T>(s, false, false, o, v, n, T(1), CTocc, n, 0, tmp, v, (long long)n * v, T(0), Y, v, (long long)o * v, nvec);
  } else {
    // Q_k = C_occ^T G_k (o x n), Y = [Q_1; ..; Q_k] C_vir
    gemm<T>(s, false, false, o, n, n, T(1), CTocc, n, 0, G, n, (long long)n * n, T(0), tmp, n, (long long)o * n, nvec);
    gemm<T>(s, false, true, nvec * o, v, n, T(1), tmp, n, 0, CTvir, n, 0, T(0), Y, v, 0, 1);
  }
}

}  // namespace

int product_batch(const DevMol& m) {
  // vectors per pass: bound the AO work arrays (R, G+, G-, tmp) to ~4 GB
  const double per = 8.0 * ((double)m.n * m.n * 3 + (double)m.n * (m.o > m.v ? m.o : m.v));
  int nb = static_cast<int>(4.0e9 / per);
  if (nb < 1) nb = 1;
  if (nb > 64) nb = 64;
  return nb;
}

void products_fp64(Ctx& c, const DevMol& m, int method, int nvec, const double* X, double* Y1, double* Y2,
                   bool triplet) {
  cudaStream_t s = c.stream;
  const int n = m.n, o = m.o, v = m.v;
  const long long ov = (long long)o * v, nn = (long long)n * n;
  const int nb = product_batch(m);
  const int chunk = nvec < nb ? nvec : nb;
  c.ws1.ensure((size_t)chunk * nn);                         // R
  c.ws2.ensure((size_t)chunk * nn);                         // G or G+
  c.ws3.ensure((size_t)chunk * nn);                         // G-
  c.ws4.ensure((size_t)chunk * n * (o > v ? o : v));        // transform scratch
  for (int k0 = 0; k0 < nvec; k0 += chunk) {
    const int k = (nvec - k0) < chunk ? (nvec - k0) : chunk;
    const double* Xk = X + k0 * ov;
    pbuild<double>(s, n, o, v, k, m.CT.get(), Xk, c.ws1.get(), c.ws4.get());
    if (method == XS_CIS) {
      gbuild<double>(s, m, c.d_par.get(), gmode(false, triplet), k, c.ws1.get(), c.ws2.get(), nullptr, c.ws0);
      backtransform<double>(s, n, o, v, k, m.CT.get(), c.ws2.get(), Y1 + k0 * ov, c.ws4.get());
      add_diag_term<double>(s, k, o, v, m.eps.get(), Xk, Y1 + k0 * ov);
    } else {
      gbuild<double>(s, m, c.d_par.get(), gmode(true, triplet), k, c.ws1.get(), c.ws2.get(), c.ws3.get(), c.ws0);
      backtransform<double>(s, n, o, v, k, m.CT.get(), c.ws2.get(), Y1 + k0 * ov, c.ws4.get());
      add_diag_term<double>(s, k, o, v, m.eps.get(), Xk, Y1 + k0 * ov);
      backtransform<double>(s, n, o, v, k, m.CT.get(), c.ws3.get(), Y2 + k0 * ov, c.ws4.get());
      add_diag_term<double>(s, k, o, v, m.eps.get(), Xk, Y2 + k0 * ov);
    }
  }
}

// float32 SIMT products: float32 coefficients, R, G and integrals, float32
// accumulation with round-to-nearest (no tensor cores); the accurate
// reference for the final Rayleigh-Ritz step of a mixed-precision solve.
void products_f32(Ctx& c, DevMol& m, int method, int nvec, const double* X, double* Y1, double* Y2, bool triplet) {
  cudaStream_t s = c.stream;
  const int n = m.n, o = m.o, v = m.v;
  const long long ov = (long long)o * v, nn = (long long)n * n;
  if (!m.Wf.get()) {
    m.Wf.alloc((size_t)m.np * m.np);
    convert_d2f(s, (long long)m.np * m.np, m.W.get(), m.Wf.get());
  }
  if (!m.CTf.get()) {
    m.CTf.alloc(nn);
    convert_d2f(s, nn, m.CT.get(), m.CTf.get());
  }
  const int nb = product_batch(m);
  const int chunk = nvec < nb ? nvec : nb;
  const size_t tmpn = (size_t)chunk * n * (o > v ? o : v);
  c.fs2.ensure((size_t)chunk * nn * 3 + tmpn + (size_t)chunk * ov * 2);
  float* R = c.fs2.get();
  float* G = R + (size_t)chunk * nn;
  float* Gm = G + (size_t)chunk * nn;
  float* tmp = Gm + (size_t)chunk * nn;
  float* Xf = tmp + tmpn;
  float* Yf = Xf + (size_t)chunk * ov;
  for (int k0 = 0; k0 < nvec; k0 += chunk) {
    const int k = (nvec - k0) < chunk ? (nvec - k0) : chunk;
    const double* Xk = X + k0 * ov;
    convert_d2f(s, k * ov, Xk, Xf);
    pbuild<float>(s, n, o, v, k, m.CTf.get(), Xf, R, tmp);
    const bool rpa = method != XS_CIS;
    gbuild<float>(s, m, c.d_par.get(), gmode(rpa, triplet), k, R, G, rpa ? Gm : nullptr, c.fs1);
    for (int pass = 0; pass < (rpa ? 2 : 1); ++pass) {
      double* Y = (pass == 0 ? Y1 : Y2) + k0 * ov;
      backtransform<float>(s, n, o, v, k, m.CTf.get(), pass == 0 ? G : Gm, Yf, tmp);
      convert_f2d(s, k * ov, Yf, Y);
      add_diag_term<double>(s, k, o, v, m.eps.get(), Xk, Y);
    }
  }
}

void products(Ctx& c, DevMol& m, int method, int precision, int nvec, const double* X, double* Y1, double* Y2,
              bool triplet, unsigned int* mx1, unsigned int* mx2) {
  if (nvec <= 0) return;
  if (precision == XS_MIXED) {
    products_mixed(c, m, method, nvec, X, Y1, Y2, triplet, mx1, mx2);
    return;
  }
  if (precision == kPrecF32) {
    products_f32(c, m, method, nvec, X, Y1, Y2, triplet);
    return;
  }
  products_fp64(c, m, method, nvec, X, Y1, Y2, triplet);
}

void gmatrix(Ctx& c, const DevMol& m, int precision, int nvec, const double* R, double* G) {
  (void)precision;
  gbuild<double>(c.stream, m, c.d_par.get(), G_CIS, nvec, R, G, nullptr, c.ws0);
}

}  // namespace xs
