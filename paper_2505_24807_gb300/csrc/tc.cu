// Mixed-precision A*X path of libxs (see tc.h).
//
// Per batch of k trial vectors (all tensor-core operands K-major TF32 pairs):
//   1. X_k (o x v)                    -> TF32 pair, v padded to 32
//   2. U_k^T (n x o) = C_vir X_k^T    (tc_gemm, epilogue writes a TF32 pair)
//   3. R_k (n x n)   = C_occ U_k      (tc_gemm, float32 out)
//   4. G_k = G(R_k)                   (float32 G build, epilogue writes the TF32 pair, n padded)
//   5. S_k^T (v x n) = C_vir^T G_k^T  (tc_gemm, TF32 pair out)
//   6. Y_k (o x v)   = C_occ^T S_k + (eps_a - eps_i) X_k   (tc_gemm, float64 out)
// For TDHF steps 5-6 run for G+ and G-.  When v < o, steps 1-3 contract the
// n x n product over v instead (2 n^2 v rather than 2 n^2 o flops):
//   1'. X_k^T (v x o) -> TF32 pair; 2'. W_k (n x v) = C_occ X_k;
//   3'. R_k = W_k C_vir^T.
// Steps 5-6 contract the n x n product over v (S^T is v x n).
#include "kernels.h"
#include "products.h"
#include "tc.h"
#include "tc_gemm.h"

namespace xs {

void products_mixed(Ctx& c, DevMol& m, int method, int nvec, const double* X, double* Y1, double* Y2, bool triplet,
                    unsigned int* mx1, unsigned int* mx2) {
  cudaStream_t s = c.stream;
  const int n = m.n, o = m.o, v = m.v;
  const int np_ = pad32(n), op = pad32(o), vp = pad32(v);
  const long long ov = (long long)o * v, nn = (long long)n * n;
  if (!m.Wf.get()) {
    m.Wf.alloc((size_t)m.np * m.np);
    convert_d2f(s, (long long)m.np * m.np, m.W.get(), m.Wf.get());
  }
  // orbital operands, cached until the orbitals change:
  //   Cvir (n x vp) = C[mu][o + a], Cocc (n x op) = C[mu][i],
  //   CTvir (v x np) = CT[o + a][mu], CTocc (o x np) = CT[i][mu]
  const size_t orb = (size_t)n * vp + (size_t)n * op + (size_t)v * np_ + (size_t)o * np_;
  if (!m.CTf_hi.get()) {
    m.CTf_hi.alloc(orb);
    m.CTf_lo.alloc(orb);
    float* h = m.CTf_hi.get();
    float* l = m.CTf_lo.get();
    const double* CT = m.CT.get();
    split_pad<double>(s, n, v, vp, CT + (size_t)o * n, n, 0, 0, 1, true, h, l);
    h += (size_t)n * vp; l += (size_t)n * vp;
    split_pad<double>(s, n, o, op, CT, n, 0, 0, 1, true, h, l);
    h += (size_t)n * op; l += (size_t)n * op;
    split_pad<double>(s, v, n, np_, CT + (size_t)o * n, n, 0, 0, 1, false, h, l);
    h += (size_t)v * np_; l += (size_t)v * np_;
    split_pad<double>(s, o, n, np_, CT, n, 0, 0, 1, false, h, l);
  }
  const float* Cvir_h = m.CTf_hi.get();
  const float* Cvir_l = m.CTf_lo.get();
  const float* Cocc_h = Cvir_h + (size_t)n * vp;
  const float* Cocc_l = Cvir_l + (size_t)n * vp;
  const float* CTvir_h = Cocc_h + (size_t)n * op;
  const float* CTvir_l = Cocc_l + (size_t)n * op;
  const float* CTocc_h = CTvir_h + (size_t)v * np_;
  const float* CTocc_l = CTvir_l + (size_t)v * np_;

  const int nb = product_batch(m);
  const int chunk = nvec < nb ? nvec : nb;
  // P build order: the n^2 contraction runs over the smaller of o and v
  //   o <= v: U^T = C_vir X^T (n x o), R = C_occ U
  //   v <  o: W = C_occ X (n x v), R = W C_vir^T
  const bool vfirst = v < o;
  // per vector: X pair (X, or X^T when vfirst), U^T or W pair, R, G+, G-, G pair, S^T pair
  // sub-buffers start on 256-byte boundaries (tensor maps need 16-byte aligned bases)
  auto up = [](size_t x) { return (x + 63) / 64 * 64; };
  const size_t sX = up((size_t)chunk * (vfirst ? (size_t)v * op : (size_t)o * vp));
  const size_t sU = up((size_t)chunk * n * (vfirst ? vp : op)), sR = up((size_t)chunk * nn);
  const size_t sG = up((size_t)chunk * n * np_), sS = up((size_t)chunk * v * np_);
  const bool rpa = method != XS_CIS;
  c.fs0.ensure(2 * sX + 2 * sU + sR + (rpa ? 4 : 2) * sG + 2 * sS);
  float* p = c.fs0.get();
  float* Xh = p; p += sX;
  float* Xl = p; p += sX;
  float* Uh = p; p += sU;
  float* Ul = p; p += sU;
  float* R = p; p += sR;
  float* Gh = p; p += sG;     // TF32 pair of G (CIS) or G+ (TDHF)
  float* Gl = p; p += sG;
  float* Gmh = nullptr;       // TF32 pair of G- (TDHF)
  float* Gml = nullptr;
  if (rpa) {
    Gmh = p; p += sG;
    Gml = p; p += sG;
  }
  float* Sh = p; p += sS;
  float* Sl = p; p += sS;
  DevBuf<int>& err = c.tc_err;
  if (!err.get()) {
    err.alloc(1);
    XS_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
  }
  if (mx1) XS_CUDA(cudaMemsetAsync(mx1, 0, sizeof(unsigned int) * nvec, s));
  if (mx2 && rpa) XS_CUDA(cudaMemsetAsync(mx2, 0, sizeof(unsigned int) * nvec, s));

  for (int k0 = 0; k0 < nvec; k0 += chunk) {
    const int k = (nvec - k0) < chunk ? (nvec - k0) : chunk;
    const double* Xk = X + k0 * ov;
    if (vfirst) {
      split_pad_t(s, v, o, op, Xk, v, ov, (long long)v * op, k, Xh, Xl);   // X^T pair: v x op
      {  // W = C_occ X : M = n, N = v, K = o
        TcOperand A{Cocc_h, Cocc_l, op, 0, false};
        TcOperand B{Xh, Xl, op, (long long)v * op, true};
        TcEpilogue e;
        e.mode = 1; e.D = Uh; e.Dlo = Ul; e.ld = vp; e.bstride = (long long)n * vp;
        tc_gemm(s, A, B, n, v, op, k, e, err.get());
      }
      {  // R = W C_vir^T : M = n, N = n, K = v
        TcOperand A{Uh, Ul, vp, (long long)n * vp, true};
        TcOperand B{Cvir_h, Cvir_l, vp, 0, false};
        TcEpilogue e;
        e.mode = 0; e.D = R; e.ld = n; e.bstride = nn;
        tc_gemm(s, A, B, n, n, vp, k, e, err.get());
      }
    } else {
      split_pad<double>(s, o, v, vp, Xk, v, ov, (long long)o * vp, k, false, Xh, Xl);
      {  // U^T = C_vir X^T : M = n, N = o, K = v
        TcOperand A{Cvir_h, Cvir_l, vp, 0, false};
        TcOperand B{Xh, Xl, vp, (long long)o * vp, true};
        TcEpilogue e;
        e.mode = 1; e.D = Uh; e.Dlo = Ul; e.ld = op; e.bstride = (long long)n * op;
        tc_gemm(s, A, B, n, o, vp, k, e, err.get());
      }
      {  // R = C_occ U : M = n, N = n, K = o
        TcOperand A{Cocc_h, Cocc_l, op, 0, false};
        TcOperand B{Uh, Ul, op, (long long)n * op, true};
        TcEpilogue e;
        e.mode = 0; e.D = R; e.ld = n; e.bstride = nn;
        tc_gemm(s, A, B, n, n, op, k, e, err.get());
      }
    }
    // G (and G-) written directly as the back-transform's TF32 pairs
    gbuild_split(s, m, c.d_par.get(), gmode(rpa, triplet), k, R, Gh, Gl, Gmh, Gml, np_, c.fs1);
    for (int pass = 0; pass < (rpa ? 2 : 1); ++pass) {
      const float* Gph = pass == 0 ? Gh : Gmh;
      const float* Gpl = pass == 0 ? Gl : Gml;
      double* Yout = (pass == 0 ? Y1 : Y2) + k0 * ov;
      unsigned int* mxo = pass == 0 ? mx1 : mx2;
      {  // S^T = C_vir^T G^T : M = v, N = n, K = n
        TcOperand A{CTvir_h, CTvir_l, np_, 0, false};
        TcOperand B{Gph, Gpl, np_, (long long)n * np_, true};
        TcEpilogue e;
        e.mode = 1; e.D = Sh; e.Dlo = Sl; e.ld = np_; e.bstride = (long long)v * np_;
        tc_gemm(s, A, B, v, n, np_, k, e, err.get());
      }
      {  // Y = C_occ^T S + d eps X : M = o, N = v, K = n
        TcOperand A{CTocc_h, CTocc_l, np_, 0, false};
        TcOperand B{Sh, Sl, np_, (long long)v * np_, true};
        TcEpilogue e;
        e.mode = 2; e.Y = Yout; e.X = Xk; e.eps = m.eps.get(); e.ld = v; e.bstride = ov; e.o = o;
        e.rowmax = mxo ? mxo + k0 : nullptr;
        tc_gemm(s, A, B, o, v, np_, k, e, err.get());
      }
    }
  }
  // the error word (bounded waits) is read by the caller at its next
  // synchronisation (check_device_error), not here: no per-product host sync
}

}  // namespace xs
