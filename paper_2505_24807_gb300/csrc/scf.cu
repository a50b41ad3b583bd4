// Ground state of libxs: restricted closed-shell SCF, F C = C eps with S = I
// (paper, Section "Ground-state wavefunction calculation", Eq. 1), started
// from the neutral-atom density (core charge spread over each atom's AOs).
//
// The two-electron Fock part reuses the excited-state G build: for the
// closed-shell density D = 2 C_occ C_occ^T, J(D) - K(D)/2 = 2 J(P) - K(P) with
// P = D/2, i.e. G_CIS(P).  Pulay DIIS on the commutator F D - D F.  The Fock
// eigenproblem of this setup step goes to cuSOLVER's dense symmetric solver
// (the excited-state path does not use it).
#include <cusolverDn.h>

#include <chrono>
#include <cmath>
#include <vector>

#include "kernels.h"
#include "scf.h"

namespace xs {

namespace {

struct Solver {
  cusolverDnHandle_t h = nullptr;
};

void check_solver(cusolverStatus_t st, const char* what) {
  if (st != CUSOLVER_STATUS_SUCCESS) throw Error(XS_ECUDA, std::string("cusolver: ") + what);
}

cusolverDnHandle_t solver_handle(Ctx& c) {
  if (!c.solver) {
    cusolverDnHandle_t h;
    check_solver(cusolverDnCreate(&h), "create");
    c.solver = h;
  }
  cusolverDnHandle_t h = static_cast<cusolverDnHandle_t>(c.solver);
  check_solver(cusolverDnSetStream(h, c.stream), "set stream");
  return h;
}

// eigenvectors of the symmetric n x n matrix in A (overwritten) as MO-major
// rows (A[p * n + mu]), eigenvalues ascending in w
void sym_eig(Ctx& c, int n, double* A, double* w, DevBuf<double>& work, DevBuf<int>& dinfo) {
  cusolverDnHandle_t h = solver_handle(c);
  int lwork = 0;
  check_solver(cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A, n, w, &lwork),
               "syevd buffer size");
  work.ensure(static_cast<size_t>(lwork));
  dinfo.ensure(1);
  check_solver(cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A, n, w, work.get(), lwork,
                                dinfo.get()),
               "syevd");
  int info = 0;
  XS_CUDA(cudaMemcpyAsync(&info, dinfo.get(), sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  XS_CUDA(cudaStreamSynchronize(c.stream));
  if (info != 0) throw Error(XS_ESCF, "Fock diagonalisation failed");
}

// D = 2 C_occ C_occ^T from the MO-major CT
void density(cudaStream_t s, int n, int o, const double* CT, double* D) {
  gemm<double>(s, true, false, n, n, o, 2.0, CT, n, 0, CT, n, 0, 0.0, D, n, 0, 1);
}

}  // namespace

void destroy_solver(Ctx& c) {
  if (c.solver) cusolverDnDestroy(static_cast<cusolverDnHandle_t>(c.solver));
  c.solver = nullptr;
}

int run_scf(Ctx& c, DevMol& m, double tol, int max_iter) {
  const int n = m.n, o = m.o;
  const size_t nn = static_cast<size_t>(n) * n;
  cudaStream_t s = c.stream;
  const int hist = 10;
  DevBuf<double> F(nn), D(nn), P(nn), T1(nn), Err(nn), Fh(hist * nn), Eh(hist * nn), Fx(nn), Dn(nn);
  DevBuf<double> work, small(64 + hist * hist + 16), gws;
  DevBuf<int> dinfo;
  m.CT.alloc(nn);
  m.eps.alloc(n);
  double* d_scal = small.get();            // [0]: max|dD|, [1]: max|err|
  double* d_coef = small.get() + 16;       // DIIS coefficients
  double* d_B = small.get() + 16 + hist;   // DIIS matrix

  // neutral-atom start: each atom's core charge spread evenly over its AOs
  {
    std::vector<double> d0(nn, 0.0);
    for (int a = 0; a < m.L.natoms; ++a)
      for (int k = 0; k < m.L.nao_atom[a]; ++k) {
        const int mu = m.L.ao_off[a] + k;
        d0[(size_t)mu * n + mu] = core_charge(m.L.Z[a]) / m.L.nao_atom[a];
      }
    XS_CUDA(cudaMemcpyAsync(D.get(), d0.data(), nn * sizeof(double), cudaMemcpyHostToDevice, s));
    XS_CUDA(cudaStreamSynchronize(s));
  }

  std::vector<int> slot_age;
  int count = 0, head = 0;
  bool converged = false;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    // F = H + G_CIS(D/2)
    XS_CUDA(cudaMemcpyAsync(P.get(), D.get(), nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    scal(s, static_cast<long long>(nn), 0.5, P.get());
    gbuild<double>(s, m, c.d_par.get(), G_CIS, 1, P.get(), F.get(), nullptr, c.ws0);
    axpy(s, static_cast<long long>(nn), 1.0, m.H.get(), F.get());
    // commutator F D - D F = T1 - T1^T with T1 = F D (both symmetric)
    gemm<double>(s, false, false, n, n, n, 1.0, F.get(), n, 0, D.get(), n, 0, 0.0, T1.get(), n, 0, 1);
    transpose(s, n, n, T1.get(), Err.get());
    scal(s, static_cast<long long>(nn), -1.0, Err.get());
    axpy(s, static_cast<long long>(nn), 1.0, T1.get(), Err.get());
    max_abs(s, static_cast<long long>(nn), Err.get(), d_scal + 1);
    // DIIS history (ring)
    XS_CUDA(cudaMemcpyAsync(Fh.get() + head * nn, F.get(), nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    XS_CUDA(cudaMemcpyAsync(Eh.get() + head * nn, Err.get(), nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    head = (head + 1) % hist;
    if (count < hist) ++count;
    const double* Fuse = F.get();
    if (count >= 2) {
      gram<double>(s, count, count, static_cast<int>(nn), Eh.get(), static_cast<int>(nn), Eh.get(),
                   static_cast<int>(nn), d_B, count, 1.0, 0.0, gws);
      std::vector<double> Bh(count * count);
      XS_CUDA(cudaMemcpyAsync(Bh.data(), d_B, sizeof(double) * count * count, cudaMemcpyDeviceToHost, s));
      XS_CUDA(cudaStreamSynchronize(s));
      // solve [B -1; -1 0][c; l] = [0; -1] by Gaussian elimination with pivoting
      int q = count + 1;
      std::vector<double> M(q * (q + 1), 0.0);
      for (int i = 0; i < count; ++i) {
        for (int j = 0; j < count; ++j) M[i * (q + 1) + j] = Bh[i * count + j];
        M[i * (q + 1) + count] = -1.0;
        M[count * (q + 1) + i] = -1.0;
      }
      M[count * (q + 1) + q] = -1.0;
      bool ok = true;
      for (int col = 0; col < q && ok; ++col) {
        int piv = col;
        for (int r = col + 1; r < q; ++r)
          if (std::fabs(M[r * (q + 1) + col]) > std::fabs(M[piv * (q + 1) + col])) piv = r;
        if (std::fabs(M[piv * (q + 1) + col]) < 1e-300) { ok = false; break; }
        if (piv != col)
          for (int k = 0; k <= q; ++k) std::swap(M[col * (q + 1) + k], M[piv * (q + 1) + k]);
        for (int r = 0; r < q; ++r) {
          if (r == col) continue;
          double f = M[r * (q + 1) + col] / M[col * (q + 1) + col];
          for (int k = col; k <= q; ++k) M[r * (q + 1) + k] -= f * M[col * (q + 1) + k];
        }
      }
      if (ok) {
        std::vector<double> coef(count);
        for (int i = 0; i < count; ++i) coef[i] = M[i * (q + 1) + q] / M[i * (q + 1) + i];
        XS_CUDA(cudaMemcpyAsync(d_coef, coef.data(), sizeof(double) * count, cudaMemcpyHostToDevice, s));
        gemm<double>(s, false, false, 1, static_cast<int>(nn), count, 1.0, d_coef, count, 0, Fh.get(),
                     static_cast<int>(nn), 0, 0.0, Fx.get(), static_cast<int>(nn), 0, 1);
        Fuse = Fx.get();
      }
    }
    XS_CUDA(cudaMemcpyAsync(m.CT.get(), Fuse, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    sym_eig(c, n, m.CT.get(), m.eps.get(), work, dinfo);
    density(s, n, o, m.CT.get(), Dn.get());
    // max |Dn - D|
    XS_CUDA(cudaMemcpyAsync(T1.get(), Dn.get(), nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    axpy(s, static_cast<long long>(nn), -1.0, D.get(), T1.get());
    max_abs(s, static_cast<long long>(nn), T1.get(), d_scal);
    std::swap(D, Dn);
    double sc[2];
    XS_CUDA(cudaMemcpyAsync(sc, d_scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
    XS_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(sc[0]) || !std::isfinite(sc[1])) throw Error(XS_ESCF, "SCF produced non-finite values");
    if (sc[0] < tol && sc[1] < 10.0 * tol) { converged = true; break; }
  }
  if (!converged) throw Error(XS_ESCF, "SCF did not converge in " + std::to_string(max_iter) + " iterations");
  // final Fock of the converged density and its eigenvectors
  XS_CUDA(cudaMemcpyAsync(P.get(), D.get(), nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  scal(s, static_cast<long long>(nn), 0.5, P.get());
  gbuild<double>(s, m, c.d_par.get(), G_CIS, 1, P.get(), F.get(), nullptr, c.ws0);
  axpy(s, static_cast<long long>(nn), 1.0, m.H.get(), F.get());
  XS_CUDA(cudaMemcpyAsync(m.CT.get(), F.get(), nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
  sym_eig(c, n, m.CT.get(), m.eps.get(), work, dinfo);
  std::vector<double> e(n);
  XS_CUDA(cudaMemcpyAsync(e.data(), m.eps.get(), sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  XS_CUDA(cudaStreamSynchronize(s));
  if (o < n && e[o] - e[o - 1] < 0.5)
    throw Error(XS_ESCF, "HOMO-LUMO gap below 0.5 eV (" + std::to_string(e[o] - e[o - 1]) + ")");
  m.scf_iterations = it;
  return it;
}

}  // namespace xs
