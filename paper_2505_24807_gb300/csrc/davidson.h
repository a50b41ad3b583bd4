// Davidson solver of libxs (davidson.cu).
#pragma once

#include "common.cuh"

namespace xs {

struct SolveStats {
  int iterations = 0;
  long long products = 0;
  int collapses = 0;
  bool converged = false;
  bool polished = false;
  bool learned = false;    // learned guess and shift were used
  bool fallback = false;   // the learned shift was dropped for a stalled residual
  double seconds_products = 0.0;
  int smax = 0;            // subspace cap in effect
  double tol_used = 0.0;   // residual threshold applied (eV)
};

// Solves molecule m; stores roots, oscillator strengths, residuals and
// amplitudes in m.  Returns XS_OK, XS_ENOCONV or XS_EUNSTABLE.
int davidson(Ctx& c, DevMol& m, const xs_ex_opts& opt, SolveStats& st);

// f (device, kk) from amplitudes U (kk x ov, X or X+Y) and omega (device, eV)
// MO dipole integrals D^x_ia (3 x nocc x nvir) of the molecule, computed once
// and kept in m.dip until the orbitals change.
void mo_dipoles(Ctx& c, DevMol& m);
void oscillator_strengths(Ctx& c, DevMol& m, int kk, const double* U, const double* omega_dev, double* f_dev);

// d omega_root / d theta for every NDDO parameter (XS_NELEM x XS_NPARAM,
// host array) of the last singlet CIS or TDHF solve of m, with the orbital
// response by one adjoint (A+B) solve (gradient.cu).
void parameter_gradient(Ctx& c, DevMol& m, int root, double* grad_host, int* cg_iterations);

}  // namespace xs
