// Host-side NDDO model of libxs: per-element parameters and the AO layout
// (the integrals and the core Hamiltonian are built on the device,
// integrals.cu).
//
// Paper, Section "Ground-state wavefunction calculation": minimal valence
// basis, three- and four-centre integrals dropped, two-centre integrals as
// classical multipole interactions, one-centre integrals as parameters.  The
// paper prints neither the parameters nor the multipole formulas; this file
// implements the stated model:
//   on-atom AO products are charge densities made from a unit Gaussian G_A of
//   width sigma_A = kappa / (sqrt(pi) gss_A) and its Cartesian derivatives
//   (rho_ss = G, rho_{s p_i} = -D1 d_i G, rho_{p_i p_j} = delta_ij G + D2^2 d_i d_j G),
//   and (mu nu|lam sig) is their Coulomb energy, built from the radial
//   Phi(R) = kappa erf(aR)/R, a = 1/sqrt(2(sA^2 + sB^2)), with R = R_B - R_A.
#pragma once

#include <cstdint>
#include <vector>

namespace xs {

constexpr double kKappa = 14.399645;          // e^2/(4 pi eps0), eV Angstrom (CODATA 2018)
constexpr double kHartreeEV = 27.211386245988;
constexpr double kBohrA = 0.529177210903;

// Slater-Koster radial model S_x(R) = a_x exp(-k_x R); k_x = mean of the two
// atoms' orbital exponents (x 1.3 for pp-pi).
constexpr double kSKss = 2.0, kSKsp = 2.4, kSKppSigma = 1.9, kSKppPi = 1.6;
constexpr double kSKPiScale = 1.3;

struct ElemParams {
  double Uss, Upp, beta_s, beta_p, gss, gsp, gpp, gp2, hsp, D1, D2, zeta_s, zeta_p;
};

// element row in the parameter table: H, C, N, O
int element_row(int Z);
double core_charge(int Z);

struct MolLayout {
  int natoms = 0;
  int nao = 0;      // AOs
  int nprod = 0;    // on-atom AO products (10 per heavy atom, 1 per H)
  int nocc = 0;
  std::vector<int> Z;
  std::vector<double> xyz;       // 3 per atom, Angstrom
  std::vector<int> ao_off;       // first AO of each atom
  std::vector<int> nao_atom;     // 4 or 1
  std::vector<int> prod_off;     // first product of each atom
  std::vector<int> elem;         // element row
  std::vector<int> ao_atom;      // atom of each AO
  std::vector<int> ao_local;     // 0 = s, 1..3 = p
};

// Builds the layout; returns false for odd electron counts or unknown elements.
bool build_layout(int natoms, const int* Z, const double* xyz, MolLayout& out);

// Product index of AOs (a, b) on one heavy atom, AO order s, px, py, pz.
int prod_index(int a, int b);

}  // namespace xs
