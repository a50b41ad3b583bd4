// Integrals and core Hamiltonian of libxs on the device (paper, Section
// "Ground-state wavefunction calculation": minimal valence basis, three- and
// four-centre integrals dropped, two-centre integrals as classical multipole
// interactions, one-centre integrals as parameters; Eq. 1's core Hamiltonian).
//
// Two-centre integrals: every on-atom AO product is a model charge density
// built from a unit Gaussian of width sigma = kappa / (sqrt(pi) gss) and its
// Cartesian derivatives (rho_ss = G, rho_{s p_i} = -D1 d_i G,
// rho_{p_i p_j} = delta_ij G + D2^2 d_i d_j G), and (mu nu|lam sig) is the
// Coulomb energy of two such densities: derivatives up to fourth order of
// Phi(R) = kappa erf(aR)/R, a = 1/sqrt(2 (sA^2 + sB^2)), R = R_B - R_A, in the
// radial form T_i = x_i g1, T_ij = d_ij g1 + x_i x_j g2, ... with
// g_n = ((1/R) d/dR)^n Phi.  One thread per unordered atom pair writes both
// blocks of the product supermatrix W (np x np, float64).
// Core Hamiltonian: U on the diagonal, core attraction -Z_B (mu nu|s_B s_B)
// summed over the other atoms (one warp per atom, fixed summation order), and
// resonance (beta_mu + beta_lam)/2 S_mu lam with the Slater-Koster overlap
// S_x(R) = a_x exp(-k_x R) (one thread per unordered pair, both blocks).
#include <cmath>

#include "kernels.h"
#include "model.h"

namespace xs {

namespace {

// parameter fields (xs.h): Uss, Upp, beta_s, beta_p, gss, gsp, gpp, gp2, hsp, D1, D2, zeta_s, zeta_p
enum { P_USS = 0, P_UPP, P_BS, P_BP, P_GSS, P_GSP, P_GPP, P_GP2, P_HSP, P_D1, P_D2, P_ZS, P_ZP };

__device__ __forceinline__ double elem_charge(int elem) {   // rows H, C, N, O
  return elem == 0 ? 1.0 : (elem == 1 ? 4.0 : (elem == 2 ? 5.0 : 6.0));
}

// Cartesian derivative of order m (indices idx[0..m)) of the radial Phi
__device__ double t_eval(const double* x, const double* g, const int* idx, int m) {
  auto d = [](int i, int j) { return i == j ? 1.0 : 0.0; };
  switch (m) {
    case 0: return g[0];
    case 1: return x[idx[0]] * g[1];
    case 2: {
      const int i = idx[0], j = idx[1];
      return d(i, j) * g[1] + x[i] * x[j] * g[2];
    }
    case 3: {
      const int i = idx[0], j = idx[1], k = idx[2];
      return (d(i, j) * x[k] + d(i, k) * x[j] + d(j, k) * x[i]) * g[2] + x[i] * x[j] * x[k] * g[3];
    }
    default: {
      const int i = idx[0], j = idx[1], k = idx[2], l = idx[3];
      const double t2 = d(i, j) * d(k, l) + d(i, k) * d(j, l) + d(i, l) * d(j, k);
      const double t3 = d(i, j) * x[k] * x[l] + d(i, k) * x[j] * x[l] + d(i, l) * x[j] * x[k] +
                        d(j, k) * x[i] * x[l] + d(j, l) * x[i] * x[k] + d(k, l) * x[i] * x[j];
      return t2 * g[2] + t3 * g[3] + x[i] * x[j] * x[k] * x[l] * g[4];
    }
  }
}

// g_0..g_4 of kappa erf(aR)/R: b_0 = erf(aR)/R,
// b_n = ((2n-1) b_{n-1} - (2a^2)^n exp(-a^2 R^2) / (a sqrt(pi))) / R^2, g_n = (-1)^n kappa b_n
__device__ void radial_g(double R, double a, double* g) {
  const double inv_sqrt_pi = 0.56418958354775628695;
  const double ex = exp(-(a * R) * (a * R));
  double b = erf(a * R) / R;
  double two_a2n = 1.0, sign = 1.0;
  g[0] = kKappa * b;
  for (int n = 1; n <= 4; ++n) {
    two_a2n *= 2.0 * a * a;
    b = ((2 * n - 1) * b - two_a2n * ex * inv_sqrt_pi / a) / (R * R);
    sign = -sign;
    g[n] = sign * kKappa * b;
  }
}

// terms of on-atom product density p: coefficient and derivative indices
struct Term {
  double c;
  int m;
  int idx[2];
};

__device__ int product_terms(bool heavy, int p, double D1, double D2, Term* out) {
  if (!heavy || p == 0) {
    out[0] = {1.0, 0, {0, 0}};
    return 1;
  }
  const int a = p < 4 ? 0 : (p < 7 ? 1 : (p < 9 ? 2 : 3));
  const int b = p < 4 ? p : (p < 7 ? p - 3 : (p < 9 ? p - 5 : 3));
  if (a == 0) {   // s p_i: a dipole of length D1 along i
    out[0] = {-D1, 1, {b - 1, 0}};
    return 1;
  }
  const int i = a - 1, j = b - 1;
  int n = 0;
  if (i == j) out[n++] = {1.0, 0, {0, 0}};
  out[n++] = {D2 * D2, 2, {i, j}};
  return n;
}

__global__ void supermatrix_kernel(int natoms, int np, const double* __restrict__ xyz, const int* __restrict__ nao,
                                   const int* __restrict__ prod_off, const int* __restrict__ elem,
                                   const double* __restrict__ par, double* __restrict__ W) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long npair = (long long)natoms * (natoms - 1) / 2;
  if (t >= npair) return;
  // unordered pair (A, B), A < B, from the row-major upper-triangle index
  int A = static_cast<int>((2.0 * natoms - 1.0 - sqrt((2.0 * natoms - 1.0) * (2.0 * natoms - 1.0) - 8.0 * t)) / 2.0);
  if (A < 0) A = 0;
  auto first = [&](int a) { return (long long)a * (2LL * natoms - a - 1) / 2; };
  while (A > 0 && first(A) > t) --A;
  while (A + 1 < natoms && first(A + 1) <= t) ++A;
  const int B = A + 1 + static_cast<int>(t - first(A));
  const double* pA = par + elem[A] * XS_NPARAM;
  const double* pB = par + elem[B] * XS_NPARAM;
  const bool hA = nao[A] == 4, hB = nao[B] == 4;
  double x[3], R2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    x[c] = xyz[3 * B + c] - xyz[3 * A + c];
    R2 += x[c] * x[c];
  }
  const double R = sqrt(R2);
  const double sqrt_pi = 1.77245385090551602730;
  const double sA = kKappa / (sqrt_pi * pA[P_GSS]), sB = kKappa / (sqrt_pi * pB[P_GSS]);
  const double a = 1.0 / sqrt(2.0 * (sA * sA + sB * sB));
  double g[5];
  radial_g(R, a, g);
  const int npA = hA ? 10 : 1, npB = hB ? 10 : 1;
  const long long rA = prod_off[A], rB = prod_off[B];
  for (int p = 0; p < npA; ++p) {
    Term ta[2];
    const int na = product_terms(hA, p, pA[P_D1], pA[P_D2], ta);
    for (int q = 0; q < npB; ++q) {
      Term tb[2];
      const int nb = product_terms(hB, q, pB[P_D1], pB[P_D2], tb);
      double acc = 0.0;
      for (int u = 0; u < na; ++u)
        for (int v = 0; v < nb; ++v) {
          int idx[4];
          int mm = 0;
          for (int k = 0; k < ta[u].m; ++k) idx[mm++] = ta[u].idx[k];
          for (int k = 0; k < tb[v].m; ++k) idx[mm++] = tb[v].idx[k];
          // densities on B enter with (-1)^order: d/dR_B acts as -d/dR
          const double sgn = (tb[v].m % 2) ? -1.0 : 1.0;
          acc += ta[u].c * tb[v].c * sgn * t_eval(x, g, idx, mm);
        }
      W[(rA + p) * np + rB + q] = acc;
      W[(rB + q) * np + rA + p] = acc;
    }
  }
}

// diagonal blocks of H: U on the diagonal and -sum_{B != A} Z_B (mu nu|s_B s_B),
// one warp per atom (lanes over B, then a fixed shuffle tree)
__global__ void core_diag_kernel(int natoms, int n, int np, const int* __restrict__ ao_off, const int* __restrict__ nao,
                                 const int* __restrict__ prod_off, const int* __restrict__ elem,
                                 const double* __restrict__ par, const double* __restrict__ W, double* __restrict__ H) {
  const int A = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (A >= natoms) return;
  const int nA = nao[A], npA = nA == 4 ? 10 : 1;
  double acc[10];
  for (int p = 0; p < 10; ++p) acc[p] = 0.0;
  for (int B = lane; B < natoms; B += 32) {
    if (B == A) continue;
    const double ZB = elem_charge(elem[B]);
    const double* row = W + (long long)prod_off[A] * np + prod_off[B];
    for (int p = 0; p < npA; ++p) acc[p] = fma(-ZB, row[(long long)p * np], acc[p]);
  }
  for (int p = 0; p < npA; ++p)
    for (int o = 16; o > 0; o >>= 1) acc[p] += __shfl_xor_sync(0xffffffffu, acc[p], o);
  if (lane != 0) return;
  const double* pA = par + elem[A] * XS_NPARAM;
  const int oA = ao_off[A];
  for (int a = 0; a < nA; ++a)
    for (int b = 0; b < nA; ++b) {
      const int p = nA == 4 ? (a <= b ? ((a * (9 - a)) >> 1) + (b - a) : ((b * (9 - b)) >> 1) + (a - b)) : 0;
      double h = acc[p];
      if (a == b) h += (a == 0) ? pA[P_USS] : pA[P_UPP];
      H[(long long)(oA + a) * n + oA + b] = h;
    }
}

// off-diagonal blocks of H: (beta_mu + beta_lam)/2 S_mu lam, both blocks of
// each unordered pair (S_BA = S_AB^T), e = (R_B - R_A)/|R|:
//   S(s_A,s_B) = Sss, S(s_A,p_Bj) = -e_j Ssp(s_A,p_B), S(p_Ai,s_B) = e_i Ssp(s_B,p_A),
//   S(p_Ai,p_Bj) = -e_i e_j Spp_sigma + (d_ij - e_i e_j) Spp_pi
__global__ void core_pair_kernel(int natoms, int n, const double* __restrict__ xyz, const int* __restrict__ ao_off,
                                 const int* __restrict__ nao, const int* __restrict__ elem,
                                 const double* __restrict__ par, double* __restrict__ H) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)natoms * natoms) return;
  const int A = static_cast<int>(t / natoms), B = static_cast<int>(t % natoms);
  if (B <= A) return;
  const double* pA = par + elem[A] * XS_NPARAM;
  const double* pB = par + elem[B] * XS_NPARAM;
  double e[3], R2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    e[c] = xyz[3 * B + c] - xyz[3 * A + c];
    R2 += e[c] * e[c];
  }
  const double R = sqrt(R2);
  for (int c = 0; c < 3; ++c) e[c] /= R;
  double S[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) S[i][j] = 0.0;
  const bool hA = nao[A] == 4, hB = nao[B] == 4;
  S[0][0] = kSKss * exp(-0.5 * (pA[P_ZS] + pB[P_ZS]) * R);
  if (hB) {
    const double v = kSKsp * exp(-0.5 * (pA[P_ZS] + pB[P_ZP]) * R);
    for (int j = 0; j < 3; ++j) S[0][1 + j] = -e[j] * v;
  }
  if (hA) {
    const double v = kSKsp * exp(-0.5 * (pB[P_ZS] + pA[P_ZP]) * R);
    for (int i = 0; i < 3; ++i) S[1 + i][0] = e[i] * v;
  }
  if (hA && hB) {
    const double kp = 0.5 * (pA[P_ZP] + pB[P_ZP]);
    const double ss = kSKppSigma * exp(-kp * R);
    const double pp = kSKppPi * exp(-kSKPiScale * kp * R);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) S[1 + i][1 + j] = -e[i] * e[j] * ss + ((i == j ? 1.0 : 0.0) - e[i] * e[j]) * pp;
  }
  const double bA[4] = {pA[P_BS], pA[P_BP], pA[P_BP], pA[P_BP]};
  const double bB[4] = {pB[P_BS], pB[P_BP], pB[P_BP], pB[P_BP]};
  const int oA = ao_off[A], oB = ao_off[B], nA = nao[A], nB = nao[B];
  for (int a = 0; a < nA; ++a)
    for (int b = 0; b < nB; ++b) {
      const double h = 0.5 * (bA[a] + bB[b]) * S[a][b];
      H[(long long)(oA + a) * n + oB + b] = h;
      H[(long long)(oB + b) * n + oA + a] = h;
    }
}

}  // namespace

void build_model(cudaStream_t s, DevMol& m, const double* d_par) {
  const int na = m.L.natoms, n = m.n, np = m.np;
  m.W.alloc((size_t)np * np);
  m.H.alloc((size_t)n * n);
  XS_CUDA(cudaMemsetAsync(m.W.get(), 0, sizeof(double) * np * np, s));
  const long long npair = (long long)na * (na - 1) / 2;
  if (npair > 0) {
    supermatrix_kernel<<<grid1(npair, 128), 128, 0, s>>>(na, np, m.xyz.get(), m.atom_nao.get(), m.atom_prod_off.get(),
                                                         m.atom_elem.get(), d_par, m.W.get());
    XS_CHECK_LAUNCH();
  }
  core_diag_kernel<<<grid1((long long)na * 32, 256), 256, 0, s>>>(na, n, np, m.atom_ao_off.get(), m.atom_nao.get(),
                                                                  m.atom_prod_off.get(), m.atom_elem.get(), d_par,
                                                                  m.W.get(), m.H.get());
  XS_CHECK_LAUNCH();
  core_pair_kernel<<<grid1((long long)na * na, 256), 256, 0, s>>>(na, n, m.xyz.get(), m.atom_ao_off.get(),
                                                                  m.atom_nao.get(), m.atom_elem.get(), d_par,
                                                                  m.H.get());
  XS_CHECK_LAUNCH();
}

}  // namespace xs
