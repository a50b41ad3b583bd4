// Host-side NDDO model of libxs (see model.h for the model statement).
#include "model.h"

#include <cmath>
#include <thread>

namespace xs {

int element_row(int Z) {
  switch (Z) {
    case 1: return 0;
    case 6: return 1;
    case 7: return 2;
    case 8: return 3;
    default: return -1;
  }
}

double core_charge(int Z) {
  switch (Z) {
    case 1: return 1.0;
    case 6: return 4.0;
    case 7: return 5.0;
    case 8: return 6.0;
    default: return 0.0;
  }
}

int prod_index(int a, int b) {
  static const int tab[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
  return tab[a][b];
}

bool build_layout(int natoms, const int* Z, const double* xyz, MolLayout& m) {
  m = MolLayout();
  m.natoms = natoms;
  m.Z.assign(Z, Z + natoms);
  m.xyz.assign(xyz, xyz + 3 * natoms);
  int nel = 0;
  for (int a = 0; a < natoms; ++a) {
    int row = element_row(Z[a]);
    if (row < 0) return false;
    m.elem.push_back(row);
    int na = (Z[a] == 1) ? 1 : 4;
    m.ao_off.push_back(m.nao);
    m.nao_atom.push_back(na);
    m.prod_off.push_back(m.nprod);
    for (int k = 0; k < na; ++k) {
      m.ao_atom.push_back(a);
      m.ao_local.push_back(k);
    }
    m.nao += na;
    m.nprod += (na == 4) ? 10 : 1;
    nel += static_cast<int>(core_charge(Z[a]));
  }
  if (nel % 2 != 0 || natoms == 0) return false;
  m.nocc = nel / 2;
  return true;
}

namespace {

// Cartesian derivative tensors of a radial function f(|R|), written with
// g_n = ((1/R) d/dR)^n f:
//   T_i    = x_i g1
//   T_ij   = d_ij g1 + x_i x_j g2
//   T_ijk  = (d_ij x_k + d_ik x_j + d_jk x_i) g2 + x_i x_j x_k g3
//   T_ijkl = (d_ij d_kl + d_ik d_jl + d_il d_jk) g2
//          + (d_ij x_k x_l + d_ik x_j x_l + d_il x_j x_k + d_jk x_i x_l
//             + d_jl x_i x_k + d_kl x_i x_j) g3 + x_i x_j x_k x_l g4
struct TTensor {
  double x[3];
  double g[5];
  double d(int i, int j) const { return i == j ? 1.0 : 0.0; }
  double eval(const int* idx, int m) const {
    switch (m) {
      case 0: return g[0];
      case 1: return x[idx[0]] * g[1];
      case 2: {
        int i = idx[0], j = idx[1];
        return d(i, j) * g[1] + x[i] * x[j] * g[2];
      }
      case 3: {
        int i = idx[0], j = idx[1], k = idx[2];
        return (d(i, j) * x[k] + d(i, k) * x[j] + d(j, k) * x[i]) * g[2] + x[i] * x[j] * x[k] * g[3];
      }
      default: {
        int i = idx[0], j = idx[1], k = idx[2], l = idx[3];
        double t2 = d(i, j) * d(k, l) + d(i, k) * d(j, l) + d(i, l) * d(j, k);
        double t3 = d(i, j) * x[k] * x[l] + d(i, k) * x[j] * x[l] + d(i, l) * x[j] * x[k] +
                    d(j, k) * x[i] * x[l] + d(j, l) * x[i] * x[k] + d(k, l) * x[i] * x[j];
        return t2 * g[2] + t3 * g[3] + x[i] * x[j] * x[k] * x[l] * g[4];
      }
    }
  }
};

// g_n of Phi(R) = kappa erf(aR)/R: b_0 = erf(aR)/R,
// b_n = ((2n-1) b_{n-1} - (2a^2)^n exp(-a^2R^2) / (a sqrt(pi))) / R^2, g_n = (-1)^n kappa b_n.
void radial(double R, double a, double* g) {
  const double inv_sqrt_pi = 0.56418958354775628695;
  double ex = std::exp(-(a * R) * (a * R));
  double b = std::erf(a * R) / R;
  double two_a2n = 1.0;
  g[0] = kKappa * b;
  double sign = 1.0;
  for (int n = 1; n <= 4; ++n) {
    two_a2n *= 2.0 * a * a;
    b = ((2 * n - 1) * b - two_a2n * ex * inv_sqrt_pi / a) / (R * R);
    sign = -sign;
    g[n] = sign * kKappa * b;
  }
}

// One term of a product density: coefficient times d^idx G.
struct Term {
  double c;
  int m;
  int idx[2];
};

int product_terms(bool heavy, int p, double D1, double D2, Term* out) {
  if (!heavy || p == 0) {
    out[0] = {1.0, 0, {0, 0}};
    return 1;
  }
  static const int pa[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
  static const int pb[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
  int a = pa[p], b = pb[p];
  if (a == 0) {  // s p_i: dipole of length D1 along i
    out[0] = {-D1, 1, {b - 1, 0}};
    return 1;
  }
  int i = a - 1, j = b - 1;
  int n = 0;
  if (i == j) out[n++] = {1.0, 0, {0, 0}};
  out[n++] = {D2 * D2, 2, {i, j}};
  return n;
}

void pair_block(const MolLayout& m, const ElemParams* par, int A, int B, double* W, int ldw) {
  const ElemParams& pA = par[m.elem[A]];
  const ElemParams& pB = par[m.elem[B]];
  bool hA = m.nao_atom[A] == 4, hB = m.nao_atom[B] == 4;
  TTensor T;
  double R2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    T.x[c] = m.xyz[3 * B + c] - m.xyz[3 * A + c];
    R2 += T.x[c] * T.x[c];
  }
  double R = std::sqrt(R2);
  const double sqrt_pi = 1.77245385090551602730;
  double sA = kKappa / (sqrt_pi * pA.gss), sB = kKappa / (sqrt_pi * pB.gss);
  double a = 1.0 / std::sqrt(2.0 * (sA * sA + sB * sB));
  radial(R, a, T.g);
  int npA = hA ? 10 : 1, npB = hB ? 10 : 1;
  for (int p = 0; p < npA; ++p) {
    Term ta[2];
    int na = product_terms(hA, p, pA.D1, pA.D2, ta);
    for (int q = 0; q < npB; ++q) {
      Term tb[2];
      int nb = product_terms(hB, q, pB.D1, pB.D2, tb);
      double acc = 0.0;
      for (int u = 0; u < na; ++u) {
        for (int v = 0; v < nb; ++v) {
          int idx[4];
          int mm = 0;
          for (int t = 0; t < ta[u].m; ++t) idx[mm++] = ta[u].idx[t];
          for (int t = 0; t < tb[v].m; ++t) idx[mm++] = tb[v].idx[t];
          // densities on B enter with (-1)^{order}: d/dR_B acts as -d/dR
          double sgn = (tb[v].m % 2) ? -1.0 : 1.0;
          acc += ta[u].c * tb[v].c * sgn * T.eval(idx, mm);
        }
      }
      W[p * ldw + q] = acc;
    }
  }
}

template <typename F>
void parallel_for(int n, F f) {
  unsigned hw = std::thread::hardware_concurrency();
  int nt = static_cast<int>(hw == 0 ? 4 : (hw > 32 ? 32 : hw));
  if (n < 64) nt = 1;
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    th.emplace_back([=]() {
      for (int i = t; i < n; i += nt) f(i);
    });
  }
  for (auto& x : th) x.join();
}

}  // namespace

void two_centre_supermatrix(const MolLayout& m, const ElemParams* par, std::vector<double>& W) {
  const int np = m.nprod;
  W.assign(static_cast<size_t>(np) * np, 0.0);
  parallel_for(m.natoms, [&](int A) {
    double blk[100];
    for (int B = A + 1; B < m.natoms; ++B) {
      pair_block(m, par, A, B, blk, 10);
      int npA = m.nao_atom[A] == 4 ? 10 : 1, npB = m.nao_atom[B] == 4 ? 10 : 1;
      for (int p = 0; p < npA; ++p)
        for (int q = 0; q < npB; ++q) {
          double v = blk[p * 10 + q];
          W[static_cast<size_t>(m.prod_off[A] + p) * np + m.prod_off[B] + q] = v;
          W[static_cast<size_t>(m.prod_off[B] + q) * np + m.prod_off[A] + p] = v;
        }
    }
  });
}

namespace {
// Slater-Koster overlap between the AOs of atoms A != B, e = (R_B - R_A)/|R|:
//   S(s_A,s_B) = Sss;  S(s_A,p_Bj) = -e_j Ssp(A_s,B_p);  S(p_Ai,s_B) = e_i Ssp(B_s,A_p);
//   S(p_Ai,p_Bj) = -e_i e_j Spp_sigma + (d_ij - e_i e_j) Spp_pi.
void sk_block(const MolLayout& m, const ElemParams* par, int A, int B, double S[4][4]) {
  const ElemParams& pA = par[m.elem[A]];
  const ElemParams& pB = par[m.elem[B]];
  double e[3], R2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    e[c] = m.xyz[3 * B + c] - m.xyz[3 * A + c];
    R2 += e[c] * e[c];
  }
  double R = std::sqrt(R2);
  for (int c = 0; c < 3; ++c) e[c] /= R;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) S[i][j] = 0.0;
  S[0][0] = kSKss * std::exp(-0.5 * (pA.zeta_s + pB.zeta_s) * R);
  bool hA = m.nao_atom[A] == 4, hB = m.nao_atom[B] == 4;
  if (hB) {
    double v = kSKsp * std::exp(-0.5 * (pA.zeta_s + pB.zeta_p) * R);
    for (int j = 0; j < 3; ++j) S[0][1 + j] = -e[j] * v;
  }
  if (hA) {
    double v = kSKsp * std::exp(-0.5 * (pB.zeta_s + pA.zeta_p) * R);
    for (int i = 0; i < 3; ++i) S[1 + i][0] = e[i] * v;
  }
  if (hA && hB) {
    double kp = 0.5 * (pA.zeta_p + pB.zeta_p);
    double ss = kSKppSigma * std::exp(-kp * R);
    double pp = kSKppPi * std::exp(-kSKPiScale * kp * R);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        S[1 + i][1 + j] = -e[i] * e[j] * ss + ((i == j ? 1.0 : 0.0) - e[i] * e[j]) * pp;
  }
}
}  // namespace

void core_hamiltonian(const MolLayout& m, const ElemParams* par, const std::vector<double>& W,
                      std::vector<double>& H) {
  const int n = m.nao, np = m.nprod;
  H.assign(static_cast<size_t>(n) * n, 0.0);
  parallel_for(m.natoms, [&](int A) {
    const ElemParams& pA = par[m.elem[A]];
    int oA = m.ao_off[A], nA = m.nao_atom[A];
    double betaA[4] = {pA.beta_s, pA.beta_p, pA.beta_p, pA.beta_p};
    // one-electron energies
    for (int a = 0; a < nA; ++a) H[static_cast<size_t>(oA + a) * n + oA + a] += (a == 0) ? pA.Uss : pA.Upp;
    for (int B = 0; B < m.natoms; ++B) {
      if (B == A) continue;
      // core attraction of B's core on the products of A: -Z_B (mu nu | s_B s_B)
      double ZB = core_charge(m.Z[B]);
      for (int a = 0; a < nA; ++a)
        for (int b = 0; b < nA; ++b) {
          int p = (nA == 4) ? prod_index(a, b) : 0;
          H[static_cast<size_t>(oA + a) * n + oA + b] -=
              ZB * W[static_cast<size_t>(m.prod_off[A] + p) * np + m.prod_off[B]];
        }
      // resonance row block A, column block B
      const ElemParams& pB = par[m.elem[B]];
      double betaB[4] = {pB.beta_s, pB.beta_p, pB.beta_p, pB.beta_p};
      double S[4][4];
      sk_block(m, par, A, B, S);
      int oB = m.ao_off[B], nB = m.nao_atom[B];
      for (int a = 0; a < nA; ++a)
        for (int b = 0; b < nB; ++b)
          H[static_cast<size_t>(oA + a) * n + oB + b] = 0.5 * (betaA[a] + betaB[b]) * S[a][b];
    }
  });
}

}  // namespace xs
