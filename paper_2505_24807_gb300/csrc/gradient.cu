// Derivatives of CIS and TDHF excitation energies with respect to the NDDO
// parameters (paper, Section "Overview of the capabilities of PySEQM": the
// model parameters are differentiable so that they can be learned).
//
// For a normalised CIS root X (nocc x nvir) of the closed-shell ground state
// (S = I, F = H + G(D/2), G(Q) = 2J(Q) - K(Q)):
//   omega = Tr(F Delta) + <R, G(R)>,
//   R = C_occ X C_vir^T,  Delta = C_vir X^T X C_vir^T - C_occ X X^T C_occ^T.
// For a TDHF root with U = X+Y, W = X-Y, U.W = 1, omega = [U^T (A+B) U +
// W^T (A-B) W] / 2 is stationary in U and W, and in the same form
//   omega = Tr(F Delta) + <Q1, G(Q1)> + <Q2, G(Q2)>,
//   Q1 = sym(C_occ U C_vir^T), Q2 = antisym(C_occ W C_vir^T),
//   Delta = C_vir (U^T U + W^T W)/2 C_vir^T - C_occ (U U^T + W W^T)/2 C_occ^T
// (G(Q2) = -K(Q2): the Coulomb part vanishes for the antisymmetric Q2).
// The orbitals move with the parameters through the SCF condition
// F_ai = 0, whose linear response is (A+B) z = -(C_occ^T dF C_vir) with the
// singlet A+B of the TDHF problem.  With the orbital gradient of omega
//   L_ia = sum over the pairs (Y, Q) = (X, R) (CIS) or (U, Q1), (W, Q2) (TDHF) of
//          2 [Y G_vv^T - G_oo^T Y]_ia,  G_vv = C_vir^T G(Q) C_vir, G_oo = C_occ^T G(Q) C_occ,
//        + 2 [C_occ^T G(Delta) C_vir]_ia,
// one adjoint solve (A+B) Z = L (conjugate gradients on the library's float64
// (A+B) products) serves every parameter:
//   d omega / d theta = Tr(dH/dtheta P) + <P, dG/dtheta(D/2)> + sum_Q <Q, dG/dtheta(Q)>,
//   P = Delta - sym(C_occ Z C_vir^T).
// The parameter derivatives are contracted directly, with no derivative
// matrices formed: the core Hamiltonian (U on the diagonal, the resonance
// (beta_mu + beta_lam)/2 S_mu lam with S_x = a_x exp(-k_x R), the core
// attraction -Z_B (mu nu|s_B s_B)), the one-centre integrals (linear in gss,
// gsp, gpp, gp2, hsp), and the two-centre integrals through the multipole
// lengths D1, D2 and the Gaussian width (gss -> sigma -> a in
// Phi = kappa erf(aR)/R), one thread per atom pair.
#include <cmath>
#include <vector>

#include "kernels.h"
#include "model.h"
#include "products.h"

namespace xs {

namespace {

enum { P_USS = 0, P_UPP, P_BS, P_BP, P_GSS, P_GSP, P_GPP, P_GP2, P_HSP, P_D1, P_D2, P_ZS, P_ZP };

__device__ __forceinline__ double elem_charge(int elem) {   // rows H, C, N, O
  return elem == 0 ? 1.0 : (elem == 1 ? 4.0 : (elem == 2 ? 5.0 : 6.0));
}

// (lo, hi) AOs of on-atom product p (s, px, py, pz order of products)
__device__ __forceinline__ int p_lo(int p) { return p < 4 ? 0 : (p < 7 ? 1 : (p < 9 ? 2 : 3)); }
__device__ __forceinline__ int p_hi(int p) { return p < 4 ? p : (p < 7 ? p - 3 : (p < 9 ? p - 5 : 3)); }

// Cartesian derivative tensor of order m of a radial function given its
// g_n = ((1/R) d/dR)^n (same formulas as the integral build)
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

// g_0..g_4 of kappa erf(aR)/R and their derivatives with respect to a:
// b_0 = erf(aR)/R, b_n = ((2n-1) b_{n-1} - (2a^2)^n e^{-a^2R^2} / (a sqrt(pi))) / R^2,
// g_n = (-1)^n kappa b_n; db_0/da = (2/sqrt(pi)) e^{-a^2R^2},
// d/da [(2a^2)^n e^{-a^2R^2} / (a sqrt(pi))] = 2^n e^{-a^2R^2} ((2n-1) a^{2n-2} - 2 R^2 a^{2n}) / sqrt(pi)
__device__ void radial_g_da(double R, double a, double* g, double* dg) {
  const double inv_sqrt_pi = 0.56418958354775628695;
  const double ex = exp(-(a * R) * (a * R));
  double b = erf(a * R) / R, db = 2.0 * inv_sqrt_pi * ex;
  double two_n = 1.0, a2n2 = 1.0 / (a * a), sign = 1.0;   // 2^n, a^(2n-2)
  g[0] = kKappa * b;
  dg[0] = kKappa * db;
  for (int n = 1; n <= 4; ++n) {
    two_n *= 2.0;
    a2n2 *= a * a;
    const double q = two_n * a2n2 * a * a * ex * inv_sqrt_pi / a;   // (2a^2)^n e / (a sqrt(pi))
    const double dq = two_n * ex * inv_sqrt_pi * ((2 * n - 1) * a2n2 - 2.0 * R * R * a2n2 * a * a);
    b = ((2 * n - 1) * b - q) / (R * R);
    db = ((2 * n - 1) * db - dq) / (R * R);
    sign = -sign;
    g[n] = sign * kKappa * b;
    dg[n] = sign * kKappa * db;
  }
}

struct Term {
  double c, dD1, dD2;   // coefficient and its derivatives with respect to D1, D2
  int m;
  int idx[2];
};

__device__ int product_terms(bool heavy, int p, double D1, double D2, Term* out) {
  if (!heavy || p == 0) {
    out[0] = {1.0, 0.0, 0.0, 0, {0, 0}};
    return 1;
  }
  const int a = p_lo(p), b = p_hi(p);
  if (a == 0) {
    out[0] = {-D1, -1.0, 0.0, 1, {b - 1, 0}};
    return 1;
  }
  const int i = a - 1, j = b - 1;
  int n = 0;
  if (i == j) out[n++] = {1.0, 0.0, 0.0, 0, {0, 0}};
  out[n++] = {D2 * D2, 0.0, 2.0 * D2, 2, {i, j}};
  return n;
}

// diagonal-block packs of the densities: for on-atom product p of atom A,
// the sum over its ordered AO pairs of Q[mu][nu], for Q = P, D/2, Q1 (the
// antisymmetric Q2 packs to zero)
__global__ void pack_kernel(int natoms, int n, const int* __restrict__ ao_off, const int* __restrict__ nao,
                            const int* __restrict__ prod_off, const double* __restrict__ P, const double* __restrict__ Dh,
                            const double* __restrict__ R, double* __restrict__ pk) {
  const int A = blockIdx.x * blockDim.x + threadIdx.x;
  if (A >= natoms) return;
  const int o = ao_off[A], np10 = nao[A] == 4 ? 10 : 1, base = prod_off[A];
  for (int p = 0; p < np10; ++p) {
    const int a = np10 == 10 ? p_lo(p) : 0, b = np10 == 10 ? p_hi(p) : 0;
    const size_t ab = (size_t)(o + a) * n + o + b, ba = (size_t)(o + b) * n + o + a;
    for (int k = 0; k < 3; ++k) {   // pk[3 (product) + k]: P, D/2, R
      const double* Q = k == 0 ? P : (k == 1 ? Dh : R);
      pk[3 * (size_t)(base + p) + k] = (a == b) ? Q[ab] : Q[ab] + Q[ba];
    }
  }
}

// one thread per unordered atom pair: two-centre integral derivatives through
// (a, D1, D2) of both atoms contracted with the pair's two-particle density,
// and the resonance derivatives (beta, zeta); per-block sums added to grad
__global__ void __launch_bounds__(128) pair_grad_kernel(int natoms, int n, const double* __restrict__ xyz,
                                                        const int* __restrict__ ao_off, const int* __restrict__ nao,
                                                        const int* __restrict__ prod_off,
                                                        const int* __restrict__ elem, const double* __restrict__ par,
                                                        const double* __restrict__ P, const double* __restrict__ Dh,
                                                        const double* __restrict__ R, const double* __restrict__ Rm,
                                                        const double* __restrict__ pk, double* __restrict__ grad) {
  __shared__ double gs[XS_NELEM * XS_NPARAM];
  for (int i = threadIdx.x; i < XS_NELEM * XS_NPARAM; i += blockDim.x) gs[i] = 0.0;
  __syncthreads();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long npair = (long long)natoms * (natoms - 1) / 2;
  if (t < npair) {
    int A = static_cast<int>((2.0 * natoms - 1.0 - sqrt((2.0 * natoms - 1.0) * (2.0 * natoms - 1.0) - 8.0 * t)) / 2.0);
    if (A < 0) A = 0;
    auto first = [&](int x) { return (long long)x * (2LL * natoms - x - 1) / 2; };
    while (A > 0 && first(A) > t) --A;
    while (A + 1 < natoms && first(A + 1) <= t) ++A;
    const int B = A + 1 + static_cast<int>(t - first(A));
    const int eA = elem[A], eB = elem[B];
    const double* pA = par + eA * XS_NPARAM;
    const double* pB = par + eB * XS_NPARAM;
    const bool hA = nao[A] == 4, hB = nao[B] == 4;
    const int oA = ao_off[A], oB = ao_off[B], nA = nao[A], nB = nao[B];
    double x[3], R2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      x[c] = xyz[3 * B + c] - xyz[3 * A + c];
      R2 += x[c] * x[c];
    }
    const double Rd = sqrt(R2);
    // off-diagonal blocks (zero past a hydrogen's single AO)
    double Pab[4][4], Pba[4][4], Dab[4][4], Dba[4][4], Rab[4][4], Rba[4][4], Sab[4][4], Sba[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const bool ok = i < nA && j < nB;
        const size_t ab = (size_t)(oA + i) * n + oB + j, ba = (size_t)(oB + j) * n + oA + i;
        Pab[i][j] = ok ? P[ab] : 0.0;
        Pba[j][i] = ok ? P[ba] : 0.0;
        Dab[i][j] = ok ? Dh[ab] : 0.0;
        Dba[j][i] = ok ? Dh[ba] : 0.0;
        Rab[i][j] = ok ? R[ab] : 0.0;
        Rba[j][i] = ok ? R[ba] : 0.0;
        Sab[i][j] = (ok && Rm) ? Rm[ab] : 0.0;
        Sba[j][i] = (ok && Rm) ? Rm[ba] : 0.0;
      }
    // two-centre integrals
    const double sqrt_pi = 1.77245385090551602730;
    const double sA = kKappa / (sqrt_pi * pA[P_GSS]), sB = kKappa / (sqrt_pi * pB[P_GSS]);
    const double a = 1.0 / sqrt(2.0 * (sA * sA + sB * sB));
    double g[5], dg[5];
    radial_g_da(Rd, a, g, dg);
    const int npA = hA ? 10 : 1, npB = hB ? 10 : 1;
    const int PA = prod_off[A], PB = prod_off[B];
    const double ZA = elem_charge(eA), ZB = elem_charge(eB);
    double Sa = 0.0, SD1A = 0.0, SD2A = 0.0, SD1B = 0.0, SD2B = 0.0;
    for (int p = 0; p < npA; ++p) {
      Term ta[2];
      const int na = product_terms(hA, p, pA[P_D1], pA[P_D2], ta);
      const int a1 = hA ? p_lo(p) : 0, a2 = hA ? p_hi(p) : 0;
      const double PpA = pk[3 * (size_t)(PA + p)], DpA = pk[3 * (size_t)(PA + p) + 1], RpA = pk[3 * (size_t)(PA + p) + 2];
      for (int q = 0; q < npB; ++q) {
        Term tb[2];
        const int nb = product_terms(hB, q, pB[P_D1], pB[P_D2], tb);
        const int b1 = hB ? p_lo(q) : 0, b2 = hB ? p_hi(q) : 0;
        const double PpB = pk[3 * (size_t)(PB + q)], DpB = pk[3 * (size_t)(PB + q) + 1],
                     RpB = pk[3 * (size_t)(PB + q) + 2];
        // two-particle density of the pair: Coulomb of <P, G(D/2)> and <R, G(R)>,
        // their exchange over the ordered AO pairs of p and q, core attraction
        double gam = 2.0 * (PpA * DpB + PpB * DpA) + 4.0 * RpA * RpB;
        for (int ca = 0; ca < 2; ++ca) {
          if (ca == 1 && a1 == a2) continue;
          const int u = ca ? a2 : a1, w = ca ? a1 : a2;
          for (int cb = 0; cb < 2; ++cb) {
            if (cb == 1 && b1 == b2) continue;
            const int y = cb ? b2 : b1, z = cb ? b1 : b2;
            gam -= Pab[u][y] * Dab[w][z] + Pba[y][u] * Dba[z][w];
            gam -= Rab[u][y] * Rab[w][z] + Rba[y][u] * Rba[z][w];
            gam -= Sab[u][y] * Sab[w][z] + Sba[y][u] * Sba[z][w];
          }
        }
        if (q == 0) gam -= ZB * PpA;
        if (p == 0) gam -= ZA * PpB;
        // derivatives of W_AB[p][q]
        double dWa = 0.0, dW1A = 0.0, dW2A = 0.0, dW1B = 0.0, dW2B = 0.0;
        for (int uu = 0; uu < na; ++uu)
          for (int vv = 0; vv < nb; ++vv) {
            int idx[4];
            int mm = 0;
            for (int k = 0; k < ta[uu].m; ++k) idx[mm++] = ta[uu].idx[k];
            for (int k = 0; k < tb[vv].m; ++k) idx[mm++] = tb[vv].idx[k];
            const double sgn = (tb[vv].m % 2) ? -1.0 : 1.0;
            const double T = t_eval(x, g, idx, mm), dT = t_eval(x, dg, idx, mm);
            dWa += ta[uu].c * tb[vv].c * sgn * dT;
            dW1A += ta[uu].dD1 * tb[vv].c * sgn * T;
            dW2A += ta[uu].dD2 * tb[vv].c * sgn * T;
            dW1B += ta[uu].c * tb[vv].dD1 * sgn * T;
            dW2B += ta[uu].c * tb[vv].dD2 * sgn * T;
          }
        Sa += gam * dWa;
        SD1A += gam * dW1A;
        SD2A += gam * dW2A;
        SD1B += gam * dW1B;
        SD2B += gam * dW2B;
      }
    }
    // a = 1/sqrt(2 (sA^2 + sB^2)), sigma = kappa / (sqrt(pi) gss): da/dgss_X = 2 a^3 sX^2 / gss_X
    atomicAdd(&gs[eA * XS_NPARAM + P_GSS], Sa * 2.0 * a * a * a * sA * sA / pA[P_GSS]);
    atomicAdd(&gs[eB * XS_NPARAM + P_GSS], Sa * 2.0 * a * a * a * sB * sB / pB[P_GSS]);
    if (hA) {
      atomicAdd(&gs[eA * XS_NPARAM + P_D1], SD1A);
      atomicAdd(&gs[eA * XS_NPARAM + P_D2], SD2A);
    }
    if (hB) {
      atomicAdd(&gs[eB * XS_NPARAM + P_D1], SD1B);
      atomicAdd(&gs[eB * XS_NPARAM + P_D2], SD2B);
    }
    // resonance H_AB = (beta_a + beta_b)/2 S_ab and its mirror: Tr(dH P) = 2 sum dH_AB P_AB
    double e[3];
    for (int c = 0; c < 3; ++c) e[c] = x[c] / Rd;
    double S[4][4], SzsA[4][4], SzsB[4][4], SzpA[4][4], SzpB[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) S[i][j] = SzsA[i][j] = SzsB[i][j] = SzpA[i][j] = SzpB[i][j] = 0.0;
    S[0][0] = kSKss * exp(-0.5 * (pA[P_ZS] + pB[P_ZS]) * Rd);
    SzsA[0][0] = SzsB[0][0] = -0.5 * Rd * S[0][0];
    if (hB) {
      const double vv = kSKsp * exp(-0.5 * (pA[P_ZS] + pB[P_ZP]) * Rd);
      for (int j = 0; j < 3; ++j) {
        S[0][1 + j] = -e[j] * vv;
        SzsA[0][1 + j] = SzpB[0][1 + j] = -0.5 * Rd * S[0][1 + j];
      }
    }
    if (hA) {
      const double vv = kSKsp * exp(-0.5 * (pB[P_ZS] + pA[P_ZP]) * Rd);
      for (int i = 0; i < 3; ++i) {
        S[1 + i][0] = e[i] * vv;
        SzsB[1 + i][0] = SzpA[1 + i][0] = -0.5 * Rd * S[1 + i][0];
      }
    }
    if (hA && hB) {
      const double kp = 0.5 * (pA[P_ZP] + pB[P_ZP]);
      const double ss = kSKppSigma * exp(-kp * Rd);
      const double pp = kSKppPi * exp(-kSKPiScale * kp * Rd);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const double ee = e[i] * e[j], dij = i == j ? 1.0 : 0.0;
          S[1 + i][1 + j] = -ee * ss + (dij - ee) * pp;
          // d/dzeta_p of either atom: dkp = 1/2
          const double dS = 0.5 * (ee * Rd * ss - (dij - ee) * kSKPiScale * Rd * pp);
          SzpA[1 + i][1 + j] = SzpB[1 + i][1 + j] = dS;
        }
    }
    const double bA[4] = {pA[P_BS], pA[P_BP], pA[P_BP], pA[P_BP]};
    const double bB[4] = {pB[P_BS], pB[P_BP], pB[P_BP], pB[P_BP]};
    double gbsA = 0.0, gbpA = 0.0, gbsB = 0.0, gbpB = 0.0, gzsA = 0.0, gzpA = 0.0, gzsB = 0.0, gzpB = 0.0;
    for (int i = 0; i < nA; ++i)
      for (int j = 0; j < nB; ++j) {
        const double w2 = 2.0 * Pab[i][j];   // both blocks of the symmetric P
        const double half = 0.5 * (bA[i] + bB[j]);
        if (i == 0) gbsA += 0.5 * S[i][j] * w2; else gbpA += 0.5 * S[i][j] * w2;
        if (j == 0) gbsB += 0.5 * S[i][j] * w2; else gbpB += 0.5 * S[i][j] * w2;
        gzsA += half * SzsA[i][j] * w2;
        gzsB += half * SzsB[i][j] * w2;
        gzpA += half * SzpA[i][j] * w2;
        gzpB += half * SzpB[i][j] * w2;
      }
    atomicAdd(&gs[eA * XS_NPARAM + P_BS], gbsA);
    atomicAdd(&gs[eB * XS_NPARAM + P_BS], gbsB);
    atomicAdd(&gs[eA * XS_NPARAM + P_ZS], gzsA);
    atomicAdd(&gs[eB * XS_NPARAM + P_ZS], gzsB);
    if (hA) {
      atomicAdd(&gs[eA * XS_NPARAM + P_BP], gbpA);
      atomicAdd(&gs[eA * XS_NPARAM + P_ZP], gzpA);
    }
    if (hB) {
      atomicAdd(&gs[eB * XS_NPARAM + P_BP], gbpB);
      atomicAdd(&gs[eB * XS_NPARAM + P_ZP], gzpB);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < XS_NELEM * XS_NPARAM; i += blockDim.x)
    if (gs[i] != 0.0) atomicAdd(&grad[i], gs[i]);
}

// one-centre (mu nu|lam sig) of a heavy atom for the parameter vector
// (gss, gsp, gpp, gp2, hsp) with hpp = (gpp - gp2)/2; a hydrogen has (ss|ss) = gss
__device__ double onec(int a, int b, int c, int d, const double* q) {
  const double gss = q[0], gsp = q[1], gpp = q[2], gp2 = q[3], hsp = q[4], hpp = 0.5 * (q[2] - q[3]);
  if (a == 0 && b == 0 && c == 0 && d == 0) return gss;
  if (a == b && c == d) {
    if (a == 0 || c == 0) return gsp;
    return a == c ? gpp : gp2;
  }
  if (a == 0 && c == 0 && b == d) return hsp;   // (s p|s p)
  if (a == 0 && d == 0 && b == c) return hsp;   // (s p|p s)
  if (b == 0 && c == 0 && a == d) return hsp;   // (p s|s p)
  if (b == 0 && d == 0 && a == c) return hsp;   // (p s|p s)
  if (a != b && a != 0 && b != 0 && ((a == c && b == d) || (a == d && b == c))) return hpp;
  return 0.0;
}

// per atom: U and the one-centre integral derivatives,
// <P, dG1(D/2)> + sum_Q <Q, dG1(Q)> with G1(Q)_mn = sum [2 (mn|ls) - (ml|ns)] Q_ls
__global__ void atom_grad_kernel(int natoms, int n, const int* __restrict__ ao_off, const int* __restrict__ nao,
                                 const int* __restrict__ elem, const double* __restrict__ P,
                                 const double* __restrict__ Dh, const double* __restrict__ R,
                                 const double* __restrict__ R2, double* __restrict__ grad) {
  const int A = blockIdx.x * blockDim.x + threadIdx.x;
  if (A >= natoms) return;
  const int e = elem[A], o = ao_off[A], na = nao[A];
  auto at = [&](const double* Q, int i, int j) { return Q[(size_t)(o + i) * n + o + j]; };
  atomicAdd(&grad[e * XS_NPARAM + P_USS], at(P, 0, 0));
  if (na == 4) {
    double s = 0.0;
    for (int i = 1; i < 4; ++i) s += at(P, i, i);
    atomicAdd(&grad[e * XS_NPARAM + P_UPP], s);
  }
  const int nk = na == 4 ? 5 : 1;
  for (int k = 0; k < nk; ++k) {
    double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    q[k] = 1.0;
    double acc = 0.0;
    for (int mu = 0; mu < na; ++mu)
      for (int nu = 0; nu < na; ++nu)
        for (int la = 0; la < na; ++la)
          for (int sg = 0; sg < na; ++sg) {
            const double coul = onec(mu, nu, la, sg, q), exch = onec(mu, la, nu, sg, q);
            if (coul == 0.0 && exch == 0.0) continue;
            acc += at(P, mu, nu) * (2.0 * coul - exch) * at(Dh, la, sg);
            acc += at(R, mu, nu) * (2.0 * coul - exch) * at(R, la, sg);
            if (R2) acc += at(R2, mu, nu) * (2.0 * coul - exch) * at(R2, la, sg);
          }
    atomicAdd(&grad[e * XS_NPARAM + P_GSS + k], acc);
  }
}

// Q = (R + sign R^T) / 2
__global__ void sym_part_kernel(int n, double sign, const double* __restrict__ R, double* __restrict__ Q) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = static_cast<int>(idx / n), j = static_cast<int>(idx % n);
  Q[idx] = 0.5 * (R[idx] + sign * R[(size_t)j * n + i]);
}

__global__ void sym_sub_kernel(int n, const double* __restrict__ Delta, const double* __restrict__ RZ,
                               double* __restrict__ P) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = static_cast<int>(idx / n), j = static_cast<int>(idx % n);
  P[idx] = Delta[idx] - 0.5 * (RZ[idx] + RZ[(size_t)j * n + i]);
}

__global__ void dot_partial_kernel(long long len, const double* __restrict__ a, const double* __restrict__ b,
                                   double* __restrict__ part) {
  __shared__ double red[8];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// z = r / de (Jacobi preconditioner of A+B)
__global__ void diag_solve_kernel(int o, int v, const double* __restrict__ eps, const double* __restrict__ r,
                                  double* __restrict__ z) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)o * v) return;
  const int i = static_cast<int>(idx / v), a = static_cast<int>(idx % v);
  z[idx] = r[idx] / (eps[o + a] - eps[i]);
}

__global__ void axpby_kernel(long long n, double alpha, const double* __restrict__ x, double beta, double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = alpha * x[i] + beta * y[i];
}

double dot(cudaStream_t s, long long len, const double* a, const double* b, DevBuf<double>& part) {
  const int blocks = static_cast<int>(std::min<long long>(256, (len + 255) / 256));
  part.ensure(blocks);
  dot_partial_kernel<<<blocks, 256, 0, s>>>(len, a, b, part.get());
  XS_CHECK_LAUNCH();
  std::vector<double> h(blocks);
  XS_CUDA(cudaMemcpyAsync(h.data(), part.get(), sizeof(double) * blocks, cudaMemcpyDeviceToHost, s));
  XS_CUDA(cudaStreamSynchronize(s));
  double t = 0.0;
  for (double x : h) t += x;
  return t;
}

}  // namespace

void parameter_gradient(Ctx& c, DevMol& m, int root, double* grad_host, int* cg_iterations) {
  cudaStream_t s = c.stream;
  const bool rpa = m.method == XS_TDHF;
  const int n = m.n, o = m.o, v = m.v;
  const long long ov = (long long)o * v, nn = (long long)n * n;
  const double* CT = m.CT.get();
  const double* CTocc = CT;
  const double* CTvir = CT + (size_t)o * n;
  // amplitudes: CIS X; TDHF U = X+Y and W = X-Y
  const double* Y1 = m.U.get() + (size_t)root * ov;
  const double* Y2 = rpa ? m.Wv.get() + (size_t)root * ov : nullptr;
  DevBuf<double> R(nn), R2(rpa ? nn : 1), Q(nn), GR(nn), Dl(nn), GD(nn), Dh(nn), tmp((size_t)n * std::max(o, v)),
      Gvv((size_t)v * v), Goo((size_t)o * o), T((size_t)std::max(o, v) * std::max(o, v)), L(ov), Z(ov), r(ov), zv(ov),
      p(ov), Ap(ov), Am(ov), RZ(nn), P(nn), pk((size_t)3 * m.np), grad((size_t)XS_NELEM * XS_NPARAM), part;
  DevBuf<double> ws;
  auto transition = [&](const double* Y, double* out) {   // C_occ Y C_vir^T
    gemm<double>(s, true, false, n, v, o, 1.0, CTocc, n, 0, Y, v, 0, 0.0, tmp.get(), v, 0, 1);
    gemm<double>(s, false, false, n, n, v, 1.0, tmp.get(), v, 0, CTvir, n, 0, 0.0, out, n, 0, 1);
  };
  // pair densities: CIS Q1 = R; TDHF Q1 = sym(R_U), Q2 = antisym(R_W)
  transition(Y1, rpa ? Q.get() : R.get());
  if (rpa) {
    sym_part_kernel<<<grid1(nn, 256), 256, 0, s>>>(n, 1.0, Q.get(), R.get());
    transition(Y2, Q.get());
    sym_part_kernel<<<grid1(nn, 256), 256, 0, s>>>(n, -1.0, Q.get(), R2.get());
    XS_CHECK_LAUNCH();
  }
  // Delta = C_vir T C_vir^T - C_occ T' C_occ^T, T = (Y1^T Y1 + Y2^T Y2) / w, T' = (Y1 Y1^T + Y2 Y2^T) / w
  const double wsc = rpa ? 0.5 : 1.0;
  gemm<double>(s, true, false, v, v, o, wsc, Y1, v, 0, Y1, v, 0, 0.0, T.get(), v, 0, 1);
  if (rpa) gemm<double>(s, true, false, v, v, o, wsc, Y2, v, 0, Y2, v, 0, 1.0, T.get(), v, 0, 1);
  gemm<double>(s, true, false, n, v, v, 1.0, CTvir, n, 0, T.get(), v, 0, 0.0, tmp.get(), v, 0, 1);
  gemm<double>(s, false, false, n, n, v, 1.0, tmp.get(), v, 0, CTvir, n, 0, 0.0, Dl.get(), n, 0, 1);
  gemm<double>(s, false, true, o, o, v, wsc, Y1, v, 0, Y1, v, 0, 0.0, T.get(), o, 0, 1);
  if (rpa) gemm<double>(s, false, true, o, o, v, wsc, Y2, v, 0, Y2, v, 0, 1.0, T.get(), o, 0, 1);
  gemm<double>(s, true, false, n, o, o, 1.0, CTocc, n, 0, T.get(), o, 0, 0.0, tmp.get(), o, 0, 1);
  gemm<double>(s, false, false, n, n, o, -1.0, tmp.get(), o, 0, CTocc, n, 0, 1.0, Dl.get(), n, 0, 1);
  gemm<double>(s, true, false, n, n, o, 1.0, CTocc, n, 0, CTocc, n, 0, 0.0, Dh.get(), n, 0, 1);
  gbuild<double>(s, m, c.d_par.get(), G_CIS, 1, Dl.get(), GD.get(), nullptr, ws);
  // L = sum_(Y, Q) 2 (Y G_vv^T - G_oo^T Y) + 2 C_occ^T G(Delta) C_vir
  XS_CUDA(cudaMemsetAsync(L.get(), 0, sizeof(double) * ov, s));
  for (int t = 0; t < (rpa ? 2 : 1); ++t) {
    const double* Yt = t == 0 ? Y1 : Y2;
    gbuild<double>(s, m, c.d_par.get(), G_CIS, 1, t == 0 ? R.get() : R2.get(), GR.get(), nullptr, ws);
    gemm<double>(s, false, true, n, v, n, 1.0, GR.get(), n, 0, CTvir, n, 0, 0.0, tmp.get(), v, 0, 1);    // G C_vir
    gemm<double>(s, false, false, v, v, n, 1.0, CTvir, n, 0, tmp.get(), v, 0, 0.0, Gvv.get(), v, 0, 1);    // G_vv
    gemm<double>(s, false, true, n, o, n, 1.0, GR.get(), n, 0, CTocc, n, 0, 0.0, tmp.get(), o, 0, 1);     // G C_occ
    gemm<double>(s, false, false, o, o, n, 1.0, CTocc, n, 0, tmp.get(), o, 0, 0.0, Goo.get(), o, 0, 1);    // G_oo
    gemm<double>(s, false, true, o, v, v, 2.0, Yt, v, 0, Gvv.get(), v, 0, 1.0, L.get(), v, 0, 1);
    gemm<double>(s, true, false, o, v, o, -2.0, Goo.get(), o, 0, Yt, v, 0, 1.0, L.get(), v, 0, 1);
  }
  gemm<double>(s, false, true, n, v, n, 1.0, GD.get(), n, 0, CTvir, n, 0, 0.0, tmp.get(), v, 0, 1);       // G(Delta) C_vir
  gemm<double>(s, false, false, o, v, n, 2.0, CTocc, n, 0, tmp.get(), v, 0, 1.0, L.get(), v, 0, 1);
  // (A+B) Z = L by preconditioned conjugate gradients on the float64 products
  const int gb = static_cast<int>((ov + 255) / 256);
  diag_solve_kernel<<<gb, 256, 0, s>>>(o, v, m.eps.get(), L.get(), Z.get());
  XS_CHECK_LAUNCH();
  products(c, m, XS_TDHF, XS_FP64, 1, Z.get(), Ap.get(), Am.get(), false);
  XS_CUDA(cudaMemcpyAsync(r.get(), L.get(), sizeof(double) * ov, cudaMemcpyDeviceToDevice, s));
  axpby_kernel<<<gb, 256, 0, s>>>(ov, -1.0, Ap.get(), 1.0, r.get());
  XS_CHECK_LAUNCH();
  diag_solve_kernel<<<gb, 256, 0, s>>>(o, v, m.eps.get(), r.get(), zv.get());
  XS_CHECK_LAUNCH();
  XS_CUDA(cudaMemcpyAsync(p.get(), zv.get(), sizeof(double) * ov, cudaMemcpyDeviceToDevice, s));
  const double bnorm = std::sqrt(dot(s, ov, L.get(), L.get(), part));
  double rz = dot(s, ov, r.get(), zv.get(), part);
  int it = 0;
  for (; it < 500; ++it) {
    const double rn = std::sqrt(dot(s, ov, r.get(), r.get(), part));
    if (!(rn > 1e-11 * bnorm)) break;
    products(c, m, XS_TDHF, XS_FP64, 1, p.get(), Ap.get(), Am.get(), false);
    const double pAp = dot(s, ov, p.get(), Ap.get(), part);
    if (!(pAp > 0.0)) throw Error(XS_EUNSTABLE, "A + B is not positive definite: unstable reference");
    const double alpha = rz / pAp;
    axpby_kernel<<<gb, 256, 0, s>>>(ov, alpha, p.get(), 1.0, Z.get());
    axpby_kernel<<<gb, 256, 0, s>>>(ov, -alpha, Ap.get(), 1.0, r.get());
    XS_CHECK_LAUNCH();
    diag_solve_kernel<<<gb, 256, 0, s>>>(o, v, m.eps.get(), r.get(), zv.get());
    XS_CHECK_LAUNCH();
    const double rz_new = dot(s, ov, r.get(), zv.get(), part);
    axpby_kernel<<<gb, 256, 0, s>>>(ov, 1.0, zv.get(), rz_new / rz, p.get());
    XS_CHECK_LAUNCH();
    rz = rz_new;
  }
  if (it >= 500) throw Error(XS_ENOCONV, "adjoint (A+B) Z = L solve did not converge");
  if (cg_iterations) *cg_iterations = it;
  // relaxed difference density P = Delta - sym(C_occ Z C_vir^T)
  gemm<double>(s, true, false, n, v, o, 1.0, CTocc, n, 0, Z.get(), v, 0, 0.0, tmp.get(), v, 0, 1);
  gemm<double>(s, false, false, n, n, v, 1.0, tmp.get(), v, 0, CTvir, n, 0, 0.0, RZ.get(), n, 0, 1);
  sym_sub_kernel<<<grid1(nn, 256), 256, 0, s>>>(n, Dl.get(), RZ.get(), P.get());
  XS_CHECK_LAUNCH();
  // contractions with the parameter derivatives
  XS_CUDA(cudaMemsetAsync(grad.get(), 0, sizeof(double) * XS_NELEM * XS_NPARAM, s));
  const int na = m.L.natoms;
  pack_kernel<<<(na + 127) / 128, 128, 0, s>>>(na, n, m.atom_ao_off.get(), m.atom_nao.get(), m.atom_prod_off.get(),
                                               P.get(), Dh.get(), R.get(), pk.get());
  XS_CHECK_LAUNCH();
  const long long npair = (long long)na * (na - 1) / 2;
  if (npair > 0) {
    pair_grad_kernel<<<grid1(npair, 128), 128, 0, s>>>(na, n, m.xyz.get(), m.atom_ao_off.get(), m.atom_nao.get(),
                                                       m.atom_prod_off.get(), m.atom_elem.get(), c.d_par.get(), P.get(),
                                                       Dh.get(), R.get(), rpa ? R2.get() : nullptr, pk.get(),
                                                       grad.get());
    XS_CHECK_LAUNCH();
  }
  atom_grad_kernel<<<(na + 127) / 128, 128, 0, s>>>(na, n, m.atom_ao_off.get(), m.atom_nao.get(), m.atom_elem.get(),
                                                    P.get(), Dh.get(), R.get(), rpa ? R2.get() : nullptr,
                                                    grad.get());
  XS_CHECK_LAUNCH();
  XS_CUDA(cudaMemcpyAsync(grad_host, grad.get(), sizeof(double) * XS_NELEM * XS_NPARAM, cudaMemcpyDeviceToHost, s));
  XS_CUDA(cudaStreamSynchronize(s));
}

}  // namespace xs
