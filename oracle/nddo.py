"""Synthetic NDDO model (oracle side; test infrastructure only).

The paper (Section "Ground-state wavefunction calculation") uses a minimal
valence basis, drops three- and four-centre integrals, keeps two-centre
integrals as classical multipole interactions and takes one-centre integrals
as tabulated parameters.  It prints neither the AM1 parameters nor the
multipole formulas, so this module implements a stated model of the same
structure:

* AO order = atom order; a heavy atom (C, N, O) carries s, px, py, pz, an H
  atom carries s.
* On-atom AO products (mu <= nu) are charge densities built from a unit
  Gaussian G_A of width sigma_A = kappa / (sqrt(pi) gss_A):
  rho_ss = G, rho_{s p_i} = -D1 d_i G, rho_{p_i p_j} = delta_ij G + D2^2 d_i d_j G.
* (mu nu | lam sig) for mu nu on A and lam sig on B is the Coulomb energy of
  the two densities: sum of c_alpha c_beta (-1)^|beta| d^(alpha+beta) Phi(R),
  R = R_B - R_A, Phi(R) = kappa erf(a R) / R, a = 1/sqrt(2 (sA^2 + sB^2)).
* One-centre integrals: gss, gsp, gpp, gp2, hsp and hpp = (gpp - gp2)/2.
* Core Hamiltonian: U on the diagonal, core attraction -Z_B (mu nu|s_B s_B),
  resonance (beta_mu + beta_lam)/2 * S_mu lam with Slater-Koster overlaps
  S_x(R) = a_x exp(-k_x R).

Energies are in eV and lengths in Angstrom.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

KAPPA = 14.399645          # e^2 / (4 pi eps0) in eV * Angstrom (CODATA 2018)
HARTREE_EV = 27.211386245988
BOHR_A = 0.529177210903

CORE_CHARGE = {1: 1.0, 6: 4.0, 7: 5.0, 8: 6.0}
ELEMENT_ROW = {1: 0, 6: 1, 7: 2, 8: 3}

# Slater-Koster radial model S_x(R) = a_x exp(-k_x R).  k_x is the mean of the
# two atoms' exponents for the orbitals involved (times 1.3 for pp-pi).
SK_PREFACTOR = {"ss_sigma": 2.0, "sp_sigma": 2.4, "pp_sigma": 1.9, "pp_pi": 1.6}
SK_PI_EXPONENT_SCALE = 1.3

# on-atom product index for mu <= nu, AO order (s, px, py, pz)
HEAVY_PAIRS = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]
PROD_INDEX = np.full((4, 4), -1, dtype=np.int64)
for _k, (_m, _n) in enumerate(HEAVY_PAIRS):
    PROD_INDEX[_m, _n] = _k
    PROD_INDEX[_n, _m] = _k


class Molecule:
    """Atoms, AO layout and parameters of one molecule."""

    def __init__(self, Z, xyz, params):
        self.Z = np.asarray(Z, dtype=np.int64)
        self.xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.params = params
        self.natoms = len(self.Z)
        self.nao_atom = np.array([1 if z == 1 else 4 for z in self.Z], dtype=np.int64)
        self.ao_offset = np.concatenate([[0], np.cumsum(self.nao_atom)[:-1]]).astype(np.int64)
        self.nao = int(self.nao_atom.sum())
        nel = int(sum(CORE_CHARGE[int(z)] for z in self.Z))
        if nel % 2:
            raise ValueError("odd electron count: only closed shells are defined")
        self.nocc = nel // 2
        self.nvir = self.nao - self.nocc
        self.ao_atom = np.repeat(np.arange(self.natoms), self.nao_atom)

    def p(self, a, field):
        return self.params[int(self.Z[a])][field]

    def sigma(self, a):
        return KAPPA / (math.sqrt(math.pi) * self.p(a, "gss"))


# ---------------------------------------------------------------------------
# radial functions of Phi(R) = kappa erf(aR)/R and Cartesian derivatives

def radial_g(R, a, nmax=4):
    """g_n(R) = ((1/R) d/dR)^n Phi(R) for n = 0..nmax, Phi = kappa erf(aR)/R.

    With b_0 = erf(aR)/R and b_n = [(2n-1) b_{n-1} - (2a^2)^n/(a sqrt(pi))
    exp(-a^2 R^2)] / R^2 one has g_n = (-1)^n kappa b_n (the screened
    multipole recursion with erf in place of erfc).
    """
    R = np.asarray(R, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    from scipy.special import erf

    ex = np.exp(-(a * R) ** 2)
    b = [erf(a * R) / R]
    for n in range(1, nmax + 1):
        b.append(((2 * n - 1) * b[n - 1] - (2 * a * a) ** n / (a * math.sqrt(math.pi)) * ex) / (R * R))
    return [((-1) ** n) * KAPPA * b[n] for n in range(nmax + 1)]


def _matchings(m):
    """All partial matchings of positions 0..m-1 as (pairs, singles)."""
    positions = list(range(m))
    all_pairs = list(itertools.combinations(positions, 2))
    out = []
    for r in range(0, m // 2 + 1):
        for combo in itertools.combinations(all_pairs, r):
            used = [p for pr in combo for p in pr]
            if len(set(used)) != len(used):
                continue
            singles = [p for p in positions if p not in used]
            out.append((list(combo), singles))
    return out


def deriv_phi(indices, x, g):
    """d/dR_{i1} ... d/dR_{im} Phi(R) for radial Phi, m <= 4.

    Sum over partial matchings P of the index list: product of delta over
    the pairs of P, product of x over the unpaired indices, times g_{m-|P|}.
    ``x`` has shape (3, P) (components of R), ``g`` is radial_g's list.
    """
    m = len(indices)
    total = np.zeros_like(g[0])
    for pairs, singles in _matchings(m):
        if any(indices[i] != indices[j] for i, j in pairs):
            continue
        term = g[m - len(pairs)].copy()
        for s in singles:
            term = term * x[indices[s]]
        total = total + term
    return total


def two_centre_block(molA_params, molB_params, RA, RB):
    """(p|q) for products p on atom A and q on atom B, vectorised over pairs.

    molA_params / molB_params: dict with 'heavy' (bool), 'D1', 'D2', 'sigma'
    (arrays over the pairs of one class); RA, RB: (P, 3) coordinates.
    Returns an array (P, npA, npB).
    """
    Rv = (np.asarray(RB) - np.asarray(RA)).T  # (3, P)
    R = np.sqrt(Rv[0] ** 2 + Rv[1] ** 2 + Rv[2] ** 2)
    a = 1.0 / np.sqrt(2.0 * (molA_params["sigma"] ** 2 + molB_params["sigma"] ** 2))
    g = radial_g(R, a, 4)
    P = R.shape[0]
    npA = 10 if molA_params["heavy"] else 1
    npB = 10 if molB_params["heavy"] else 1
    W = np.zeros((P, npA, npB))
    # coefficients differ per pair (D1, D2 per atom): expand symbolically with
    # per-pair coefficient arrays
    expA = _product_terms(molA_params)
    expB = _product_terms(molB_params)
    cache = {}
    for p in range(npA):
        for q in range(npB):
            acc = np.zeros(P)
            for ia, ca in expA[p]:
                for ib, cb in expB[q]:
                    key = tuple(sorted(ia + ib))
                    if key not in cache:
                        cache[key] = deriv_phi(list(key), Rv, g)
                    acc = acc + ca * cb * ((-1) ** len(ib)) * cache[key]
            W[:, p, q] = acc
    return W


def _product_terms(pp):
    """Per product: list of (index tuple, coefficient array over pairs)."""
    if not pp["heavy"]:
        return [[((), 1.0)]]
    D1 = pp["D1"]
    D2 = pp["D2"]
    out = []
    for (mu, nu) in HEAVY_PAIRS:
        if mu == 0 and nu == 0:
            out.append([((), 1.0)])
        elif mu == 0:
            out.append([((nu - 1,), -D1)])
        else:
            i, j = mu - 1, nu - 1
            terms = []
            if i == j:
                terms.append(((), 1.0))
            terms.append(((i, j), D2 * D2))
            out.append(terms)
    return out


def one_centre_tensor(p, heavy):
    """(mu nu | lam sig) with all four AOs on one atom, shape (n, n, n, n)."""
    if not heavy:
        t = np.zeros((1, 1, 1, 1))
        t[0, 0, 0, 0] = p["gss"]
        return t
    gss, gsp, gpp, gp2, hsp = p["gss"], p["gsp"], p["gpp"], p["gp2"], p["hsp"]
    hpp = 0.5 * (gpp - gp2)
    t = np.zeros((4, 4, 4, 4))
    t[0, 0, 0, 0] = gss
    for i in range(1, 4):
        t[0, 0, i, i] = t[i, i, 0, 0] = gsp
        t[i, i, i, i] = gpp
        t[0, i, 0, i] = t[0, i, i, 0] = t[i, 0, 0, i] = t[i, 0, i, 0] = hsp
        for j in range(1, 4):
            if i != j:
                t[i, i, j, j] = gp2
                t[i, j, i, j] = t[i, j, j, i] = hpp
    return t


class Integrals:
    """Two-centre blocks of a molecule, grouped by the AO counts of the pair.

    For every unordered atom pair A < B the block w[(mu nu | lam sig)] with
    mu, nu on A and lam, sig on B is stored as a 4-index array (nA, nA, nB,
    nB).  Pairs with the same (nA, nB) are stacked in one class.
    """

    def __init__(self, mol: Molecule):
        self.mol = mol
        nat = mol.natoms
        iu, ju = np.triu_indices(nat, k=1)
        heavy = mol.nao_atom == 4
        self.classes = {}
        self.pair_index = {}
        for hA in (True, False):
            for hB in (True, False):
                sel = (heavy[iu] == hA) & (heavy[ju] == hB)
                A = iu[sel]
                B = ju[sel]
                if A.size == 0:
                    continue
                pa = dict(heavy=hA, D1=np.array([mol.p(x, "D1") for x in A]),
                          D2=np.array([mol.p(x, "D2") for x in A]),
                          sigma=np.array([mol.sigma(x) for x in A]))
                pb = dict(heavy=hB, D1=np.array([mol.p(x, "D1") for x in B]),
                          D2=np.array([mol.p(x, "D2") for x in B]),
                          sigma=np.array([mol.sigma(x) for x in B]))
                W = two_centre_block(pa, pb, mol.xyz[A], mol.xyz[B])
                nA = 4 if hA else 1
                nB = 4 if hB else 1
                w4 = _expand_w(W, nA, nB)
                self.classes[(nA, nB)] = (A, B, W, w4)
                for k, (a, b) in enumerate(zip(A.tolist(), B.tolist())):
                    self.pair_index[(a, b)] = ((nA, nB), k)
        self.one_centre = [one_centre_tensor(mol.params[int(z)], z != 1) for z in mol.Z]

    def pair_block(self, A, B):
        """(mu nu | lam sig) for atoms A != B as an (nA, nA, nB, nB) array."""
        if A > B:
            return np.transpose(self.pair_block(B, A), (2, 3, 0, 1))
        cls, k = self.pair_index[(int(A), int(B))]
        return self.classes[cls][3][k]


def _expand_w(W, nA, nB):
    if nA == 4:
        ia = PROD_INDEX
    else:
        ia = np.zeros((1, 1), dtype=np.int64)
    if nB == 4:
        ib = PROD_INDEX
    else:
        ib = np.zeros((1, 1), dtype=np.int64)
    return W[:, ia[:, :, None, None], ib[None, None, :, :]]


def full_eri(mol: Molecule, ints: Integrals):
    """Dense (mu nu | lam sig) over all n AOs -- tiny molecules only (n^4)."""
    n = mol.nao
    eri = np.zeros((n, n, n, n))
    off = mol.ao_offset
    na = mol.nao_atom
    for A in range(mol.natoms):
        sA = slice(off[A], off[A] + na[A])
        eri[sA, sA, sA, sA] = ints.one_centre[A]
        for B in range(mol.natoms):
            if B == A:
                continue
            sB = slice(off[B], off[B] + na[B])
            eri[sA, sA, sB, sB] = ints.pair_block(A, B)
    return eri


# ---------------------------------------------------------------------------
# one-electron part

def sk_overlap_block(mol: Molecule, A, B):
    """Overlap S between the AOs of atoms A != B (Slater-Koster two-centre form).

    With e = (R_B - R_A)/|R_B - R_A|:
      S(s_A, s_B)   = S_ss
      S(s_A, p_Bj)  = -e_j S_sp(s on A, p on B)
      S(p_Ai, s_B)  = +e_i S_sp(s on B, p on A)
      S(p_Ai, p_Bj) = -e_i e_j S_pp_sigma + (delta_ij - e_i e_j) S_pp_pi
    where every radial S_x(R) > 0 is the overlap of the lobes that point at
    each other.
    """
    Rv = mol.xyz[B] - mol.xyz[A]
    R = math.sqrt(float(Rv @ Rv))
    e = Rv / R
    zsA, zpA = mol.p(A, "zeta_s"), mol.p(A, "zeta_p")
    zsB, zpB = mol.p(B, "zeta_s"), mol.p(B, "zeta_p")
    nA, nB = int(mol.nao_atom[A]), int(mol.nao_atom[B])
    S = np.zeros((nA, nB))
    S[0, 0] = SK_PREFACTOR["ss_sigma"] * math.exp(-0.5 * (zsA + zsB) * R)
    if nB == 4:
        s_sp = SK_PREFACTOR["sp_sigma"] * math.exp(-0.5 * (zsA + zpB) * R)
        for j in range(3):
            S[0, 1 + j] = -e[j] * s_sp
    if nA == 4:
        s_ps = SK_PREFACTOR["sp_sigma"] * math.exp(-0.5 * (zsB + zpA) * R)
        for i in range(3):
            S[1 + i, 0] = e[i] * s_ps
    if nA == 4 and nB == 4:
        kp = 0.5 * (zpA + zpB)
        s_sig = SK_PREFACTOR["pp_sigma"] * math.exp(-kp * R)
        s_pi = SK_PREFACTOR["pp_pi"] * math.exp(-SK_PI_EXPONENT_SCALE * kp * R)
        for i in range(3):
            for j in range(3):
                S[1 + i, 1 + j] = -e[i] * e[j] * s_sig + ((1.0 if i == j else 0.0) - e[i] * e[j]) * s_pi
    return S


def core_hamiltonian(mol: Molecule, ints: Integrals):
    """H_core: U_mu delta - sum_{B != A} Z_B (mu nu | s_B s_B) on the diagonal
    blocks, (beta_mu + beta_lam)/2 * S_mu lam on the off-diagonal blocks."""
    n = mol.nao
    H = np.zeros((n, n))
    off = mol.ao_offset
    na = mol.nao_atom
    def beta(a):
        return np.array([mol.p(a, "beta_s")] + [mol.p(a, "beta_p")] * (na[a] - 1))

    for A in range(mol.natoms):
        sA = slice(off[A], off[A] + na[A])
        U = [mol.p(A, "Uss")] + [mol.p(A, "Upp")] * (na[A] - 1)
        H[sA, sA] += np.diag(U)
    for A in range(mol.natoms):
        sA = slice(off[A], off[A] + na[A])
        for B in range(A + 1, mol.natoms):
            sB = slice(off[B], off[B] + na[B])
            w = ints.pair_block(A, B)  # (mu nu | lam sig), mu nu on A, lam sig on B
            H[sA, sA] -= CORE_CHARGE[int(mol.Z[B])] * w[:, :, 0, 0]
            H[sB, sB] -= CORE_CHARGE[int(mol.Z[A])] * w[0, 0, :, :]
            S = sk_overlap_block(mol, A, B)
            H[sA, sB] = 0.5 * (beta(A)[:, None] + beta(B)[None, :]) * S
            H[sB, sA] = H[sA, sB].T
    return H


def dipole_integrals(mol: Molecule):
    """<mu| r |nu> in Angstrom, shape (3, n, n): R_A on the diagonal plus the
    one-centre s-p term <s|r_i|p_i> = D1 (the dipole of rho_{s p_i})."""
    n = mol.nao
    d = np.zeros((3, n, n))
    for A in range(mol.natoms):
        o = mol.ao_offset[A]
        for mu in range(mol.nao_atom[A]):
            d[:, o + mu, o + mu] = mol.xyz[A]
        if mol.nao_atom[A] == 4:
            D1 = mol.p(A, "D1")
            for i in range(3):
                d[i, o, o + 1 + i] = D1
                d[i, o + 1 + i, o] = D1
    return d
