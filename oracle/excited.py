"""CIS and TDHF/RPA excitations (oracle; test infrastructure only).

Paper, Section "TDHF and CIS equations":
  Eq. rpa_eqn        [[A, B], [B, A]] [X; Y] = omega diag(I, -I) [X; Y]
  Eq. A_matrix_elem  A_ia,jb = (eps_a - eps_i) d_ij d_ab + (ia|jb) - (ij|ab),
                     B_ia,jb = (ia|jb) - (ib|ja)   ("spin indices omitted")
  Eq. cis_eqn        A X = omega X (B = 0, Tamm-Dancoff)
Section "GPU Implementation":
  Eq. cis_matrix_vector  (A V)_ia = (eps_a - eps_i) V_ia + sum C_mu,i Ft_mu,nu C_nu,a
  Eq. ftilde             Ft = sum [(mu nu|lam sig) - (mu lam|nu sig)] R_lam sig,
                         R = C_occ V C_vir^T
  Coulomb with the symmetrised R, exchange called with the symmetrised and
  the antisymmetrised R.

Reading of the omitted spin factors (the paper validates against ORCA's
closed-shell singlets): singlet spin adaptation,
  A = d eps + 2 (ia|jb) - (ij|ab),   B = 2 (ia|jb) - (ib|ja).
Then with J(R), K(R) of ``scf.coulomb_exchange``:
  A X       = d eps X + C_occ^T [2 J(R) - K(R)] C_vir
  (A + B) X = d eps X + C_occ^T [4 J(Rs) - 2 K(Rs)] C_vir
  (A - B) X = d eps X - C_occ^T [2 K(Ra)] C_vir
with Rs, Ra the symmetric and antisymmetric parts of R.

Amplitude layout: X[i, a] with i over occupied and a over virtual orbitals;
flattened index ia = i * nvir + a.
"""
from __future__ import annotations

import numpy as np

from .nddo import BOHR_A, HARTREE_EV, dipole_integrals
from .scf import coulomb_exchange

SQRT2 = np.sqrt(2.0)


# ---------------------------------------------------------------------------
# the A*V product through the AO transition density (Eqs. cis_matrix_vector, ftilde)

def transition_density(C, nocc, X):
    """R = C_occ X C_vir^T for one amplitude matrix X (nocc x nvir)."""
    return C[:, :nocc] @ X @ C[:, nocc:].T


def g_cis(mol, ints, R):
    J, K = coulomb_exchange(mol, ints, R)
    return 2.0 * J - K


def g_plus(mol, ints, R):
    Rs = 0.5 * (R + R.T)
    J, K = coulomb_exchange(mol, ints, Rs)
    return 4.0 * J - 2.0 * K


def g_minus(mol, ints, R):
    Ra = 0.5 * (R - R.T)
    _, K = coulomb_exchange(mol, ints, Ra)
    return -2.0 * K


# Triplet excitations (not computed in the paper, which treats closed-shell
# singlets; the spin-adapted triplet combinations are the textbook ones, e.g.
# Dreuw and Head-Gordon, Chem. Rev. 105, 4009 (2005)): the Coulomb-type
# 2(ia|jb) terms drop out, A_T = de - (ij|ab), B_T = -(ib|ja).  Through the AO
# transition density: A_T X uses -K(R), (A+B)_T X uses -2K(R_s), and
# (A-B)_T = (A-B) (the same -2K(R_a) as the singlet).

def g_cis_triplet(mol, ints, R):
    _, K = coulomb_exchange(mol, ints, R)
    return -K


def g_plus_triplet(mol, ints, R):
    Rs = 0.5 * (R + R.T)
    _, K = coulomb_exchange(mol, ints, Rs)
    return -2.0 * K


def delta_eps(eps, nocc):
    """(eps_a - eps_i) as an (nocc, nvir) matrix."""
    return eps[None, nocc:] - eps[:nocc, None]


def apply_kind(mol, ints, C, eps, nocc, X, kind):
    """Products for a stack of amplitude matrices X (k, nocc, nvir).

    kind: 'A' (CIS), 'ApB' (A + B), 'AmB' (A - B), their triplet forms
    'A_T', 'ApB_T', 'AmB_T' (the last equal to 'AmB'), or 'G' (returns the
    AO matrix G_CIS(R) for each R = X given directly as an n x n matrix).
    """
    X = np.asarray(X, dtype=np.float64)
    if kind == "G":
        return np.stack([g_cis(mol, ints, R) for R in X])
    de = delta_eps(eps, nocc)
    Co, Cv = C[:, :nocc], C[:, nocc:]
    out = np.empty_like(X)
    for k in range(X.shape[0]):
        R = transition_density(C, nocc, X[k])
        if kind == "A":
            G = g_cis(mol, ints, R)
        elif kind == "ApB":
            G = g_plus(mol, ints, R)
        elif kind in ("AmB", "AmB_T"):
            G = g_minus(mol, ints, R)
        elif kind == "A_T":
            G = g_cis_triplet(mol, ints, R)
        elif kind == "ApB_T":
            G = g_plus_triplet(mol, ints, R)
        else:
            raise ValueError(kind)
        out[k] = de * X[k] + Co.T @ G @ Cv
    return out


# ---------------------------------------------------------------------------
# explicit matrices (tiny molecules only)

def mo_eri(eri, C):
    return np.einsum("mnls,mp,nq,lr,st->pqrt", eri, C, C, C, C, optimize=True)


def explicit_AB(eps, C, nocc, eri):
    """Singlet A and B as (ov, ov) matrices from the dense AO integrals."""
    n = C.shape[0]
    o, v = nocc, n - nocc
    mo = mo_eri(eri, C)
    ov_ov = mo[:o, o:, :o, o:]                       # (ia|jb) as [i, a, j, b]
    oo_vv = mo[:o, :o, o:, o:].transpose(0, 2, 1, 3)  # (ij|ab) as [i, a, j, b]
    ib_ja = ov_ov.transpose(0, 3, 2, 1)              # (ib|ja) as [i, a, j, b]
    de = delta_eps(eps, nocc).reshape(-1)
    A = np.diag(de) + (2.0 * ov_ov - oo_vv).reshape(o * v, o * v)
    B = (2.0 * ov_ov - ib_ja).reshape(o * v, o * v)
    return A, B


def explicit_AB_triplet(eps, C, nocc, eri):
    """Triplet A and B as (ov, ov) matrices: A_T = de - (ij|ab), B_T = -(ib|ja)."""
    n = C.shape[0]
    o, v = nocc, n - nocc
    mo = mo_eri(eri, C)
    ov_ov = mo[:o, o:, :o, o:]
    oo_vv = mo[:o, :o, o:, o:].transpose(0, 2, 1, 3)
    ib_ja = ov_ov.transpose(0, 3, 2, 1)
    de = delta_eps(eps, nocc).reshape(-1)
    A = np.diag(de) - oo_vv.reshape(o * v, o * v)
    B = -ib_ja.reshape(o * v, o * v)
    return A, B


def cis_bruteforce(A, k):
    w, V = np.linalg.eigh(A)
    return w[:k], V[:, :k]


def rpa_bruteforce(A, B, k):
    """Lowest k RPA roots from M = (A-B)^(1/2) (A+B) (A-B)^(1/2).

    Returns omega, U = X+Y and W = X-Y (columns), normalised U.W = 1.
    Raises LinAlgError when A - B is not positive definite (unstable
    reference).
    """
    AmB = A - B
    ApB = A + B
    np.linalg.cholesky(AmB)
    lam, Q = np.linalg.eigh(AmB)
    S = (Q * np.sqrt(lam)) @ Q.T
    Si = (Q / np.sqrt(lam)) @ Q.T
    M = S @ ApB @ S
    w2, Z = np.linalg.eigh(0.5 * (M + M.T))
    w2, Z = w2[:k], Z[:, :k]
    omega = np.sqrt(w2)
    U = S @ Z / np.sqrt(omega)
    W = Si @ Z * np.sqrt(omega)
    return omega, U, W


def rpa_full_spectrum(A, B):
    """All eigenvalues of the non-Hermitian [[A, B], [-B, -A]] (Eq. rpa_eqn)."""
    top = np.hstack([A, B])
    bot = np.hstack([-B, -A])
    return np.linalg.eigvals(np.vstack([top, bot]))


# ---------------------------------------------------------------------------
# Davidson (the paper's batched steps 1-6 for one molecule)

def _guess(diag, nguess):
    order = np.argsort(diag, kind="stable")  # ties: lower flattened index (i, then a) first
    V = np.zeros((diag.size, nguess))
    V[order[:nguess], np.arange(nguess)] = 1.0
    return V


def _precondition(r, theta, diag):
    denom = theta - diag
    small = np.abs(denom) < 1e-4
    denom = np.where(small, np.where(denom < 0, -1e-4, 1e-4), denom)
    return r / denom


def _orthonormalise_new(V, T, drop=1e-8):
    """Classical Gram-Schmidt, twice, of the columns of T against V and each other."""
    kept = []
    for t in T.T:
        t = t / np.linalg.norm(t)
        for _ in range(2):
            t = t - V @ (V.T @ t)
            for q in kept:
                t = t - q * (q @ t)
        nrm = np.linalg.norm(t)
        if nrm >= drop:
            kept.append(t / nrm)
    if not kept:
        return np.zeros((V.shape[0], 0))
    return np.stack(kept, axis=1)


def davidson_cis(apply, diag, k, *, tol=1e-6, max_iter=200, max_sub=None, nguess=None):
    """Lowest k eigenpairs of the symmetric A from products apply(V) only.

    Steps (paper, Section "GPU Implementation", steps 1-6): orthonormal
    start V; AV; a = V^T A V, diagonalise, keep the lowest k; X = V x;
    r = AX - omega X, converged when every ||r||_2 <= tol; precondition the
    unconverged residuals by (omega - d eps)^-1 (denominator clamped to
    1e-4 eV); orthonormalise against V (Gram-Schmidt twice), append, repeat.
    When V would exceed max_sub columns it collapses to the 2k lowest Ritz
    vectors.
    Guess: unit vectors on the min(ov, 2k) lowest d eps.
    """
    ov = diag.size
    nguess = min(ov, 2 * k) if nguess is None else min(ov, nguess)
    max_sub = max_sub or min(ov, 40 * k)
    V = _guess(diag, nguess)
    AV = apply(V)
    n_products = V.shape[1]
    for it in range(1, max_iter + 1):
        a = V.T @ AV
        a = 0.5 * (a + a.T)
        theta, s = np.linalg.eigh(a)
        kk = min(k, theta.size)
        X = V @ s[:, :kk]
        AX = AV @ s[:, :kk]
        r = AX - X * theta[:kk]
        norms = np.linalg.norm(r, axis=0)
        if np.all(norms <= tol):
            return dict(omega=theta[:kk], X=X, residual=norms, iterations=it, products=n_products,
                        converged=True)
        T = np.stack([_precondition(r[:, j], theta[j], diag) for j in range(kk) if norms[j] > tol],
                     axis=1)
        if V.shape[1] + T.shape[1] > max_sub:
            keep = min(2 * k, theta.size)
            V = V @ s[:, :keep]
            AV = AV @ s[:, :keep]
        Tn = _orthonormalise_new(V, T)
        if Tn.shape[1] == 0:
            break
        V = np.hstack([V, Tn])
        AV = np.hstack([AV, apply(Tn)])
        n_products += Tn.shape[1]
    return dict(omega=theta[:kk], X=X, residual=norms, iterations=it, products=n_products,
                converged=False)


def davidson_rpa(apply_pm, diag, k, *, tol=1e-6, max_iter=200, max_sub=None, nguess=None):
    """Lowest k RPA roots by the symmetric subspace form of Stratmann,
    Scuseria and Frisch (J. Chem. Phys. 109, 8218 (1998)); the paper names
    Davidson for RPA without giving the variant.

    apply_pm(V) returns ((A+B) V, (A-B) V).  In the orthonormal space V:
    a+ = V^T (A+B) V, a- = V^T (A-B) V, a- = L L^T, L^T a+ L z = omega^2 z,
    u~ = L z, w~ = a+ u~ / omega, scaled so u~.w~ = 1; X+Y = V u~,
    X-Y = V w~.  Residuals r1 = (A+B)(X+Y) - omega (X-Y) and
    r2 = (A-B)(X-Y) - omega (X+Y); a root is converged when both norms are
    <= tol.  Both preconditioned residuals of every unconverged root are
    appended.
    """
    ov = diag.size
    nguess = min(ov, 2 * k) if nguess is None else min(ov, nguess)
    max_sub = max_sub or min(ov, 40 * k)
    V = _guess(diag, nguess)
    P, M = apply_pm(V)
    n_products = V.shape[1]
    for it in range(1, max_iter + 1):
        ap = V.T @ P
        am = V.T @ M
        ap = 0.5 * (ap + ap.T)
        am = 0.5 * (am + am.T)
        L = np.linalg.cholesky(am)
        w2, z = np.linalg.eigh(L.T @ ap @ L)
        kk = min(k, w2.size)
        omega = np.sqrt(w2[:kk])
        ut = L @ z[:, :kk]
        wt = ap @ ut / omega
        scale = 1.0 / np.sqrt(np.sum(ut * wt, axis=0))
        ut = ut * scale
        wt = wt * scale
        U = V @ ut
        W = V @ wt
        r1 = P @ ut - W * omega
        r2 = M @ wt - U * omega
        n1 = np.linalg.norm(r1, axis=0)
        n2 = np.linalg.norm(r2, axis=0)
        norms = np.maximum(n1, n2)
        if np.all(norms <= tol):
            return dict(omega=omega, U=U, W=W, residual=norms, iterations=it, products=n_products,
                        converged=True)
        cols = []
        for j in range(kk):
            if norms[j] > tol:
                cols.append(_precondition(r1[:, j], omega[j], diag))
                cols.append(_precondition(r2[:, j], omega[j], diag))
        T = np.stack(cols, axis=1)
        if V.shape[1] + T.shape[1] > max_sub:
            # collapse onto the current X+Y and X-Y of the lowest roots
            basis = _orthonormalise_new(np.zeros((ov, 0)), np.hstack([U, W]))
            c = V.T @ basis
            V, P, M = basis, P @ c, M @ c
        Tn = _orthonormalise_new(V, T)
        if Tn.shape[1] == 0:
            break
        Pn, Mn = apply_pm(Tn)
        V = np.hstack([V, Tn])
        P = np.hstack([P, Pn])
        M = np.hstack([M, Mn])
        n_products += Tn.shape[1]
    return dict(omega=omega, U=U, W=W, residual=norms, iterations=it, products=n_products,
                converged=False)


# ---------------------------------------------------------------------------
# transition dipoles and oscillator strengths (Section "Results and discussion")

def oscillator_strengths(mol, C, nocc, omega, U):
    """f_n = 2/3 omega_n |d_n|^2 in atomic units, d_n = sqrt(2) sum (X+Y)_ia <i|r|a>.

    U: (k, nocc, nvir) amplitudes X (CIS, ||X|| = 1) or X+Y (RPA,
    (X+Y).(X-Y) = 1).  <mu|r|nu> is the model's dipole matrix.
    """
    dip = dipole_integrals(mol)
    dmo = np.einsum("xmn,mi,na->xia", dip, C[:, :nocc], C[:, nocc:])
    d = SQRT2 * np.einsum("kia,xia->kx", U, dmo) / BOHR_A
    return (2.0 / 3.0) * (np.asarray(omega) / HARTREE_EV) * np.sum(d * d, axis=1)


# ---------------------------------------------------------------------------
# the whole excited-state solve for one molecule

def solve(mol, ints, scf_result, method="CIS", nroots=5, tol=1e-6, max_sub=None, spin="singlet"):
    """Davidson solve on top of a converged SCF; returns omega (eV), f, amplitudes.

    spin: 'singlet' or 'triplet' (triplets are dipole-forbidden: f = 0).
    """
    if spin not in ("singlet", "triplet"):
        raise ValueError(spin)
    sfx = "_T" if spin == "triplet" else ""
    C, eps = scf_result.C, scf_result.eps
    o, v = mol.nocc, mol.nvir
    diag = delta_eps(eps, o).reshape(-1)

    def unflat(Vc):
        return Vc.T.reshape(-1, o, v)

    def flat(Xs):
        return Xs.reshape(Xs.shape[0], -1).T

    if method == "CIS":
        res = davidson_cis(lambda Vc: flat(apply_kind(mol, ints, C, eps, o, unflat(Vc), "A" + sfx)),
                           diag, nroots, tol=tol, max_sub=max_sub)
        Xs = unflat(res["X"])
        f = oscillator_strengths(mol, C, o, res["omega"], Xs) if not sfx else np.zeros(len(res["omega"]))
        return dict(omega=res["omega"], f=f, X=Xs, Y=None, residual=res["residual"],
                    iterations=res["iterations"], products=res["products"], converged=res["converged"])
    if method in ("RPA", "TDHF"):
        def apm(Vc):
            Xs = unflat(Vc)
            return (flat(apply_kind(mol, ints, C, eps, o, Xs, "ApB" + sfx)),
                    flat(apply_kind(mol, ints, C, eps, o, Xs, "AmB" + sfx)))
        res = davidson_rpa(apm, diag, nroots, tol=tol, max_sub=max_sub)
        U, W = unflat(res["U"]), unflat(res["W"])
        f = oscillator_strengths(mol, C, o, res["omega"], U) if not sfx else np.zeros(len(res["omega"]))
        return dict(omega=res["omega"], f=f, X=0.5 * (U + W), Y=0.5 * (U - W), residual=res["residual"],
                    iterations=res["iterations"], products=res["products"], converged=res["converged"])
    raise ValueError(method)
