"""Coulomb / exchange builds and the closed-shell SCF (oracle; test infrastructure only).

Paper, Section "Ground-state wavefunction calculation", Eq. 1: F C = C eps
with S = I under NDDO, restricted closed shell, N doubly occupied orbitals.
Section "GPU Implementation", Eq. ftilde: the two-electron contraction with a
(possibly nonsymmetric) density R has a Coulomb part sum (mu nu|lam sig) R_lam sig
and an exchange part sum (mu lam|nu sig) R_lam sig.
"""
from __future__ import annotations

import numpy as np

from .nddo import CORE_CHARGE, Integrals, Molecule, core_hamiltonian, full_eri


def coulomb_exchange(mol: Molecule, ints: Integrals, R):
    """J(R)_{mu nu} = sum (mu nu|lam sig) R_{lam sig} and
    K(R)_{mu nu} = sum (mu lam|nu sig) R_{lam sig}, for any (nonsymmetric) R,
    with the NDDO restriction that both AOs of a bra or ket sit on one atom.

    J lives on the diagonal atom blocks; K has one-centre terms on the
    diagonal blocks and two-centre terms on the off-diagonal blocks.
    """
    R = np.asarray(R, dtype=np.float64)
    n = mol.nao
    J = np.zeros((n, n))
    K = np.zeros((n, n))
    off = mol.ao_offset
    na = mol.nao_atom
    for A in range(mol.natoms):
        sA = slice(off[A], off[A] + na[A])
        t = ints.one_centre[A]
        RA = R[sA, sA]
        J[sA, sA] += np.einsum("mnls,ls->mn", t, RA)
        K[sA, sA] += np.einsum("mlns,ls->mn", t, RA)
    for (nA, nB), (Aidx, Bidx, _W, w4) in ints.classes.items():
        ia = off[Aidx][:, None] + np.arange(nA)[None, :]
        ib = off[Bidx][:, None] + np.arange(nB)[None, :]
        R_AA = R[ia[:, :, None], ia[:, None, :]]
        R_BB = R[ib[:, :, None], ib[:, None, :]]
        R_AB = R[ia[:, :, None], ib[:, None, :]]
        R_BA = R[ib[:, :, None], ia[:, None, :]]
        # Coulomb on the diagonal blocks of both atoms
        JA = np.einsum("pmnls,pls->pmn", w4, R_BB)
        JB = np.einsum("pmnls,pmn->pls", w4, R_AA)
        _scatter_add(J, ia[:, :, None] * n + ia[:, None, :], JA)
        _scatter_add(J, ib[:, :, None] * n + ib[:, None, :], JB)
        # exchange on the off-diagonal blocks AB and BA
        # K_{m l} (m on A, l on B) = sum_{n on A, s on B} (m n | l s) R_{n s}
        KAB = np.einsum("pmnls,pns->pml", w4, R_AB)
        # K_{l m} (l on B, m on A) = sum_{s on B, n on A} (l s | m n) R_{s n}
        KBA = np.einsum("pmnls,psn->plm", w4, R_BA)
        K[ia[:, :, None], ib[:, None, :]] += KAB
        K[ib[:, :, None], ia[:, None, :]] += KBA
    return J, K


def _scatter_add(M, flat_index, values):
    """M.flat[flat_index] += values, accumulating repeated indices."""
    M += np.bincount(flat_index.reshape(-1), weights=values.reshape(-1),
                     minlength=M.size).reshape(M.shape)


def coulomb_exchange_bruteforce(eri, R):
    """J and K straight from the dense n^4 integral tensor (Eq. ftilde)."""
    J = np.einsum("mnls,ls->mn", eri, R)
    K = np.einsum("mlns,ls->mn", eri, R)
    return J, K


def fock_two_electron(mol, ints, D):
    """Closed-shell two-electron Fock part G(D) = J(D) - K(D)/2, D = 2 C_occ C_occ^T."""
    J, K = coulomb_exchange(mol, ints, D)
    return J - 0.5 * K


class SCFResult:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def scf(mol: Molecule, ints: Integrals | None = None, *, tol_density=1e-10, tol_commutator=1e-9,
        max_iter=300, diis_size=10, min_gap=0.5, D0=None):
    """Restricted closed-shell SCF with Pulay DIIS (error F D - D F, S = I).

    Converged when max|D_new - D| < tol_density and max|F D - D F| <
    tol_commutator (eV).  The returned C, eps diagonalise F(D) of the
    converged D.  Raises if the HOMO-LUMO gap is below ``min_gap`` eV.
    The start is ``D0`` if given, else the neutral-atom density: each atom's
    core charge spread evenly over its valence AOs (diagonal).
    """
    if ints is None:
        ints = Integrals(mol)
    Hc = core_hamiltonian(mol, ints)
    o = mol.nocc
    if D0 is None:
        occ = np.concatenate([np.full(na, CORE_CHARGE[int(z)] / na) for z, na in zip(mol.Z, mol.nao_atom)])
        D = np.diag(occ)
    else:
        D = np.array(D0, dtype=np.float64)
    Fs, Es = [], []
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        F = Hc + fock_two_electron(mol, ints, D)
        err = F @ D - D @ F
        Fs.append(F)
        Es.append(err)
        if len(Fs) > diis_size:
            Fs.pop(0)
            Es.pop(0)
        m = len(Fs)
        if m >= 2:
            B = -np.ones((m + 1, m + 1))
            B[m, m] = 0.0
            for i in range(m):
                for j in range(m):
                    B[i, j] = np.sum(Es[i] * Es[j])
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            try:
                c = np.linalg.solve(B, rhs)[:m]
                Fx = sum(ci * Fi for ci, Fi in zip(c, Fs))
            except np.linalg.LinAlgError:
                Fx = F
        else:
            Fx = F
        eps, C = np.linalg.eigh(Fx)
        Dn = 2.0 * C[:, :o] @ C[:, :o].T
        dD = np.max(np.abs(Dn - D))
        D = Dn
        if dD < tol_density and np.max(np.abs(err)) < tol_commutator:
            converged = True
            break
    if not converged:
        raise RuntimeError("SCF did not converge")
    F = Hc + fock_two_electron(mol, ints, D)
    eps, C = np.linalg.eigh(F)
    D = 2.0 * C[:, :o] @ C[:, :o].T
    gap = eps[o] - eps[o - 1] if o < mol.nao else np.inf
    if gap < min_gap:
        raise RuntimeError(f"HOMO-LUMO gap {gap:.3f} eV below {min_gap} eV")
    energy = 0.5 * np.sum(D * (Hc + F))
    return SCFResult(C=C, eps=eps, D=D, F=F, Hcore=Hc, energy=energy, iterations=it, gap=gap,
                     ints=ints, mol=mol)


def electronic_energy(mol, ints, Hc, C):
    """E = 1/2 sum D (H + F(D)) for the determinant of the first nocc columns of C."""
    o = mol.nocc
    D = 2.0 * C[:, :o] @ C[:, :o].T
    F = Hc + fock_two_electron(mol, ints, D)
    return 0.5 * np.sum(D * (Hc + F))


__all__ = ["coulomb_exchange", "coulomb_exchange_bruteforce", "fock_two_electron", "scf",
           "electronic_energy", "full_eri", "SCFResult"]
