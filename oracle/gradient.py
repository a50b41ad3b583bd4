"""Derivatives of excitation energies with respect to the NDDO parameters
(oracle; test infrastructure only).

The paper (Section "Overview of the capabilities of PySEQM") builds its
semiempirical models so that the parameters can be learned: excitation
energies differentiated with respect to them.  The oracle takes the plain
definition of that derivative: a central finite difference of the lowest
roots of the explicit A (CIS) or of the RPA problem (brute force), each after
a fresh SCF at the displaced parameter -- so the orbital response of the
ground state is included by construction.  Five-point stencil (truncation
error O(h^4)); the SCF restarts from the undisplaced density.
"""
from __future__ import annotations

import copy

import numpy as np

from . import excited, nddo, scf

FIELDS = ("Uss", "Upp", "beta_s", "beta_p", "gss", "gsp", "gpp", "gp2", "hsp", "D1", "D2", "zeta_s", "zeta_p")


def excitation_energies(Z, xyz, params, method="CIS", k=1, D0=None):
    """Lowest k singlet excitation energies (eV) by brute force, and the density;
    method "CIS" (Tamm-Dancoff) or anything else for the RPA (TDHF)."""
    mol = nddo.Molecule(Z, xyz, params)
    ints = nddo.Integrals(mol)
    res = scf.scf(mol, ints, D0=D0, tol_density=1e-12, tol_commutator=1e-11)
    A, B = excited.explicit_AB(res.eps, res.C, mol.nocc, nddo.full_eri(mol, ints))
    if method == "CIS":
        w = excited.cis_bruteforce(A, k)[0]
    else:
        w = excited.rpa_bruteforce(A, B, k)[0]
    return np.asarray(w), res.D


def domega_dparam(Z, xyz, params, z, field, method="CIS", k=1, h=1e-3):
    """d omega_n / d params[z][field] for the lowest k roots (eV per unit of the
    parameter), five-point central difference with step h."""
    _, D0 = excitation_energies(Z, xyz, params, method, k)
    vals = []
    for s in (-2, -1, 1, 2):
        p = copy.deepcopy(params)
        p[z][field] = params[z][field] + s * h
        vals.append(excitation_energies(Z, xyz, p, method, k, D0=D0)[0])
    m2, m1, p1, p2 = vals
    return (m2 - 8.0 * m1 + 8.0 * p1 - p2) / (12.0 * h)
