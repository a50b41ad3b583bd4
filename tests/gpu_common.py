"""Shared helpers of the GPU parity tests."""
import numpy as np

import molgen
from paper_2505_24807_gb300 import xs


def context(params=None):
    if params is None:
        params = molgen.make_params(0)
    return xs.Context(0, molgen.params_table(params))


def oracle_ground_state(Z, xyz, params):
    from oracle import nddo, scf
    mol = nddo.Molecule(Z, xyz, params)
    ints = nddo.Integrals(mol)
    res = scf.scf(mol, ints)
    return mol, ints, res


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
