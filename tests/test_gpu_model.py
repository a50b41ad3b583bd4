"""The device-built model (two-centre product supermatrix W and core
Hamiltonian H) against the oracle element by element.

Paper, Section "Ground-state wavefunction calculation": two-centre integrals
as classical multipole interactions of the on-atom AO products, one-centre
integrals as parameters, core Hamiltonian of Eq. 1.  The library evaluates
the multipole derivatives with explicit T-tensor formulas on the GPU, the
oracle with the partial-matching formula on the CPU; both in float64.
"""
import numpy as np
import pytest

import molgen
from tests.gpu_common import context

pytestmark = pytest.mark.gpu
xs = pytest.importorskip("paper_2505_24807_gb300.xs")


def oracle_supermatrix(mol, ints):
    from oracle import nddo
    nprod = np.where(mol.nao_atom == 4, 10, 1)
    off = np.concatenate([[0], np.cumsum(nprod)[:-1]])
    W = np.zeros((nprod.sum(), nprod.sum()))
    for A in range(mol.natoms):
        for B in range(mol.natoms):
            if A == B:
                continue
            w = ints.pair_block(A, B)    # (nA, nA, nB, nB)
            for p in range(nprod[A]):
                mu, nu = nddo.HEAVY_PAIRS[p] if nprod[A] == 10 else (0, 0)
                for q in range(nprod[B]):
                    lam, sig = nddo.HEAVY_PAIRS[q] if nprod[B] == 10 else (0, 0)
                    W[off[A] + p, off[B] + q] = w[mu, nu, lam, sig]
    return W


@pytest.mark.parametrize("case", ["small", "hydrocarbon"])
def test_device_model_matches_oracle(case):
    from oracle import nddo
    params = molgen.make_params(0)
    Z, xyz = molgen.config_small(3) if case == "small" else molgen.make_chain(7, 20, 30)
    mol = nddo.Molecule(Z, xyz, params)
    ints = nddo.Integrals(mol)
    W_ref = oracle_supermatrix(mol, ints)
    H_ref = nddo.core_hamiltonian(mol, ints)
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, [(Z, xyz)])
        W, H = xs.xs_get_model(ctx.h, 0)
    finally:
        ctx.close()
    assert W.shape == W_ref.shape and H.shape == H_ref.shape
    assert np.abs(W - W_ref).max() <= 1e-12 * np.abs(W_ref).max()
    assert np.abs(H - H_ref).max() <= 1e-12 * np.abs(H_ref).max()
    assert np.array_equal(W, W.T)
