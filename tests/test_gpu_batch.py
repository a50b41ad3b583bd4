"""Batched solves: many molecules of uneven size advance together.

Batch membership must not change a molecule's roots (the paper's batched
steps 1-6 solve each molecule's own problem), and the batched roots match the
oracle for each molecule.  Two forms: the lock-step batch (batched = 1: one
captured graph per Davidson iteration for all molecules, ragged device-side
work lists) runs its own kernels, so it agrees with the one-molecule solver
to the accuracy of converged roots (energy errors quadratic in the 1e-7 eV
residual, oscillator strengths linear in it); the concurrent form (batched =
2) runs the one-molecule solver on several streams and agrees to rounding.
"""
import numpy as np
import pytest

import molgen
from tests.gpu_common import context

pytestmark = pytest.mark.gpu
xs = pytest.importorskip("paper_2505_24807_gb300.xs")


def _mols():
    return [molgen.config_sized(100 + s, n) for s, n in enumerate((20, 33, 47, 26, 58, 21))]


@pytest.mark.parametrize("method", [0, 1])
def test_lockstep_batch_equals_one_at_a_time(method):
    params = molgen.make_params(0)
    mols = _mols()
    k = 4
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, mols)
        batched = xs.xs_excited(ctx.h, method=method, nroots=k, tol=1e-7, batched=1, n_mol=len(mols))
        seq = xs.xs_excited(ctx.h, method=method, nroots=k, tol=1e-7, batched=0, n_mol=len(mols))
    finally:
        ctx.close()
    assert batched["info"]["converged"] == 1
    assert batched["info"]["graph_launches"] >= batched["info"]["iterations"]
    assert np.abs(batched["omega"] - seq["omega"]).max() < 1e-9
    assert np.abs(batched["osc"] - seq["osc"]).max() < 1e-6
    assert np.all(batched["resid"] <= 1e-7)
    # each molecule on its own context
    for i, (Z, xyz) in enumerate(mols[:3]):
        c1 = context(params)
        try:
            xs.xs_ground_state(c1.h, [(Z, xyz)])
            solo = xs.xs_excited(c1.h, method=method, nroots=k, tol=1e-7)
        finally:
            c1.close()
        assert np.abs(solo["omega"][0] - batched["omega"][i]).max() < 1e-9


@pytest.mark.parametrize("method", [0, 1])
def test_concurrent_batch_equals_one_at_a_time(method):
    params = molgen.make_params(0)
    mols = _mols()
    k = 4
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, mols)
        conc = xs.xs_excited(ctx.h, method=method, nroots=k, tol=1e-7, batched=2, n_mol=len(mols))
        seq = xs.xs_excited(ctx.h, method=method, nroots=k, tol=1e-7, batched=0, n_mol=len(mols))
    finally:
        ctx.close()
    assert np.abs(conc["omega"] - seq["omega"]).max() < 1e-10
    assert np.abs(conc["osc"] - seq["osc"]).max() < 1e-10


@pytest.mark.parametrize("method", ["CIS", "RPA"])
@pytest.mark.parametrize("precision", [0, 1])
def test_batched_roots_match_oracle(method, precision):
    from oracle import excited, nddo, scf
    params = molgen.make_params(0)
    mols = _mols()[:4]
    k = 6
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, mols)
        out = xs.xs_excited(ctx.h, method=xs.XS_CIS if method == "CIS" else xs.XS_TDHF, nroots=k, tol=1e-5,
                            precision=precision, batched=1, n_mol=len(mols))
    finally:
        ctx.close()
    assert out["info"]["converged"] == 1
    for i, (Z, xyz) in enumerate(mols):
        mol = nddo.Molecule(Z, xyz, params)
        ints = nddo.Integrals(mol)
        res = scf.scf(mol, ints)
        ref = excited.solve(mol, ints, res, method, k, tol=1e-7)
        tol = 1e-6 if precision == 0 else 1e-5
        assert np.abs(out["omega"][i] - ref["omega"]).max() < tol, i
        assert np.abs(out["osc"][i] - ref["f"]).max() < 1e-4, i


@pytest.mark.parametrize("method", ["CIS", "RPA"])
def test_batched_triplets_match_bruteforce(method):
    from oracle import excited, nddo, scf
    params = molgen.make_params(0)
    mols = _mols()[:3]
    k = 4
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, mols)
        out = xs.xs_excited(ctx.h, method=xs.XS_CIS if method == "CIS" else xs.XS_TDHF, nroots=k, tol=1e-7,
                            batched=1, n_mol=len(mols), spin=xs.XS_TRIPLET)
    finally:
        ctx.close()
    for i, (Z, xyz) in enumerate(mols):
        mol = nddo.Molecule(Z, xyz, params)
        ints = nddo.Integrals(mol)
        res = scf.scf(mol, ints)
        A, B = excited.explicit_AB_triplet(res.eps, res.C, mol.nocc, nddo.full_eri(mol, ints))
        w = excited.cis_bruteforce(A, k)[0] if method == "CIS" else excited.rpa_bruteforce(A, B, k)[0]
        assert np.abs(out["omega"][i] - w).max() < 1e-6, i
        assert np.all(out["osc"][i] == 0.0)


def test_batched_amplitudes_are_normalised_eigenvectors():
    """xs_get_amplitudes after a lock-step solve returns each molecule's own
    Ritz vectors: unit norm (CIS) and A X = omega X to the residual."""
    from oracle import excited, nddo, scf
    params = molgen.make_params(0)
    mols = _mols()[:3]
    k = 3
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, mols)
        out = xs.xs_excited(ctx.h, method=xs.XS_CIS, nroots=k, tol=1e-7, batched=1, n_mol=len(mols))
        for i, (Z, xyz) in enumerate(mols):
            Cm, eps = xs.xs_get_orbitals(ctx.h, i)
            mol = nddo.Molecule(Z, xyz, params)
            ints = nddo.Integrals(mol)
            for r in range(k):
                X, _ = xs.xs_get_amplitudes(ctx.h, i, r)
                assert abs(np.linalg.norm(X) - 1.0) < 1e-10
                AX = excited.apply_kind(mol, ints, Cm, eps, mol.nocc, X[None], "A")[0]
                assert np.linalg.norm(AX - out["omega"][i][r] * X) < 2e-7
    finally:
        ctx.close()
