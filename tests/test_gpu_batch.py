"""Batched solves: many molecules of uneven size advance together.

Batch membership must not change a molecule's roots (the paper's batched
steps 1-6 solve each molecule's own problem), and the batched roots match the
oracle for each molecule.
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
def test_batched_equals_solo(method):
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
    assert np.abs(batched["omega"] - seq["omega"]).max() < 1e-10
    assert np.abs(batched["osc"] - seq["osc"]).max() < 1e-10
    # each molecule on its own
    for i, (Z, xyz) in enumerate(mols[:3]):
        c1 = context(params)
        try:
            xs.xs_ground_state(c1.h, [(Z, xyz)])
            solo = xs.xs_excited(c1.h, method=method, nroots=k, tol=1e-7)
        finally:
            c1.close()
        assert np.abs(solo["omega"][0] - batched["omega"][i]).max() < 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_roots_match_oracle(precision):
    from oracle import excited, nddo, scf
    params = molgen.make_params(0)
    mols = _mols()[:4]
    k = 6
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, mols)
        out = xs.xs_excited(ctx.h, method=xs.XS_CIS, nroots=k, tol=1e-5, precision=precision, batched=1,
                            n_mol=len(mols))
    finally:
        ctx.close()
    for i, (Z, xyz) in enumerate(mols):
        mol = nddo.Molecule(Z, xyz, params)
        ints = nddo.Integrals(mol)
        res = scf.scf(mol, ints)
        ref = excited.solve(mol, ints, res, "CIS", k, tol=1e-7)
        tol = 1e-6 if precision == 0 else 1e-5
        assert np.abs(out["omega"][i] - ref["omega"]).max() < tol, i
        assert np.abs(out["osc"][i] - ref["f"]).max() < 1e-4, i
