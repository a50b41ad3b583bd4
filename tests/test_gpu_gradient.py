"""Parameter derivatives of CIS and TDHF excitation energies on the GPU (adjoint
orbital response) against the oracle's central finite differences of
brute-force roots after a fresh SCF at each displaced parameter (paper,
Section "Overview of the capabilities of PySEQM": learned semiempirical
parameters).  62-AO molecule, lowest root; every parameter that its elements
carry."""
import numpy as np
import pytest

import molgen
from tests.gpu_common import context

pytestmark = pytest.mark.gpu
xs = pytest.importorskip("paper_2505_24807_gb300.xs")

FIELDS = ("Uss", "Upp", "beta_s", "beta_p", "gss", "gsp", "gpp", "gp2", "hsp", "D1", "D2", "zeta_s", "zeta_p")
ROWS = {1: 0, 6: 1, 7: 2, 8: 3}


@pytest.mark.parametrize("method", ["CIS", "RPA"])
def test_parameter_gradient_matches_finite_differences(method):
    from oracle import gradient
    params = molgen.make_params(0)
    Z, xyz = molgen.config_small(1)
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, [(Z, xyz)], scf_tol=1e-12)
        xs.xs_excited(ctx.h, method=xs.XS_CIS if method == "CIS" else xs.XS_TDHF, nroots=2, tol=1e-9)
        g, its = xs.xs_gradient(ctx.h, 0, 0)
    finally:
        ctx.close()
    assert its > 0
    present = sorted(set(int(z) for z in Z))
    checked = 0
    for z in present:
        fields = ("Uss", "beta_s", "gss", "zeta_s") if z == 1 else FIELDS
        for f in fields:
            fd = gradient.domega_dparam(Z, xyz, params, z, f, method, k=1, h=1e-3)[0]
            got = g[ROWS[z], FIELDS.index(f)]
            assert abs(got - fd) <= 2e-6 * max(1.0, abs(fd)), (z, f, got, fd)
            checked += 1
    # hydrogen has no p orbitals and no multipole lengths
    for f in ("Upp", "beta_p", "gsp", "gpp", "gp2", "hsp", "D1", "D2", "zeta_p"):
        assert g[0, FIELDS.index(f)] == 0.0
    assert checked >= 20


@pytest.mark.parametrize("method", ["CIS", "RPA"])
def test_gradient_after_lockstep_batch(method):
    """The lock-step batch keeps each molecule's amplitudes, so xs_gradient
    after a batched solve equals xs_gradient after a per-molecule solve of the
    same molecule (both float64, converged far below the gradient's
    sensitivity)."""
    params = molgen.make_params(0)
    mols = [molgen.config_small(2), molgen.config_small(1)]
    meth = xs.XS_CIS if method == "CIS" else xs.XS_TDHF
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, mols, scf_tol=1e-12)
        xs.xs_excited(ctx.h, method=meth, nroots=2, tol=1e-9, precision=xs.XS_FP64, batched=1, n_mol=2)
        g_batch, _ = xs.xs_gradient(ctx.h, 1, 0)
    finally:
        ctx.close()
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, [mols[1]], scf_tol=1e-12)
        xs.xs_excited(ctx.h, method=meth, nroots=2, tol=1e-9, precision=xs.XS_FP64)
        g_solo, _ = xs.xs_gradient(ctx.h, 0, 0)
    finally:
        ctx.close()
    assert np.abs(g_batch - g_solo).max() <= 1e-6 * max(1.0, np.abs(g_solo).max())
