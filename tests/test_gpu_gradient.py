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
