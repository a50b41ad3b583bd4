"""Full-size parity of the A.X product: the large workload (400 C/N/O + 600 H,
2200 AOs, nocc = 1201) in the configuration the benchmark times (TDHF, mixed
precision, tensor-core transforms) and in float64, on outputs the oracle
computes directly: two seeded trial vectors with seeded orthonormal orbitals
given to both sides (the library receives them through xs_set_orbitals, so no
input of the oracle comes from the GPU path).

Tolerances as in the small-size parity tests: float64 products to 1e-10
relative to the largest element (rounding order only), mixed products within
mixed_product_tol(2200) of the non-diagonal part (tests/gpu_common.py).
"""
import numpy as np
import pytest

import molgen
from tests.gpu_common import context, mixed_product_err, mixed_product_tol, rel_err

pytestmark = pytest.mark.gpu

xs = pytest.importorskip("paper_2505_24807_gb300.xs")


@pytest.fixture(scope="module")
def large_case():
    from oracle import excited, nddo
    params = molgen.make_params(0)
    Z, xyz = molgen.config_large(0)
    mol = nddo.Molecule(Z, xyz, params)
    ints = nddo.Integrals(mol)
    Cm = molgen.orthonormal_matrix(11, mol.nao)
    eps = np.sort(np.random.default_rng(3).uniform(-40.0, 10.0, mol.nao))
    X = molgen.trial_vectors(5, 2, mol.nocc, mol.nvir)
    ref = {kind: excited.apply_kind(mol, ints, Cm, eps, mol.nocc, X, kind) for kind in ("ApB", "AmB")}
    ctx = context(params)
    xs.xs_ground_state(ctx.h, [(Z, xyz)])
    xs.xs_set_orbitals(ctx.h, 0, Cm, eps)
    yield dict(ctx=ctx, X=X.reshape(2, -1), ref=ref, nocc=mol.nocc, nao=mol.nao, eps=eps)
    ctx.close()


@pytest.mark.parametrize("kind,okind", [("ApB", xs.XS_KIND_APB), ("AmB", xs.XS_KIND_AMB)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_products_match_oracle(large_case, kind, okind, precision):
    c = large_case
    n, o, _ = xs.xs_get_sizes(c["ctx"].h, 0)
    assert (n, o) == (c["nao"], c["nocc"]) == (2200, 1201)
    prec = xs.XS_MIXED if precision == "mixed" else xs.XS_FP64
    got = xs.xs_apply(c["ctx"].h, 0, okind, c["X"], precision=prec)
    ref = c["ref"][kind].reshape(2, -1)
    if precision == "mixed":
        assert mixed_product_err(got, ref, c["X"], c["eps"], c["nocc"]) < mixed_product_tol(c["nao"])
    else:
        assert rel_err(got, ref) < 1e-10
