"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: float64 products agree to 1e-11 relative (rounding order only);
mixed-precision products within mixed_product_tol(n) (tests/gpu_common.py:
the truncation and split errors of four TF32x3 GEMMs over n terms); excitation energies to 1e-6 eV in
float64 and 1e-5 eV in mixed precision (the stated target); oscillator
strengths to 1e-4 absolute.
"""
import numpy as np
import pytest

import molgen
from tests.gpu_common import context, mixed_product_err, mixed_product_tol, oracle_ground_state, rel_err

pytestmark = pytest.mark.gpu

xs = pytest.importorskip("paper_2505_24807_gb300.xs")


@pytest.fixture(scope="module")
def small_case():
    params = molgen.make_params(0)
    Z, xyz = molgen.config_small(1)
    mol, ints, res = oracle_ground_state(Z, xyz, params)
    ctx = context(params)
    xs.xs_ground_state(ctx.h, [(Z, xyz)])
    yield dict(params=params, Z=Z, xyz=xyz, mol=mol, ints=ints, res=res, ctx=ctx)
    ctx.close()


def test_scf_matches_oracle(small_case):
    c = small_case
    Cg, eps = xs.xs_get_orbitals(c["ctx"].h, 0)
    assert np.abs(eps - c["res"].eps).max() < 1e-7
    o = c["mol"].nocc
    D = 2 * Cg[:, :o] @ Cg[:, :o].T
    assert np.abs(D - c["res"].D).max() < 1e-7


def test_gbuild_matches_oracle(small_case):
    from oracle import excited
    c = small_case
    n = c["mol"].nao
    R = np.random.default_rng(5).uniform(-1, 1, size=(3, n, n))
    G = xs.xs_apply(c["ctx"].h, 0, xs.XS_KIND_G, R)
    ref = excited.apply_kind(c["mol"], c["ints"], None, None, None, R, "G")
    assert rel_err(G, ref) < 1e-12


@pytest.mark.parametrize("kind,okind", [(0, "A"), (1, "ApB"), (2, "AmB")])
@pytest.mark.parametrize("precision", [0, 1])
def test_products_match_oracle(small_case, kind, okind, precision):
    from oracle import excited
    c = small_case
    mol, res = c["mol"], c["res"]
    # run on the oracle's own orbitals so elementwise comparison is meaningful
    xs.xs_set_orbitals(c["ctx"].h, 0, res.C, res.eps)
    X = molgen.trial_vectors(7, 4, mol.nocc, mol.nvir)
    Y = xs.xs_apply(c["ctx"].h, 0, kind, X.reshape(4, -1), precision=precision).reshape(X.shape)
    ref = excited.apply_kind(mol, c["ints"], res.C, res.eps, mol.nocc, X, okind)
    if precision == 0:
        assert rel_err(Y, ref) < 1e-11
    else:
        assert mixed_product_err(Y, ref, X, res.eps, mol.nocc) < mixed_product_tol(mol.nao)


@pytest.mark.parametrize("kind,okind", [(0, "A"), (1, "ApB"), (2, "AmB")])
def test_mixed_products_hydrocarbon(kind, okind):
    """An alkane has nocc == nvir, so the mixed path builds R = C_occ X C_vir^T
    contracting its n x n product over nocc (molecules with N or O, nvir <
    nocc, contract over nvir): the other branch of the contraction order."""
    from oracle import excited
    params = molgen.make_params(0)
    Z, xyz = molgen.make_chain(3, 12, 26)
    mol, ints, res = oracle_ground_state(Z, xyz, params)
    assert mol.nocc == mol.nvir
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, [(Z, xyz)])
        xs.xs_set_orbitals(ctx.h, 0, res.C, res.eps)
        X = molgen.trial_vectors(9, 3, mol.nocc, mol.nvir)
        Y = xs.xs_apply(ctx.h, 0, kind, X.reshape(3, -1), precision=1).reshape(X.shape)
        ref = excited.apply_kind(mol, ints, res.C, res.eps, mol.nocc, X, okind)
        assert mixed_product_err(Y, ref, X, res.eps, mol.nocc) < mixed_product_tol(mol.nao)
    finally:
        ctx.close()


@pytest.mark.parametrize("method", ["CIS", "RPA"])
@pytest.mark.parametrize("precision", [0, 1])
def test_roots_match_bruteforce(small_case, method, precision):
    from oracle import excited, nddo
    c = small_case
    mol, res = c["mol"], c["res"]
    eri = nddo.full_eri(mol, c["ints"])
    A, B = excited.explicit_AB(res.eps, res.C, mol.nocc, eri)
    k = 5
    if method == "CIS":
        w, V = excited.cis_bruteforce(A, k)
        f = excited.oscillator_strengths(mol, res.C, mol.nocc, w, V.T.reshape(k, mol.nocc, mol.nvir))
    else:
        w, U, W = excited.rpa_bruteforce(A, B, k)
        f = excited.oscillator_strengths(mol, res.C, mol.nocc, w, U.T.reshape(k, mol.nocc, mol.nvir))
    ctx = context(c["params"])
    try:
        xs.xs_ground_state(ctx.h, [(c["Z"], c["xyz"])])
        out = xs.xs_excited(ctx.h, method=xs.XS_CIS if method == "CIS" else xs.XS_TDHF, nroots=k, tol=1e-6,
                            precision=precision)
    finally:
        ctx.close()
    tol = 1e-6 if precision == 0 else 1e-5
    assert np.abs(out["omega"][0] - w).max() < tol
    assert np.abs(out["osc"][0] - f).max() < 1e-4
    assert out["info"]["converged"] == 1


@pytest.mark.parametrize("method", ["CIS", "RPA"])
def test_many_roots_match_bruteforce(small_case, method):
    """33 roots: the new-block Gram matrices (up to 66 x 66 for TDHF) take the
    global-memory Jacobi, the subspace (up to 16 x 33) the global-memory
    eigensolver and Cholesky -- the paths beyond the shared-memory sizes."""
    from oracle import excited, nddo
    c = small_case
    mol, res = c["mol"], c["res"]
    eri = nddo.full_eri(mol, c["ints"])
    A, B = excited.explicit_AB(res.eps, res.C, mol.nocc, eri)
    k = 33
    w = excited.cis_bruteforce(A, k)[0] if method == "CIS" else excited.rpa_bruteforce(A, B, k)[0]
    ctx = context(c["params"])
    try:
        xs.xs_ground_state(ctx.h, [(c["Z"], c["xyz"])])
        out = xs.xs_excited(ctx.h, method=xs.XS_CIS if method == "CIS" else xs.XS_TDHF, nroots=k, tol=1e-6)
    finally:
        ctx.close()
    assert np.abs(out["omega"][0] - w).max() < 1e-6
    assert out["info"]["converged"] == 1


def test_amplitudes_normalised(small_case):
    c = small_case
    ctx = context(c["params"])
    try:
        xs.xs_ground_state(ctx.h, [(c["Z"], c["xyz"])])
        xs.xs_excited(ctx.h, method=xs.XS_TDHF, nroots=3, tol=1e-7)
        for r in range(3):
            X, Y = xs.xs_get_amplitudes(ctx.h, 0, r)
            assert abs(np.sum(X * X) - np.sum(Y * Y) - 1.0) < 1e-8
    finally:
        ctx.close()


def test_h2_two_orbital_edge_case():
    from oracle import excited, nddo, scf
    params = molgen.make_params(0)
    Z = np.array([1, 1])
    xyz = np.array([[0.0, 0.0, 0.0], [0.9, 0.0, 0.0]])
    mol = nddo.Molecule(Z, xyz, params)
    ints = nddo.Integrals(mol)
    res = scf.scf(mol, ints, min_gap=0.0)
    ref = excited.solve(mol, ints, res, "RPA", 1, tol=1e-10)
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, [(Z, xyz)])
        out = xs.xs_excited(ctx.h, method=xs.XS_TDHF, nroots=3, tol=1e-9)
    finally:
        ctx.close()
    assert abs(out["omega"][0, 0] - ref["omega"][0]) < 1e-9
    assert np.all(out["omega"][0, 1:] == 0.0)   # only one root exists (ov = 1)


def test_odd_electron_count_rejected():
    params = molgen.make_params(0)
    ctx = context(params)
    try:
        with pytest.raises(xs.XSError) as e:
            xs.xs_ground_state(ctx.h, [(np.array([1, 1, 1]), np.array([[0, 0, 0], [1.0, 0, 0], [0, 1.2, 0]]))])
        assert e.value.status == xs.XS_EINVAL
    finally:
        ctx.close()


def test_unstable_reference_reported():
    # an all-oxygen chain with weakened resonance integrals has an A - B with a
    # negative eigenvalue (checked here with the oracle): TDHF must refuse it
    import copy
    from oracle import excited, nddo
    params = copy.deepcopy(molgen.make_params(0))
    for z in params:
        params[z]["beta_s"] *= 0.6
        params[z]["beta_p"] *= 0.6
    Z, xyz = molgen.config_small(0)
    Z = Z.copy()
    Z[Z > 1] = 8
    mol, ints, res = oracle_ground_state(Z, xyz, params)
    A, B = excited.explicit_AB(res.eps, res.C, mol.nocc, nddo.full_eri(mol, ints))
    assert np.linalg.eigvalsh(A - B)[0] < -0.1
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, [(Z, xyz)])
        with pytest.raises(xs.XSError) as e:
            xs.xs_excited(ctx.h, method=xs.XS_TDHF, nroots=5, tol=1e-6)
        assert e.value.status == xs.XS_EUNSTABLE
        # CIS (B = 0) is still defined for this reference
        out = xs.xs_excited(ctx.h, method=xs.XS_CIS, nroots=3, tol=1e-6)
        w, _ = excited.cis_bruteforce(A, 3)
        assert np.abs(out["omega"][0] - w).max() < 1e-6
    finally:
        ctx.close()


def test_spectrum_matches_oracle():
    """Gaussian-broadened absorption spectrum (paper width 0.1 eV) against the
    oracle on seeded lines, and on a solved molecule's own roots."""
    from oracle.spectrum import absorption_spectrum
    rng = np.random.default_rng(4)
    omega = rng.uniform(3.0, 8.0, 37)
    f = rng.uniform(0.0, 1.5, 37)
    grid = np.linspace(2.0, 9.0, 3001)
    ctx = context(molgen.make_params(0))
    try:
        got = xs.xs_spectrum(ctx.h, omega, f, grid, 0.1)
        ref = absorption_spectrum(omega, f, grid, 0.1)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.all(xs.xs_spectrum(ctx.h, [], [], grid, 0.1) == 0.0)
        with pytest.raises(xs.XSError):
            xs.xs_spectrum(ctx.h, omega, f, grid, 0.0)
    finally:
        ctx.close()


def test_spectrum_of_solved_molecule(small_case):
    """The library's spectrum of its own CIS roots equals the oracle's spectrum
    of the brute-force roots within what the 1e-6 eV root tolerance allows."""
    from oracle import excited, nddo
    from oracle.spectrum import absorption_spectrum
    c = small_case
    mol, res = c["mol"], c["res"]
    eri = nddo.full_eri(mol, c["ints"])
    A, _ = excited.explicit_AB(res.eps, res.C, mol.nocc, eri)
    k = 5
    w, V = excited.cis_bruteforce(A, k)
    fo = excited.oscillator_strengths(mol, res.C, mol.nocc, w, V.T.reshape(k, mol.nocc, mol.nvir))
    grid = np.linspace(w[0] - 1.0, w[-1] + 1.0, 2001)
    ref = absorption_spectrum(w, fo, grid)
    ctx = context(c["params"])
    try:
        xs.xs_ground_state(ctx.h, [(c["Z"], c["xyz"])])
        out = xs.xs_excited(ctx.h, method=xs.XS_CIS, nroots=k, tol=1e-6)
        got = xs.xs_spectrum(ctx.h, out["omega"][0], out["osc"][0], grid)
    finally:
        ctx.close()
    # |dS| <= sum_n (|df_n| peak + f_n |d omega_n| max slope), peak = 1/(sigma sqrt(2 pi))
    peak = 1.0 / (0.1 * np.sqrt(2 * np.pi))
    bound = k * (1e-4 * peak + fo.max() * 1e-6 * peak / (0.1 * np.sqrt(np.e)))
    assert np.abs(got - ref).max() <= bound


def test_memory_bounded_subspace(small_case):
    """A memory budget lowers the subspace cap (more restarts, same roots); a
    budget below the guess block plus one new block is XS_ENOMEM."""
    from oracle import excited, nddo
    c = small_case
    mol, res = c["mol"], c["res"]
    eri = nddo.full_eri(mol, c["ints"])
    A, _ = excited.explicit_AB(res.eps, res.C, mol.nocc, eri)
    k = 5
    w = excited.cis_bruteforce(A, k)[0]
    per_vec = 8.0 * 2 * mol.nocc * mol.nvir   # V and A V in float64
    ctx = context(c["params"])
    try:
        xs.xs_ground_state(ctx.h, [(c["Z"], c["xyz"])])
        free = xs.xs_excited(ctx.h, method=xs.XS_CIS, nroots=k, tol=1e-6)
        tight = xs.xs_excited(ctx.h, method=xs.XS_CIS, nroots=k, tol=1e-6, memory_limit=20.5 * per_vec)
        assert free["info"]["max_subspace_used"] == 50
        assert tight["info"]["max_subspace_used"] == 20
        assert np.abs(tight["omega"][0] - w).max() < 1e-6
        assert tight["info"]["converged"] == 1
        with pytest.raises(xs.XSError) as e:
            xs.xs_excited(ctx.h, method=xs.XS_CIS, nroots=k, tol=1e-6, memory_limit=10 * per_vec)
        assert e.value.status == xs.XS_ENOMEM
    finally:
        ctx.close()


@pytest.mark.parametrize("kind,okind", [(4, "A_T"), (5, "ApB_T")])
@pytest.mark.parametrize("precision", [0, 1])
def test_triplet_products_match_oracle(small_case, kind, okind, precision):
    from oracle import excited
    c = small_case
    mol, res = c["mol"], c["res"]
    xs.xs_set_orbitals(c["ctx"].h, 0, res.C, res.eps)
    X = molgen.trial_vectors(8, 4, mol.nocc, mol.nvir)
    Y = xs.xs_apply(c["ctx"].h, 0, kind, X.reshape(4, -1), precision=precision).reshape(X.shape)
    ref = excited.apply_kind(mol, c["ints"], res.C, res.eps, mol.nocc, X, okind)
    if precision == 0:
        assert rel_err(Y, ref) < 1e-11
    else:
        assert mixed_product_err(Y, ref, X, res.eps, mol.nocc) < mixed_product_tol(mol.nao)


@pytest.mark.parametrize("method", ["CIS", "RPA"])
@pytest.mark.parametrize("precision", [0, 1])
def test_triplet_roots_match_bruteforce(small_case, method, precision):
    from oracle import excited, nddo
    c = small_case
    mol, res = c["mol"], c["res"]
    eri = nddo.full_eri(mol, c["ints"])
    At, Bt = excited.explicit_AB_triplet(res.eps, res.C, mol.nocc, eri)
    k = 5
    w = excited.cis_bruteforce(At, k)[0] if method == "CIS" else excited.rpa_bruteforce(At, Bt, k)[0]
    ctx = context(c["params"])
    try:
        xs.xs_ground_state(ctx.h, [(c["Z"], c["xyz"])])
        out = xs.xs_excited(ctx.h, method=xs.XS_CIS if method == "CIS" else xs.XS_TDHF, nroots=k, tol=1e-6,
                            precision=precision, spin=xs.XS_TRIPLET, guess=xs.XS_GUESS_LEARNED)
    finally:
        ctx.close()
    assert np.abs(out["omega"][0] - w).max() < (1e-6 if precision == 0 else 1e-5)
    assert np.all(out["osc"][0] == 0.0)
    assert out["info"]["converged"] == 1 and out["info"]["learned"] == 0
