"""Pins for the oracle's SCF, A*X products, Davidson and oscillator strengths (CPU only).

What fixes each result: brute force on tiny inputs (the n^4 integral tensor
and explicit A, B), the Tamm-Dancoff reduction (B = 0 gives CIS), the +/-omega
pairing of the RPA spectrum, closed forms for the two-site H2 model,
invariances (rigid motion, atom order, far-apart fragments) and the
variational character of the SCF.
"""
import math

import numpy as np
import pytest

import molgen
from oracle import excited, nddo, scf


@pytest.fixture(scope="module")
def small(params0):
    Z, xyz = molgen.config_small(1)
    mol = nddo.Molecule(Z, xyz, params0)
    ints = nddo.Integrals(mol)
    res = scf.scf(mol, ints)
    eri = nddo.full_eri(mol, ints)
    A, B = excited.explicit_AB(res.eps, res.C, mol.nocc, eri)
    return mol, ints, res, eri, A, B


def test_blocked_coulomb_exchange_equals_bruteforce(small):
    mol, ints, res, eri, A, B = small
    R = np.random.default_rng(0).uniform(-1, 1, size=(mol.nao, mol.nao))
    J, K = scf.coulomb_exchange(mol, ints, R)
    J2, K2 = scf.coulomb_exchange_bruteforce(eri, R)
    assert np.abs(J - J2).max() < 1e-11
    assert np.abs(K - K2).max() < 1e-11
    # K(R^T) = K(R)^T, linearity, symmetric G for symmetric R
    _, Kt = scf.coulomb_exchange(mol, ints, R.T)
    assert np.abs(Kt - K.T).max() < 1e-12
    Rs = R + R.T
    G = excited.g_cis(mol, ints, Rs)
    assert np.abs(G - G.T).max() < 1e-11
    G1 = excited.g_cis(mol, ints, R)
    G2 = excited.g_cis(mol, ints, 2.0 * R)
    assert np.abs(G2 - 2 * G1).max() < 1e-11


def test_scf_invariants(small):
    mol, ints, res, eri, A, B = small
    P = res.D / 2
    assert np.abs(P @ P - P).max() < 1e-10
    assert abs(np.trace(res.D) - 2 * mol.nocc) < 1e-10
    assert np.abs(res.F @ res.D - res.D @ res.F).max() < 1e-8
    # the excited-state kernel at the ground-state density reproduces F - H:
    # J(D) - K(D)/2 = 2 J(D/2) - K(D/2) = G_CIS(D/2)
    assert np.abs(excited.g_cis(mol, ints, res.D / 2) - (res.F - res.Hcore)).max() < 1e-10
    # the energy is stationary (a minimum) under small orbital rotations
    rng = np.random.default_rng(3)
    Kr = rng.normal(size=(mol.nao, mol.nao))
    Kr = Kr - Kr.T
    E0 = scf.electronic_energy(mol, ints, res.Hcore, res.C)
    for t in (1e-3, 2e-3):
        from scipy.linalg import expm
        E = scf.electronic_energy(mol, ints, res.Hcore, res.C @ expm(t * Kr))
        assert E - E0 > -1e-9
    e1 = scf.electronic_energy(mol, ints, res.Hcore, res.C @ expm(1e-3 * Kr)) - E0
    e2 = scf.electronic_energy(mol, ints, res.Hcore, res.C @ expm(2e-3 * Kr)) - E0
    assert abs(e2 / e1 - 4.0) < 0.05   # quadratic, no linear term


def test_products_equal_explicit_matrices(small):
    mol, ints, res, eri, A, B = small
    o, v = mol.nocc, mol.nvir
    X = np.random.default_rng(1).uniform(-1, 1, size=(3, o, v))
    flat = X.reshape(3, -1).T
    for kind, M in (("A", A), ("ApB", A + B), ("AmB", A - B)):
        Y = excited.apply_kind(mol, ints, res.C, res.eps, o, X, kind).reshape(3, -1).T
        ref = M @ flat
        assert np.abs(Y - ref).max() <= 1e-12 * np.abs(ref).max(), kind


def test_explicit_matrices_structure(small):
    mol, ints, res, eri, A, B = small
    assert np.abs(A - A.T).max() < 1e-12
    assert np.abs(B - B.T).max() < 1e-12
    assert np.linalg.eigvalsh(A - B)[0] > 0
    assert np.linalg.eigvalsh(A + B)[0] > 0


def test_davidson_cis_equals_bruteforce(small):
    mol, ints, res, eri, A, B = small
    w, _ = excited.cis_bruteforce(A, 5)
    out = excited.solve(mol, ints, res, "CIS", 5, tol=1e-6)
    assert out["converged"]
    assert np.abs(out["omega"] - w).max() < 1e-8


def test_davidson_rpa_equals_bruteforce_and_pairs(small):
    mol, ints, res, eri, A, B = small
    om, U, W = excited.rpa_bruteforce(A, B, 5)
    out = excited.solve(mol, ints, res, "RPA", 5, tol=1e-6)
    assert out["converged"]
    assert np.abs(out["omega"] - om).max() < 1e-8
    ev = excited.rpa_full_spectrum(A, B)
    assert np.abs(ev.imag).max() < 1e-8
    pos = np.sort(ev.real[ev.real > 0])
    neg = np.sort(-ev.real[ev.real < 0])
    assert np.abs(pos - neg).max() < 1e-8
    assert np.abs(pos[:5] - om).max() < 1e-8
    # oscillator strengths agree between brute force and Davidson
    f_b = excited.oscillator_strengths(mol, res.C, mol.nocc, om, U.T.reshape(5, mol.nocc, mol.nvir))
    assert np.abs(out["f"] - f_b).max() < 1e-7


def test_tda_reduces_rpa_to_cis(small):
    mol, ints, res, eri, A, B = small
    w, _ = excited.cis_bruteforce(A, 5)
    om, _, _ = excited.rpa_bruteforce(A, np.zeros_like(B), 5)
    assert np.abs(om - w).max() < 1e-10
    diag = excited.delta_eps(res.eps, mol.nocc).reshape(-1)
    out = excited.davidson_rpa(lambda V: (A @ V, A @ V), diag, 5, tol=1e-7)
    assert np.abs(out["omega"] - w).max() < 1e-9


def _h2(params, R):
    Z = np.array([1, 1])
    xyz = np.array([[0.0, 0.0, 0.0], [R, 0.0, 0.0]])
    mol = nddo.Molecule(Z, xyz, params)
    ints = nddo.Integrals(mol)
    return mol, ints


def test_h2_closed_forms(params0):
    R = 0.9
    mol, ints = _h2(params0, R)
    res = scf.scf(mol, ints, min_gap=0.0)
    gss = params0[1]["gss"]
    gamma = ints.pair_block(0, 1)[0, 0, 0, 0]
    t = res.Hcore[0, 1]
    de = -2 * t + gamma
    assert abs((res.eps[1] - res.eps[0]) - de) < 1e-10
    Acf = de + 0.5 * gss - 1.5 * gamma
    Bcf = 0.5 * (gss - gamma)
    cis = excited.solve(mol, ints, res, "CIS", 1, tol=1e-10)
    rpa = excited.solve(mol, ints, res, "RPA", 1, tol=1e-10)
    assert abs(cis["omega"][0] - Acf) < 1e-10
    assert abs(rpa["omega"][0] - math.sqrt(Acf ** 2 - Bcf ** 2)) < 1e-10
    Rb = R / nddo.BOHR_A
    w_cis = Acf / nddo.HARTREE_EV
    w_rpa = math.sqrt(Acf ** 2 - Bcf ** 2) / nddo.HARTREE_EV
    assert abs(cis["f"][0] - w_cis * Rb ** 2 / 3) < 1e-10
    assert abs(rpa["f"][0] - w_rpa ** 2 * Rb ** 2 / (3 * (Acf + Bcf) / nddo.HARTREE_EV)) < 1e-10


def _solve(Z, xyz, params, method="CIS", k=4, D0=None):
    mol = nddo.Molecule(Z, xyz, params)
    ints = nddo.Integrals(mol)
    res = scf.scf(mol, ints, D0=D0)
    out = excited.solve(mol, ints, res, method, k, tol=1e-7)
    out["D"] = res.D
    return out


def test_rigid_motion_and_reordering_invariance(params0):
    Z, xyz = molgen.make_chain(11, 6, 9)
    ref = _solve(Z, xyz, params0, "RPA")
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    moved = xyz @ Q.T + np.array([3.0, -1.0, 2.5])
    out = _solve(Z, moved, params0, "RPA")
    assert np.abs(out["omega"] - ref["omega"]).max() < 1e-9
    assert np.abs(out["f"] - ref["f"]).max() < 1e-9
    perm = rng.permutation(len(Z))
    out2 = _solve(Z[perm], xyz[perm], params0, "RPA")
    assert np.abs(out2["omega"] - ref["omega"]).max() < 1e-9
    assert np.abs(out2["f"] - ref["f"]).max() < 1e-9


def test_far_fragments_spectrum_is_union(params0):
    Z1, x1 = molgen.make_chain(21, 3, 5)
    Z2, x2 = molgen.make_chain(31, 3, 5)   # both LUMOs above both HOMOs: no charge transfer
    a = _solve(Z1, x1, params0, "CIS", 3)
    b = _solve(Z2, x2, params0, "CIS", 3)
    Z = np.concatenate([Z1, Z2])
    xyz = np.vstack([x1, x2 + np.array([1000.0, 0.0, 0.0])])
    if sum(nddo.CORE_CHARGE[int(z)] for z in Z) % 2:
        pytest.skip("odd combined electron count")
    # start from the fragments' own densities: at 1000 Angstrom the charge
    # would otherwise slosh between the nearly decoupled fragments
    D0 = np.zeros((molgen.n_orbitals(Z),) * 2)
    n1 = molgen.n_orbitals(Z1)
    D0[:n1, :n1] = a["D"]
    D0[n1:, n1:] = b["D"]
    ab = _solve(Z, xyz, params0, "CIS", 3, D0=D0)
    union = np.sort(np.concatenate([a["omega"], b["omega"]]))[:3]
    assert np.abs(ab["omega"] - union).max() < 1e-6


def test_generator_sizes():
    Z, xyz = molgen.config_small(0)
    assert molgen.n_orbitals(Z) == 62
    Z, xyz = molgen.config_medium(0)
    assert molgen.n_orbitals(Z) == 600
    Z2, xyz2 = molgen.config_medium(0)
    assert np.array_equal(Z, Z2) and np.array_equal(xyz, xyz2)


# ---- triplets (spin-adapted A_T = de - (ij|ab), B_T = -(ib|ja)) -------------

@pytest.fixture(scope="module")
def small_triplet(small):
    mol, ints, res, eri, A, B = small
    At, Bt = excited.explicit_AB_triplet(res.eps, res.C, mol.nocc, eri)
    return At, Bt


def test_triplet_products_equal_explicit_matrices(small, small_triplet):
    mol, ints, res, eri, A, B = small
    At, Bt = small_triplet
    o, v = mol.nocc, mol.nvir
    X = np.random.default_rng(2).uniform(-1, 1, size=(3, o, v))
    flat = X.reshape(3, -1).T
    for kind, M in (("A_T", At), ("ApB_T", At + Bt), ("AmB_T", At - Bt)):
        Y = excited.apply_kind(mol, ints, res.C, res.eps, o, X, kind).reshape(3, -1).T
        ref = M @ flat
        assert np.abs(Y - ref).max() <= 1e-12 * np.abs(ref).max(), kind


def test_triplet_matrix_structure(small, small_triplet):
    mol, ints, res, eri, A, B = small
    At, Bt = small_triplet
    # A - B is spin-independent; A - A_T = 2 (ia|jb) and B - B_T = 2 (ia|jb)
    # (the model's two-electron matrix need not be positive semidefinite, so no
    # ordering of singlets and triplets is implied)
    assert np.abs((A - B) - (At - Bt)).max() < 1e-12
    assert np.abs((A - At) - (B - Bt)).max() < 1e-12
    assert np.abs(At - At.T).max() < 1e-12 and np.abs(Bt - Bt.T).max() < 1e-12


def test_davidson_triplets_equal_bruteforce(small, small_triplet):
    mol, ints, res, eri, A, B = small
    At, Bt = small_triplet
    w, _ = excited.cis_bruteforce(At, 5)
    out = excited.solve(mol, ints, res, "CIS", 5, tol=1e-6, spin="triplet")
    assert out["converged"]
    assert np.abs(out["omega"] - w).max() < 1e-8
    assert np.all(out["f"] == 0.0)
    if np.linalg.eigvalsh(At + Bt)[0] > 0:   # triplet-stable reference
        om, _, _ = excited.rpa_bruteforce(At, Bt, 5)
        out = excited.solve(mol, ints, res, "RPA", 5, tol=1e-6, spin="triplet")
        assert np.abs(out["omega"] - om).max() < 1e-8


def test_h2_triplet_closed_form(params0):
    # two-site H2: (ii|aa) = (gss + gamma)/2, (ia|ia) = (gss - gamma)/2, so
    # A_T = de - (gss + gamma)/2 and B_T = -(gss - gamma)/2
    R = 0.9
    mol, ints = _h2(params0, R)
    res = scf.scf(mol, ints, min_gap=0.0)
    gss = params0[1]["gss"]
    gamma = ints.pair_block(0, 1)[0, 0, 0, 0]
    de = res.eps[1] - res.eps[0]
    At = de - 0.5 * (gss + gamma)
    Bt = -0.5 * (gss - gamma)
    cis = excited.solve(mol, ints, res, "CIS", 1, tol=1e-10, spin="triplet")
    assert abs(cis["omega"][0] - At) < 1e-10
    if (At - Bt) > 0 and (At + Bt) > 0:
        rpa = excited.solve(mol, ints, res, "RPA", 1, tol=1e-10, spin="triplet")
        assert abs(rpa["omega"][0] - math.sqrt(At ** 2 - Bt ** 2)) < 1e-10
