"""Pins for the oracle's synthetic NDDO integrals (CPU only).

Each check compares against something other than the oracle's own formula:
finite differences, point-multipole electrostatics, limits and symmetries.
"""
import math

import numpy as np
import pytest

import molgen
from oracle import nddo


def test_radial_recursion_matches_finite_differences():
    # g_{n+1} = (1/R) d g_n / dR, checked by central differences
    R = np.linspace(0.9, 9.0, 25)
    a = 0.83
    h = 1e-5
    g = nddo.radial_g(R, a)
    gp = nddo.radial_g(R + h, a)
    gm = nddo.radial_g(R - h, a)
    for n in range(4):
        fd = (gp[n] - gm[n]) / (2 * h) / R
        assert np.allclose(g[n + 1], fd, rtol=1e-6, atol=1e-9), n


def test_radial_zero_limit_is_gss():
    # sigma = kappa / (sqrt(pi) gss) makes the R -> 0 limit of (ss|ss) equal gss
    gss = 12.7
    s = nddo.KAPPA / (math.sqrt(math.pi) * gss)
    a = 1.0 / math.sqrt(2 * (2 * s * s))
    g0 = nddo.radial_g(np.array([1e-7]), a)[0]
    assert abs(g0[0] - gss) < 1e-6


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_cartesian_derivatives_by_finite_differences(order):
    rng = np.random.default_rng(order)
    a = 0.7
    h = 1e-4
    for _ in range(6):
        Rv = rng.uniform(-2.5, 2.5, size=3)
        if np.linalg.norm(Rv) < 1.0:
            Rv *= 1.5 / np.linalg.norm(Rv)
        idx = list(rng.integers(0, 3, size=order))

        def d(indices, v):
            x = v.reshape(3, 1)
            g = nddo.radial_g(np.array([np.linalg.norm(v)]), a)
            return nddo.deriv_phi(indices, x, g)[0]

        j = idx[-1]
        e = np.zeros(3)
        e[j] = h
        fd = (d(idx[:-1], Rv + e) - d(idx[:-1], Rv - e)) / (2 * h)
        assert abs(d(idx, Rv) - fd) <= 1e-6 * max(1.0, abs(fd)), (idx, Rv)


def _point_charges(heavy, product, D1, D2, h):
    """Point-charge stand-in for an on-atom product density (limit h -> 0)."""
    if not heavy or product == 0:
        return [(np.zeros(3), 1.0)]
    mu, nu = nddo.HEAVY_PAIRS[product]
    if mu == 0:
        i = nu - 1
        e = np.zeros(3)
        e[i] = h
        q = D1 / (2 * h)
        return [(e, q), (-e, -q)]
    i, j = mu - 1, nu - 1
    out = []
    if i == j:
        out.append((np.zeros(3), 1.0))
        e = np.zeros(3)
        e[i] = h
        c = D2 * D2 / (h * h)
        out += [(e, c), (-e, c), (np.zeros(3), -2 * c)]
    else:
        ei = np.zeros(3)
        ei[i] = h
        ej = np.zeros(3)
        ej[j] = h
        c = D2 * D2 / (4 * h * h)
        out += [(ei + ej, c), (-ei - ej, c), (ei - ej, -c), (-ei + ej, -c)]
    return out


def test_two_centre_block_matches_point_multipoles_far_apart():
    rng = np.random.default_rng(5)
    D1A, D2A, D1B, D2B = 0.55, 0.45, 0.35, 0.62
    RA = np.zeros(3)
    RB = rng.normal(size=3)
    RB *= 8.0 / np.linalg.norm(RB)
    pa = dict(heavy=True, D1=np.array([D1A]), D2=np.array([D2A]), sigma=np.array([0.6]))
    pb = dict(heavy=True, D1=np.array([D1B]), D2=np.array([D2B]), sigma=np.array([0.7]))
    W = nddo.two_centre_block(pa, pb, RA[None], RB[None])[0]
    h = 0.01
    for p in range(10):
        for q in range(10):
            E = 0.0
            for ra, qa in _point_charges(True, p, D1A, D2A, h):
                for rb, qb in _point_charges(True, q, D1B, D2B, h):
                    E += nddo.KAPPA * qa * qb / np.linalg.norm(RB + rb - RA - ra)
            assert abs(W[p, q] - E) <= 2e-5 * abs(E) + 1e-7, (p, q, W[p, q], E)


def test_dipole_sign_convention():
    # the s-px product has its dipole along +x; a charge at +x sees more repulsion
    pa = dict(heavy=True, D1=np.array([0.5]), D2=np.array([0.5]), sigma=np.array([0.6]))
    pb = dict(heavy=False, D1=np.array([0.0]), D2=np.array([0.0]), sigma=np.array([0.6]))
    W = nddo.two_centre_block(pa, pb, np.zeros((1, 3)), np.array([[3.0, 0.0, 0.0]]))[0]
    assert W[1, 0] > 0 and W[2, 0] == pytest.approx(0.0, abs=1e-14)


def test_eri_permutational_symmetry(params0):
    Z, xyz = molgen.make_chain(3, 4, 6)
    mol = nddo.Molecule(Z, xyz, params0)
    eri = nddo.full_eri(mol, nddo.Integrals(mol))
    assert np.allclose(eri, eri.transpose(1, 0, 2, 3), atol=1e-13)
    assert np.allclose(eri, eri.transpose(0, 1, 3, 2), atol=1e-13)
    assert np.allclose(eri, eri.transpose(2, 3, 0, 1), atol=1e-13)


def test_one_centre_block_positive_definite(params0):
    for z in (6, 7, 8):
        t = nddo.one_centre_tensor(params0[z], True)
        G = np.array([[t[a, a, b, b] for b in range(4)] for a in range(4)])
        assert np.all(np.linalg.eigvalsh(G) > 0)


def test_overlap_rotational_covariance(params0):
    # S between two atoms transforms as s (scalar) and p (vector) under rotation
    Z = np.array([6, 8])
    xyz = np.array([[0.1, -0.2, 0.3], [1.0, 0.7, -0.4]])
    mol = nddo.Molecule(Z, xyz, params0)
    S = nddo.sk_overlap_block(mol, 0, 1)
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    mol2 = nddo.Molecule(Z, xyz @ Q.T, params0)
    S2 = nddo.sk_overlap_block(mol2, 0, 1)
    T = np.eye(4)
    T[1:, 1:] = Q
    assert np.allclose(S2, T @ S @ T.T, atol=1e-13)
    # antisymmetry of the s-p part under exchange of the atoms
    S21 = nddo.sk_overlap_block(mol, 1, 0)
    assert np.allclose(S21, S.T, atol=1e-14)


def test_one_centre_dipole_term_is_the_product_density_dipole(params0):
    # <s|r_j|p_i> of the dipole integrals must be the dipole moment of the
    # model density rho_{s p_i}, whose Coulomb field defines the two-centre
    # integrals: far from atom A, (s p_i | s_B s_B) -> kappa d_i . (R_B - R_A) / R^3
    # (erf(aR) = 1 to ~1e-40 at R = 12 Angstrom).  A flipped sign or a wrong
    # scale of the one-centre term in dipole_integrals fails here.
    rng = np.random.default_rng(17)
    dirs = rng.normal(size=(4, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    RA = np.array([0.3, -0.2, 0.1])
    for z in (6, 7, 8):
        Z = np.array([z] + [1] * len(dirs) + ([1] if (nddo.CORE_CHARGE[z] + len(dirs)) % 2 else []))
        far = [RA + 12.0 * d for d in dirs]
        extra = [RA + np.array([0.0, 0.0, 40.0])] if len(Z) > 1 + len(dirs) else []
        xyz = np.array([RA] + far + extra)
        mol = nddo.Molecule(Z, xyz, params0)
        ints = nddo.Integrals(mol)
        dip = nddo.dipole_integrals(mol)
        o = mol.ao_offset[0]
        for B in range(1, 1 + len(dirs)):
            Rv = mol.xyz[B] - mol.xyz[0]
            R = np.linalg.norm(Rv)
            w = ints.pair_block(0, B)          # (mu nu | s_B s_B), mu nu on the heavy atom
            for i in range(3):
                d_si = dip[:, o, o + 1 + i]    # <s| r |p_i>, Angstrom
                expected = nddo.KAPPA * float(d_si @ Rv) / R ** 3
                assert w[0, 1 + i, 0, 0] == pytest.approx(expected, rel=1e-9, abs=1e-12), (z, B, i)
                # and the matrix is symmetric in s, p_i
                assert np.allclose(dip[:, o + 1 + i, o], d_si, atol=0.0)
