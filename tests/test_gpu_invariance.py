"""Invariances and degenerate cases of the GPU solver (paper, Sections "TDHF
and CIS equations" and "GPU Implementation"; what the method fixes without
reference to any implementation):

* excitation energies and oscillator strengths do not change under a
  reordering of the atoms (which also regroups the hydrogens of the
  super-atom G build) or a rigid rotation and translation of the molecule;
* two copies of a molecule 1000 Angstrom apart have the monomer's spectrum
  with every root doubled: exactly degenerate pairs for the eigensolver and
  the Davidson iteration, and oscillator strengths that add up per pair;
* input edges: fewer amplitudes than requested roots, and rejected inputs.
"""
import numpy as np
import pytest

import molgen
from tests.gpu_common import context

pytestmark = pytest.mark.gpu
xs = pytest.importorskip("paper_2505_24807_gb300.xs")


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q *= np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1.0
    return q


def _solve(params, mols, method, precision, k, tol):
    ctx = context(params)
    try:
        xs.xs_ground_state(ctx.h, mols, scf_tol=1e-11)
        out = xs.xs_excited(ctx.h, method=method, nroots=k, tol=tol, precision=precision, n_mol=len(mols))
        return out["omega"], out["osc"]
    finally:
        ctx.close()


@pytest.mark.parametrize("method", ["CIS", "RPA"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_roots_invariant_under_reordering_and_rigid_motion(method, precision):
    params = molgen.make_params(0)
    Z, xyz = molgen.config_small(4)
    rng = np.random.default_rng(17)
    perm = rng.permutation(len(Z))
    moved = (xyz[perm] - xyz.mean(axis=0)) @ _rotation(rng).T + np.array([3.7, -11.2, 25.0])
    meth = xs.XS_CIS if method == "CIS" else xs.XS_TDHF
    prec = xs.XS_FP64 if precision == "fp64" else xs.XS_MIXED
    tol = 1e-8 if precision == "fp64" else 1e-5
    w, f = _solve(params, [(Z, xyz), (Z[perm], moved)], meth, prec, 6, tol)
    # float64: rounding order only; mixed: each side within its product
    # rounding of the exact roots (the reordered molecule rounds differently)
    dw = 1e-9 if precision == "fp64" else 2e-5
    df = 1e-7 if precision == "fp64" else 1e-4
    assert np.abs(w[0] - w[1]).max() < dw
    assert np.abs(f[0] - f[1]).max() < df


@pytest.mark.parametrize("method", ["CIS", "RPA"])
@pytest.mark.parametrize("batched", [0, 1])
def test_separated_fragments_double_every_root(method, batched):
    params = molgen.make_params(0)
    Z, xyz = molgen.config_small(5)
    rng = np.random.default_rng(23)
    far = (xyz - xyz.mean(axis=0)) @ _rotation(rng).T + np.array([1000.0, 0.0, 0.0])
    dimer = (np.concatenate([Z, Z]), np.concatenate([xyz, far]))
    meth = xs.XS_CIS if method == "CIS" else xs.XS_TDHF
    k = 5
    # 2k + 2 roots: no degenerate pair is cut at the last requested root;
    # batched = 1 solves monomer and dimer together in the lock-step batch
    if batched:
        ctx = context(params)
        try:
            xs.xs_ground_state(ctx.h, [(Z, xyz), dimer], scf_tol=1e-11)
            out = xs.xs_excited(ctx.h, method=meth, nroots=2 * k + 2, tol=1e-9, precision=xs.XS_FP64, batched=1,
                                n_mol=2)
        finally:
            ctx.close()
        wm, fm = out["omega"][:1, :k], out["osc"][:1, :k]
        wd, fd = out["omega"][1][:2 * k], out["osc"][1][:2 * k]
    else:
        wm, fm = _solve(params, [(Z, xyz)], meth, xs.XS_FP64, k, 1e-9)
        wd, fd = _solve(params, [dimer], meth, xs.XS_FP64, 2 * k + 2, 1e-9)
        wd, fd = wd[0][:2 * k], fd[0][:2 * k]
    # at 1000 Angstrom the other fragment's field and the exciton coupling move
    # the roots by ~1e-7 eV at most
    assert np.abs(wd[0::2] - wm[0]).max() < 1e-6
    assert np.abs(wd[1::2] - wm[0]).max() < 1e-6
    # oscillator strengths are invariant only summed over each degenerate pair
    assert np.abs(fd[0::2] + fd[1::2] - 2.0 * fm[0]).max() < 1e-6


def test_more_roots_than_amplitudes():
    """H2 in the minimal basis has one occupied and one virtual orbital: one
    root, the rest of the requested entries are 0."""
    params = molgen.make_params(0)
    h2 = (np.array([1, 1]), np.array([[0.0, 0.0, 0.0], [0.74, 0.0, 0.0]]))
    from oracle import excited, nddo, scf
    mol = nddo.Molecule(h2[0], h2[1], params)
    ints = nddo.Integrals(mol)
    res = scf.scf(mol, ints)
    A, B = excited.explicit_AB(res.eps, res.C, mol.nocc, nddo.full_eri(mol, ints))
    for method, meth, ref in (("CIS", xs.XS_CIS, excited.cis_bruteforce(A, 1)[0]),
                              ("RPA", xs.XS_TDHF, excited.rpa_bruteforce(A, B, 1)[0])):
        w, f = _solve(params, [h2], meth, xs.XS_FP64, 3, 1e-9)
        assert abs(w[0][0] - ref[0]) < 1e-9, method
        assert np.all(w[0][1:] == 0.0) and np.all(f[0][1:] == 0.0), method


def test_rejected_inputs():
    params = molgen.make_params(0)
    ctx = context(params)
    try:
        with pytest.raises(xs.XSError) as e:
            xs.xs_excited(ctx.h, method=xs.XS_CIS, nroots=2, tol=1e-6)
        assert e.value.status == xs.XS_ESTATE          # no ground state yet
        assert xs.load().xs_ground_state(ctx.h, 0, None, None, None, 1e-10, 300, None) == xs.XS_EINVAL   # no molecule
        xs.xs_ground_state(ctx.h, [molgen.config_small(1)])
        for bad in (dict(nroots=0), dict(tol=0.0), dict(precision=7), dict(method=5), dict(batched=3)):
            kw = dict(method=xs.XS_CIS, nroots=2, tol=1e-6)
            kw.update(bad)
            with pytest.raises(xs.XSError) as e:
                xs.xs_excited(ctx.h, **kw)
            assert e.value.status == xs.XS_EINVAL, bad
    finally:
        ctx.close()
