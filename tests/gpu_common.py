"""Shared helpers of the GPU parity tests."""
import numpy as np

import molgen
from paper_2505_24807_gb300 import xs


def context(params=None):
    if params is None:
        params = molgen.make_params(0)
    return xs.Context(0, molgen.params_table(params))


def oracle_ground_state(Z, xyz, params):
    from oracle import nddo, scf
    mol = nddo.Molecule(Z, xyz, params)
    ints = nddo.Integrals(mol)
    res = scf.scf(mol, ints)
    return mol, ints, res


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def mixed_product_tol(n):
    """Bound on max|Y - ref| / max|ref - de X| for the mixed-precision product
    (split-TF32 tensor-core transforms, float32 G build) of an n-AO molecule.

    The product chains four split-TF32 GEMMs, each contracting over at most n
    terms.  The tensor cores add every 8-term MMA step into a float32
    accumulator with truncation, which biases a sum of K terms by about
    (K / 8) steps x half an ulp (2^-24) x 2/3 of its final magnitude (the mean
    running sum): (K / 12) 2^-24 relative.  The GEMM promotes its accumulator
    every 128 terms into round-to-nearest float32 registers, so K is at most
    128 in that bias, and the sqrt(K / 128) promoting additions add about half
    an ulp each.  Each GEMM also drops lo*lo (2^-22 relative) and reads lo
    rounded to TF32 (2 x 2^-22; lo is rounded to nearest TF32 when split, so
    this part is unbiased), and stores its output in float32.  Summed over
    the four GEMMs, with a factor 2 of headroom.  The exact float64 term de*X
    carries no rounding, so the error is measured against the rest of the
    product (C_occ^T G C_vir).  Measured on a GB300: 2.1e-6 at n = 62,
    4.1e-6 at n = 600, 3.6e-6 at n = 2200 (this bound: 8.4e-6, 1.1e-5,
    1.2e-5; with one float32 accumulator over all of K and an unrounded lo the
    same products were 1.9e-6, 1.3e-5 and 4.7e-5 off)."""
    k = min(n, 128)
    per_gemm = (k / 12.0) * 2.0 ** -24 + (n / 128.0) ** 0.5 * 2.0 ** -25 + 3.0 * 2.0 ** -22
    return 2.0 * 4.0 * per_gemm


def mixed_product_err(Y, ref, X, eps, nocc):
    """max|Y - ref| / max|ref - de X| (see mixed_product_tol)."""
    from oracle import excited
    Y = np.asarray(Y).reshape(len(X), -1)
    ref = np.asarray(ref).reshape(len(X), -1)
    de = excited.delta_eps(eps, nocc).reshape(-1)
    g_part = ref - de[None, :] * np.asarray(X).reshape(len(X), -1)
    return float(np.abs(Y - ref).max() / np.abs(g_part).max())
