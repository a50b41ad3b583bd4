"""Float64 subspace products of the Davidson step (projections V^T A V,
Gram-Schmidt against V, Ritz vectors and residuals V x) on the tensor cores
by exact digit splitting, against numpy float64 and the float64-pipe path.

The bound for a float64 dot product of length L is about L u sum|a||b|
(u = 2^-53); the digit-split products must stay within a small multiple of
u sum|a||b| (they are exact up to the 2^-55 relative truncation of each
input and the final float64 additions)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2505_24807_gb300 import xs
    h = xs.xs_create(0)
    yield h
    xs.xs_destroy(h)


U = 2.0 ** -53


def _mixed(rng, shape, spread=10.0):
    """Gaussian entries with per-row scales over 10 decades and elementwise
    magnitudes over `spread` decades, a few exact zeros."""
    x = rng.standard_normal(shape)
    x *= 10.0 ** rng.uniform(-spread, 0.0, size=shape)
    x *= 10.0 ** rng.uniform(-5, 5, size=(shape[0], 1))
    x[rng.random(shape) < 0.01] = 0.0
    return x


# N = 37, 40 and 81 reach the 320-column Gram tile (up to 40 B vectors per
# launch, a partly filled second 160-row box for 37, three launches for 81)
@pytest.mark.parametrize("M,N,L", [(37, 5, 5000 + 37), (3, 33, 4096), (160, 20, 100_003), (1, 1, 1),
                                   (50, 40, 30_011), (17, 37, 9000), (5, 81, 5000)])
def test_gram_matches_float64(ctx, M, N, L):
    from paper_2505_24807_gb300 import xs
    rng = np.random.default_rng(M * 1000 + N + L)
    A = _mixed(rng, (M, L))
    B = _mixed(rng, (N, L))
    ref = A @ B.T
    bound = np.abs(A) @ np.abs(B).T
    got = xs.xs_subspace_gram(ctx, A, B, emulated=True)
    simt = xs.xs_subspace_gram(ctx, A, B, emulated=False)
    # both are within a few u of the exact product; numpy itself is off by up to ~sqrt(L) u
    tol = 8 * U * np.sqrt(L) * bound + 1e-300
    assert np.all(np.abs(got - ref) <= tol)
    assert np.all(np.abs(simt - ref) <= tol)


def test_gram_integers_exact(ctx):
    """Integer inputs whose products sum below 2^53: the digit-split product
    is exact, so it equals the integer result bit for bit (the float32
    tensor-core accumulation of digit products is exact)."""
    from paper_2505_24807_gb300 import xs
    rng = np.random.default_rng(7)
    L = 20_000
    A = rng.integers(-2**16, 2**16, size=(19, L))
    B = rng.integers(-2**16, 2**16, size=(9, L))
    exact = A @ B.T
    assert np.abs(exact).max() < 2**53
    got = xs.xs_subspace_gram(ctx, A.astype(np.float64), B.astype(np.float64), emulated=True)
    assert np.array_equal(got, exact.astype(np.float64))


def test_gram_integers_exact_wide(ctx):
    """The 320-column Gram tile (40 B vectors, one pass over A) is exact on
    integer inputs like the narrower tiles."""
    from paper_2505_24807_gb300 import xs
    rng = np.random.default_rng(11)
    L = 12_345
    A = rng.integers(-2**16, 2**16, size=(23, L))
    B = rng.integers(-2**16, 2**16, size=(40, L))
    exact = A @ B.T
    assert np.abs(exact).max() < 2**53
    got = xs.xs_subspace_gram(ctx, A.astype(np.float64), B.astype(np.float64), emulated=True)
    assert np.array_equal(got, exact.astype(np.float64))


@pytest.mark.parametrize("nb,S,nout,L", [(3, 170, 40, 3005), (2, 20, 20, 129), (1, 1, 1, 1), (3, 64, 7, 70_001)])
def test_combine_matches_float64(ctx, nb, S, nout, L):
    from paper_2505_24807_gb300 import xs
    rng = np.random.default_rng(nb * 100 + S + nout + L)
    X = np.stack([_mixed(rng, (S, L)) for _ in range(nb)])
    coef = np.stack([_mixed(rng, (S, nout), spread=6.0) for _ in range(nb)])
    ref = np.einsum("bmk,bml->kl", coef, X)
    bound = np.einsum("bmk,bml->kl", np.abs(coef), np.abs(X))
    got = xs.xs_subspace_combine(ctx, X, coef, emulated=True)
    simt = xs.xs_subspace_combine(ctx, X, coef, emulated=False)
    assert np.all(np.abs(simt - ref) <= 8 * U * np.sqrt(nb * S) * bound + 1e-300)
    # The digit products keep the pairs i + j <= 9 of the eight digits of
    # each side, so the error is bounded relative to each row's largest entry
    # (the scale its digits are taken against), not elementwise:
    # |err_kl| <~ u sqrt(S) sum_m |coef_mk| max_l' |X_m,l'|
    rowmax = np.abs(X).max(axis=2)                                  # nb x S
    scale = np.einsum("bmk,bm->k", np.abs(coef), rowmax)[:, None]   # nout x 1
    assert np.all(np.abs(got - ref) <= 16 * U * np.sqrt(nb * S) * scale + 1e-300)


def test_combine_integers_exact(ctx):
    from paper_2505_24807_gb300 import xs
    rng = np.random.default_rng(11)
    X = rng.integers(-2**18, 2**18, size=(3, 150, 777))
    coef = rng.integers(-2**18, 2**18, size=(3, 150, 24))
    exact = np.einsum("bmk,bml->kl", coef, X)
    assert np.abs(exact).max() < 2**53
    got = xs.xs_subspace_combine(ctx, X.astype(np.float64), coef.astype(np.float64), emulated=True)
    assert np.array_equal(got, exact.astype(np.float64))


def test_rejects_non_finite(ctx):
    from paper_2505_24807_gb300 import xs
    A = np.ones((4, 100))
    A[2, 50] = np.nan
    with pytest.raises(RuntimeError):
        xs.xs_subspace_gram(ctx, A, np.ones((2, 100)), emulated=True)
    # the context stays usable
    got = xs.xs_subspace_gram(ctx, np.ones((4, 100)), np.ones((2, 100)), emulated=True)
    assert np.array_equal(got, np.full((4, 2), 100.0))


@pytest.mark.parametrize("method", ["CIS", "TDHF"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_davidson_emulated_subspace_matches_float64_pipe(method, precision):
    """The whole solve with the subspace products on the tensor cores (exact
    digit splitting) against the float64-pipe subspace: the same roots to
    well below the 1e-5 eV target, the same oscillator strengths."""
    import molgen
    from paper_2505_24807_gb300 import xs
    params = molgen.make_params(0)
    Z, xyz = molgen.make_chain(3, 40, 60)
    with xs.Context(0, molgen.params_table(params)) as h:
        xs.xs_ground_state(h, [(Z, xyz)])
        m = xs.XS_TDHF if method == "TDHF" else xs.XS_CIS
        p = xs.XS_MIXED if precision == "mixed" else xs.XS_FP64
        tol = 1e-5 if precision == "mixed" else 1e-7
        # the same subspace cap for both (the default depends on the subspace arithmetic)
        ref = xs.xs_excited(h, method=m, nroots=6, tol=tol, precision=p, subspace=xs.XS_SUBSPACE_FP64,
                            max_subspace=72)
        emu = xs.xs_excited(h, method=m, nroots=6, tol=tol, precision=p, subspace=xs.XS_SUBSPACE_EMULATED,
                            max_subspace=72)
        assert ref["info"]["converged"] and emu["info"]["converged"]
        # float64 products: the two solves agree to rounding; mixed products
        # carry ~1e-7 relative noise, so the two solves stop at different
        # points inside the 1e-5 eV target
        bound = 1e-5 if precision == "mixed" else 1e-9
        assert np.abs(emu["omega"] - ref["omega"]).max() < bound
        assert np.abs(emu["osc"] - ref["osc"]).max() < 1e-6
        assert abs(int(emu["iters"][0]) - int(ref["iters"][0])) <= 3


def _spectrum_matrix(rng, lam):
    S = lam.size
    q, r = np.linalg.qr(rng.standard_normal((S, S)))
    q *= np.sign(np.diag(r))
    return (q * lam) @ q.T


def _eig_cases():
    rng = np.random.default_rng(41)
    cases = {}
    M = rng.standard_normal((97, 97))
    cases["random"] = (0.5 * (M + M.T), 12)
    base = np.sort(rng.uniform(5.0, 20.0, 60))
    pairs = np.repeat(base, 2)                                 # exactly degenerate pairs
    cases["pairs"] = (_spectrum_matrix(rng, pairs), 12)
    for split in (1e-12, 1e-9, 1e-7, 1e-5, 1e-4):              # nearly degenerate pairs (relative to |A| ~ 20)
        lam = np.sort(np.concatenate([base, base + split * 20.0]))
        cases["split%g" % split] = (_spectrum_matrix(rng, lam), 14)
    lam = np.sort(np.concatenate([np.full(3, 7.0), np.full(5, 9.0), rng.uniform(10.0, 30.0, 100)]))
    cases["clusters3+5"] = (_spectrum_matrix(rng, lam), 10)   # a cluster larger than the rotation limit
    lam = np.sort(np.concatenate([np.full(4, 11.0), rng.uniform(3.0, 10.9, 9), rng.uniform(12.0, 30.0, 60)]))
    cases["cut"] = (_spectrum_matrix(rng, lam), 11)           # the cut falls inside a 4-fold cluster
    return cases


@pytest.mark.parametrize("name", sorted(_eig_cases()))
def test_subspace_eigensolver(ctx, name):
    """The Davidson step's eigensolver against numpy: eigenvalues, residuals
    |A z - lambda z| and orthonormality (degenerate eigenvectors are not
    unique, so they are compared through what the step uses)."""
    from paper_2505_24807_gb300 import xs
    A, k = _eig_cases()[name]
    w, Z = xs.xs_subspace_eig(ctx, A, k)
    ref = np.linalg.eigvalsh(A)[:k]
    scale = np.abs(A).max() * A.shape[0]
    assert np.abs(w - ref).max() <= 1e-13 * scale, name
    assert np.abs(A @ Z - Z * w).max() <= 1e-12 * scale, name
    # eigenvectors of one cluster are orthogonalised as they are found; across
    # clusters orthogonality comes from the Rayleigh-quotient shifted solves
    # (measured: 1e-14 to 8e-12, 5e-10 between exactly degenerate pairs 0.01 apart)
    assert np.abs(Z.T @ Z - np.eye(k)).max() <= 1e-9, name
