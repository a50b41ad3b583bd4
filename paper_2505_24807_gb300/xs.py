"""ctypes binding of libxs (argument marshalling only; see include/xs.h).

Array arguments may be numpy arrays (host memory) or CUDA tensors / objects
with ``data_ptr()`` (device memory); the library resolves either through
unified addressing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libxs.so")

XS_OK, XS_EINVAL, XS_ENOMEM, XS_ESCF, XS_EUNSTABLE, XS_ENOCONV, XS_ECUDA, XS_ETIMEOUT, XS_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
XS_CIS, XS_TDHF = 0, 1
XS_FP64, XS_MIXED = 0, 1
XS_KIND_A, XS_KIND_APB, XS_KIND_AMB, XS_KIND_G, XS_KIND_A_TRIPLET, XS_KIND_APB_TRIPLET = 0, 1, 2, 3, 4, 5
XS_SINGLET, XS_TRIPLET = 0, 1
XS_GUESS_PLAIN, XS_GUESS_LEARNED = 0, 1
XS_SUBSPACE_AUTO, XS_SUBSPACE_FP64, XS_SUBSPACE_EMULATED = 0, 1, 2
XS_NPARAM, XS_NELEM = 13, 4
XS_MLP_FEATURES = 11

STATUS_NAMES = {0: "XS_OK", -1: "XS_EINVAL", -2: "XS_ENOMEM", -3: "XS_ESCF", -4: "XS_EUNSTABLE",
                -5: "XS_ENOCONV", -6: "XS_ECUDA", -7: "XS_ETIMEOUT", -8: "XS_ESTATE"}


class XSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class xs_gs_info(C.Structure):
    _fields_ = [("n_mol", C.c_int), ("max_scf_iter_used", C.c_int), ("seconds", C.c_double)]


class xs_ex_opts(C.Structure):
    _fields_ = [("method", C.c_int), ("nroots", C.c_int), ("tol", C.c_double), ("precision", C.c_int),
                ("guess", C.c_int), ("max_subspace", C.c_int), ("max_iter", C.c_int), ("batched", C.c_int),
                ("subspace", C.c_int), ("memory_limit", C.c_double), ("spin", C.c_int)]


class xs_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("products", C.c_longlong), ("converged", C.c_int),
                ("polished", C.c_int), ("learned", C.c_int), ("fallback", C.c_int), ("seconds", C.c_double),
                ("seconds_products", C.c_double), ("max_subspace_used", C.c_int),
                ("tol_used", C.c_double), ("graph_launches", C.c_longlong)]


class xs_prof_entry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int), ("ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


_lib = None


def load():
    """Load libxs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libxs.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    sig = {
        "xs_create": (i, [C.POINTER(vp), i, vp]),
        "xs_destroy": (i, [vp]),
        "xs_last_error": (C.c_char_p, [vp]),
        "xs_set_params": (i, [vp, vp, i]),
        "xs_ground_state": (i, [vp, i, vp, vp, vp, d, i, C.POINTER(xs_gs_info)]),
        "xs_get_sizes": (i, [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
        "xs_get_orbitals": (i, [vp, i, vp, vp]),
        "xs_get_model": (i, [vp, i, vp, vp, C.POINTER(i)]),
        "xs_set_orbitals": (i, [vp, i, vp, vp]),
        "xs_apply": (i, [vp, i, i, i, vp, vp, i]),
        "xs_excited": (i, [vp, C.POINTER(xs_ex_opts), vp, vp, vp, vp, C.POINTER(xs_solve_info)]),
        "xs_get_amplitudes": (i, [vp, i, i, vp, vp, sz]),
        "xs_profile": (i, [vp, i]),
        "xs_gbuild_noalloc": (i, [vp, i, i, vp, vp]),
        "xs_subspace_gram": (i, [vp, i, i, C.c_longlong, vp, vp, vp, i]),
        "xs_subspace_combine": (i, [vp, i, i, i, C.c_longlong, vp, vp, vp, i]),
        "xs_subspace_eig": (i, [vp, i, i, vp, vp, vp]),
        "xs_spectrum": (i, [vp, i, vp, vp, d, i, vp, vp]),
        "xs_gradient": (i, [vp, i, i, vp, C.POINTER(i)]),
        "xs_mlp_nparams": (i, []),
        "xs_mlp_init": (i, [vp, C.c_ulonglong]),
        "xs_mlp_get_weights": (i, [vp, vp]),
        "xs_mlp_set_weights": (i, [vp, vp]),
        "xs_mlp_features": (i, [vp, i, i, vp, vp, C.POINTER(i)]),
        "xs_mlp_targets": (i, [vp, i, i, vp, vp]),
        "xs_mlp_forward": (i, [vp, i, vp, vp]),
        "xs_mlp_train": (i, [vp, i, vp, vp, i, i, C.c_float, vp]),
        "xs_mlp_grad": (i, [vp, i, vp, vp, vp, C.POINTER(C.c_float)]),
        "xs_profile_read": (i, [vp, C.POINTER(xs_prof_entry), i, C.POINTER(i)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported array type {type(x)}")


def _check(ctx, rc, allow=()):
    if rc != XS_OK and rc not in allow:
        raise XSError(rc, xs_last_error(ctx))
    return rc


def xs_create(device: int = 0, stream=None):
    lib = load()
    h = C.c_void_p()
    rc = lib.xs_create(C.byref(h), int(device), C.c_void_p(stream) if stream else None)
    if rc != XS_OK:
        raise XSError(rc, "xs_create failed")
    return h


def xs_destroy(ctx):
    return load().xs_destroy(ctx)


def xs_last_error(ctx) -> str:
    r = load().xs_last_error(ctx)
    return r.decode() if r else ""


def xs_set_params(ctx, table):
    t = np.ascontiguousarray(table, dtype=np.float64)
    return _check(ctx, load().xs_set_params(ctx, _ptr(t), int(t.shape[0])))


def xs_ground_state(ctx, molecules, scf_tol=1e-10, max_iter=300):
    """molecules: list of (Z, xyz); returns xs_gs_info as a dict."""
    natoms = np.array([len(z) for z, _ in molecules], dtype=np.int32)
    Z = np.ascontiguousarray(np.concatenate([np.asarray(z, dtype=np.int32) for z, _ in molecules]))
    xyz = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).reshape(-1, 3) for _, x in molecules]))
    info = xs_gs_info()
    _check(ctx, load().xs_ground_state(ctx, len(molecules), _ptr(natoms), _ptr(Z), _ptr(xyz), float(scf_tol),
                                       int(max_iter), C.byref(info)))
    return {"n_mol": info.n_mol, "max_scf_iter_used": info.max_scf_iter_used, "seconds": info.seconds}


def xs_get_sizes(ctx, mol=0):
    nao, nocc, nat = C.c_int(), C.c_int(), C.c_int()
    _check(ctx, load().xs_get_sizes(ctx, int(mol), C.byref(nao), C.byref(nocc), C.byref(nat)))
    return nao.value, nocc.value, nat.value


def xs_get_model(ctx, mol=0):
    """Two-centre product supermatrix W (nprod x nprod) and core Hamiltonian H (n x n)."""
    n, _, _ = xs_get_sizes(ctx, mol)
    npr = C.c_int()
    _check(ctx, load().xs_get_model(ctx, int(mol), None, None, C.byref(npr)))
    W = np.empty((npr.value, npr.value))
    H = np.empty((n, n))
    _check(ctx, load().xs_get_model(ctx, int(mol), _ptr(W), _ptr(H), None))
    return W, H


def xs_get_orbitals(ctx, mol=0):
    n, _, _ = xs_get_sizes(ctx, mol)
    Cm = np.empty((n, n))
    eps = np.empty(n)
    _check(ctx, load().xs_get_orbitals(ctx, int(mol), _ptr(Cm), _ptr(eps)))
    return Cm, eps


def xs_set_orbitals(ctx, mol, Cm, eps):
    Cm = np.ascontiguousarray(Cm, dtype=np.float64)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    return _check(ctx, load().xs_set_orbitals(ctx, int(mol), _ptr(Cm), _ptr(eps)))


def xs_apply(ctx, mol, kind, x, precision=XS_FP64, out=None):
    """Products of nvec vectors x (nvec x ov or nvec x n x n for XS_KIND_G)."""
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float64)
        if out is None:
            out = np.empty_like(x)
    elif out is None:
        out = x.new_empty(x.shape)
    nvec = x.shape[0]
    _check(ctx, load().xs_apply(ctx, int(mol), int(kind), int(nvec), _ptr(x), _ptr(out), int(precision)))
    return out


def xs_excited(ctx, method=XS_CIS, nroots=5, tol=1e-6, precision=XS_FP64, guess=XS_GUESS_PLAIN, max_subspace=0,
               max_iter=0, batched=0, n_mol=1, outputs=None, allow=(), subspace=0, memory_limit=0.0,
               spin=0):
    """Returns dict(omega, osc, iters, resid, info, status); arrays of shape (n_mol, nroots)."""
    o = xs_ex_opts(int(method), int(nroots), float(tol), int(precision), int(guess), int(max_subspace),
                   int(max_iter), int(batched), int(subspace), float(memory_limit), int(spin))
    if outputs is None:
        outputs = dict(omega=np.zeros((n_mol, nroots)), osc=np.zeros((n_mol, nroots)),
                       iters=np.zeros(n_mol, dtype=np.int32), resid=np.zeros((n_mol, nroots)))
    info = xs_solve_info()
    rc = load().xs_excited(ctx, C.byref(o), _ptr(outputs["omega"]), _ptr(outputs["osc"]), _ptr(outputs["iters"]),
                           _ptr(outputs["resid"]), C.byref(info))
    _check(ctx, rc, allow=allow)
    out = dict(outputs)
    out["status"] = rc
    out["info"] = {f: getattr(info, f) for f, _ in xs_solve_info._fields_}
    return out


def xs_get_amplitudes(ctx, mol, root):
    n, o, _ = xs_get_sizes(ctx, mol)
    ov = o * (n - o)
    X = np.empty(ov)
    Y = np.empty(ov)
    _check(ctx, load().xs_get_amplitudes(ctx, int(mol), int(root), _ptr(X), _ptr(Y), ov))
    return X.reshape(o, n - o), Y.reshape(o, n - o)


def xs_gbuild_noalloc(ctx, mol, R, G):
    """G(R) into caller-owned device arrays, no device allocation (see xs.h).
    Asynchronous on the context's stream."""
    return _check(ctx, load().xs_gbuild_noalloc(ctx, int(mol), int(R.shape[0]), _ptr(R), _ptr(G)))


def xs_subspace_gram(ctx, A, B, emulated=True):
    """C = A B^T (float64) for A (M x L) and B (N x L): on the tensor cores by
    exact digit splitting (emulated=True) or on the float64 pipe."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, L = A.shape
    N = B.shape[0]
    Cm = np.empty((M, N))
    _check(ctx, load().xs_subspace_gram(ctx, M, N, L, _ptr(A), _ptr(B), _ptr(Cm), int(bool(emulated))))
    return Cm


def xs_subspace_eig(ctx, A, k):
    """k lowest eigenpairs of the symmetric float64 matrix A with the Davidson
    step's eigensolver: (w ascending, Z with the eigenvectors in columns)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    S = A.shape[0]
    w = np.empty(k)
    Z = np.empty((S, k))
    _check(ctx, load().xs_subspace_eig(ctx, S, int(k), _ptr(A), _ptr(w), _ptr(Z)))
    return w, Z


def xs_subspace_combine(ctx, X, coef, emulated=True):
    """Y[k] = sum_b sum_m coef[b][m][k] X[b][m] for X (nb x S x L) and coef
    (nb x S x nout), nb <= 3."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    nb, S, L = X.shape
    nout = coef.shape[2]
    Y = np.empty((nout, L))
    _check(ctx, load().xs_subspace_combine(ctx, nb, S, nout, L, _ptr(X), _ptr(coef), _ptr(Y), int(bool(emulated))))
    return Y


def xs_gradient(ctx, mol=0, root=0):
    """d omega_root / d parameter (XS_NELEM x XS_NPARAM, eV per parameter unit)
    of the last singlet CIS or TDHF solve; returns (grad, adjoint iterations)."""
    g = np.zeros((XS_NELEM, XS_NPARAM))
    its = C.c_int()
    _check(ctx, load().xs_gradient(ctx, int(mol), int(root), _ptr(g), C.byref(its)))
    return g, its.value


def xs_spectrum(ctx, omega, f, grid, width=0.1):
    """Absorption spectrum on the energy grid (eV): the oscillator strengths f
    of the states at omega (eV) broadened by unit-area Gaussians of standard
    deviation width (eV)."""
    omega = np.ascontiguousarray(omega, dtype=np.float64).ravel()
    f = np.ascontiguousarray(f, dtype=np.float64).ravel()
    grid = np.ascontiguousarray(grid, dtype=np.float64).ravel()
    if omega.shape != f.shape:
        raise ValueError("omega and f differ in length")
    out = np.empty_like(grid)
    _check(ctx, load().xs_spectrum(ctx, len(omega), _ptr(omega), _ptr(f), float(width), len(grid), _ptr(grid),
                                   _ptr(out)))
    return out


def xs_mlp_nparams():
    return int(load().xs_mlp_nparams())


def xs_mlp_init(ctx, seed=0):
    return _check(ctx, load().xs_mlp_init(ctx, int(seed)))


def xs_mlp_get_weights(ctx):
    w = np.empty(xs_mlp_nparams(), dtype=np.float32)
    _check(ctx, load().xs_mlp_get_weights(ctx, _ptr(w)))
    return w


def xs_mlp_set_weights(ctx, w):
    w = np.ascontiguousarray(w, dtype=np.float32)
    return _check(ctx, load().xs_mlp_set_weights(ctx, _ptr(w)))


def xs_mlp_features(ctx, mol, npairs):
    F = np.empty((npairs, XS_MLP_FEATURES), dtype=np.float32)
    P = np.empty(npairs, dtype=np.int64)
    cnt = C.c_int()
    _check(ctx, load().xs_mlp_features(ctx, int(mol), int(npairs), _ptr(F), _ptr(P), C.byref(cnt)))
    return F[: cnt.value], P[: cnt.value]


def xs_mlp_targets(ctx, mol, pairs):
    pairs = np.ascontiguousarray(pairs, dtype=np.int64)
    T = np.empty((pairs.size, 2), dtype=np.float32)
    _check(ctx, load().xs_mlp_targets(ctx, int(mol), int(pairs.size), _ptr(pairs), _ptr(T)))
    return T


def xs_mlp_forward(ctx, features):
    F = np.ascontiguousarray(features, dtype=np.float32)
    out = np.empty((F.shape[0], 2), dtype=np.float32)
    _check(ctx, load().xs_mlp_forward(ctx, int(F.shape[0]), _ptr(F), _ptr(out)))
    return out


def xs_mlp_grad(ctx, features, targets):
    F = np.ascontiguousarray(features, dtype=np.float32)
    T = np.ascontiguousarray(targets, dtype=np.float32)
    g = np.empty(xs_mlp_nparams(), dtype=np.float32)
    loss = C.c_float()
    _check(ctx, load().xs_mlp_grad(ctx, int(F.shape[0]), _ptr(F), _ptr(T), _ptr(g), C.byref(loss)))
    return g, loss.value


def xs_mlp_train(ctx, features, targets, epochs=10, batch=4096, lr=1e-3):
    F = np.ascontiguousarray(features, dtype=np.float32)
    T = np.ascontiguousarray(targets, dtype=np.float32)
    loss = np.zeros(int(epochs), dtype=np.float32)
    _check(ctx, load().xs_mlp_train(ctx, int(F.shape[0]), _ptr(F), _ptr(T), int(epochs), int(batch), float(lr),
                                    _ptr(loss)))
    return loss


def xs_profile(ctx, enable=True):
    """enable: True / 1 (CUDA-event timing), 2 (counts only), False / 0 (off)."""
    return _check(ctx, load().xs_profile(ctx, int(enable)))


def xs_profile_read(ctx):
    """dict name -> dict(launches, ms, bytes, flops) of the instrumented kernels."""
    n = C.c_int()
    _check(ctx, load().xs_profile_read(ctx, None, 0, C.byref(n)))
    arr = (xs_prof_entry * max(n.value, 1))()
    _check(ctx, load().xs_profile_read(ctx, arr, n.value, C.byref(n)))
    return {arr[k].name.decode(): dict(launches=arr[k].launches, ms=arr[k].ms, bytes=arr[k].bytes,
                                       flops=arr[k].flops) for k in range(n.value)}


class Context:
    """Owns one libxs context: ``with Context() as ctx: ...``."""

    def __init__(self, device=0, params=None):
        self.h = xs_create(device)
        if params is not None:
            xs_set_params(self.h, params)

    def __enter__(self):
        return self.h

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if self.h is not None:
            xs_destroy(self.h)
            self.h = None
