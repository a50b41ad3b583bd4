"""Small, self-contained invocations of single libxs kernel families through
the public API, sized for profiling one or a few launches (Nsight Compute
captures of the full workload would hold ~12 GB on the device):

  python -m paper_2505_24807_gb300.kernel_cases oz      # digit-product kernel: combination, then Gram
  python -m paper_2505_24807_gb300.kernel_cases tc      # TF32 transforms: one TDHF product, large molecule
  python -m paper_2505_24807_gb300.kernel_cases gbuild  # G build: one TDHF product, medium molecule
  python -m paper_2505_24807_gb300.kernel_cases slice   # digit split of 3 x 20 vectors of 600k amplitudes
  python -m paper_2505_24807_gb300.kernel_cases batch   # one lock-step batched CIS solve, 256 molecules of 20-200 atoms

Inputs are seeded; each case prints one line with a checksum.
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import molgen  # noqa: E402
from paper_2505_24807_gb300 import xs  # noqa: E402


def case_oz():
    ctx = xs.xs_create(0)
    rng = np.random.default_rng(0)
    L = 300_000
    X = rng.standard_normal((3, 160, L))
    coef = rng.standard_normal((3, 160, 20))
    A = rng.standard_normal((160, L))
    B = rng.standard_normal((20, L))
    for _ in range(2):
        Y = xs.xs_subspace_combine(ctx, X, coef, emulated=True)
        C = xs.xs_subspace_gram(ctx, A, B, emulated=True)
    return float(np.abs(Y).max()), float(np.abs(C).max())


def _product_case(gen, nvec):
    ctx = xs.xs_create(0)
    xs.xs_set_params(ctx, molgen.params_table(molgen.make_params(0)))
    Z, xyz = gen(0)
    xs.xs_ground_state(ctx, [(Z, xyz)])
    n, o, _ = xs.xs_get_sizes(ctx, 0)
    X = np.random.default_rng(1).standard_normal((nvec, o * (n - o)))
    Y = xs.xs_apply(ctx, 0, xs.XS_KIND_APB, X, precision=xs.XS_MIXED)
    return (float(np.abs(Y).max()),)


def case_slice():
    ctx = xs.xs_create(0)
    X = np.random.default_rng(0).standard_normal((3, 20, 600_000))
    coef = np.random.default_rng(1).standard_normal((3, 20, 4))
    Y = xs.xs_subspace_combine(ctx, X, coef, emulated=True)
    return (float(np.abs(Y).max()),)


def case_batch():
    ctx = xs.xs_create(0)
    xs.xs_set_params(ctx, molgen.params_table(molgen.make_params(0)))
    mols = [molgen.config_batch(s) for s in range(256)]
    xs.xs_ground_state(ctx, mols)
    out = xs.xs_excited(ctx, method=xs.XS_CIS, nroots=6, tol=1e-5, precision=xs.XS_MIXED, batched=1, n_mol=len(mols))
    return float(out["omega"].sum()), int(out["info"]["iterations"])


CASES = {
    "oz": case_oz,
    "tc": lambda: _product_case(molgen.config_large, 10),
    "gbuild": lambda: _product_case(molgen.config_medium, 8),
    "slice": case_slice,
    "batch": case_batch,
}


def main():
    name = sys.argv[1] if len(sys.argv) > 1 else "oz"
    if name not in CASES:
        raise SystemExit(f"unknown case {name!r}; one of {sorted(CASES)}")
    print("ok", name, *CASES[name](), flush=True)


if __name__ == "__main__":
    main()
