"""Writes the oracle's reference excitation energies for the seeded workloads.

Calls only ``oracle/`` and ``molgen``: every stored value here comes from the
FP64 CPU oracle.  Usage: python tests/golden/make_golden.py [medium|large ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import molgen  # noqa: E402
from oracle import excited, nddo, scf  # noqa: E402

WORKLOADS = {
    # name: (generator, methods, nroots, tol)
    "medium": (molgen.config_medium, ("CIS", "RPA"), 10, 1e-6),
    "large": (molgen.config_large, ("RPA",), 10, 1e-6),
}


def run(name):
    gen, methods, k, tol = WORKLOADS[name]
    params = molgen.make_params(0)
    Z, xyz = gen(0)
    t0 = time.time()
    mol = nddo.Molecule(Z, xyz, params)
    ints = nddo.Integrals(mol)
    res = scf.scf(mol, ints)
    out = dict(workload=name, seed=0, param_seed=0, natoms=int(len(Z)), nao=mol.nao, nocc=mol.nocc,
               homo_lumo_eV=[float(res.eps[mol.nocc - 1]), float(res.eps[mol.nocc])],
               scf_iterations=int(res.iterations), scf_seconds=time.time() - t0, tol=tol, roots={})
    for meth in methods:
        t1 = time.time()
        r = excited.solve(mol, ints, res, meth, k, tol=tol)
        out["roots"][meth] = dict(omega=[float(x) for x in r["omega"]], f=[float(x) for x in r["f"]],
                                  residual=[float(x) for x in r["residual"]], iterations=int(r["iterations"]),
                                  products=int(r["products"]), converged=bool(r["converged"]),
                                  seconds=time.time() - t1)
        print(name, meth, np.round(r["omega"], 6), r["iterations"], f"{time.time() - t1:.1f}s", flush=True)
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(WORKLOADS)):
        run(name)
