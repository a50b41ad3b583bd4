"""Parity at the benchmark sizes: roots and oscillator strengths of the CUDA
path against the oracle's stored values (tests/golden/*.json, written by
tests/golden/make_golden.py, which calls only the oracle).

Tolerances: 1e-6 eV (float64 path) and 1e-5 eV (mixed precision) on the
excitation energies -- the stated target -- and 1e-4 on oscillator strengths.
"""
import json
import os

import numpy as np
import pytest

import molgen
from tests.gpu_common import context

pytestmark = pytest.mark.gpu
xs = pytest.importorskip("paper_2505_24807_gb300.xs")

HERE = os.path.dirname(os.path.abspath(__file__))
GEN = {"medium": molgen.config_medium, "large": molgen.config_large}


def golden(name):
    path = os.path.join(HERE, "golden", f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle values for {name}")
    with open(path) as f:
        return json.load(f)


CASES = [("medium", "CIS", 0), ("medium", "CIS", 1), ("medium", "RPA", 0), ("medium", "RPA", 1),
         ("large", "RPA", 1)]


@pytest.mark.parametrize("name,method,precision", CASES)
def test_roots_match_stored_oracle(name, method, precision):
    g = golden(name)
    if method not in g["roots"]:
        pytest.skip("method not stored")
    ref = g["roots"][method]
    Z, xyz = GEN[name](g["seed"])
    ctx = context(molgen.make_params(g["param_seed"]))
    try:
        xs.xs_ground_state(ctx.h, [(Z, xyz)])
        nao, nocc, _ = xs.xs_get_sizes(ctx.h, 0)
        assert (nao, nocc) == (g["nao"], g["nocc"])
        k = len(ref["omega"])
        out = xs.xs_excited(ctx.h, method=xs.XS_CIS if method == "CIS" else xs.XS_TDHF, nroots=k, tol=1e-5,
                            precision=precision)
    finally:
        ctx.close()
    tol = 1e-6 if precision == 0 else 1e-5
    d_omega = np.abs(out["omega"][0] - np.array(ref["omega"]))
    d_f = np.abs(out["osc"][0] - np.array(ref["f"]))
    print(name, method, precision, "max |d omega| (eV):", d_omega.max(), "max |d f|:", d_f.max())
    assert d_omega.max() < tol
    assert d_f.max() < 1e-4
