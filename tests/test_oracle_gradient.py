"""Pins of the oracle's parameter derivatives of excitation energies (CPU only).

The oracle differentiates by five-point central differences of brute-force
roots after a fresh SCF at each displaced parameter.  Pinned here against
the two-site H2 closed forms (omega_CIS = -2t + gss/2 - gamma/2 with
t = beta_s S_ss and gamma = kappa erf(aR)/R, a = sqrt(pi) gss / (2 kappa)):
  d omega / d Uss(H)    = 0          (both sites shift together)
  d omega / d beta_s(H) = -2 S_ss
  d omega / d gss(H)    = 1/2 - exp(-a^2 R^2) / 2
and against step-size independence on a heavy-atom molecule.
"""
import math

import numpy as np

import molgen
from oracle import gradient, nddo


def _h2(R):
    return np.array([1, 1]), np.array([[0.0, 0.0, 0.0], [R, 0.0, 0.0]])


def test_h2_closed_form_derivatives(params0):
    R = 0.9
    Z, xyz = _h2(R)
    gss = params0[1]["gss"]
    zeta = params0[1]["zeta_s"]
    S = nddo.SK_PREFACTOR["ss_sigma"] * math.exp(-zeta * R)
    a = math.sqrt(math.pi) * gss / (2.0 * nddo.KAPPA)
    d_U = gradient.domega_dparam(Z, xyz, params0, 1, "Uss")[0]
    d_beta = gradient.domega_dparam(Z, xyz, params0, 1, "beta_s")[0]
    d_gss = gradient.domega_dparam(Z, xyz, params0, 1, "gss")[0]
    assert abs(d_U) < 1e-8
    assert abs(d_beta - (-2.0 * S)) < 1e-8
    assert abs(d_gss - (0.5 - 0.5 * math.exp(-(a * R) ** 2))) < 1e-8


def test_step_size_independence(params0):
    Z, xyz = molgen.make_chain(2, 3, 4)
    for field in ("gsp", "D1", "zeta_p"):
        g1 = gradient.domega_dparam(Z, xyz, params0, 6, field, k=2, h=1e-3)
        g2 = gradient.domega_dparam(Z, xyz, params0, 6, field, k=2, h=2e-3)
        assert np.abs(g1 - g2).max() <= 1e-6 * max(1.0, np.abs(g1).max()), field


def test_h2_closed_form_rpa_derivatives(params0):
    """Two-site H2 in the RPA: A = omega_CIS, B = (ia|ia) = (gss - gamma)/2,
    omega = sqrt(A^2 - B^2), so d omega = (A dA - B dB) / omega with
    dA/dbeta_s = -2 S_ss, dB/dbeta_s = 0 and dA/dgss = dB/dgss = (1 - exp(-a^2 R^2))/2."""
    R = 0.9
    Z, xyz = _h2(R)
    gss = params0[1]["gss"]
    beta = params0[1]["beta_s"]
    zeta = params0[1]["zeta_s"]
    S = nddo.SK_PREFACTOR["ss_sigma"] * math.exp(-zeta * R)
    a = math.sqrt(math.pi) * gss / (2.0 * nddo.KAPPA)
    gamma = nddo.KAPPA * math.erf(a * R) / R
    A = -2.0 * beta * S + 0.5 * gss - 0.5 * gamma
    B = 0.5 * (gss - gamma)
    w = math.sqrt(A * A - B * B)
    w_or = gradient.excitation_energies(Z, xyz, params0, "RPA", k=1)[0][0]
    assert abs(w_or - w) < 1e-9
    d_U = gradient.domega_dparam(Z, xyz, params0, 1, "Uss", "RPA")[0]
    d_beta = gradient.domega_dparam(Z, xyz, params0, 1, "beta_s", "RPA")[0]
    d_gss = gradient.domega_dparam(Z, xyz, params0, 1, "gss", "RPA")[0]
    dg = 0.5 - 0.5 * math.exp(-(a * R) ** 2)
    assert abs(d_U) < 1e-8
    assert abs(d_beta - (-2.0 * S) * A / w) < 1e-8
    assert abs(d_gss - (A - B) * dg / w) < 1e-8
