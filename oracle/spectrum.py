"""Absorption spectrum of computed excited states, plain float64 (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows arXiv:2505.24807, Section "Results and discussion" (the simulated
absorption spectra of the molecular sets): each excited state contributes its
oscillator strength, broadened by a Gaussian of width 0.1 eV.  Reading of
"width": the Gaussian's standard deviation sigma, each line normalised to unit
area, so the spectrum integrates to the sum of the oscillator strengths:

    S(E) = sum_n f_n exp(-(E - omega_n)^2 / (2 sigma^2)) / (sigma sqrt(2 pi))

Pinned by tests/test_oracle_spectrum.py: integral = sum f, single-line peak
height and full width at half maximum (2 sqrt(2 ln 2) sigma), linearity in f,
translation covariance, and a brute-force term-by-term sum.
"""
from __future__ import annotations

import math

import numpy as np

PAPER_WIDTH_EV = 0.1


def absorption_spectrum(omega, f, grid, width=PAPER_WIDTH_EV):
    """S(E) on the energy grid (eV) for excitation energies omega (eV) and
    oscillator strengths f; width = Gaussian standard deviation (eV)."""
    omega = np.asarray(omega, dtype=np.float64).ravel()
    f = np.asarray(f, dtype=np.float64).ravel()
    grid = np.asarray(grid, dtype=np.float64).ravel()
    if omega.shape != f.shape:
        raise ValueError("omega and f differ in length")
    if not width > 0.0:
        raise ValueError("width must be positive")
    norm = 1.0 / (width * math.sqrt(2.0 * math.pi))
    x = (grid[:, None] - omega[None, :]) / width
    return (np.exp(-0.5 * x * x) * f[None, :]).sum(axis=1) * norm
