"""Pins of the oracle's absorption spectrum (Gaussian broadening of the
excited states, paper Section "Results and discussion", width 0.1 eV)."""
import math

import numpy as np
import pytest

from oracle.spectrum import PAPER_WIDTH_EV, absorption_spectrum


def test_single_line_peak_and_fwhm():
    sigma = PAPER_WIDTH_EV
    grid = np.linspace(2.0, 4.0, 200001)
    S = absorption_spectrum([3.0], [0.5], grid, sigma)
    # peak value f / (sigma sqrt(2 pi)) at E = omega
    assert S.max() == pytest.approx(0.5 / (sigma * math.sqrt(2 * math.pi)), rel=1e-12)
    assert grid[np.argmax(S)] == pytest.approx(3.0, abs=1e-5)
    # full width at half maximum 2 sqrt(2 ln 2) sigma
    above = grid[S >= 0.5 * S.max()]
    assert above[-1] - above[0] == pytest.approx(2 * math.sqrt(2 * math.log(2)) * sigma, abs=2e-5)


def test_integral_equals_total_oscillator_strength():
    rng = np.random.default_rng(0)
    omega = rng.uniform(3.0, 7.0, 12)
    f = rng.uniform(0.0, 1.0, 12)
    grid = np.linspace(0.0, 10.0, 100001)
    S = absorption_spectrum(omega, f, grid)
    assert np.trapezoid(S, grid) == pytest.approx(f.sum(), rel=1e-10)


def test_linear_in_f_and_translation_covariant():
    rng = np.random.default_rng(1)
    omega = rng.uniform(3.0, 5.0, 5)
    f1, f2 = rng.uniform(0, 1, 5), rng.uniform(0, 1, 5)
    grid = np.linspace(2.0, 6.0, 401)
    S = absorption_spectrum(omega, 2.0 * f1 + 3.0 * f2, grid)
    assert np.allclose(S, 2.0 * absorption_spectrum(omega, f1, grid) + 3.0 * absorption_spectrum(omega, f2, grid),
                       rtol=1e-13, atol=0.0)
    shifted = absorption_spectrum(omega + 0.37, f1, grid + 0.37)
    assert np.allclose(shifted, absorption_spectrum(omega, f1, grid), rtol=1e-12, atol=1e-300)


def test_matches_term_by_term_sum():
    omega, f = [2.5, 2.55, 4.0], [0.1, 0.2, 0.05]
    sigma = 0.2
    for E in (2.4, 2.52, 3.3, 4.1):
        ref = 0.0
        for w, fn in zip(omega, f):
            ref += fn * math.exp(-((E - w) ** 2) / (2 * sigma * sigma)) / (sigma * math.sqrt(2 * math.pi))
        assert absorption_spectrum(omega, f, [E], sigma)[0] == pytest.approx(ref, rel=1e-14)


def test_rejects_bad_input():
    with pytest.raises(ValueError):
        absorption_spectrum([1.0, 2.0], [0.1], [1.0])
    with pytest.raises(ValueError):
        absorption_spectrum([1.0], [0.1], [1.0], width=0.0)
