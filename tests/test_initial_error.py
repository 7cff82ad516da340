"""Pins of the oracle's closed-form Fourier coefficients of g1 (Sec. 3.4): quadrature and Parseval (no GPU)."""

import math

import numpy as np
import pytest

from oracle import initial_error as X


def _quad(h, c, gamma, m=200000):
    x = (np.arange(m) + 0.5) / m                       # midpoint rule, error O(m^-2)
    f = np.exp(-((2 * np.pi * x - c) ** 2) / gamma) * np.exp(-2j * np.pi * h * x)
    return f.mean()


@pytest.mark.parametrize("gamma", [1.0, 0.1, 0.01])
@pytest.mark.parametrize("c", [1.5 * math.pi, math.pi])
def test_g1_factor_equals_quadrature(gamma, c):
    hs = np.array([0, 1, -1, 3, 7, -12, 25])
    got = X.g1_factor(hs, c, gamma)
    ref = np.array([_quad(h, c, gamma) for h in hs])
    assert np.allclose(got, ref, rtol=0, atol=1e-9)


def test_g1_factor_large_frequencies_stay_finite_and_small():
    got = X.g1_factor(np.array([200, 1000, -5000]), 1.5 * math.pi, 1.0)
    assert np.all(np.isfinite(got)) and np.all(np.abs(got) < 1e-2)


def test_g1_norm_and_parseval():
    """sum_h |ghat(h)|^2 over a large box equals the unit norm (Parseval on the torus)."""
    gamma = 1.0
    assert abs(X.g1_norm_factor(math.pi, gamma) - _quad(0, math.pi, gamma / 2).real) < 1e-9
    hs = np.arange(-400, 401)
    H = np.stack(np.meshgrid(hs, hs, indexing="ij"), axis=-1).reshape(-1, 2)
    g = X.g1_coefficients(H, gamma)
    assert abs(np.sum(np.abs(g) ** 2) - 1.0) < 1e-4
