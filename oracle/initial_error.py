"""Exact Fourier coefficients of the paper's initial function g1 (Sec. 3.4).

TEST INFRASTRUCTURE ONLY (see the oracle package docstring).  Sec. 3.4 measures the
initial discretisation error e_total = ||g1 - g1_a|| of the lattice interpolant g1_a;
its exact side is g1's Fourier coefficients on the torus, a product over coordinates
of the one-dimensional integrals below.  Pinned against midpoint quadrature and
Parseval in tests/test_initial_error.py.

g1(x) = c prod_j exp(-(2 pi x_j - c_j)^2 / gamma) on [0, 1)^d (Sec. 3.2), with centres
c_1 = 3 pi / 2 and c_j = pi for j > 1, normalised to unit L2 norm.
"""

from __future__ import annotations

import math

import numpy as np


def g1_factor(h, c: float, gamma: float):
    """I(h) = int_0^1 exp(-(2 pi x - c)^2 / gamma) exp(-2 pi i h x) dx, closed form.

    With y = 2 pi x - c and the square completed,
        I(h) = exp(-i h c) / (2 pi) * sqrt(pi gamma) / 2 * [E(y)]_{y=-c}^{2 pi - c},
        E(y) = exp(-gamma h^2 / 4) erf((y + i gamma h / 2) / sqrt(gamma)),
    and E is evaluated through the Faddeeva function w (erf z = 1 - exp(-z^2) w(i z) for
    Re z >= 0, odd symmetry otherwise), so that no factor overflows for large h.
    """
    from scipy.special import wofz
    h = np.asarray(h, dtype=np.float64)
    sg = math.sqrt(gamma)
    es = np.exp(-gamma * h * h / 4.0)

    def E(y):
        z = (y + 0.5j * gamma * h) / sg
        tail = np.exp(-y * y / gamma - 1j * h * y)             # exp(-gamma h^2 / 4 - z^2)
        return es - tail * wofz(1j * z) if y >= 0 else -(es - tail * wofz(-1j * z))

    return np.exp(-1j * h * c) / (2.0 * math.pi) * (math.sqrt(math.pi * gamma) / 2.0) * (E(2 * math.pi - c) - E(-c))


def g1_norm_factor(c: float, gamma: float) -> float:
    """int_0^1 exp(-2 (2 pi x - c)^2 / gamma) dx (one factor of ||g1||^2 before normalisation)."""
    from scipy.special import erf
    a = math.sqrt(2.0 / gamma)
    return (1.0 / (2.0 * math.pi)) * math.sqrt(math.pi * gamma / 2.0) / 2.0 * (erf(a * (2 * math.pi - c)) - erf(-a * c))


def g1_centres(d: int):
    return [1.5 * math.pi] + [math.pi] * (d - 1)


def g1_coefficients(H, gamma: float):
    """Exact Fourier coefficients ghat(h) of g1 with unit L2 norm on [0,1)^d, for the rows h of H."""
    H = np.asarray(H)
    d = H.shape[1]
    cs = g1_centres(d)
    norm2 = 1.0
    for c in cs:
        norm2 *= g1_norm_factor(c, gamma)
    out = np.full(H.shape[0], 1.0 / math.sqrt(norm2), dtype=np.complex128)
    for j in range(d):
        lo, hi = int(H[:, j].min()), int(H[:, j].max())
        tab = g1_factor(np.arange(lo, hi + 1), cs[j], gamma)
        out *= tab[H[:, j] - lo]
    return out


def g1_samples(points, gamma: float):
    """g1 with unit L2 norm at the rows of points."""
    cs = np.array(g1_centres(points.shape[1]))
    norm2 = 1.0
    for c in cs:
        norm2 *= g1_norm_factor(float(c), gamma)
    return np.exp(-np.sum((2.0 * np.pi * points - cs) ** 2, axis=1) / gamma) / math.sqrt(norm2)


def e_total(ghat_exact, ghat_lattice) -> float:
    """Sec. 3.4: with ||g1|| = 1, e_total^2 = 1 - sum_A |ghat|^2 + sum_A |ghat - ghat_a|^2."""
    inside = float(np.sum(np.abs(ghat_exact) ** 2))
    alias = float(np.sum(np.abs(ghat_exact - ghat_lattice) ** 2))
    return math.sqrt(max(0.0, 1.0 - inside) + alias)
