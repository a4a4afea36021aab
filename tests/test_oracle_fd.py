"""Pins of the oracle's finite-difference weights (sixth-order, 7-point; Sec. 5.2).

Checked against: the textbook closed-form centred weights, and exactness on
monomials of degree <= 6 by a Vandermonde check written here in numpy.
"""
import math

import numpy as np
import pytest

import oracle as O


def test_centred_weights_closed_form():
    xs = np.arange(-3, 4, dtype=float)
    c = O.fornberg(0.0, xs, 2)
    d1 = np.array([-1, 9, -45, 0, 45, -9, 1]) / 60.0
    d2 = np.array([2, -27, 270, -490, 270, -27, 2]) / 180.0
    np.testing.assert_allclose(c[1], d1, atol=1e-15)
    np.testing.assert_allclose(c[2], d2, atol=1e-14)
    np.testing.assert_allclose(c[0], [0, 0, 0, 1, 0, 0, 0], atol=1e-15)


@pytest.mark.parametrize("z", [-1.0, -0.5, 0.0, 0.3, 2.0, 3.0, 5.0])
def test_offcentre_weights_exact_on_monomials(z):
    # nodes of a shifted window on a uniform grid, evaluation point anywhere
    xs = np.array([-1, 0, 1, 2, 3, 4, 5], dtype=float) * 0.125
    zz = z * 0.125
    c = O.fornberg(zz, xs, 2)
    for q in range(7):
        f = xs ** q
        d1 = q * zz ** (q - 1) if q >= 1 else 0.0
        d2 = q * (q - 1) * zz ** (q - 2) if q >= 2 else 0.0
        assert abs(c[0] @ f - zz ** q) < 1e-13
        assert abs(c[1] @ f - d1) < 1e-11 * max(1, abs(d1))
        assert abs(c[2] @ f - d2) < 1e-9 * max(1, abs(d2))


def test_weights_match_vandermonde_solution():
    # Independent construction: weights w solve sum_i w_i (x_i - z)^q / q! = [q == d].
    xs = np.linspace(0.0, 0.75, 7)
    for z in [0.0, 0.125, 0.5, 0.75]:
        V = np.array([[(x - z) ** q / math.factorial(q) for x in xs] for q in range(7)])
        c = O.fornberg(z, xs, 2)
        for d in range(3):
            e = np.zeros(7); e[d] = 1.0
            w = np.linalg.solve(V, e)
            np.testing.assert_allclose(c[d], w, rtol=1e-9, atol=1e-9 * np.abs(w).max())


@pytest.mark.parametrize("nz", [7, 9, 17, 33])
def test_sigma_window(nz):
    for j in range(-1, nz):
        s = O.sigma_window(nz, j)
        assert -1 <= s and s + 6 <= nz - 1
        assert s <= j <= s + 6
        if 2 <= j <= nz - 4:
            assert s == j - 3      # centred where it fits
