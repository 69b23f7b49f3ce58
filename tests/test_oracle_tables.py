"""Pins of the oracle's 1D tables (Sec. 2.1, Sec. 3.2, Appendix A)."""
import os
from fractions import Fraction
from math import sqrt  # noqa: F401  (used by eval of golden expressions)

import numpy as np
import pytest

from oracle.tables import Tables, gauss_legendre, midpoint_weights, lagrange, lagrange_deriv

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_gauss_legendre_closed_forms(k):
    rows = [r for r in _rows("gauss_legendre.txt") if int(r[0]) == k]
    xs = np.array([eval(r[1]) for r in rows])
    ws = np.array([eval(r[2]) for r in rows])
    x, w = gauss_legendre(k)
    np.testing.assert_allclose(x, xs, atol=1e-15)
    np.testing.assert_allclose(w, ws, atol=1e-15)


def test_midpoint_weights_match_paper_k3():
    rows = _rows("midpoint_weights_k3.txt")
    G_paper = np.array([float(Fraction(r[1])) for r in rows])
    w_paper = np.array([float(Fraction(r[2])) for r in rows])
    G, w = midpoint_weights(3)
    np.testing.assert_allclose(G, G_paper, rtol=0, atol=1e-16)
    np.testing.assert_allclose(w, w_paper, rtol=0, atol=1e-14)


def test_midpoint_weights_k2_closed_form():
    G, w = midpoint_weights(2)
    np.testing.assert_allclose(w, [3 / 8, 1 / 4, 3 / 8], atol=1e-16)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_midpoint_rule_exact_to_degree_k(k):
    G, w = midpoint_weights(k)
    for m in range(k + 1):
        assert abs(np.sum(w * G ** m) - 1.0 / (m + 1)) < 1e-15


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_lagrange_basis_and_derivatives(k):
    t = Tables(k)
    np.testing.assert_allclose(lagrange(t.xi, t.xi), np.eye(k + 1), atol=1e-15)
    xs = np.linspace(-1, 1, 7)
    # polynomials of degree <= k are reproduced, derivatives exactly
    for m in range(k + 1):
        vals = t.xi ** m
        np.testing.assert_allclose(lagrange(t.xi, xs) @ vals, xs ** m, atol=1e-13)
        dm = m * t.xi ** (m - 1) if m > 0 else 0 * t.xi
        np.testing.assert_allclose(t.D @ vals, dm, atol=1e-12)
        assert abs(t.lp @ vals - 1.0) < 1e-13
        assert abs(t.lm @ vals - (-1.0) ** m) < 1e-13
        assert abs(t.dlp @ vals - m) < 1e-11
        assert abs(t.dlm @ vals - (m * (-1.0) ** (m - 1) if m > 0 else 0)) < 1e-11


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_transfer_matrix_interpolates_and_inverts(k):
    t = Tables(k)
    np.testing.assert_allclose(t.c, -1 + (2 * np.arange(k + 1) + 1) / (k + 1), atol=1e-16)
    for m in range(k + 1):
        np.testing.assert_allclose(t.V @ t.xi ** m, t.c ** m, atol=1e-14)
    np.testing.assert_allclose(t.Vinv @ t.V, np.eye(k + 1), atol=1e-13)


def test_fig_subcell_centres_k3():
    # FV centres of Fig. lgl_fv_points: -0.75, -0.25, 0.25, 0.75
    np.testing.assert_allclose(Tables(3).c, [-0.75, -0.25, 0.25, 0.75], atol=0)
