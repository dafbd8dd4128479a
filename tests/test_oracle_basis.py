"""Pins of the oracle's B-spline basis, quadrature and mass matrices (Sec. 3.1)
against library routines (scipy B-splines, numpy Gauss--Legendre) and closed
forms; none of these re-use the oracle's own formulas."""
import json
import os

import numpy as np
import pytest
import scipy.interpolate as si

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("d", [0, 1, 2, 3, 4, 5])
def test_cardinal_bspline_matches_scipy(d):
    ref = si.BSpline.basis_element(np.arange(d + 2, dtype=float), extrapolate=False)
    rng = np.random.default_rng(d)
    s = rng.uniform(0.0, d + 1.0, 200)
    ours = np.array([O.cardinal_bspline(d, v) for v in s])
    np.testing.assert_allclose(ours, np.nan_to_num(ref(s)), rtol=0, atol=1e-14)
    # outside the support
    assert O.cardinal_bspline(d, -0.25) == 0.0
    assert O.cardinal_bspline(d, d + 1.0) == 0.0


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5])
def test_partition_of_unity_and_symmetry(d):
    for t in np.linspace(0.0, 1.0, 37, endpoint=False):
        v = O.basis(d, t)
        assert abs(v.sum() - 1.0) < 4e-16
        assert np.all(v >= 0.0)
    for s in np.linspace(0.0, d + 1.0, 41):
        assert abs(O.cardinal_bspline(d, s) - O.cardinal_bspline(d, d + 1.0 - s)) < 1e-15


@pytest.mark.parametrize("k", [2, 3, 5])
def test_derivative_relation(k):
    """d/dx Lambda^0_j = (Lambda^1_j - Lambda^1_{j+1}) / dx (Sec. 3.1), checked
    with central differences of the degree-k basis on the cardinal line."""
    h = 1e-6
    for s in np.linspace(0.05, k + 0.95, 53):
        fd = (O.cardinal_bspline(k, s + h) - O.cardinal_bspline(k, s - h)) / (2 * h)
        rel = O.cardinal_bspline(k - 1, s) - O.cardinal_bspline(k - 1, s - 1.0)
        assert abs(fd - rel) < 1e-8


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_gauss_legendre(n):
    xi, w = O.gauss_legendre(n)
    rx, rw = np.polynomial.legendre.leggauss(n)
    order = np.argsort(xi)
    np.testing.assert_allclose(xi[order], rx, atol=1e-15)
    np.testing.assert_allclose(w[order], rw, atol=1e-15)
    for m in range(2 * n):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.sum(w * xi ** m) - exact) < 1e-14


def test_mass_rows_closed_form():
    """(M_d)_{0,r} = dx N^{2d+1}(d+1+r): the autocorrelation of the cardinal
    B-spline; for d = 3 and 2 these are the classical integer tables."""
    with open(os.path.join(GOLDEN, "mass_rows.json")) as f:
        g = json.load(f)
    dx = 0.37
    M = 16
    for key, rec in g["rows"].items():
        d = int(key)
        row = O.mass_row(d, M, dx)
        num = np.array(rec["numerators"], dtype=float) / rec["denominator"]
        np.testing.assert_allclose(row[: len(num)], dx * num, rtol=0, atol=1e-15)
        np.testing.assert_allclose(row[M - len(num) + 1:], dx * num[1:][::-1], rtol=0, atol=1e-15)
        assert np.all(row[len(num): M - len(num) + 1] == 0.0)
        assert abs(row.sum() - dx) < 1e-15


@pytest.mark.parametrize("d", [1, 4, 5])
def test_mass_rows_vs_scipy_autocorrelation(d):
    ref = si.BSpline.basis_element(np.arange(2 * d + 3, dtype=float), extrapolate=False)
    dx, M = 0.21, 32
    row = O.mass_row(d, M, dx)
    for r in range(d + 1):
        assert abs(row[r] - dx * float(ref(d + 1.0 + r))) < 1e-15
