"""Pins of the oracle's path integral of the 1-form basis (Sec. 4.2, subsystem I:
int Lambda_1(x(tau)) dtau along the straight path x^n -> x^{n+1})."""
import numpy as np
import pytest
import scipy.interpolate as si

from oracle import oracle as O


def periodic_integral_scipy(k, M, dx, i, x0, x1):
    """int_{x0}^{x1} Lambda^1_i by scipy's exact B-spline antiderivative, summing
    the periodic images of N^{k-1}_i."""
    L = M * dx
    lo, hi = min(x0, x1), max(x0, x1)
    total = 0.0
    nmin = int(np.floor((lo - (i + k) * dx) / L)) - 1
    nmax = int(np.ceil((hi - i * dx) / L)) + 1
    for n in range(nmin, nmax + 1):
        knots = (i + np.arange(k + 1)) * dx + n * L
        b = si.BSpline.basis_element(knots, extrapolate=False)
        a, c = max(lo, knots[0]), min(hi, knots[-1])
        if c > a:
            total += float(b.integrate(a, c, extrapolate=False))
    return total if x1 >= x0 else -total


@pytest.mark.parametrize("k", [2, 3, 5])
def test_path_integral_vs_scipy(k):
    rng = np.random.default_rng(10 + k)
    M, dx = 12, 0.3
    L = M * dx
    for trial in range(25):
        x0 = rng.uniform(0, L)
        ncross = trial % 21          # 0..20 crossed cells, both directions
        x1 = x0 + (1 if trial % 2 else -1) * (ncross + rng.uniform(0, 1)) * dx * 0.7
        mean, integ = O.path_integral(k, M, dx, x0, x1)
        ref = np.array([periodic_integral_scipy(k, M, dx, i, x0, x1) for i in range(M)])
        np.testing.assert_allclose(integ, ref, rtol=0, atol=2e-15 * max(1.0, abs(x1 - x0)))


@pytest.mark.parametrize("k", [2, 3, 5])
def test_path_integral_antiderivative_identity(k):
    """int_{x0}^{x1} Lambda^1_i = dx [sum_{j>=i} Lambda^0_j]_{x0}^{x1} on the
    unwrapped line (the telescoping of Remark 2, Sec. 4.2); checked with the
    oracle's cardinal B-spline values on a grid large enough not to wrap."""
    M, dx = 64, 0.1
    rng = np.random.default_rng(k)

    def S(i, x):   # sum_{j >= i} Lambda^0_j(x), unwrapped
        u = x / dx
        return sum(O.cardinal_bspline(k, u - j) for j in range(i, M + 2 * k))

    for _ in range(10):
        x0 = rng.uniform(20 * dx, 40 * dx)
        x1 = x0 + rng.uniform(-8, 8) * dx
        _, integ = O.path_integral(k, M, dx, x0, x1)
        for i in range(10, 50):
            assert abs(integ[i] - dx * (S(i, x1) - S(i, x0))) < 1e-15


def test_zero_length_path_mean_is_point_value():
    k, M, dx = 3, 10, 0.25
    for x0 in [0.0, 0.3, 1.0, 2.4999]:
        mean, integ = O.path_integral(k, M, dx, x0, x0)
        assert np.all(integ == 0.0)
        u = x0 / dx
        c = int(np.floor(u))
        v = O.basis(k - 1, u - c)
        ref = np.zeros(M)
        for r in range(k):
            ref[(c - r) % M] += v[r]
        np.testing.assert_allclose(mean, ref, atol=1e-15)


def test_difference_quotient_reading():
    """(A(x1) - A(x0)) / (x1 - x0) = sum_i m_i (G a)_i: the exact path mean of
    d/dx A_h (reading of the 0/0 remark of Sec. 4.2)."""
    k, M, L = 3, 16, 4.0
    dx = L / M
    rng = np.random.default_rng(3)
    a = rng.normal(size=M)
    G = O.derivative_matrix(M, dx)
    ga = G @ a
    b = si.BSpline(np.arange(-k, M + 2 * k + 1) * dx, np.concatenate([a[-k:], a, a[:2 * k]]), k)
    for _ in range(20):
        x0 = rng.uniform(0.5 * L, 0.6 * L)
        x1 = x0 + rng.uniform(-1, 1) * 3 * dx
        mean, _ = O.path_integral(k, M, dx, x0, x1)
        dq = (b(x1) - b(x0)) / (x1 - x0)
        assert abs(mean @ ga - dq) < 1e-12
