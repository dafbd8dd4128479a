"""Pins of the two-dimensional subsystem-I oracle (Sec. 3.2 spaces, Sec. 4.3
subsystem I) against what the mathematics fixes: path integrals of the V1 basis
against scipy quadrature of scipy B-splines, the discrete gradient identity
G^T int Lambda_1 . dx = Lambda_0(x^{n+1}) - Lambda_0(x^n), the coordinate-increment
difference quotients against scipy derivatives and their telescoping sum, exact
energy conservation, and the reductions to the (separately pinned) one-dimensional
oracle when the grid has one cell in the other direction."""
import math

import numpy as np
import pytest
import scipy.integrate as sint
import scipy.interpolate as si

from oracle import oracle as O
from oracle import oracle2d as O2


def periodic_basis(d, M, dx, i, x):
    """N^d_i(x) summed over the periodic images, from scipy's B-spline."""
    L = M * dx
    s = 0.0
    for n in range(-2, 3):
        knots = (i + np.arange(d + 2)) * dx + n * L
        b = si.BSpline.basis_element(knots, extrapolate=False)
        v = b(x)
        if np.isfinite(v):
            s += float(v)
    return s


def periodic_basis_deriv(d, M, dx, i, x):
    L = M * dx
    s = 0.0
    for n in range(-2, 3):
        knots = (i + np.arange(d + 2)) * dx + n * L
        b = si.BSpline.basis_element(knots, extrapolate=False).derivative()
        v = b(x)
        if np.isfinite(v):
            s += float(v)
    return s


def scipy_path_means(g, P0, P1, comp, node):
    i1, i2 = node // g.M[1], node % g.M[1]
    k = g.k
    d1, d2 = (k - 1, k) if comp == 0 else (k, k - 1)

    def f(s):
        x1 = P0[0] + s * (P1[0] - P0[0])
        x2 = P0[1] + s * (P1[1] - P0[1])
        return periodic_basis(d1, g.M[0], g.dx[0], i1, x1) * periodic_basis(d2, g.M[1], g.dx[1], i2, x2)
    # breakpoints: knot crossings of either coordinate
    pts = []
    for q in range(2):
        du = (P1[q] - P0[q]) / g.dx[q]
        u0 = P0[q] / g.dx[q]
        if du != 0:
            lo, hi = sorted((u0, u0 + du))
            pts += [(n - u0) / du for n in range(math.floor(lo) + 1, math.ceil(hi))]
    val, _ = sint.quad(f, 0.0, 1.0, points=sorted(p for p in pts if 0 < p < 1) or None, limit=200,
                       epsabs=1e-15, epsrel=1e-13)
    return val


@pytest.mark.parametrize("k", [2, 3])
def test_path_means_vs_scipy(k):
    g = O2.Grid2D(3.0, 2.2, 5, 4, k)
    rng = np.random.default_rng(7 + k)
    for trial in range(4):
        P0 = np.array([rng.uniform(0, 3.0), rng.uniform(0, 2.2)])
        P1 = P0 + rng.normal(0, 1.0, 2) * np.array(g.dx) * (1 + trial)
        if trial == 0:
            P1[1] = P0[1]                      # along x1 only
        mx, my = g.path_means(P0, P1)
        for comp, m in ((0, mx), (1, my)):
            ref = np.array([scipy_path_means(g, P0, P1, comp, i) for i in range(g.N)])
            np.testing.assert_allclose(m, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_gradient_identity(k):
    """G^T (dx1 m_x, dx2 m_y) = Lambda_0(P1) - Lambda_0(P0): the discrete de Rham
    property that makes the scheme keep the Gauss law."""
    g = O2.Grid2D(4.0, 3.0, 6, 5, k)
    rng = np.random.default_rng(3 * k)
    for _ in range(6):
        P0 = np.array([rng.uniform(0, 4.0), rng.uniform(0, 3.0)])
        P1 = P0 + rng.normal(0, 1.5, 2) * np.array(g.dx)
        mx, my = g.path_means(P0, P1)
        lhs = g.Gx.T @ ((P1[0] - P0[0]) * mx) + g.Gy.T @ ((P1[1] - P0[1]) * my)
        rhs = g.basis0(P1[0], P1[1]) - g.basis0(P0[0], P0[1])
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13)


@pytest.mark.parametrize("k", [2, 3])
def test_difference_quotients(k):
    g = O2.Grid2D(4.0, 3.0, 6, 5, k)
    rng = np.random.default_rng(11 * k)
    a = rng.normal(0, 1, g.N)
    for trial in range(5):
        P0 = np.array([rng.uniform(0, 4.0), rng.uniform(0, 3.0)])
        P1 = P0 + rng.normal(0, 1.2, 2) * np.array(g.dx)
        D1, D2 = g.dA_means(a, P0, P1)
        # telescoping: D . (P1 - P0) = A(P1) - A(P0)
        dA = g.value0(a, P1[0], P1[1]) - g.value0(a, P0[0], P0[1])
        assert abs(D1 * (P1[0] - P0[0]) + D2 * (P1[1] - P0[1]) - dA) < 1e-13
        # each component against scipy: mean of dA/dx1 along x1 at x2 = P1[1]
        def A_dx1(x1):
            return sum(a[i] * periodic_basis_deriv(k, g.M[0], g.dx[0], i // g.M[1], x1)
                       * periodic_basis(k, g.M[1], g.dx[1], i % g.M[1], P1[1]) for i in range(g.N))

        def A_dx2(x2):
            return sum(a[i] * periodic_basis(k, g.M[0], g.dx[0], i // g.M[1], P0[0])
                       * periodic_basis_deriv(k, g.M[1], g.dx[1], i % g.M[1], x2) for i in range(g.N))
        def knots_between(lo, hi, h):
            lo, hi = sorted((lo, hi))
            return [n * h for n in range(math.floor(lo / h) + 1, math.ceil(hi / h))] or None
        r1 = sint.quad(A_dx1, P0[0], P1[0], points=knots_between(P0[0], P1[0], g.dx[0]), limit=200,
                       epsabs=1e-15, epsrel=1e-13)[0] / (P1[0] - P0[0])
        r2 = sint.quad(A_dx2, P0[1], P1[1], points=knots_between(P0[1], P1[1], g.dx[1]), limit=200,
                       epsabs=1e-15, epsrel=1e-13)[0] / (P1[1] - P0[1])
        assert abs(D1 - r1) < 1e-10 * max(1.0, abs(r1))
        assert abs(D2 - r2) < 1e-10 * max(1.0, abs(r2))


def _random_case(seed, M1, M2, k, npart, L1=4.0, L2=3.0, amp=0.3, vth=0.2):
    rng = np.random.default_rng(seed)
    orc = O2.Oracle2D(L1, L2, M1, M2, k, w=L1 * L2 / npart, dt=0.1)
    g = orc.g
    x = np.column_stack([rng.uniform(0, L1, npart), rng.uniform(0, L2, npart)])
    p = rng.normal(0, vth, (npart, 2))
    a = amp * rng.normal(0, 1, g.N)
    ex = 0.05 * rng.normal(0, 1, g.N)
    ey = 0.05 * rng.normal(0, 1, g.N)
    return orc, x, p, ex, ey, a


@pytest.mark.parametrize("k", [2, 3])
def test_energy_conserved(k):
    orc, x, p, ex, ey, a = _random_case(5 + k, 6, 5, k, 24)
    H0 = orc.energy(x, p, ex, ey, a)["total"]
    for _ in range(2):
        x, p, ex, ey, it = orc.substep1(x, p, ex, ey, a)
    H1 = orc.energy(x, p, ex, ey, a)["total"]
    assert abs(H1 - H0) < 1e-12 * abs(H0)
    assert it >= 3


def test_gauss_law_kept():
    """G^T M1 (e^{n+1} - e^n) = -(rho^{n+1} - rho^n): the scheme keeps the discrete
    Poisson equation."""
    orc, x, p, ex, ey, a = _random_case(21, 5, 4, 3, 16)
    g = orc.g
    x1, p1, ex1, ey1, _ = orc.substep1(x, p, ex, ey, a)
    lhs = g.Gx.T @ (g.M1x @ (ex1 - ex)) + g.Gy.T @ (g.M1y @ (ey1 - ey))
    rhs = -(g.charge(x1, orc.w) - g.charge(x, orc.w))
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12)


@pytest.mark.parametrize("axis", [0, 1])
def test_reduces_to_one_dimension(axis):
    """With one cell across the other direction (its basis is then identically 1)
    and no momentum across it, the 2D step is the 1D oracle's subsystem I with
    A_y = 0 and A_z = the 2D A_z, the weight scaled by the other length."""
    k, M, npart = 3, 8, 20
    L, Lo = 5.0, 1.7
    rng = np.random.default_rng(31 + axis)
    xs = rng.uniform(0, L, npart)
    ps = rng.normal(0, 0.2, npart)
    az = 0.3 * rng.normal(0, 1, M)
    e1 = 0.05 * rng.normal(0, 1, M)
    w1 = L / npart
    dt = 0.1
    orc1 = O.Oracle(L, M, k, w1, dt)
    s0 = O.initial_state(orc1, xs, ps, np.zeros(M), az, None, None)
    s0.ex = e1.copy()
    s1, it1 = orc1.substep1(s0)
    yo = rng.uniform(0, Lo, npart)
    if axis == 0:
        orc2 = O2.Oracle2D(L, Lo, M, 1, k, w=w1 * Lo, dt=dt)
        x = np.column_stack([xs, yo])
        p = np.column_stack([ps, np.zeros(npart)])
        ex, ey = e1.copy(), np.zeros(M)
    else:
        orc2 = O2.Oracle2D(Lo, L, 1, M, k, w=w1 * Lo, dt=dt)
        x = np.column_stack([yo, xs])
        p = np.column_stack([np.zeros(npart), ps])
        ex, ey = np.zeros(M), e1.copy()
    x2, p2, ex2, ey2, it2 = orc2.substep1(x, p, ex, ey, az.copy())
    np.testing.assert_allclose(x2[:, axis], s1.x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(x2[:, 1 - axis], yo, rtol=0, atol=0)
    np.testing.assert_allclose(p2[:, axis], s1.p, rtol=0, atol=1e-12)
    np.testing.assert_allclose(p2[:, 1 - axis], 0.0, rtol=0, atol=0)
    e2 = ex2 if axis == 0 else ey2
    np.testing.assert_allclose(e2, s1.ex, rtol=0, atol=1e-12)
    assert abs(it1 - it2) <= 1


# ---------------- spin terms (hbar != 0) ----------------

@pytest.mark.parametrize("k", [2, 3])
def test_quotients_telescope_and_match_scipy(k):
    """Coordinate-increment quotients of the three Zeeman fields (dA/dx2 on degrees
    (k, k-1), dA/dx1 on (k-1, k), B_z on (k-1, k-1)): Q . (P1 - P0) = f(P1) - f(P0),
    and each component against scipy's derivative of the periodic B-splines."""
    g = O2.Grid2D(4.0, 3.0, 6, 5, k)
    rng = np.random.default_rng(100 + k)
    a = rng.normal(0, 1, g.N)
    bz = rng.normal(0, 1, g.N)
    fields = ((g.Gy @ a, k, k - 1), (g.Gx @ a, k - 1, k), (bz, k - 1, k - 1))
    for _ in range(4):
        P0 = np.array([rng.uniform(0, 4.0), rng.uniform(0, 3.0)])
        P1 = P0 + rng.normal(0, 1.2, 2) * np.array(g.dx)
        for c, d1, d2 in fields:
            Q1, Q2 = g.quotients(c, d1, d2, P0, P1)
            df = g.value(c, d1, d2, P1[0], P1[1]) - g.value(c, d1, d2, P0[0], P0[1])
            assert abs(Q1 * (P1[0] - P0[0]) + Q2 * (P1[1] - P0[1]) - df) < 1e-12
            # Q1 = (f(P1) - f(P0[0], P1[1])) / dx1 from scipy's periodic B-splines
            def f_sc(x1, x2):
                return sum(c[i] * periodic_basis(d1, g.M[0], g.dx[0], i // g.M[1], x1)
                           * periodic_basis(d2, g.M[1], g.dx[1], i % g.M[1], x2) for i in range(g.N))
            r1 = (f_sc(P1[0], P1[1]) - f_sc(P0[0], P1[1])) / (P1[0] - P0[0])
            r2 = (f_sc(P0[0], P1[1]) - f_sc(P0[0], P0[1])) / (P1[1] - P0[1])
            assert abs(Q1 - r1) < 1e-11 * max(1.0, abs(r1))
            assert abs(Q2 - r2) < 1e-11 * max(1.0, abs(r2))


@pytest.mark.parametrize("k", [2, 3])
def test_energy_conserved_with_spin(k):
    rng = np.random.default_rng(55 + k)
    orc, x, p, ex, ey, a = _random_case(9 + k, 6, 5, k, 20)
    orc.hbar = 0.1
    s = rng.normal(0, 1, (20, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    bz = 0.3 * rng.normal(0, 1, orc.g.N)
    E0 = orc.energy(x, p, ex, ey, a, s, bz)
    assert abs(E0["zeeman"]) > 1e-4 * abs(E0["total"])
    for _ in range(2):
        x, p, ex, ey, it = orc.substep1(x, p, ex, ey, a, s=s, bz=bz)
    E1 = orc.energy(x, p, ex, ey, a, s, bz)
    assert abs(E1["total"] - E0["total"]) < 1e-12 * abs(E0["total"])


def test_spin_reduces_to_one_dimension():
    """M2 = 1, A_y = 0, B_z = 0: the 2D Zeeman term -hbar s_y dA_z/dx1 is the 1D
    oracle's hbar s_y dA_z/dx with the spin's y component reversed (the printed 1D
    and 2D Hamiltonians carry opposite signs of s . B)."""
    k, M, npart = 3, 8, 20
    L, Lo = 5.0, 1.7
    rng = np.random.default_rng(77)
    xs = rng.uniform(0, L, npart)
    ps = rng.normal(0, 0.2, npart)
    az = 0.3 * rng.normal(0, 1, M)
    e1 = 0.05 * rng.normal(0, 1, M)
    sp = rng.normal(0, 1, (npart, 3))
    sp /= np.linalg.norm(sp, axis=1, keepdims=True)
    w1, dt, hbar = L / npart, 0.1, 0.1
    orc1 = O.Oracle(L, M, k, w1, dt, hbar=hbar)
    s0 = O.initial_state(orc1, xs, ps, np.zeros(M), az, None, None, spin=(sp[:, 0], sp[:, 1], sp[:, 2]))
    s0.ex = e1.copy()
    s1, _ = orc1.substep1(s0)
    orc2 = O2.Oracle2D(L, Lo, M, 1, k, w=w1 * Lo, dt=dt, hbar=hbar)
    x = np.column_stack([xs, rng.uniform(0, Lo, npart)])
    p = np.column_stack([ps, np.zeros(npart)])
    s2 = sp * np.array([1.0, -1.0, 1.0])
    x2, p2, ex2, ey2, _ = orc2.substep1(x, p, e1.copy(), np.zeros(M), az.copy(), s=s2, bz=np.zeros(M))
    np.testing.assert_allclose(x2[:, 0], s1.x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(p2[:, 0], s1.p, rtol=0, atol=1e-12)
    np.testing.assert_allclose(ex2, s1.ex, rtol=0, atol=1e-12)
