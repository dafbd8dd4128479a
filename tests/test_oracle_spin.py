"""Pins of the oracle's spin terms (hbar != 0, Sec. 4.2): subsystem III's exact
rotation (Eq. spin_rodrigue) against a matrix exponential, its invariants, the
Zeeman source of subsystem II against B-spline derivatives evaluated by scipy,
subsystem I's momentum update with the discrete gradient of the Zeeman term
against a Newton solve of the implicit equations written independently, and
energy / Gauss-law conservation of whole steps."""
import math

import numpy as np
import scipy.interpolate as si
import scipy.linalg as sla
import scipy.optimize as so

from oracle import oracle as O
from paper_2203_06513_gb300 import inputs as I


def _periodic_spline(coef, k, M, dx):
    """scipy BSpline of the periodic V0 function sum_j coef_j N^k_j(x/dx - j), valid on
    [-dx, L + dx] (periodic images of the coefficients on both sides)."""
    ext = 2 * k + 2
    knots = np.arange(-ext, M + ext + k + 2) * dx
    idx = np.arange(-ext, M + ext + 1) % M
    return si.BSpline(knots, coef[idx], k)


def _spin_case(M=16, k=3, npart=300, seed=4, hbar=0.1):
    w = I.Workload("sp", L=2 * math.pi * math.sqrt(2), nx=M, degree=k, np=npart, dt=0.05, vth=0.1,
                   pump=0.3, seed=seed)
    orc = O.Oracle(w.L, M, k, w.weight, w.dt, 1e-13, hbar=hbar)
    x, p = I.particles(w)
    rng = np.random.default_rng(seed)
    ay = 0.4 * np.cos(2 * np.pi * np.arange(M) / M) + 0.05 * rng.normal(size=M)
    az = 0.4 * np.sin(2 * np.pi * np.arange(M) / M) + 0.05 * rng.normal(size=M)
    s = rng.normal(size=(3, npart))
    s /= np.linalg.norm(s, axis=0)
    st = O.initial_state(orc, x, p, ay, az, spin=(s[0], s[1], s[2]))
    return orc, st


def test_rotation_matches_matrix_exponential():
    orc, st = _spin_case(npart=40)
    out = orc.substep3(st)
    Ay = _periodic_spline(st.ay, orc.k, orc.M, orc.dx).derivative()
    Az = _periodic_spline(st.az, orc.k, orc.M, orc.dx).derivative()
    for a in range(40):
        Y, Z = float(Ay(st.x[a])), float(Az(st.x[a]))
        rhat = np.array([[0.0, Y, Z], [-Y, 0.0, 0.0], [-Z, 0.0, 0.0]])
        want = sla.expm(orc.dt * rhat) @ np.array([st.sx[a], st.sy[a], st.sz[a]])
        got = np.array([out.sx[a], out.sy[a], out.sz[a]])
        np.testing.assert_allclose(got, want, atol=2e-15)
    # |s| and r.s (the Zeeman energy of each marker) are invariants of the rotation
    n0 = st.sx ** 2 + st.sy ** 2 + st.sz ** 2
    n1 = out.sx ** 2 + out.sy ** 2 + out.sz ** 2
    assert np.max(np.abs(n1 - n0)) < 1e-15
    assert abs(orc.spin_energy(out) - orc.spin_energy(st)) < 1e-15 * orc.w * 40
    np.testing.assert_array_equal(out.x, st.x)
    np.testing.assert_array_equal(out.p, st.p)


def test_zero_field_rotation_is_identity():
    orc, st = _spin_case(npart=20)
    st.ay[:] = 1.25          # constant A: dA/dx = 0, r = 0
    st.az[:] = -0.5
    out = orc.substep3(st)
    np.testing.assert_array_equal(out.sy, st.sy)
    np.testing.assert_array_equal(out.sz, st.sz)


def test_zeeman_source_is_the_derivative_of_the_basis():
    """(G^T Lambda_1(X)^T W S)_j = sum_a w s_a dLambda^0_j/dx(x_a) (derivative relation),
    with the derivative of each basis function evaluated by scipy."""
    orc, st = _spin_case(M=12, npart=50)
    d = orc.G.T @ orc.spin_deposit(st.x, st.sz)
    want = np.zeros(orc.M)
    for j in range(orc.M):
        e = np.zeros(orc.M)
        e[j] = 1.0
        dN = _periodic_spline(e, orc.k, orc.M, orc.dx).derivative()
        want[j] = orc.w * np.sum(st.sz * dN(st.x))
    np.testing.assert_allclose(d, want, atol=1e-13)


def test_energy_has_the_zeeman_term():
    orc, st = _spin_case(npart=60)
    Ay = _periodic_spline(st.ay, orc.k, orc.M, orc.dx).derivative()
    Az = _periodic_spline(st.az, orc.k, orc.M, orc.dx).derivative()
    want = orc.hbar * orc.w * np.sum(st.sy * Az(st.x) - st.sz * Ay(st.x))
    assert abs(orc.energy(st)["spin"] - want) < 1e-14


def test_path_mean_of_degree_d_is_exact():
    """Mean of N^d_i over a path = its integral (scipy antiderivative) / length."""
    M, L = 10, 5.0
    dx = L / M
    rng = np.random.default_rng(3)
    for d in (0, 1, 2, 3):
        for _ in range(10):
            x0 = rng.uniform(0, L)
            x1 = x0 + rng.uniform(-3, 3) * dx
            m = O.path_mean_deg(d, M, dx, x0, x1)
            want = np.zeros(M)
            for i in range(M):
                e = np.zeros(M)
                e[i] = 1.0
                F = _periodic_spline(e, d, M, dx).antiderivative()
                want[i] = (F(x1) - F(x0)) / (x1 - x0) if x1 != x0 else 0.0
            np.testing.assert_allclose(m, want, atol=1e-13)


def test_subsystem1_with_spin_brute_force_newton():
    """Tiny case: the oracle's Picard fixed point equals a Newton solve of the
    subsystem-I equations with the Zeeman term's difference quotients
    (dA/dx(x1) - dA/dx(x0)) / (x1 - x0) written literally."""
    M, k, L, dt, hbar = 8, 3, 2.0, 0.2, 0.7
    x = np.array([0.1, 1.05, 1.93])
    p = np.array([-1.7, 0.9, 2.5])
    rng = np.random.default_rng(11)
    orc = O.Oracle(L, M, k, 0.35, dt, tol=1e-14, hbar=hbar)
    ay, az = 0.3 * rng.normal(size=M), 0.2 * rng.normal(size=M)
    sp = rng.normal(size=(3, 3))
    sp /= np.linalg.norm(sp, axis=0)
    s = O.initial_state(orc, x, p, ay, az, spin=(sp[0], sp[1], sp[2]))
    s1, _ = orc.substep1(s)
    dx = orc.dx
    Ay, Az = _periodic_spline(ay, k, M, dx), _periodic_spline(az, k, M, dx)
    dAy, dAz = Ay.derivative(), Az.derivative()

    def A(xx):
        xx = np.mod(xx, L)
        return np.array([Ay(xx), Az(xx)])

    def dA(xx):
        xx = np.mod(xx, L)
        return np.array([dAy(xx), dAz(xx)])

    def path_int(x0, x1):
        out = np.zeros(M)
        for i in range(M):
            e = np.zeros(M)
            e[i] = 1.0
            F = _periodic_spline(e, k - 1, M, dx).antiderivative()
            # the periodic integral over the straight path (|x1 - x0| < L)
            tot = 0.0
            a, b = x0, x1
            while True:
                lo = np.floor(a / L) * L
                c = min(b, lo + L) if b > a else max(b, lo)
                if c == a:
                    c = min(b, lo + L) if b > a else max(b, lo - L)
                tot += F(c - lo) - F(a - lo)
                if c == b:
                    break
                a = c
            out[i] = tot
        return out

    def gam(pp, AA):
        return np.sqrt(1 + pp * pp + AA @ AA)

    n = 3

    def resid(u):
        x1, p1, e1 = u[:n], u[n:2 * n], u[2 * n:]
        r = np.zeros_like(u)
        J = np.zeros(M)
        for a in range(n):
            x0, p0 = s.x[a], s.p[a]
            A0, A1 = A(x0), A(x1[a])
            Ip = path_int(x0, x1[a])
            J += orc.w * Ip
            r[a] = x1[a] - x0 - dt * (p0 + p1[a]) / (gam(p0, A1) + gam(p1[a], A1))
            h = x1[a] - x0
            dq = (A1 - A0) / h
            d2 = (dA(x1[a]) - dA(x0)) / h
            r[n + a] = (p1[a] - p0 - Ip @ (0.5 * (s.ex + e1)) / h * dt
                        + dt * ((A1 + A0) @ dq) / (gam(p0, A1) + gam(p0, A0))
                        + dt * hbar * (s.sy[a] * d2[1] - s.sz[a] * d2[0]))
        r[2 * n:] = orc.M1 @ (e1 - s.ex) + J
        return r

    sol = so.root(resid, np.concatenate([s.x + dt * s.p, s.p, s.ex]), method="hybr", tol=1e-15)
    assert np.max(np.abs(resid(sol.x))) < 1e-12
    d = np.mod(s1.x - sol.x[:n] + L / 2, L) - L / 2
    assert np.max(np.abs(d)) < 1e-12
    np.testing.assert_allclose(s1.p, sol.x[n:2 * n], atol=1e-12)
    np.testing.assert_allclose(s1.ex, sol.x[2 * n:], atol=1e-12)


def test_steps_with_spin_conserve_energy_and_gauss():
    orc, st = _spin_case(M=32, npart=2000, hbar=0.1)
    H0 = orc.energy(st)["total"]
    s, hist = orc.run(st, 5, diagnostics=True)
    assert max(abs(h[0] - H0) / abs(H0) for h in hist) < 1e-12
    assert max(h[1] for h in hist) < 1e-13
    # the spin moves, and its length does not change
    assert np.max(np.abs(s.sz - st.sz)) > 1e-6
    n = s.sx ** 2 + s.sy ** 2 + s.sz ** 2
    assert np.max(np.abs(n - 1.0)) < 1e-14
    # each substep conserves the energy on its own
    for sub in (lambda q: orc.substep1(q)[0], lambda q: orc.substep2(q)[0], orc.substep3):
        E0 = orc.energy(s)["total"]
        s = sub(s)
        assert abs(orc.energy(s)["total"] - E0) / abs(E0) < 1e-13


def test_hbar_zero_ignores_spin():
    w = I.Workload("z", nx=16, np=200, seed=2, pump=0.2)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    sp = np.ones((3, w.np)) / math.sqrt(3)
    o1 = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt)
    o2 = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, hbar=0.0)
    a = o1.step(O.initial_state(o1, x, p, ay, az, ey, ez))
    b = o2.step(O.initial_state(o2, x, p, ay, az, ey, ez, spin=(sp[0], sp[1], sp[2])))
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.ey, b.ey)
    np.testing.assert_array_equal(b.sz, sp[2])
