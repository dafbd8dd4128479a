"""Pins of the oracle's time stepping (Sec. 4.2 subsystems I and II, Sec. 5
Lie--Trotter) against closed forms, invariants the paper states, and a
brute-force Newton solve of the implicit equations written independently."""
import math

import numpy as np
import pytest
import scipy.interpolate as si
import scipy.optimize as so

from oracle import oracle as O
from paper_2203_06513_gb300 import inputs as I


def small_case(M=16, k=3, npart=400, seed=1, pump=0.1, vth=0.1, dt=0.05, L=4 * math.pi):
    w = I.Workload("t", L=L, nx=M, degree=k, np=npart, dt=dt, vth=vth, pump=pump, seed=seed)
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, 1e-13)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    rng = np.random.default_rng(seed)
    az = 0.05 * rng.normal(size=M)   # exercise both transverse components
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    return orc, s


def test_poisson_vs_least_squares():
    orc, s = small_case(M=24)
    r = -orc.charge(s.x) + orc.dx
    A = np.vstack([orc.G.T @ orc.M1, np.ones((1, orc.M))])
    e_ls = np.linalg.lstsq(A, np.concatenate([r, [0.0]]), rcond=None)[0]
    np.testing.assert_allclose(s.ex, e_ls, atol=1e-13)
    assert np.max(np.abs(orc.gauss_residual(s.x, s.ex))) < 1e-14


def test_free_streaming_closed_form():
    """w = 0, e = 0, a = 0: p is constant and x^{n+1} = x^n + dt p / sqrt(1+p^2)."""
    M, k, L, dt = 12, 3, 3.0, 0.1
    orc = O.Oracle(L, M, k, 0.0, dt)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, L, 50)
    p = rng.normal(0, 2.0, 50)
    z = np.zeros(M)
    s = O.State(x, p, z.copy(), z.copy(), z.copy(), z.copy(), z.copy())
    s1, _ = orc.substep1(s)
    np.testing.assert_allclose(s1.p, p, atol=0)
    ref = np.mod(x + dt * p / np.sqrt(1 + p * p), L)
    d = np.abs(s1.x - ref)
    assert np.max(np.minimum(d, L - d)) < 1e-14


def test_uniform_field_exact_relativistic_motion():
    """w = 0, uniform E_x = E0 (sum_i Lambda^1_i = 1), a = 0: the scheme gives
    p^{n+1} = p^n + dt E0 and x^{n+1} - x^n = (gamma^{n+1} - gamma^n)/E0, the
    exact relativistic motion under a constant force."""
    M, k, L, dt, E0 = 10, 3, 5.0, 0.2, 0.7
    orc = O.Oracle(L, M, k, 0.0, dt)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, L, 30)
    p = rng.normal(0, 1.0, 30)
    z = np.zeros(M)
    s = O.State(x, p, np.full(M, E0), z.copy(), z.copy(), z.copy(), z.copy())
    s1, _ = orc.substep1(s)
    np.testing.assert_allclose(s1.p, p + dt * E0, atol=1e-14)
    dx_ref = (np.sqrt(1 + s1.p ** 2) - np.sqrt(1 + p ** 2)) / E0
    d = np.mod(s1.x - x - dx_ref + L / 2, L) - L / 2
    assert np.max(np.abs(d)) < 1e-13


def test_test_particle_in_static_potential_conserves_gamma():
    """w = 0, e = 0, static A_perp: each particle keeps gamma(p, A(x)) (its
    energy) to the fixed-point tolerance."""
    M, k, L, dt = 16, 3, 2 * math.pi, 0.1
    orc = O.Oracle(L, M, k, 0.0, dt, tol=1e-14)
    rng = np.random.default_rng(2)
    ay = rng.normal(0, 0.5, M)
    az = rng.normal(0, 0.5, M)
    x = rng.uniform(0, L, 40)
    p = rng.normal(0, 0.8, 40)
    z = np.zeros(M)
    s = O.State(x, p, z.copy(), z.copy(), z.copy(), ay, az)
    g0 = np.sqrt(1 + p ** 2 + orc.gather(k, x, ay) ** 2 + orc.gather(k, x, az) ** 2)
    for _ in range(5):
        s, _ = orc.substep1(s)
    g1 = np.sqrt(1 + s.p ** 2 + orc.gather(k, s.x, ay) ** 2 + orc.gather(k, s.x, az) ** 2)
    assert np.max(np.abs(g1 - g0)) < 1e-12


@pytest.mark.parametrize("k", [2, 3, 5])
def test_subsystem1_energy_and_gauss(k):
    orc, s = small_case(k=k, npart=300)
    E0 = orc.energy(s)
    s1, it = orc.substep1(s)
    E1 = orc.energy(s1)
    assert abs(E1["total"] - E0["total"]) / E0["total"] < 1e-13
    assert np.max(np.abs(orc.gauss_residual(s1.x, s1.ex))) < 1e-14
    assert E1["eperp"] == E0["eperp"] and E1["aperp"] == E0["aperp"]


@pytest.mark.parametrize("k", [2, 3, 5])
def test_subsystem2_energy(k):
    orc, s = small_case(k=k, npart=300, pump=0.3)
    E0 = orc.energy(s)
    s2, it = orc.substep2(s)
    E1 = orc.energy(s2)
    assert abs(E1["total"] - E0["total"]) / E0["total"] < 1e-13
    np.testing.assert_array_equal(s2.x, s.x)
    np.testing.assert_array_equal(s2.ex, s.ex)
    assert not np.allclose(s2.ay, s.ay)


def test_subsystem2_vacuum_is_crank_nicolson_per_mode():
    """w = 0: subsystem II is the Crank--Nicolson scheme of the linear wave.
    Per Fourier mode theta, with the circulant symbols mu(theta) of M0 and
    kappa(theta) = (2 - 2cos theta)/dx^2 * mu1(theta) of G^T M1 G (from the
    closed-form mass rows), e1 = [(mu - c kappa) e0 + dt kappa a0]/(mu + c kappa)."""
    M, k, L, dt = 32, 3, 6.0, 0.07
    dx = L / M
    orc = O.Oracle(L, M, k, 0.0, dt)
    rng = np.random.default_rng(5)
    ey, ay = rng.normal(size=M), rng.normal(size=M)
    z = np.zeros(M)
    s = O.State(np.zeros(1), np.zeros(1), z.copy(), ey, z.copy(), ay, z.copy())
    s2, _ = orc.substep2(s)
    th = 2 * np.pi * np.arange(M) / M
    mu = dx * (2416 + 2 * 1191 * np.cos(th) + 2 * 120 * np.cos(2 * th) + 2 * np.cos(3 * th)) / 5040
    mu1 = dx * (66 + 2 * 26 * np.cos(th) + 2 * np.cos(2 * th)) / 120
    kap = (2 - 2 * np.cos(th)) / dx ** 2 * mu1
    c = dt * dt / 4
    E0, A0 = np.fft.fft(ey), np.fft.fft(ay)
    E1 = ((mu - c * kap) * E0 + dt * kap * A0) / (mu + c * kap)
    A1 = A0 - dt / 2 * (E0 + E1)
    np.testing.assert_allclose(s2.ey, np.fft.ifft(E1).real, atol=1e-12)
    np.testing.assert_allclose(s2.ay, np.fft.ifft(A1).real, atol=1e-12)


def _brute_force_subsystem1(orc, s):
    """Newton (scipy hybr) on the implicit equations of subsystem I, written
    literally: difference quotient of A, path integrals from scipy's B-spline
    antiderivative, and M1 (e1 - e0) = -sum_a w int Lambda_1."""
    M, k, dx, dt, w, L = orc.M, orc.k, orc.dx, orc.dt, orc.w, orc.L
    n = s.x.shape[0]
    ext = 2 * k + 2                       # periodic images on both sides
    knots0 = np.arange(-ext, M + ext + k + 2) * dx
    idx = np.arange(-ext, M + ext + 1) % M

    def spline(coef):                     # base interval covers [-(ext-k) dx, (M+ext) dx)
        return si.BSpline(knots0, coef[idx], k)

    Ay, Az = spline(s.ay), spline(s.az)

    def path_int(x0, x1):
        out = np.zeros(M)
        for i in range(M):
            lo, hi = min(x0, x1), max(x0, x1)
            tot = 0.0
            for nimg in range(-2, 3):
                kn = (i + np.arange(k + 1)) * dx + nimg * L
                a, c = max(lo, kn[0]), min(hi, kn[-1])
                if c > a:
                    tot += float(si.BSpline.basis_element(kn, extrapolate=False).integrate(a, c, extrapolate=False))
            out[i] = tot if x1 >= x0 else -tot
        return out

    def gam(p, A):
        return np.sqrt(1 + p * p + A @ A)

    def resid(u):
        x1, p1, e1 = u[:n], u[n:2 * n], u[2 * n:]
        r = np.zeros_like(u)
        J = np.zeros(M)
        for a in range(n):
            x0, p0 = s.x[a], s.p[a]
            A0 = np.array([Ay(x0), Az(x0)])
            A1 = np.array([Ay(x1[a]), Az(x1[a])])
            I_ = path_int(x0, x1[a])
            J += w * I_
            r[a] = x1[a] - x0 - dt * (p0 + p1[a]) / (gam(p0, A1) + gam(p1[a], A1))
            dq = (A1 - A0) / (x1[a] - x0)
            r[n + a] = (p1[a] - p0 - I_ @ (0.5 * (s.ex + e1)) / (x1[a] - x0) * dt
                        + dt * ((A1 + A0) @ dq) / (gam(p0, A1) + gam(p0, A0)))
        r[2 * n:] = orc.M1 @ (e1 - s.ex) + J
        return r

    u0 = np.concatenate([s.x + dt * s.p, s.p, s.ex])
    sol = so.root(resid, u0, method="hybr", tol=1e-15)
    assert np.max(np.abs(resid(sol.x))) < 1e-13
    return sol.x[:n], sol.x[n:2 * n], sol.x[2 * n:]


def test_subsystem1_brute_force_newton():
    """Tiny case (M = 8, 3 markers with fast momenta so paths cross knots and
    the periodic boundary): Picard in the oracle == Newton on the equations."""
    M, k, L, dt = 8, 3, 2.0, 0.2
    rng = np.random.default_rng(11)
    x = np.array([0.1, 1.05, 1.93])
    p = np.array([-1.7, 0.9, 2.5])
    orc = O.Oracle(L, M, k, 0.35, dt, tol=1e-14)
    ay, az = 0.3 * rng.normal(size=M), 0.2 * rng.normal(size=M)
    s = O.initial_state(orc, x, p, ay, az)
    s1, it = orc.substep1(s)
    xb, pb, eb = _brute_force_subsystem1(orc, s)
    d = np.mod(s1.x - xb + L / 2, L) - L / 2
    assert np.max(np.abs(d)) < 1e-13
    np.testing.assert_allclose(s1.p, pb, atol=1e-13)
    np.testing.assert_allclose(s1.ex, eb, atol=1e-13)
