"""Plain FP64 CPU oracle of subsystem I of the two-dimensional scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module.  It shares no
code with the CUDA library under ``paper_2203_06513_gb300/``.

What it computes (paper, Sec. 3.2 for the spaces and Sec. 4.3, subsystem I of the
two-dimensional splitting), written with plain numpy and pure-Python marker loops
(small cases only):

* the tensor-product spline spaces on a uniform periodic M1 x M2 grid, node index
  i = i1 M2 + i2: V0 basis N^k(x1/dx1 - i1) N^k(x2/dx2 - i2) (A_z), the two V1
  components N^{k-1} x N^k (E_x) and N^k x N^{k-1} (E_y);
* the V1 mass matrix M1 = diag(M1_x (x) M0_y, M0_x (x) M1_y) from the 1D circulant
  mass matrices, and the gradient G = (G_x (x) I; I (x) G_y) with the 1D
  derivative matrices of the one-dimensional oracle;
* subsystem I (markers x, p in R^2, field e_xy; A_z, b_z and the spins frozen):
      x^{n+1} - x^n = dt (p^n + p^{n+1}) / (g(p^n, A(x^{n+1})) + g(p^{n+1}, A(x^{n+1}))),
      p^{n+1} - p^n = int Lambda_1^T(x(t)) dt e_bar
                      - dt (A(x^{n+1}) + A(x^n)) D / (g(p^n, A(x^{n+1})) + g(p^n, A(x^n))),
      e^{n+1} - e^n = -M1^{-1} sum_a w int_{x^n}^{x^{n+1}} Lambda_1 . dx,
  g(p, A) = sqrt(1 + |p|^2 + A^2), e_bar = (e^n + e^{n+1}) / 2, x(t) the straight
  path, D the coordinate-increment difference quotients of A_z: first along x1 at
  x2^{n+1}, then along x2 at x1^n;
* the discrete energy of the subsystem, sum_a w (g(p_a, A(x_a)) - 1) + e^T M1 e / 2.

Readings (where the paper is silent): the difference quotients of D are the exact
path means of dA/dx1 along x1 (at x2^{n+1}) and of dA/dx2 along x2 (at x1^n), so no
0/0 arises; path integrals of the V1 basis are split at every knot crossing of
either coordinate and integrated on each piece by k-point Gauss--Legendre (the
integrand is a polynomial of degree 2k - 1 in the path parameter, so the rule is
exact); the fixed point is Picard on the positions from x^(0) = x^n, p^(0) = p^n,
one global e_xy update per sweep, stopped when the position, momentum and field
increments are all at most tol.  With hbar != 0 the Zeeman term's discrete gradient
uses the same coordinate increments, with the sign of the printed 2D Hamiltonian
(+ hbar s . B, B = (dA_z/dx2, -dA_z/dx1, B_z)).
Parity status: every function here is pinned by tests/test_oracle_2d.py.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O


def bvals(d: int, u: float):
    """(cell c, [N^d(r + t) for r = 0..d]) at the cell coordinate u = x / dx."""
    c = math.floor(u)
    return c, O.basis(d, u - c)


class Grid2D:
    """Spaces, mass matrices and gradient on a uniform periodic M1 x M2 grid."""

    def __init__(self, L1: float, L2: float, M1: int, M2: int, k: int):
        self.L = (float(L1), float(L2))
        self.M = (int(M1), int(M2))
        self.k = int(k)
        self.dx = (self.L[0] / self.M[0], self.L[1] / self.M[1])
        self.N = self.M[0] * self.M[1]
        m0 = [O.circulant(O.mass_row(k, self.M[q], self.dx[q])) for q in range(2)]
        m1 = [O.circulant(O.mass_row(k - 1, self.M[q], self.dx[q])) for q in range(2)]
        self.M1x = np.kron(m1[0], m0[1])            # E_x block: N^{k-1} x N^k
        self.M1y = np.kron(m0[0], m1[1])            # E_y block: N^k x N^{k-1}
        self.M0 = np.kron(m0[0], m0[1])
        g = [O.derivative_matrix(self.M[q], self.dx[q]) for q in range(2)]
        self.Gx = np.kron(g[0], np.eye(self.M[1]))
        self.Gy = np.kron(np.eye(self.M[0]), g[1])

    def idx(self, i1: int, i2: int) -> int:
        return (i1 % self.M[0]) * self.M[1] + (i2 % self.M[1])

    # ---------------- point values ----------------
    def value0(self, a: np.ndarray, x1: float, x2: float) -> float:
        """A_h(x) = sum_i a_i Lambda^0_i(x)."""
        c1, v1 = bvals(self.k, x1 / self.dx[0])
        c2, v2 = bvals(self.k, x2 / self.dx[1])
        s = 0.0
        for r1 in range(self.k + 1):
            for r2 in range(self.k + 1):
                s += a[self.idx(c1 - r1, c2 - r2)] * v1[r1] * v2[r2]
        return s

    def basis0(self, x1: float, x2: float) -> np.ndarray:
        """Lambda^0(x) as a vector over the V0 nodes."""
        out = np.zeros(self.N)
        c1, v1 = bvals(self.k, x1 / self.dx[0])
        c2, v2 = bvals(self.k, x2 / self.dx[1])
        for r1 in range(self.k + 1):
            for r2 in range(self.k + 1):
                out[self.idx(c1 - r1, c2 - r2)] += v1[r1] * v2[r2]
        return out

    # ---------------- path integrals ----------------
    def path_means(self, P0, P1):
        """(m_x, m_y): int_0^1 Lambda^1_{1,i}(x(s)) ds and int_0^1 Lambda^1_{2,i}(x(s)) ds
        along x(s) = P0 + s (P1 - P0), as vectors over the nodes.  P0, P1 in length
        units, unwrapped (the indices wrap)."""
        k = self.k
        u0 = (P0[0] / self.dx[0], P0[1] / self.dx[1])
        du = ((P1[0] - P0[0]) / self.dx[0], (P1[1] - P0[1]) / self.dx[1])
        # breakpoints: parameter values where a coordinate crosses a knot
        cuts = [0.0, 1.0]
        for q in range(2):
            if du[q] != 0.0:
                lo, hi = sorted((u0[q], u0[q] + du[q]))
                for n in range(math.floor(lo) + 1, math.ceil(hi)):
                    cuts.append((n - u0[q]) / du[q])
        cuts = sorted(set(c for c in cuts if 0.0 <= c <= 1.0))
        xi, wq = O.gauss_legendre(k)
        mx, my = np.zeros(self.N), np.zeros(self.N)
        for sa, sb in zip(cuts[:-1], cuts[1:]):
            if sb <= sa:
                continue
            sm = 0.5 * (sa + sb)
            cell = [math.floor(u0[q] + sm * du[q]) for q in range(2)]
            for g in range(k):
                s = sm + 0.5 * (sb - sa) * xi[g]
                wgt = 0.5 * (sb - sa) * wq[g]
                t = [u0[q] + s * du[q] - cell[q] for q in range(2)]
                b1k, b1m = O.basis(k, t[0]), O.basis(k - 1, t[0])
                b2k, b2m = O.basis(k, t[1]), O.basis(k - 1, t[1])
                for r1 in range(k + 1):
                    for r2 in range(k + 1):
                        if r1 < k:
                            mx[self.idx(cell[0] - r1, cell[1] - r2)] += wgt * b1m[r1] * b2k[r2]
                        if r2 < k:
                            my[self.idx(cell[0] - r1, cell[1] - r2)] += wgt * b1k[r1] * b2m[r2]
        return mx, my

    def dA_means(self, a: np.ndarray, P0, P1):
        """D = (mean of dA/dx1 along x1 from x1^0 to x1^1 at x2 = x2^1,
                mean of dA/dx2 along x2 from x2^0 to x2^1 at x1 = x1^0):
        the coordinate-increment difference quotients of A_h, as exact path means."""
        k = self.k
        ga_x = self.Gx @ a
        ga_y = self.Gy @ a
        # along x1 at fixed x2 = P1[1]: means of N^{k-1} in x1, point values N^k in x2
        m1 = O.path_mean_deg(k - 1, self.M[0], self.dx[0], P0[0], P1[0])
        c2, v2 = bvals(k, P1[1] / self.dx[1])
        D1 = 0.0
        for i1 in range(self.M[0]):
            if m1[i1] == 0.0:
                continue
            for r2 in range(k + 1):
                D1 += ga_x[self.idx(i1, c2 - r2)] * m1[i1] * v2[r2]
        # along x2 at fixed x1 = P0[0]
        m2 = O.path_mean_deg(k - 1, self.M[1], self.dx[1], P0[1], P1[1])
        c1, v1 = bvals(k, P0[0] / self.dx[0])
        D2 = 0.0
        for i2 in range(self.M[1]):
            if m2[i2] == 0.0:
                continue
            for r1 in range(k + 1):
                D2 += ga_y[self.idx(c1 - r1, i2)] * v1[r1] * m2[i2]
        return D1, D2

    # ---------------- any tensor-product spline ----------------
    def value(self, c: np.ndarray, d1: int, d2: int, x1: float, x2: float) -> float:
        """f(x) = sum_i c_i N^{d1}(x1/dx1 - i1) N^{d2}(x2/dx2 - i2)."""
        c1, v1 = bvals(d1, x1 / self.dx[0])
        c2, v2 = bvals(d2, x2 / self.dx[1])
        s = 0.0
        for r1 in range(d1 + 1):
            for r2 in range(d2 + 1):
                s += c[self.idx(c1 - r1, c2 - r2)] * v1[r1] * v2[r2]
        return s

    def quotients(self, c: np.ndarray, d1: int, d2: int, P0, P1):
        """Coordinate-increment difference quotients of f (degrees d1, d2), as exact
        path means: (mean of df/dx1 along x1 at x2 = x2^1, mean of df/dx2 along x2 at
        x1 = x1^0).  df/dx1 has coefficients G_x c on degrees (d1 - 1, d2)."""
        fx = self.Gx @ c
        fy = self.Gy @ c
        m1 = O.path_mean_deg(d1 - 1, self.M[0], self.dx[0], P0[0], P1[0])
        c2, v2 = bvals(d2, P1[1] / self.dx[1])
        Q1 = 0.0
        for i1 in range(self.M[0]):
            if m1[i1] != 0.0:
                for r2 in range(d2 + 1):
                    Q1 += fx[self.idx(i1, c2 - r2)] * m1[i1] * v2[r2]
        m2 = O.path_mean_deg(d2 - 1, self.M[1], self.dx[1], P0[1], P1[1])
        c1, v1 = bvals(d1, P0[0] / self.dx[0])
        Q2 = 0.0
        for i2 in range(self.M[1]):
            if m2[i2] != 0.0:
                for r1 in range(d1 + 1):
                    Q2 += fy[self.idx(c1 - r1, i2)] * v1[r1] * m2[i2]
        return Q1, Q2

    # ---------------- grid algebra ----------------
    def solve_M1(self, jx, jy):
        return np.linalg.solve(self.M1x, jx), np.linalg.solve(self.M1y, jy)

    def field_energy(self, ex, ey) -> float:
        return 0.5 * (ex @ self.M1x @ ex + ey @ self.M1y @ ey)

    def charge(self, x, w: float) -> np.ndarray:
        rho = np.zeros(self.N)
        for a in range(x.shape[0]):
            rho += w * self.basis0(x[a, 0], x[a, 1])
        return rho


class Oracle2D:
    """Subsystem I of the two-dimensional scheme, plain FP64.  With hbar != 0 the
    markers carry spins s (Np x 3, frozen in this subsystem) and b_z (the 2-form,
    degrees k-1, k-1) enters through the Zeeman term of the Hamiltonian
    (Eq. discrete_H2d): hbar sum_a w (s_x dA_z/dx2 - s_y dA_z/dx1 + s_z B_z)(x_a),
    whose coordinate-increment discrete gradient joins the momentum update."""

    def __init__(self, L1, L2, M1, M2, k, w, dt, tol=1e-13, max_iter=100, hbar=0.0):
        self.g = Grid2D(L1, L2, M1, M2, k)
        self.w, self.dt = float(w), float(dt)
        self.tol, self.max_iter = float(tol), int(max_iter)
        self.hbar = float(hbar)

    def zeeman(self, x, a, s, bz) -> float:
        """hbar sum_a w (s_x dA/dx2 - s_y dA/dx1 + s_z B_z)(x_a)."""
        if self.hbar == 0.0 or s is None:
            return 0.0
        g, k = self.g, self.g.k
        ay, ax = g.Gy @ a, g.Gx @ a          # dA/dx2 on (k, k-1), dA/dx1 on (k-1, k)
        tot = 0.0
        for q in range(x.shape[0]):
            x1, x2 = x[q]
            tot += s[q, 0] * g.value(ay, k, k - 1, x1, x2) - s[q, 1] * g.value(ax, k - 1, k, x1, x2) \
                + s[q, 2] * g.value(bz, k - 1, k - 1, x1, x2)
        return self.hbar * self.w * tot

    def kinetic(self, x, p, a) -> float:
        s = 0.0
        for q in range(x.shape[0]):
            A = self.g.value0(a, x[q, 0], x[q, 1])
            s += self.w * (math.sqrt(1.0 + p[q, 0] ** 2 + p[q, 1] ** 2 + A * A) - 1.0)
        return s

    def energy(self, x, p, ex, ey, a, s=None, bz=None) -> dict:
        kin = self.kinetic(x, p, a)
        fe = self.g.field_energy(ex, ey)
        ze = self.zeeman(x, a, s, bz)
        return {"kinetic": kin, "field": fe, "zeeman": ze, "total": kin + fe + ze}

    def substep1(self, x, p, ex, ey, a, dt=None, s=None, bz=None):
        """One discrete-gradient step of subsystem I.  x, p: (Np, 2); s (Np, 3) and
        bz with hbar != 0; returns (x^{n+1} wrapped into the box, p^{n+1}, e_x^{n+1},
        e_y^{n+1}, sweeps)."""
        g = self.g
        k = g.k
        spin = self.hbar != 0.0 and s is not None
        if spin:
            ay, ax = g.Gy @ a, g.Gx @ a
        dt = self.dt if dt is None else float(dt)
        x = np.asarray(x, dtype=np.float64)
        pn = np.asarray(p, dtype=np.float64)
        npart = x.shape[0]
        d = np.zeros((npart, 2))
        pk = pn.copy()
        exk, eyk = ex.copy(), ey.copy()
        A0 = np.array([g.value0(a, x[q, 0], x[q, 1]) for q in range(npart)])
        for it in range(1, self.max_iter + 1):
            ebx, eby = 0.5 * (ex + exk), 0.5 * (ey + eyk)
            jx, jy = np.zeros(g.N), np.zeros(g.N)
            dmax = pmax = 0.0
            for q in range(npart):
                P0 = x[q]
                Pk = x[q] + d[q]
                A1 = g.value0(a, Pk[0], Pk[1])
                mx, my = g.path_means(P0, Pk)
                Ebar = np.array([ebx @ mx, eby @ my])
                D = np.array(g.dA_means(a, P0, Pk))
                p2 = pn[q] @ pn[q]
                g0 = math.sqrt(1.0 + p2 + A0[q] ** 2)
                g1 = math.sqrt(1.0 + p2 + A1 * A1)
                pnew = pn[q] + dt * Ebar - dt * (A1 + A0[q]) * D / (g1 + g0)
                if spin:
                    # discrete gradient of the Zeeman term (coordinate increments)
                    Qy = np.array(g.quotients(ay, k, k - 1, P0, Pk))
                    Qx = np.array(g.quotients(ax, k - 1, k, P0, Pk))
                    Qb = np.array(g.quotients(bz, k - 1, k - 1, P0, Pk))
                    pnew = pnew - dt * self.hbar * (s[q, 0] * Qy - s[q, 1] * Qx + s[q, 2] * Qb)
                g2 = math.sqrt(1.0 + pnew @ pnew + A1 * A1)
                dnew = dt * (pn[q] + pnew) / (g1 + g2)
                # current of the new path x^n -> x^n + dnew
                mx1, my1 = g.path_means(P0, P0 + dnew)
                jx += self.w * dnew[0] * mx1
                jy += self.w * dnew[1] * my1
                dmax = max(dmax, float(np.max(np.abs(dnew - d[q]))))
                pmax = max(pmax, float(np.max(np.abs(pnew - pk[q]))))
                d[q] = dnew
                pk[q] = pnew
            sx, sy = g.solve_M1(jx, jy)
            exn, eyn = ex - sx, ey - sy
            emax = max(float(np.max(np.abs(exn - exk))), float(np.max(np.abs(eyn - eyk))))
            exk, eyk = exn, eyn
            if dmax <= self.tol and pmax <= self.tol and emax <= self.tol:
                break
        else:
            raise O.NoConvergence(f"2D subsystem I: no convergence in {self.max_iter} sweeps")
        xn = x + d
        for q in range(2):
            xn[:, q] = np.mod(xn[:, q], g.L[q])
            xn[xn[:, q] >= g.L[q], q] -= g.L[q]
        return xn, pk, exk, eyk, it
