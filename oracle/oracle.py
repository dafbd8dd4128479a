"""Plain FP64 CPU oracle of the energy-conserving PIC scheme (hbar = 0).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library under ``paper_2203_06513_gb300/``; the two meet only through the
seeded input generator ``paper_2203_06513_gb300.inputs``, which holds no
arithmetic of the method.

The particle loops are plain C (``pic_oracle.c``); the grid side is dense
linear algebra here (numpy / scipy LAPACK), written as the paper states it:

* mass matrices M0, M1 and the derivative matrix G (Sec. 3.1, the relation
  d/dx Lambda^0_j = (Lambda^1_j - Lambda^1_{j+1}) / dx),
* the discrete Poisson equation G^T M1 e_x = -Lambda_0(X)^T W 1 + dx 1
  (Remark 2 of Sec. 4.2 with the neutralising unit background),
* subsystem I (Sec. 4.2): Picard iteration on the particle positions, one
  global e_x update per sweep,
* subsystem II (Sec. 4.2): the fixed point on e_y, e_z with the exact solve of
  (M0 + dt^2/4 G^T M1 G),
* the Lie--Trotter step Phi_II(dt) o Phi_I(dt) (Sec. 5),
* the discrete Hamiltonian (Eq. discrete_H) and the Gauss-law residual.

Where the paper is silent or its printed schemes disagree, this module reads it so:
the V1 basis is the plain B-spline N^{k-1} with (G v)_j = (v_j - v_{j-1}) / dx; a
marker in cell c touches Lambda^0_{c-k..c}, a knot belonging to the cell on its
right; Poisson is G^T M1 e_x = -rho + dx (neutralising background) with sum e_x = 0;
subsystem I iterates on positions from x^(0) = x^n (or a given warm start) with
p^(0) = p^n; the difference quotient of A is the exact path mean of dA/dx, so no
0/0 arises; subsystem II uses Lambda^0 and solves (M0 + dt^2/4 K) exactly each
sweep; the stray M0^{-1} and the dot in the printed schemes are typos and the
hbar terms vanish; the Lie--Trotter order is subsystem I first; each loop stops
when the position and field increments are both at most tol = 1e-13; path
integrals are split at every crossed knot and integrated by ceil(k/2)-point
Gauss--Legendre on each piece.
Parity status: every function here is pinned by tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libpic_oracle.so")
_SRC = os.path.join(_HERE, "pic_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C particle loops (plain gcc, IEEE double, no FMA contraction
    so that x86 and Arm hosts round identically)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                               "-ffp-contract=off", "-fno-fast-math",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_cardinal_bspline.restype = ctypes.c_double
            L.orc_cardinal_bspline.argtypes = [ctypes.c_int, ctypes.c_double]
            L.orc_basis.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            L.orc_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
            L.orc_mass_row.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, dp]
            L.orc_path_integral.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, dp, dp]
            L.orc_gather.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_long,
                                     dp, dp, dp]
            L.orc_charge.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_long,
                                     dp, ctypes.c_double, dp]
            L.orc_kinetic.restype = ctypes.c_double
            L.orc_kinetic.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_long,
                                      dp, dp, ctypes.c_double, dp, dp]
            L.orc_sweep1.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_long, dp, dp, dp, dp, dp, dp, dp,
                                     dp, dp, dp, dp, dp, dp]
            L.orc_sweep2.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_long, dp, dp, dp, dp, dp, dp, dp, dp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# B-splines and mass matrices (Sec. 3.1)
# --------------------------------------------------------------------------

def cardinal_bspline(d: int, s: float) -> float:
    """N^d(s): cardinal B-spline of degree d on integer knots (Cox--de Boor)."""
    return lib().orc_cardinal_bspline(d, float(s))


def basis(d: int, t: float) -> np.ndarray:
    """[N^d(r + t) for r = 0..d]: the d+1 nonzero basis values in a cell."""
    out = np.zeros(d + 1)
    lib().orc_basis(d, float(t), _p(out))
    return out


def gauss_legendre(n: int):
    xi, w = np.zeros(n), np.zeros(n)
    assert lib().orc_gauss_legendre(n, _p(xi), _p(w)) == 0
    return xi, w


def mass_row(d: int, M: int, dx: float) -> np.ndarray:
    """First row of the circulant mass matrix of the degree-d periodic spline
    space: (M_d)_{0j} = int Lambda_0 Lambda_j dx."""
    row = np.zeros(M)
    assert lib().orc_mass_row(d, M, dx, _p(row)) == 0
    return row


def circulant(row: np.ndarray) -> np.ndarray:
    """Dense matrix A_{ij} = row[(j - i) mod M]."""
    M = row.shape[0]
    idx = (np.arange(M)[None, :] - np.arange(M)[:, None]) % M
    return row[idx]


def derivative_matrix(M: int, dx: float) -> np.ndarray:
    """G (N1 x N0): d/dx (Lambda^0)(x) = (Lambda^1)(x) G, i.e. G_{jj} = 1/dx,
    G_{j+1,j} = -1/dx (mod M), from d/dx Lambda^0_j = (Lambda^1_j - Lambda^1_{j+1})/dx."""
    G = np.zeros((M, M))
    for j in range(M):
        G[j, j] += 1.0 / dx
        G[(j + 1) % M, j] -= 1.0 / dx
    return G


def path_integral(k: int, M: int, dx: float, x0: float, x1: float):
    """(mean, integral) of every Lambda^1_i along the straight path x0 -> x1."""
    mean, integ = np.zeros(M), np.zeros(M)
    lib().orc_path_integral(k, M, dx, float(x0), float(x1), _p(mean), _p(integ))
    return mean, integ


# --------------------------------------------------------------------------
# The discrete system
# --------------------------------------------------------------------------

@dataclass
class State:
    x: np.ndarray   # positions in [0, L)
    p: np.ndarray   # longitudinal momenta
    ex: np.ndarray  # E_x coefficients (V1)
    ey: np.ndarray  # E_y coefficients (V0)
    ez: np.ndarray
    ay: np.ndarray  # A_y coefficients (V0)
    az: np.ndarray

    def copy(self) -> "State":
        return State(*(a.copy() for a in (self.x, self.p, self.ex, self.ey, self.ez,
                                          self.ay, self.az)))


class NoConvergence(RuntimeError):
    pass


class Oracle:
    """Plain FP64 oracle on one uniform periodic grid.

    L: domain length, M: cells, k: V0 degree (V1 has degree k-1), w: equal
    particle weight, dt: time step, tol: absolute fixed-point tolerance on the
    max-norm of the increments, max_iter: iteration cap.
    """

    def __init__(self, L: float, M: int, k: int, w: float, dt: float,
                 tol: float = 1e-13, max_iter: int = 100):
        self.L, self.M, self.k, self.w, self.dt = float(L), int(M), int(k), float(w), float(dt)
        self.tol, self.max_iter = float(tol), int(max_iter)
        self.dx = self.L / self.M
        self.M0 = circulant(mass_row(self.k, self.M, self.dx))
        self.M1 = circulant(mass_row(self.k - 1, self.M, self.dx))
        self.G = derivative_matrix(self.M, self.dx)
        self.K = self.G.T @ self.M1 @ self.G
        c = self.dt * self.dt / 4.0
        self.P_plus = self.M0 + c * self.K
        self.P_minus = self.M0 - c * self.K
        self._M1_lu = sla.lu_factor(self.M1)
        self._P_lu = sla.lu_factor(self.P_plus)
        self._scratch = np.zeros(self.M)
        self.last_iters = (0, 0)

    # ---------------- particle loops (C) ----------------
    def charge(self, x) -> np.ndarray:
        x = _f64(x)
        rho = np.zeros(self.M)
        lib().orc_charge(self.k, self.M, self.dx, x.shape[0], _p(x), self.w, _p(rho))
        return rho

    def gather(self, degree: int, x, coef) -> np.ndarray:
        x, coef = _f64(x), _f64(coef)
        out = np.zeros_like(x)
        lib().orc_gather(degree, self.M, self.dx, x.shape[0], _p(x), _p(coef), _p(out))
        return out

    def kinetic(self, x, p, ay, az) -> float:
        x, p, ay, az = map(_f64, (x, p, ay, az))
        return lib().orc_kinetic(self.k, self.M, self.dx, x.shape[0], _p(x), _p(p), self.w,
                                 _p(ay), _p(az))

    # ---------------- Poisson (Remark 2, Sec. 4.2) ----------------
    def poisson(self, x) -> np.ndarray:
        """e_x with G^T M1 e_x = -rho + dx 1 and sum_j e_x,j = 0.  With d = M1 e_x
        the equation reads (d_j - d_{j+1})/dx = r_j: a running sum, made
        mean-free, then one M1 solve."""
        r = -self.charge(x) + self.dx
        d = np.zeros(self.M)
        for j in range(self.M - 1):
            d[j + 1] = d[j] - self.dx * r[j]
        d -= d.mean()
        return sla.lu_solve(self._M1_lu, d)

    def gauss_residual(self, x, ex) -> np.ndarray:
        """G^T M1 e_x + rho - dx 1 (zero when the discrete Poisson equation holds)."""
        return self.G.T @ (self.M1 @ _f64(ex)) + self.charge(x) - self.dx

    # ---------------- energy (Eq. discrete_H) ----------------
    def energy(self, s: State) -> dict:
        kin = self.kinetic(s.x, s.p, s.ay, s.az)
        eex = 0.5 * s.ex @ self.M1 @ s.ex
        eeperp = 0.5 * (s.ey @ self.M0 @ s.ey + s.ez @ self.M0 @ s.ez)
        eaperp = 0.5 * (s.ay @ self.K @ s.ay + s.az @ self.K @ s.az)
        return {"kinetic": kin, "ex": eex, "eperp": eeperp, "aperp": eaperp,
                "total": kin + eex + eeperp + eaperp}

    # ---------------- subsystem I (Sec. 4.2) ----------------
    def substep1(self, s: State, delta0=None, return_history=False):
        """Advance (X, P, e_x) by dt with the discrete-gradient scheme of
        subsystem I.  Picard on the positions: x^(0) = x^n (or x^n + delta0),
        sweep -> deposit -> e^(k+1) = e^n - M1^{-1} j -> test."""
        x, pn, en = s.x, s.p, s.ex
        npart = x.shape[0]
        delta = np.zeros(npart) if delta0 is None else _f64(delta0).copy()
        pk = pn.copy()
        ek = en.copy()
        ga_y = self.G @ s.ay
        ga_z = self.G @ s.az
        dmax, pmax = ctypes.c_double(), ctypes.c_double()
        hist = []
        for it in range(1, self.max_iter + 1):
            ebar = 0.5 * (en + ek)
            j = np.zeros(self.M)
            lib().orc_sweep1(self.k, self.M, self.dx, self.dt, self.w, npart,
                             _p(x), _p(pn), _p(delta), _p(pk), _p(ebar), _p(ga_y), _p(ga_z),
                             _p(s.ay), _p(s.az), _p(j), ctypes.byref(dmax), ctypes.byref(pmax),
                             _p(self._scratch))
            enew = en - sla.lu_solve(self._M1_lu, j)
            emax = float(np.max(np.abs(enew - ek)))
            ek = enew
            hist.append((dmax.value, pmax.value, emax))
            if dmax.value <= self.tol and pmax.value <= self.tol and emax <= self.tol:
                break
        else:
            raise NoConvergence(f"subsystem I: no convergence in {self.max_iter} sweeps: {hist[-1]}")
        xn = np.mod(x + delta, self.L)
        xn[xn >= self.L] -= self.L
        out = State(xn, pk, ek, s.ey.copy(), s.ez.copy(), s.ay.copy(), s.az.copy())
        if return_history:
            return out, it, hist
        return out, it

    # ---------------- subsystem II (Sec. 4.2) ----------------
    def substep2(self, s: State, return_history=False):
        """Advance (e_y, e_z, a_y, a_z) by dt with particles frozen:
        (M0 + dt^2/4 K) e^{n+1} = (M0 - dt^2/4 K) e^n + dt K a^n + dt s(a^{n+1}),
        a^{n+1} = a^n - dt/2 (e^n + e^{n+1}), by fixed-point iteration."""
        dt = self.dt
        x, p = s.x, s.p
        b_y = self.P_minus @ s.ey + dt * (self.K @ s.ay)
        b_z = self.P_minus @ s.ez + dt * (self.K @ s.az)
        ek_y, ek_z = s.ey.copy(), s.ez.copy()
        hist = []
        for it in range(1, self.max_iter + 1):
            ak_y = s.ay - 0.5 * dt * (s.ey + ek_y)
            ak_z = s.az - 0.5 * dt * (s.ez + ek_z)
            sy, sz = np.zeros(self.M), np.zeros(self.M)
            lib().orc_sweep2(self.k, self.M, self.dx, self.w, x.shape[0], _p(x), _p(p),
                             _p(s.ay), _p(s.az), _p(ak_y), _p(ak_z), _p(sy), _p(sz))
            en_y = sla.lu_solve(self._P_lu, b_y + dt * sy)
            en_z = sla.lu_solve(self._P_lu, b_z + dt * sz)
            emax = float(max(np.max(np.abs(en_y - ek_y)), np.max(np.abs(en_z - ek_z))))
            ek_y, ek_z = en_y, en_z
            hist.append(emax)
            if emax <= self.tol:
                break
        else:
            raise NoConvergence(f"subsystem II: no convergence in {self.max_iter} sweeps: {hist[-1]}")
        ay = s.ay - 0.5 * dt * (s.ey + ek_y)
        az = s.az - 0.5 * dt * (s.ez + ek_z)
        out = State(s.x.copy(), s.p.copy(), s.ex.copy(), ek_y, ek_z, ay, az)
        if return_history:
            return out, it, hist
        return out, it

    # ---------------- Lie--Trotter step (Sec. 5) ----------------
    def step(self, s: State) -> State:
        s1, i1 = self.substep1(s)
        s2, i2 = self.substep2(s1)
        self.last_iters = (i1, i2)
        return s2

    def run(self, s: State, nsteps: int, diagnostics: bool = False):
        hist = []
        for _ in range(nsteps):
            s = self.step(s)
            if diagnostics:
                hist.append((self.energy(s)["total"],
                             float(np.max(np.abs(self.gauss_residual(s.x, s.ex)))),
                             self.last_iters))
        return (s, hist) if diagnostics else s


def initial_state(orc: Oracle, x, p, ay, az, ey=None, ez=None) -> State:
    """Initial state with e_x from the discrete Poisson equation."""
    x, p, ay, az = map(_f64, (x, p, ay, az))
    ey = np.zeros(orc.M) if ey is None else _f64(ey)
    ez = np.zeros(orc.M) if ez is None else _f64(ez)
    return State(x.copy(), p.copy(), orc.poisson(x), ey.copy(), ez.copy(), ay.copy(), az.copy())
