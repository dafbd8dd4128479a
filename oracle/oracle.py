"""Plain FP64 CPU oracle of the energy-conserving PIC scheme.

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
* the Lie--Trotter step Phi_II(dt) o Phi_I(dt) (Sec. 5), and its symmetric
  (Strang) variant Phi_I(dt/2) o Phi_II(dt) o Phi_I(dt/2),
* the discrete Hamiltonian (Eq. discrete_H) and the Gauss-law residual,
* with hbar != 0, the spin: the Zeeman term of the Hamiltonian, its discrete
  gradient in subsystem I, its source in subsystem II, and subsystem III (the
  exact Rodrigues rotation of every spin); the Lie--Trotter step is then
  Phi_III o Phi_II o Phi_I.

Where the paper is silent or its printed schemes disagree, this module reads it so:
the V1 basis is the plain B-spline N^{k-1} with (G v)_j = (v_j - v_{j-1}) / dx; a
marker in cell c touches Lambda^0_{c-k..c}, a knot belonging to the cell on its
right; Poisson is G^T M1 e_x = -rho + dx (neutralising background) with sum e_x = 0;
subsystem I iterates on positions from x^(0) = x^n (or a given warm start) with
p^(0) = p^n; the difference quotient of A is the exact path mean of dA/dx, so no
0/0 arises; subsystem II uses Lambda^0 and solves (M0 + dt^2/4 K) exactly each
sweep; the stray M0^{-1} and the dot in the printed schemes are typos; with
hbar != 0 the spin terms follow the Hamiltonian's Zeeman term (momentum update
- dt hbar (s_y D2_z - s_z D2_y) with D2 the exact path mean of d^2A/dx^2, the
printed sign of the second gradient term and its missing weight read as typos;
subsystem II's right side - dt hbar G^T Lambda_1^T W S_z for y and + dt hbar
G^T Lambda_1^T W S_y for z, without the printed M0^{-1}); the Lie--Trotter order
is subsystem I first, then II, then III; each loop stops
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
            L.orc_path_mean_deg.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, dp]
            L.orc_sweep1_spin.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_long] + [dp] * 18
            L.orc_spin_deposit.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_long, dp,
                                           ctypes.c_double, dp, dp]
            L.orc_spin_rotate.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_long, dp, dp, dp, dp, dp, dp]
            L.orc_spin_energy.restype = ctypes.c_double
            L.orc_spin_energy.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_long, dp,
                                          ctypes.c_double, dp, dp, dp, dp]
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


def path_mean_deg(d: int, M: int, dx: float, x0: float, x1: float) -> np.ndarray:
    """Path mean of every degree-d basis function N^d_i along x0 -> x1."""
    mean = np.zeros(M)
    lib().orc_path_mean_deg(d, M, dx, float(x0), float(x1), _p(mean))
    return mean


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
    sx: np.ndarray | None = None   # spin components (hbar != 0 only)
    sy: np.ndarray | None = None
    sz: np.ndarray | None = None

    def copy(self) -> "State":
        return State(*(None if a is None else a.copy()
                       for a in (self.x, self.p, self.ex, self.ey, self.ez, self.ay, self.az,
                                 self.sx, self.sy, self.sz)))

    def spin(self):
        return (self.sx, self.sy, self.sz)


class NoConvergence(RuntimeError):
    pass


class LocalComm:
    """Reductions over the holders of the markers when one process holds them all."""

    def sum(self, a: np.ndarray) -> np.ndarray:
        return a

    def max(self, v: float) -> float:
        return v


class Oracle:
    """Plain FP64 oracle on one uniform periodic grid.

    L: domain length, M: cells, k: V0 degree (V1 has degree k-1), w: equal
    particle weight, dt: time step, tol: absolute fixed-point tolerance on the
    max-norm of the increments, max_iter: iteration cap, splitting: "lie" or
    "strang".

    Markers may be split over several holders (processes), each with its own
    state arrays x, p and the same fields: every grid sum over markers (charge,
    current and susceptibility deposits, kinetic energy) then goes through
    comm.sum and every max over markers (the increments of the fixed-point test)
    through comm.max, so that all holders take the same steps.  threads > 1 runs
    the marker loops of this process on contiguous slices in parallel (for
    timing; the slices' deposits are added, which changes only the order of the
    additions); threads = 1 is the plain serial loop.
    """

    def __init__(self, L: float, M: int, k: int, w: float, dt: float,
                 tol: float = 1e-13, max_iter: int = 100, splitting: str = "lie",
                 comm=None, threads: int = 1, hbar: float = 0.0):
        self.L, self.M, self.k, self.w, self.dt = float(L), int(M), int(k), float(w), float(dt)
        self.tol, self.max_iter = float(tol), int(max_iter)
        assert splitting in ("lie", "strang")
        self.splitting = splitting
        self.hbar = float(hbar)
        assert self.hbar == 0.0 or splitting == "lie", "spin runs use the Lie--Trotter step"
        self.comm = LocalComm() if comm is None else comm
        self.threads = max(1, int(threads))
        self._pool = None
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
    def _slices(self, n: int):
        """Contiguous marker ranges of this process's loops."""
        t = self.threads if n >= 64 * self.threads else 1
        b = [n * i // t for i in range(t + 1)]
        return [(b[i], b[i + 1]) for i in range(t)]

    def _run(self, fn, n: int):
        """fn(lo, hi) on each slice (the C loops release the interpreter lock)."""
        sl = self._slices(n)
        if len(sl) == 1:
            return [fn(*sl[0])]
        if self._pool is None:
            import concurrent.futures as cf
            self._pool = cf.ThreadPoolExecutor(max_workers=self.threads)
        return list(self._pool.map(lambda r: fn(*r), sl))

    def charge(self, x) -> np.ndarray:
        x = _f64(x)

        def part(lo, hi):
            rho = np.zeros(self.M)
            xs = x[lo:hi]
            lib().orc_charge(self.k, self.M, self.dx, xs.shape[0], _p(xs), self.w, _p(rho))
            return rho
        parts = self._run(part, x.shape[0])
        rho = parts[0]
        for q in parts[1:]:
            rho = rho + q
        return self.comm.sum(rho)

    def gather(self, degree: int, x, coef) -> np.ndarray:
        x, coef = _f64(x), _f64(coef)
        out = np.zeros_like(x)
        lib().orc_gather(degree, self.M, self.dx, x.shape[0], _p(x), _p(coef), _p(out))
        return out

    def kinetic(self, x, p, ay, az) -> float:
        x, p, ay, az = map(_f64, (x, p, ay, az))

        def part(lo, hi):
            xs, ps = x[lo:hi], p[lo:hi]
            return lib().orc_kinetic(self.k, self.M, self.dx, xs.shape[0], _p(xs), _p(ps), self.w,
                                     _p(ay), _p(az))
        return float(self.comm.sum(np.array([sum(self._run(part, x.shape[0]))]))[0])

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
        spin = self.spin_energy(s) if self._spin(s) else 0.0
        return {"kinetic": kin, "ex": eex, "eperp": eeperp, "aperp": eaperp, "spin": spin,
                "total": kin + eex + eeperp + eaperp + spin}

    # ---------------- spin (hbar != 0) ----------------
    def _spin(self, s: State) -> bool:
        return self.hbar != 0.0 and s.sy is not None

    def spin_energy(self, s: State) -> float:
        """Zeeman term of Eq. discrete_H:
        hbar sum_a w (s_y dA_z/dx - s_z dA_y/dx)(x_a) = hbar (a_z^T G^T Lambda_1^T W S_y
        - a_y^T G^T Lambda_1^T W S_z)."""
        x, sy, sz = map(_f64, (s.x, s.sy, s.sz))
        ga_y, ga_z = self.G @ s.ay, self.G @ s.az

        def part(lo, hi):
            xs, ys, zs = x[lo:hi], sy[lo:hi], sz[lo:hi]
            return lib().orc_spin_energy(self.k, self.M, self.dx, xs.shape[0], _p(xs), self.w,
                                         _p(ys), _p(zs), _p(ga_y), _p(ga_z))
        return self.hbar * float(self.comm.sum(np.array([sum(self._run(part, x.shape[0]))]))[0])

    def spin_deposit(self, x, comp) -> np.ndarray:
        """Lambda_1(X)^T W S_comp: sum_a w s_a Lambda^1_i(x_a)."""
        x, comp = _f64(x), _f64(comp)

        def part(lo, hi):
            d = np.zeros(self.M)
            xs, cs = x[lo:hi], comp[lo:hi]
            lib().orc_spin_deposit(self.k, self.M, self.dx, xs.shape[0], _p(xs), self.w, _p(cs), _p(d))
            return d
        parts = self._run(part, x.shape[0])
        d = parts[0]
        for q in parts[1:]:
            d = d + q
        return self.comm.sum(d)

    def substep3(self, s: State, dt=None) -> State:
        """Subsystem III (Sec. 4.2, Eq. spin_rodrigue): every spin rotated exactly by
        exp(dt r^), r = (0, dA_z/dx, -dA_y/dx) at the (frozen) marker position."""
        dt = self.dt if dt is None else float(dt)
        out = s.copy()
        ga_y, ga_z = self.G @ s.ay, self.G @ s.az
        x = _f64(out.x)

        def part(lo, hi):
            lib().orc_spin_rotate(self.k, self.M, self.dx, dt, hi - lo, _p(x[lo:hi]), _p(ga_y), _p(ga_z),
                                  _p(out.sx[lo:hi]), _p(out.sy[lo:hi]), _p(out.sz[lo:hi]))
        self._run(part, x.shape[0])
        return out

    # ---------------- subsystem I (Sec. 4.2) ----------------
    def substep1(self, s: State, delta0=None, return_history=False, dt=None):
        """Advance (X, P, e_x) by dt (default: the oracle's dt) with the
        discrete-gradient scheme of subsystem I.  Picard on the positions:
        x^(0) = x^n (or x^n + delta0), sweep -> deposit -> e^(k+1) = e^n - M1^{-1} j
        -> test."""
        dt = self.dt if dt is None else float(dt)
        x, pn, en = s.x, s.p, s.ex
        npart = x.shape[0]
        spin = self._spin(s)
        if spin:
            gga_y = self.G @ (self.G @ s.ay)     # coefficients of d^2A/dx^2 in the degree-(k-2) space
            gga_z = self.G @ (self.G @ s.az)
            sy, sz = _f64(s.sy), _f64(s.sz)
        delta = np.zeros(npart) if delta0 is None else _f64(delta0).copy()
        pk = pn.copy()
        ek = en.copy()
        ga_y = self.G @ s.ay
        ga_z = self.G @ s.az
        dmax, pmax = ctypes.c_double(), ctypes.c_double()
        hist = []
        for it in range(1, self.max_iter + 1):
            ebar = 0.5 * (en + ek)

            def part(lo, hi):
                j = np.zeros(self.M)
                scratch = self._scratch if lo == 0 else np.zeros(self.M)
                dm, pm = ctypes.c_double(), ctypes.c_double()
                if spin:
                    lib().orc_sweep1_spin(self.k, self.M, self.dx, dt, self.w, self.hbar, hi - lo,
                                          _p(x[lo:hi]), _p(pn[lo:hi]), _p(sy[lo:hi]), _p(sz[lo:hi]),
                                          _p(delta[lo:hi]), _p(pk[lo:hi]), _p(ebar), _p(ga_y), _p(ga_z),
                                          _p(gga_y), _p(gga_z), _p(s.ay), _p(s.az), _p(j),
                                          ctypes.byref(dm), ctypes.byref(pm), _p(scratch), _p(np.zeros(self.M)))
                else:
                    lib().orc_sweep1(self.k, self.M, self.dx, dt, self.w, hi - lo,
                                     _p(x[lo:hi]), _p(pn[lo:hi]), _p(delta[lo:hi]), _p(pk[lo:hi]),
                                     _p(ebar), _p(ga_y), _p(ga_z), _p(s.ay), _p(s.az), _p(j),
                                     ctypes.byref(dm), ctypes.byref(pm), _p(scratch))
                return j, dm.value, pm.value
            parts = self._run(part, npart)
            j = parts[0][0]
            for q in parts[1:]:
                j = j + q[0]
            j = self.comm.sum(j)
            dmax.value = self.comm.max(max(q[1] for q in parts))
            pmax.value = self.comm.max(max(q[2] for q in parts))
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
        out = State(xn, pk, ek, s.ey.copy(), s.ez.copy(), s.ay.copy(), s.az.copy(),
                    *(None if a is None else a.copy() for a in s.spin()))
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
        if self._spin(s):
            # the Zeeman term is linear in a: - dt hbar G^T Lambda_1^T W S_z in the
            # y equation, + dt hbar G^T Lambda_1^T W S_y in the z equation
            b_y = b_y - dt * self.hbar * (self.G.T @ self.spin_deposit(x, s.sz))
            b_z = b_z + dt * self.hbar * (self.G.T @ self.spin_deposit(x, s.sy))
        ek_y, ek_z = s.ey.copy(), s.ez.copy()
        hist = []
        for it in range(1, self.max_iter + 1):
            ak_y = s.ay - 0.5 * dt * (s.ey + ek_y)
            ak_z = s.az - 0.5 * dt * (s.ez + ek_z)

            def part(lo, hi):
                sy, sz = np.zeros(self.M), np.zeros(self.M)
                lib().orc_sweep2(self.k, self.M, self.dx, self.w, hi - lo, _p(x[lo:hi]), _p(p[lo:hi]),
                                 _p(s.ay), _p(s.az), _p(ak_y), _p(ak_z), _p(sy), _p(sz))
                return np.concatenate([sy, sz])
            parts = self._run(part, x.shape[0])
            ss = parts[0]
            for q in parts[1:]:
                ss = ss + q
            ss = self.comm.sum(ss)
            sy, sz = ss[: self.M], ss[self.M:]
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
        out = State(s.x.copy(), s.p.copy(), s.ex.copy(), ek_y, ek_z, ay, az,
                    *(None if a is None else a.copy() for a in s.spin()))
        if return_history:
            return out, it, hist
        return out, it

    # ---------------- splitting steps (Sec. 5) ----------------
    def step(self, s: State) -> State:
        """One step: Lie--Trotter Phi_II(dt) o Phi_I(dt) as in Sec. 5, or with
        splitting = "strang" the symmetric composition Phi_I(dt/2) o Phi_II(dt) o
        Phi_I(dt/2) of the same two energy-conserving substeps."""
        if self.splitting == "strang":
            s1, i1 = self.substep1(s, dt=0.5 * self.dt)
            s2, i2 = self.substep2(s1)
            s3, i3 = self.substep1(s2, dt=0.5 * self.dt)
            self.last_iters = (i1 + i3, i2)
            return s3
        s1, i1 = self.substep1(s)
        s2, i2 = self.substep2(s1)
        self.last_iters = (i1, i2)
        if self._spin(s2):
            return self.substep3(s2)
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


def initial_state(orc: Oracle, x, p, ay, az, ey=None, ez=None, spin=None) -> State:
    """Initial state with e_x from the discrete Poisson equation; spin = (sx, sy, sz)
    per marker or None."""
    x, p, ay, az = map(_f64, (x, p, ay, az))
    ey = np.zeros(orc.M) if ey is None else _f64(ey)
    ez = np.zeros(orc.M) if ez is None else _f64(ez)
    sp = (None, None, None) if spin is None else tuple(_f64(c).copy() for c in spin)
    return State(x.copy(), p.copy(), orc.poisson(x), ey.copy(), ez.copy(), ay.copy(), az.copy(), *sp)
