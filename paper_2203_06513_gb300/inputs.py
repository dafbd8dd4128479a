"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the method: it only draws marker positions
and momenta and writes the initial field coefficients of the workloads the
library is measured on.  Both sides (CUDA library and CPU oracle) take these
arrays as given.

Recipe (one electron species on a neutralising unit ion background):
* positions x in [0, L): inverse CDF of the density (1 + eps cos(kappa x)) / L,
  i.e. x + (eps/kappa) sin(kappa x) = u L with u ~ U[0,1), solved by Newton;
* momenta p ~ N(0, vth^2) (a Maxwellian in p with c = 1);
* equal weights w = L / Np, so that sum w = L balances the background;
* pump A_y = amp cos(k0 x), A_z = 0, E_y = E_z = 0 (released from rest); or,
  for the paper's parametric-instability runs (Sec. 5), the circularly
  polarised wave E_y = E0 cos(k0 x), E_z = E0 sin(k0 x), A_y = -E0 sin(k0 x),
  A_z = E0 cos(k0 x).  Coefficients are the values of the fields at the
  Greville abscissae x_j + (k+1) dx / 2 of the degree-k basis (the Schoenberg
  quasi-interpolant, one reading of the projector Pi_0 of Sec. 3.1);
* spins (runs with hbar != 0): every marker starts with s = (0, 0, 1);
* E_x is not an input: each side solves the discrete Poisson equation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    L: float = 4.0 * math.pi
    nx: int = 128
    degree: int = 3
    np: int = 20000
    dt: float = 0.05
    steps: int = 50
    tol: float = 1e-13
    eps: float = 0.01          # density perturbation amplitude
    kappa: float = 0.5         # density perturbation wavenumber
    vth: float = 0.1
    pump: float = 0.1          # A_y amplitude
    k0_mode: int = 4           # k0 = 2 pi k0_mode / L
    seed: int = 0
    max_iter: int = 100
    pump_kind: str = "standing"   # "standing": A_y = pump cos(k0 x); "circular": the wave of Sec. 5
    hbar: float = 0.0          # normalised Planck constant (spin runs)

    @property
    def dx(self) -> float:
        return self.L / self.nx

    @property
    def k0(self) -> float:
        return 2.0 * math.pi * self.k0_mode / self.L

    @property
    def weight(self) -> float:
        return self.L / self.np


# The five measured workloads (1D periodic, L = 4 pi, k0 = 2 pi 4 / L = 2).
WORKLOADS = {
    # plain method, FP64: the parity workload
    "C1": Workload("C1", nx=128, degree=3, np=20000, dt=0.05, steps=50, tol=1e-13,
                   vth=0.1, pump=0.1),
    # plain method at scale (FP32 particle state, FP64 grid)
    "C2": Workload("C2", nx=2048, degree=3, np=100_000_000, dt=0.05, steps=1000,
                   vth=0.1, pump=0.2),
    # precision sweep: quintic splines
    "C3": Workload("C3", nx=4096, degree=5, np=400_000_000, dt=0.05, steps=1000,
                   vth=0.05, pump=0.3),
    # learned warm start: C2 shape
    "C5": Workload("C5", nx=2048, degree=3, np=100_000_000, dt=0.05, steps=1000,
                   vth=0.1, pump=0.2),
    # the paper's runs (Sec. 5): parametric instability of a circularly polarised
    # wave, E0 = sqrt(3), k = 1/sqrt(2), L = 2 pi / k, T = 3/511 (vth = sqrt(T)),
    # homogeneous density, M = 128, cubic V0, dt = 0.02; without spin to t = 80
    # with 4e3 markers, with spin (hbar = 0.1, s = (0, 0, 1)) to t = 200 with 1e4
    "P1": Workload("P1", L=2.0 * math.pi * math.sqrt(2.0), nx=128, degree=3, np=4000, dt=0.02,
                   steps=4000, eps=0.0, vth=math.sqrt(3.0 / 511.0), pump=math.sqrt(3.0), k0_mode=1,
                   pump_kind="circular"),
    "P2": Workload("P2", L=2.0 * math.pi * math.sqrt(2.0), nx=128, degree=3, np=10000, dt=0.02,
                   steps=10000, eps=0.0, vth=math.sqrt(3.0 / 511.0), pump=math.sqrt(3.0), k0_mode=1,
                   pump_kind="circular", hbar=0.1),
}


def workload(name: str, **overrides) -> Workload:
    return replace(WORKLOADS[name], **overrides)


def ensemble_members(n_runs: int = 256, seed: int = 0, np_scale: float = 1.0):
    """The batched-ensemble workload: per run r, nx ~ U{256,512,1024,2048},
    Np = floor(exp(U[ln 1e5, ln 4e6])) (times np_scale), pump ~ U[0.01, 0.3],
    vth ~ U[0.02, 0.15], seed r.  Cubic splines, dt = 0.05."""
    rng = np.random.default_rng(seed + 7919)
    out = []
    for r in range(n_runs):
        nx = int(rng.choice([256, 512, 1024, 2048]))
        npart = int(math.floor(math.exp(rng.uniform(math.log(1e5), math.log(4e6)))))
        npart = max(64, int(npart * np_scale))
        pump = float(rng.uniform(0.01, 0.3))
        vth = float(rng.uniform(0.02, 0.15))
        out.append(Workload(f"E{r}", nx=nx, degree=3, np=npart, dt=0.05, steps=1,
                            vth=vth, pump=pump, seed=1000 + r))
    return out


def _inverse_cdf(u: np.ndarray, L: float, eps: float, kappa: float) -> np.ndarray:
    """Solve x + (eps/kappa) sin(kappa x) = u L for x in [0, L) (Newton)."""
    target = u * L
    x = target.copy()
    if eps != 0.0:
        a = eps / kappa
        for _ in range(60):
            f = x + a * np.sin(kappa * x) - target
            fp = 1.0 + eps * np.cos(kappa * x)
            step = f / fp
            x -= step
            if np.max(np.abs(step)) < 1e-15 * L:
                break
    x = np.where(x < 0.0, x + L, x)
    x = np.where(x >= L, x - L, x)
    return x


# markers per independently seeded chunk of the generator
CHUNK = 1 << 22


def _chunk(job):
    seed, c, n, L, eps, kappa, vth = job
    rng = np.random.default_rng(np.random.SeedSequence([seed, c]))
    u = rng.random(n)
    return _inverse_cdf(u, L, eps, kappa), rng.normal(0.0, vth, n)


def particles(w: Workload, np_override: int | None = None, workers: int = 1):
    """(x, p) as float64 arrays.  Chunk c (CHUNK markers) is drawn from its own
    seed (w.seed, c), so the arrays do not depend on how many processes draw
    them; workers > 1 uses a pool of spawned processes (safe after CUDA start)."""
    n = w.np if np_override is None else int(np_override)
    return particles_range(w, 0, n, workers=workers, total=n)


def particles_range(w: Workload, lo: int, hi: int, workers: int = 1, total: int | None = None):
    """Markers [lo, hi) of the plasma of `total` (default w.np) markers: the same
    values as particles() at those indices, drawing only the chunks they lie in."""
    total = w.np if total is None else int(total)
    if not 0 <= lo <= hi <= total:
        raise ValueError("bad marker range")
    x = np.empty(hi - lo, dtype=np.float64)
    p = np.empty(hi - lo, dtype=np.float64)
    c0, c1 = lo // CHUNK, (hi + CHUNK - 1) // CHUNK
    starts = [c * CHUNK for c in range(c0, c1)]
    jobs = [(w.seed, c, min(CHUNK, total - c * CHUNK), w.L, w.eps, w.kappa, w.vth) for c in range(c0, c1)]

    def place(s, xc, pc):
        a, b = max(s, lo), min(s + xc.size, hi)
        if b > a:
            x[a - lo:b - lo] = xc[a - s:b - s]
            p[a - lo:b - lo] = pc[a - s:b - s]
    if workers > 1 and len(jobs) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=min(workers, len(jobs)),
                                    mp_context=mp.get_context("spawn")) as ex:
            results = ex.map(_chunk, jobs)
            for s, (xc, pc) in zip(starts, results):
                place(s, xc, pc)
    else:
        for s, job in zip(starts, jobs):
            xc, pc = _chunk(job)
            place(s, xc, pc)
    return x, p


def fields(w: Workload):
    """(ay, az, ey, ez) initial coefficients, float64 arrays of length nx."""
    j = np.arange(w.nx, dtype=np.float64)
    greville = (j + 0.5 * (w.degree + 1)) * w.dx
    if w.pump_kind == "circular":
        kx = w.k0 * greville
        return -w.pump * np.sin(kx), w.pump * np.cos(kx), w.pump * np.cos(kx), w.pump * np.sin(kx)
    ay = w.pump * np.cos(w.k0 * greville)
    az = np.zeros(w.nx)
    ey = np.zeros(w.nx)
    ez = np.zeros(w.nx)
    return ay, az, ey, ez


def spins(w: Workload):
    """(sx, sy, sz) initial spins of the markers: s = (0, 0, 1) (Sec. 5)."""
    return np.zeros(w.np), np.zeros(w.np), np.ones(w.np)


# ---------------------------------------------------------------------------
# Two-dimensional subsystem I (measurement workload): markers uniform in the box
# [0, L1) x [0, L2), p ~ N(0, vth^2) in each component, equal weights L1 L2 / Np;
# A_z = amp cos(k0 x1) cos(x2 2 pi / L2) at the Greville abscissae of the
# degree-k tensor-product basis; e_x = e_y = 0.
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload2D:
    L1: float = 4.0 * math.pi
    L2: float = 4.0 * math.pi
    M1: int = 64
    M2: int = 64
    degree: int = 3
    np: int = 2_000_000
    dt: float = 0.05
    vth: float = 0.1
    amp: float = 0.2
    k0: float = 2.0
    seed: int = 0

    @property
    def weight(self) -> float:
        return self.L1 * self.L2 / self.np


def particles2d(w: Workload2D):
    """(x, p), each np x 2, seeded."""
    rng = np.random.default_rng([w.seed, 2])
    x = np.empty((w.np, 2))
    x[:, 0] = rng.uniform(0.0, w.L1, w.np)
    x[:, 1] = rng.uniform(0.0, w.L2, w.np)
    p = rng.normal(0.0, w.vth, (w.np, 2))
    return x, p


def fields2d(w: Workload2D):
    """(e_x, e_y, a_z) coefficients, node index i1 * M2 + i2."""
    g1 = (np.arange(w.M1) + 0.5 * (w.degree + 1)) * (w.L1 / w.M1)
    g2 = (np.arange(w.M2) + 0.5 * (w.degree + 1)) * (w.L2 / w.M2)
    az = w.amp * np.outer(np.cos(w.k0 * g1), np.cos(2.0 * math.pi * g2 / w.L2)).ravel()
    n = w.M1 * w.M2
    return np.zeros(n), np.zeros(n), az
