"""Parity at the full workload sizes, in the launch configuration bench.py times.

The oracle cannot run these workloads (1e8 and 4e8 markers) step by step, so the
GPU step is checked through what the oracle can compute at any size:

* a sample of markers, one by one: fed the GPU's converged displacement, momentum
  and fields, the oracle's subsystem-I sweep (Sec. 4.2) must return them
  unchanged, up to the stopping tolerance of the form;
* the discrete Gauss law (Sec. 4.2, Remark 2) after subsystem I, with the charge
  deposited by the oracle from every marker;
* the subsystem-II equations (Sec. 4.2), with the susceptibility deposited by the
  oracle from every marker: P e^{n+1} = (M0 - dt^2/4 K) e^n + dt K a^n + dt s and
  a^{n+1} = a^n - dt/2 (e^n + e^{n+1});
* the discrete energy (Sec. 3.1), evaluated by the oracle before and after the step.

The oracle's particle loops run in a pool of spawned processes over chunks of
markers (tests/_oracle_pool.py).
"""
import ctypes
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_06513_gb300 import inputs as I
from paper_2203_06513_gb300 import pic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from _oracle_pool import Pool  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2203_06513_gb300", "data", "warm_mlp.npz")
WORKERS = max(1, min(16, os.cpu_count() or 1))


def circ(row, v):
    """Circulant product y_i = sum_j row[(j - i) mod M] v_j (row: first row)."""
    y = np.zeros_like(v)
    for d in np.nonzero(row)[0]:
        y += row[d] * np.roll(v, -d)
    return y


class Grid:
    """Banded operators of the oracle (mass rows from its C code)."""

    def __init__(self, w):
        self.M, self.k, self.dx, self.dt = w.nx, w.degree, w.dx, w.dt
        self.m0 = O.mass_row(self.k, self.M, self.dx)
        self.m1 = O.mass_row(self.k - 1, self.M, self.dx)

    def G(self, v):                     # (G v)_j = (v_j - v_{j-1}) / dx
        return (v - np.roll(v, 1)) / self.dx

    def GT(self, u):                    # (G^T u)_j = (u_j - u_{j+1}) / dx
        return (u - np.roll(u, -1)) / self.dx

    def K(self, v):
        return self.GT(circ(self.m1, self.G(v)))

    def field_energy(self, st):
        return (0.5 * st["ex"] @ circ(self.m1, st["ex"])
                + 0.5 * (st["ey"] @ circ(self.m0, st["ey"]) + st["ez"] @ circ(self.m0, st["ez"]))
                + 0.5 * (st["ay"] @ self.K(st["ay"]) + st["az"] @ self.K(st["az"])))


def energy(pool, grid, w, st):
    kin = pool.kinetic(w.degree, w.nx, w.dx, w.weight, st["x"], st["p"], st["ay"], st["az"])
    return kin + grid.field_energy(st)


def sampled_sweep1(w, st0, st1, n_sample=4096, seed=11):
    """Largest change the oracle's sweep makes to the GPU's converged iterate, on a
    sample: (max |delta' - delta| / (dx max(1, |delta|/dx)), max |p' - p| / max|p|)."""
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(st0["x"].shape[0], n_sample, replace=False))
    x0 = np.ascontiguousarray(st0["x"][idx])
    p0 = np.ascontiguousarray(st0["p"][idx])
    L = w.L
    delta = np.mod(st1["x"][idx] - x0 + 0.5 * L, L) - 0.5 * L
    d_in = delta.copy()
    pk = np.ascontiguousarray(st1["p"][idx])
    p_in = pk.copy()
    ebar = 0.5 * (st0["ex"] + st1["ex"])
    ga_y = (st0["ay"] - np.roll(st0["ay"], 1)) / w.dx
    ga_z = (st0["az"] - np.roll(st0["az"], 1)) / w.dx
    j = np.zeros(w.nx)
    scratch = np.zeros(w.nx)
    dmax, pmax = ctypes.c_double(), ctypes.c_double()
    P = O._p
    O.lib().orc_sweep1(w.degree, w.nx, w.dx, w.dt, w.weight, n_sample, P(x0), P(p0), P(delta), P(pk),
                       P(ebar), P(ga_y), P(ga_z), P(np.ascontiguousarray(st0["ay"])),
                       P(np.ascontiguousarray(st0["az"])), P(j), ctypes.byref(dmax), ctypes.byref(pmax),
                       P(scratch))
    dscale = w.dx * np.maximum(1.0, np.abs(d_in) / w.dx)
    return float(np.max(np.abs(delta - d_in) / dscale)), float(np.max(np.abs(pk - p_in)) / np.max(np.abs(p_in)))


def gauss_residual(pool, grid, w, st):
    rho = pool.charge(w.degree, w.nx, w.dx, w.weight, st["x"])
    return float(np.max(np.abs(grid.GT(circ(grid.m1, st["ex"])) + rho - w.dx))), rho


def subsystem2_residual(pool, grid, w, st1, st2):
    s = pool.sweep2(w.degree, w.nx, w.dx, w.weight, st1["x"], st1["p"], st1["ay"], st1["az"], st2["ay"],
                    st2["az"])
    dt = w.dt
    q = dt * dt / 4.0
    worst_e, worst_a = 0.0, 0.0
    for c, comp in enumerate(("y", "z")):
        en, e1 = st1["e" + comp], st2["e" + comp]
        an, a1 = st1["a" + comp], st2["a" + comp]
        lhs = circ(grid.m0, e1) + q * grid.K(e1)
        rhs = circ(grid.m0, en) - q * grid.K(en) + dt * grid.K(an) + dt * s[c]
        scale = max(np.max(np.abs(dt * s[c])), 1e-300)
        worst_e = max(worst_e, float(np.max(np.abs(lhs - rhs)) / scale))
        worst_a = max(worst_a, float(np.max(np.abs(a1 - (an - 0.5 * dt * (en + e1))))
                                     / max(np.max(np.abs(a1)), 1e-300)))
    return worst_e, worst_a


def run_one_step(cfg, arrays, mlp=None):
    x, p, ay, az, ey, ez = arrays
    g = pic.Pic(cfg, x, p, ay, az, ey, ez)
    if mlp is not None:
        mlp.attach(g)
    st0 = g.state_numpy()
    g.substep(pic.PIC_SUBSYSTEM_I)
    st1 = g.state_numpy()
    g.substep(pic.PIC_SUBSYSTEM_II)
    st2 = g.state_numpy()
    gpu_gauss = g.energy()["gauss"]
    g.close()
    return st0, st1, st2, gpu_gauss


def check_step(pool, w, st0, st1, st2, tol_sweep, tol_energy, tol_gauss, tol_ii):
    grid = Grid(w)
    dd, dp = sampled_sweep1(w, st0, st1)
    assert dd <= tol_sweep and dp <= tol_sweep, (dd, dp)
    res, rho = gauss_residual(pool, grid, w, st1)
    assert res <= tol_gauss * np.max(np.abs(rho)), res
    re, ra = subsystem2_residual(pool, grid, w, st1, st2)
    assert re <= tol_ii and ra <= 1e-14, (re, ra)
    H0, H2 = energy(pool, grid, w, st0), energy(pool, grid, w, st2)
    assert abs(H2 - H0) / abs(H0) <= tol_energy, (H0, H2)
    return {"sweep_delta": dd, "sweep_p": dp, "gauss": res, "ii_residual": re,
            "rel_energy": abs(H2 - H0) / abs(H0)}


@pytest.fixture(scope="module")
def pool():
    p = Pool(WORKERS)
    yield p
    p.close()


def test_c2_full_size_fp32_learned(pool):
    """C2 (M=2048, k=3, 1e8 markers) in the configuration of the bench's value:
    FP32 form, learned warm start, sort every 2 steps; one full step."""
    w = I.workload("C2")
    x, p = I.particles(w, workers=WORKERS)
    ay, az, ey, ez = I.fields(w)
    mlp = None
    warm = pic.PIC_WARM_EXPLICIT
    if os.path.exists(WEIGHTS):
        d = np.load(WEIGHTS)
        mlp = pic.Mlp(d["norm"], d["params"])
        warm = pic.PIC_WARM_MLP
    cfg = pic.Config.from_workload(w, precision=pic.PIC_FP32, warm_start=warm, sort_every=2, warm_field=1)
    st0, st1, st2, _ = run_one_step(cfg, (x, p, ay, az, ey, ez), mlp)
    del x, p
    # FP32 stopping rule: position estimate <= 1e-6 cells relative; float state.
    # Measured: sweep 2.4e-7, Gauss 1.6e-9 max|rho|, subsystem II 1.7e-9, energy 2e-14.
    out = check_step(pool, w, st0, st1, st2, tol_sweep=1e-6, tol_energy=1e-12, tol_gauss=5e-9, tol_ii=5e-9)
    print("C2 FP32 full size:", out)


def test_c3_full_size_fp64_and_fp32(pool):
    """C3 (M=4096, k=5, 4e8 markers): the FP64 form and the FP32 form from the same
    markers, one step each; every check above, and the FP32 fields against FP64."""
    w = I.workload("C3")
    x, p = I.particles(w, workers=WORKERS)
    ay, az, ey, ez = I.fields(w)
    arrays = (x, p, ay, az, ey, ez)
    res = {}
    fields = {}
    # FP32 measured: sweep 4.8e-7, energy 1.6e-12, Gauss 1.4e-9 max|rho|, subsystem II 2.9e-9
    for prec, name, tols in ((pic.PIC_FP64, "fp64", (1e-10, 1e-12, 1e-12, 1e-9)),
                             (pic.PIC_FP32, "fp32", (2e-6, 5e-12, 5e-9, 1e-8))):
        cfg = pic.Config.from_workload(w, precision=prec, warm_start=pic.PIC_WARM_EXPLICIT, sort_every=2)
        st0, st1, st2, _ = run_one_step(cfg, arrays)
        res[name] = check_step(pool, w, st0, st1, st2, *tols)
        fields[name] = {k: st2[k] for k in ("ex", "ey", "ez", "ay", "az")}
        del st0, st1, st2
    diff = max(float(np.max(np.abs(fields["fp32"][k] - fields["fp64"][k])) / np.max(np.abs(fields["fp64"][k])))
               for k in ("ex", "ey", "ay"))
    print("C3 full size:", res, "FP32 vs FP64 fields, relative:", diff)
    assert diff <= 3e-7          # measured 9.9e-8
