"""Pins of the oracle's symmetric splitting Phi_I(dt/2) o Phi_II(dt) o Phi_I(dt/2),
the Strang variant of the Lie--Trotter composition the paper uses (Sec. 5).

Each substep is the paper's energy-conserving scheme (Sec. 4.2), so the composed
step conserves the discrete energy and the discrete Gauss law like the
Lie--Trotter step.  What distinguishes the two compositions is the order in dt
of the splitting error: halving dt must divide the error of Lie--Trotter by
about 2 and that of the symmetric composition by about 4 (a composition with the
wrong substep lengths, or a missing half step, is first order or inconsistent).
"""
import math

import numpy as np

from oracle import oracle as O
from paper_2203_06513_gb300 import inputs as I


def _run(dt, splitting, T=0.4):
    w = I.Workload("s", L=4 * math.pi, nx=16, degree=3, np=64, dt=dt, vth=0.2, pump=0.5, seed=3)
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, dt, 1e-13, splitting=splitting)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    ey = 0.3 * np.sin(w.k0 * np.arange(w.nx) * w.dx)      # a transverse field that moves the markers
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    for _ in range(int(round(T / dt))):
        s = orc.step(s)
    return s


def _err(s, ref):
    return max(np.max(np.abs(s.p - ref.p)), np.max(np.abs(s.ey - ref.ey)), np.max(np.abs(s.ex - ref.ex)))


def test_splitting_orders():
    ref = _run(0.4 / 256, "strang")
    lie = [_err(_run(dt, "lie"), ref) for dt in (0.1, 0.05, 0.025)]
    strang = [_err(_run(dt, "strang"), ref) for dt in (0.1, 0.05, 0.025)]
    for e in (lie, strang):
        assert e[0] > e[1] > e[2]
    r_lie = [lie[i] / lie[i + 1] for i in range(2)]
    r_str = [strang[i] / strang[i + 1] for i in range(2)]
    assert all(1.7 < r < 3.0 for r in r_lie), r_lie
    assert all(3.5 < r < 4.5 for r in r_str), r_str
    assert strang[2] < 0.5 * lie[2]


def test_strang_conserves_energy_and_gauss():
    w = I.Workload("s", nx=32, degree=3, np=2000, dt=0.05, pump=0.2, seed=8)
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, 1e-13, splitting="strang")
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    H0 = orc.energy(s)["total"]
    s, hist = orc.run(s, 6, diagnostics=True)
    assert max(abs(h[0] - H0) / H0 for h in hist) < 1e-12
    assert max(h[1] for h in hist) < 1e-13
    # two subsystem-I loops a step
    assert all(h[2][0] >= 4 for h in hist)
