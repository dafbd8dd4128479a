"""The paper's claims on a full run of the plain FP64 workload (Sec. 5): the
relative energy error stays at the level of the iteration tolerance and the
discrete Poisson equation holds at every step."""
import numpy as np

from oracle import oracle as O
from paper_2203_06513_gb300 import inputs as I


def test_c1_fifty_steps_energy_and_gauss():
    w = I.workload("C1")
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, w.tol)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    H0 = orc.energy(s)["total"]
    s, hist = orc.run(s, w.steps, diagnostics=True)
    rel = np.array([abs(h[0] - H0) / H0 for h in hist])
    gauss = np.array([h[1] for h in hist])
    assert rel.max() < 1e-12
    assert gauss.max() < 1e-13
    iters = np.array([h[2] for h in hist])
    assert iters.max() < 20 and iters.min() >= 2
    # the pump does work on the plasma: energy moves between parts
    E = orc.energy(s)
    assert E["eperp"] > 0.0
