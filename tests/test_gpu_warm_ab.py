"""What the trained warm-start network gains over the method without it: on the
C2 grid (M = 2048, cubic, pump 0.2, vth 0.1, dt = 0.05), the same markers stepped
three ways at identical tolerance -- x^(0) = x^n (the plain method), the explicit
predictor, and the trained network, each proposal with the field of its path
(warm_field) -- with the mean subsystem-I sweeps a step and the final states
compared, in the FP32 form (2e7 markers) and in the FP64 form (2e6 markers,
tolerance 1e-13 on the increments).  The counts are printed for the design notes;
the network must save at least a sweep a step over the plain method, and all
three must reach the same fixed point."""
import os

import numpy as np
import pytest

from paper_2203_06513_gb300 import inputs as I
from paper_2203_06513_gb300 import pic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2203_06513_gb300", "data", "warm_mlp.npz")


def test_learned_warm_start_ab_fp64():
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained weights")
    w = I.workload("C5", np=2_000_000)
    x, p = I.particles(w, workers=8)
    ay, az, ey, ez = I.fields(w)
    d = np.load(WEIGHTS)
    mlp = pic.Mlp(d["norm"], d["params"])
    steps = 4
    res = {}
    for name, warm in (("none", pic.PIC_WARM_NONE), ("explicit", pic.PIC_WARM_EXPLICIT),
                       ("learned", pic.PIC_WARM_MLP)):
        g = pic.Pic(pic.Config.from_workload(w, sort_every=2, warm_start=warm,
                                             warm_field=int(warm != pic.PIC_WARM_NONE)), x, p, ay, az, ey, ez)
        if warm == pic.PIC_WARM_MLP:
            mlp.attach(g)
        i1, i2 = g.step(steps)
        res[name] = (i1 / steps, g.state_numpy())
        g.close()
    print("\nsubsystem-I sweeps a step (C2 grid, 2e6 markers, FP64, tol 1e-13): "
          + ", ".join(f"{k} {v[0]:.2f}" for k, v in res.items()))
    assert res["learned"][0] <= res["none"][0] - 1
    ref = res["none"][1]
    for name in ("explicit", "learned"):
        st = res[name][1]
        dx = np.abs(np.mod(st["x"] - ref["x"] + 0.5 * w.L, w.L) - 0.5 * w.L)
        assert np.max(dx) < 1e-10 * w.L, name
        assert np.max(np.abs(st["p"] - ref["p"])) < 1e-10, name


def test_learned_warm_start_ab():
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained weights")
    w = I.workload("C5", np=20_000_000)
    x, p = I.particles(w, workers=8)
    ay, az, ey, ez = I.fields(w)
    d = np.load(WEIGHTS)
    mlp = pic.Mlp(d["norm"], d["params"])
    steps = 6
    res = {}
    for name, warm in (("none", pic.PIC_WARM_NONE), ("explicit", pic.PIC_WARM_EXPLICIT),
                       ("learned", pic.PIC_WARM_MLP)):
        g = pic.Pic(pic.Config.from_workload(w, precision=pic.PIC_FP32, warm_start=warm, sort_every=2,
                                             warm_field=int(warm != pic.PIC_WARM_NONE)),
                    x, p, ay, az, ey, ez)
        if warm == pic.PIC_WARM_MLP:
            mlp.attach(g)
        H0 = g.energy()["total"]
        i1, i2 = g.step(steps)
        E = g.energy()
        st = g.state_numpy()
        g.close()
        res[name] = (i1 / steps, i2 / steps, abs(E["total"] - H0) / H0, st)
    print("\nsubsystem-I sweeps a step (C2 grid, 2e7 markers, FP32): "
          + ", ".join(f"{k} {v[0]:.2f}" for k, v in res.items()))
    assert res["learned"][0] <= res["none"][0] - 1
    ref = res["none"][3]
    for name in ("explicit", "learned"):
        st = res[name][3]
        dx = np.abs(np.mod(st["x"] - ref["x"] + 0.5 * w.L, w.L) - 0.5 * w.L)
        assert np.max(dx) < 1e-4 * w.dx, name       # same fixed point to the FP32 stopping rule
        assert np.max(np.abs(st["ex"] - ref["ex"])) < 1e-4 * np.max(np.abs(ref["ex"])), name
        assert res[name][2] < 1e-10, name
