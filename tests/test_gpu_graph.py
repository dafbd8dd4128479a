"""Steps as CUDA graphs with device-ended loops (pic_step after its first step)
against the same kernels driven from the host (one readback per sweep): the same
state to rounding, the same sweep counts, for the FP64 and FP32 forms, both warm
starts, the symmetric splitting, and across marker sorts (one graph per marker
copy)."""
import os

import numpy as np
import pytest

from paper_2203_06513_gb300 import inputs as I
from paper_2203_06513_gb300 import pic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _run(w, cfg, steps, no_graph):
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    if no_graph:
        os.environ["PIC_NO_GRAPH"] = "1"
    try:
        g = pic.Pic(cfg, x, p, ay, az, ey, ez)
        its = [g.step(1)]
        its.append(g.step(steps - 1))
        st = g.state_numpy()
        E = g.energy()
        g.close()
    finally:
        os.environ.pop("PIC_NO_GRAPH", None)
    return st, its, E


@pytest.mark.parametrize("case", ["fp64", "fp32_explicit", "fp32_none", "strang", "fp32_predicted", "fp64_predicted"])
def test_graph_steps_match_host_loops(case):
    w = I.Workload("g", nx=96, degree=3, np=30011, seed=23, vth=0.15, pump=0.25)
    kw = {"sort_every": 2}
    if case == "fp64":
        cfg = pic.Config.from_workload(w, **kw)
    elif case == "fp32_explicit":
        cfg = pic.Config.from_workload(w, precision=pic.PIC_FP32, warm_start=pic.PIC_WARM_EXPLICIT, **kw)
    elif case == "fp32_none":
        cfg = pic.Config.from_workload(w, precision=pic.PIC_FP32, **kw)
    elif case == "fp32_predicted":
        cfg = pic.Config.from_workload(w, precision=pic.PIC_FP32, warm_start=pic.PIC_WARM_EXPLICIT, warm_field=1,
                                       **kw)
    elif case == "fp64_predicted":
        cfg = pic.Config.from_workload(w, warm_start=pic.PIC_WARM_EXPLICIT, warm_field=1, **kw)
    else:
        cfg = pic.Config.from_workload(w, splitting=pic.PIC_SPLIT_STRANG, **kw)
    a, ia, Ea = _run(w, cfg, 7, no_graph=False)
    b, ib, Eb = _run(w, cfg, 7, no_graph=True)
    tol = 1e-12 if cfg.precision == pic.PIC_FP64 else 1e-6
    if cfg.precision == pic.PIC_FP64:
        assert ia == ib
    else:   # float decisions near the noise floor may differ by a sweep (atomics order)
        for (a1, a2), (b1, b2) in zip(ia, ib):
            assert abs(a1 - b1) <= 7 and abs(a2 - b2) <= 7
    d = np.abs(np.mod(a["x"] - b["x"] + 0.5 * w.L, w.L) - 0.5 * w.L)
    assert np.max(d) / w.L < tol
    for key in ("p", "ex", "ey", "ay"):
        assert np.max(np.abs(a[key] - b[key])) <= tol * np.max(np.abs(b[key])), key
    assert abs(Ea["total"] - Eb["total"]) < (1e-13 if cfg.precision == pic.PIC_FP64 else 1e-10) * Eb["total"]
