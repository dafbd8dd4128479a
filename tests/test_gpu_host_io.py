"""Host arrays in and out of the C ABI: page-locked host arrays (read and written by
the load and store kernels directly) give the same state, bit for bit, as pageable
ones (staged through device buffers and copies), in both precision forms."""
import numpy as np
import pytest

from paper_2203_06513_gb300 import inputs as I
from paper_2203_06513_gb300 import pic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_FP32])
def test_pinned_host_arrays_match_pageable(precision):
    w = I.Workload("io", nx=64, degree=3, np=5003, seed=3, pump=0.2)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    cfg = pic.Config.from_workload(w, precision=precision, warm_start=pic.PIC_WARM_EXPLICIT, sort_every=2)
    g1 = pic.Pic(cfg, x, p, ay, az, ey, ez)
    g2 = pic.Pic(cfg, _pinned(x), _pinned(p), ay, az, ey, ez)
    # input: the loaded markers are the same bits (the fields come from a charge
    # deposit with atomics, whose order differs between any two handles)
    s1, s2 = g1.state_numpy(), g2.state_numpy()
    for k in ("x", "p"):
        np.testing.assert_array_equal(s2[k], s1[k], err_msg=k)
    i1, i2 = g1.step(3), g2.step(3)
    # output: one handle read into page-locked and into pageable arrays, same bits
    ref = g2.state_numpy()
    out = {k: _pinned(np.zeros(w.np)) for k in ("x", "p")}
    out.update({k: np.zeros(w.nx) for k in ("ex", "ey", "ez", "ay", "az")})
    g2.get_state(**out)
    for k in ref:
        np.testing.assert_array_equal(out[k], ref[k], err_msg=k)
    # the two handles after three steps: equal up to the order of the atomics
    tol = 1e-12 if precision == pic.PIC_FP64 else 1e-5
    s1 = g1.state_numpy()
    d = np.abs(np.mod(s1["x"] - ref["x"] + 0.5 * w.L, w.L) - 0.5 * w.L)
    assert np.max(d) / w.L <= tol
    assert np.max(np.abs(s1["p"] - ref["p"])) <= tol * np.max(np.abs(ref["p"]))
    assert abs(i1[0] - i2[0]) <= 1 and abs(i1[1] - i2[1]) <= 1
    g1.close()
    g2.close()
