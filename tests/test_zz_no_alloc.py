"""GPU test of pic_deposit_current_noalloc, the deposit for callers that cannot
allocate device memory (a memory pool that must not grow, a device heap owned by
another component).  It needs no handle and uses only the library's fixed
scratch array, so two calls in a row must each reproduce the handle-based
pic_deposit(PIC_DEP_CURRENT) on their own inputs: the second call must not see
anything the first left in the shared scratch.

This file is collected last (test_zz_*), so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2203_06513_gb300 import inputs as I
from paper_2203_06513_gb300 import pic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(L, w, x_dev, d_dev, out_dev):
    lib = pic.load()
    f = lib.pic_deposit_current_noalloc
    f.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    rc = f(w.L, w.nx, w.degree, w.np, w.weight, ctypes.c_void_p(x_dev.data_ptr()),
           ctypes.c_void_p(d_dev.data_ptr()), ctypes.c_void_p(out_dev.data_ptr()), None)
    if rc != pic.PIC_OK:
        raise pic.PicError(rc, lib.pic_last_error(None).decode())


@pytest.mark.parametrize("k", [3, 5])
def test_noalloc_deposit_matches_handle_deposit_twice(k):
    w = I.Workload("na", nx=48, degree=k, np=6007, seed=11)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    # a handle whose dt puts 6.5-cell displacements inside its halo
    cfg = pic.Config(w.L, w.nx, k, w.np, w.weight, 8 * w.dx)
    g = pic.Pic(cfg, x, p, ay, az, ey, ez)
    x_dev = torch.from_numpy(x).cuda()
    rng = np.random.default_rng(k)
    # the same tolerance as the handle-based deposit test (double arithmetic)
    tol = 1e-13
    for call in range(2):
        disp = rng.uniform(-6.5, 6.5, w.np) * w.dx * (rng.random(w.np) < 0.6)
        d_dev = torch.from_numpy(disp).cuda()
        ref = torch.zeros(w.nx, dtype=torch.float64, device="cuda")
        g.deposit(pic.PIC_DEP_CURRENT, d_dev, ref)
        out = torch.full((w.nx,), float("nan"), dtype=torch.float64, device="cuda")
        _noalloc(w.L, w, x_dev, d_dev, out)
        scale = w.weight * np.sum(np.abs(disp))
        err = float((out - ref).abs().max())
        assert err < tol * scale, (call, err, scale)
    g.close()


def test_noalloc_rejects_oversized_grid():
    w = I.Workload("na", nx=16384, degree=3, np=1)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(16384, dtype=torch.float64, device="cuda")
    with pytest.raises(pic.PicError) as e:
        _noalloc(w.L, w, x, x, out)
    assert e.value.code == pic.PIC_ERR_INVALID
