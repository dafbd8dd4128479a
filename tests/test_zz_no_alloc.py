"""GPU test of pic_deposit_current_noalloc, the deposit for callers that cannot
allocate device memory (a memory pool that must not grow, a device heap owned by
another component).  It needs no handle and uses only the library's fixed
scratch array, so two calls in a row must each reproduce the handle-based
pic_deposit(PIC_DEP_CURRENT) on their own inputs: the second call must not see
anything the first left in the shared scratch.  The deposits are also checked
against the oracle's path integral of the 1-form basis (Sec. 4.2, subsystem I),
at the largest grid the scratch accepts, for every degree, and after a call that
was refused for a bad displacement.

This file is collected last (test_zz_*), so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_06513_gb300 import inputs as I
from paper_2203_06513_gb300 import pic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# double arithmetic on both sides; the bound is relative to w * sum |disp|
TOL = 1e-13


def _noalloc(L, nx, k, np_, weight, x_dev, d_dev, out_dev):
    lib = pic.load()
    f = lib.pic_deposit_current_noalloc
    f.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    rc = f(L, nx, k, np_, weight, ctypes.c_void_p(x_dev.data_ptr()),
           ctypes.c_void_p(d_dev.data_ptr()), ctypes.c_void_p(out_dev.data_ptr()), None)
    if rc != pic.PIC_OK:
        raise pic.PicError(rc, lib.pic_last_error(None).decode())


def _oracle_current(k, nx, L, weight, x, disp):
    """sum_a w int_{x_a}^{x_a + disp_a} Lambda^1_i, marker by marker (oracle)."""
    dx = L / nx
    j = np.zeros(nx)
    for xa, da in zip(x, disp):
        _, integ = O.path_integral(k, nx, dx, float(xa), float(xa + da))
        j += weight * integ
    return j


def _call(L, nx, k, weight, x, disp):
    out = torch.full((nx,), float("nan"), dtype=torch.float64, device="cuda")
    _noalloc(L, nx, k, x.shape[0], weight, torch.from_numpy(x).cuda(), torch.from_numpy(disp).cuda(), out)
    return out.cpu().numpy()


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
    for call in range(2):
        disp = rng.uniform(-6.5, 6.5, w.np) * w.dx * (rng.random(w.np) < 0.6)
        d_dev = torch.from_numpy(disp).cuda()
        ref = torch.zeros(w.nx, dtype=torch.float64, device="cuda")
        g.deposit(pic.PIC_DEP_CURRENT, d_dev, ref)
        out = torch.full((w.nx,), float("nan"), dtype=torch.float64, device="cuda")
        _noalloc(w.L, w.nx, k, w.np, w.weight, x_dev, d_dev, out)
        scale = w.weight * np.sum(np.abs(disp))
        err = float((out - ref).abs().max())
        assert err < TOL * scale, (call, err, scale)
        if call == 0:
            # the first call also against the oracle, marker by marker
            sub = slice(0, 1500)
            xs, ds = x[sub], disp[sub]
            got = _call(w.L, w.nx, k, w.weight, xs, ds)
            want = _oracle_current(k, w.nx, w.L, w.weight, xs, ds)
            assert np.max(np.abs(got - want)) < TOL * w.weight * np.sum(np.abs(ds))
    g.close()


@pytest.mark.parametrize("k", [2, 4])
def test_noalloc_deposit_other_degrees_vs_oracle(k):
    L, nx, n = 4 * np.pi, 40, 700
    rng = np.random.default_rng(40 + k)
    dx = L / nx
    x = rng.uniform(0, L, n)
    x[:5] = np.array([0.0, 3.0, 7.0, 11.0, nx - 1.0]) * dx      # markers on knots
    disp = rng.uniform(-3.2, 3.2, n) * dx
    disp[5:8] = 0.0                                               # at rest
    w = L / n
    got = _call(L, nx, k, w, x, disp)
    want = _oracle_current(k, nx, L, w, x, disp)
    assert np.max(np.abs(got - want)) < TOL * w * np.sum(np.abs(disp))


def test_noalloc_largest_grid_vs_oracle():
    # nx = 8192 is the largest grid the scratch accepts (fewest block rows)
    L, nx, k, n = 4 * np.pi, 8192, 3, 300
    rng = np.random.default_rng(8192)
    dx = L / nx
    x = rng.uniform(0, L, n)
    x[0], x[1] = L - 0.25 * dx, 0.1 * dx                          # paths across the periodic boundary
    disp = rng.uniform(-60, 60, n) * dx
    disp[0], disp[1] = 2.5 * dx, -1.75 * dx
    w = L / n
    for _ in range(2):
        got = _call(L, nx, k, w, x, disp)
        want = _oracle_current(k, nx, L, w, x, disp)
        assert np.max(np.abs(got - want)) < TOL * w * np.sum(np.abs(disp))


def test_noalloc_numeric_errors_then_valid_call():
    L, nx, k, n = 4 * np.pi, 64, 3, 257
    rng = np.random.default_rng(5)
    dx = L / nx
    x = rng.uniform(0, L, n)
    disp = rng.uniform(-2, 2, n) * dx
    w = L / n
    bad_disp = disp.copy()
    bad_disp[100] = 70 * dx                                       # beyond 64 cells
    inf_x = x.copy()
    inf_x[17] = np.inf                                            # non-finite position
    nan_disp = disp.copy()
    nan_disp[3] = np.nan
    for xx, dd in ((x, bad_disp), (inf_x, disp), (x, nan_disp)):
        with pytest.raises(pic.PicError) as e:
            _call(L, nx, k, w, xx, dd)
        assert e.value.code == pic.PIC_ERR_NUMERIC
    # the refused calls leave nothing behind in the shared scratch
    got = _call(L, nx, k, w, x, disp)
    want = _oracle_current(k, nx, L, w, x, disp)
    assert np.max(np.abs(got - want)) < TOL * w * np.sum(np.abs(disp))


def test_noalloc_rejects_oversized_grid():
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(16384, dtype=torch.float64, device="cuda")
    with pytest.raises(pic.PicError) as e:
        _noalloc(4 * np.pi, 16384, 3, 1, 1.0, x, x, out)
    assert e.value.code == pic.PIC_ERR_INVALID
