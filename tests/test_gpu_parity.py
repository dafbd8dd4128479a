"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 form: the parity bar is a relative 1e-10 in particle state and field
coefficients over the 50 steps of the plain workload; single kernels and single
substeps are held to 1e-12..1e-13 (both sides solve the same fixed point to
tol = 1e-13, and differ only in rounding order: atomics, and the kernel's exact
midpoint-Taylor path means against the oracle's Gauss--Legendre rule).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_06513_gb300 import inputs as I
from paper_2203_06513_gb300 import pic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def pdist(a, b, L):
    d = np.mod(a - b + 0.5 * L, L) - 0.5 * L
    return np.abs(d)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def setup(w, precision=pic.PIC_FP64, az_seed=None, **kw):
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    if az_seed is not None:
        az = 0.05 * np.random.default_rng(az_seed).normal(size=w.nx)
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, w.tol, w.max_iter)
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    cfg = pic.Config.from_workload(w, precision=precision, **kw)
    g = pic.Pic(cfg, x, p, ay, az, ey, ez)
    return orc, s, g


def small(M=32, k=3, npart=3001, seed=3, **kw):
    return I.Workload("t", nx=M, degree=k, np=npart, seed=seed, **kw)


def compare_state(g, s, L, tx, tp, te):
    st = g.state_numpy()
    assert np.max(pdist(st["x"], s.x, L)) / L <= tx
    assert rel(st["p"], s.p) <= tp
    for k in ("ex", "ey", "ez", "ay", "az"):
        ref = getattr(s, k)
        if np.max(np.abs(ref)) > 0:
            assert rel(st[k], ref) <= te, k
        else:
            assert np.max(np.abs(st[k])) <= te
    return st


@pytest.mark.parametrize("k", [2, 3, 5])
def test_init_poisson_and_gathers(k):
    w = small(k=k, M=24, npart=2049)
    orc, s, g = setup(w, az_seed=1)
    st = g.state_numpy()
    np.testing.assert_array_equal(st["p"], s.p)
    assert np.max(pdist(st["x"], s.x, w.L)) < 1e-14 * w.L
    assert rel(st["ex"], s.ex) < 1e-12
    dev = torch.empty(w.np, dtype=torch.float64, device="cuda")
    for field, deg, coef in [(pic.PIC_FIELD_EX, k - 1, s.ex), (pic.PIC_FIELD_AY, k, s.ay),
                             (pic.PIC_FIELD_AZ, k, s.az)]:
        g.gather(field, dev)
        ref = orc.gather(deg, s.x, coef)
        assert np.max(np.abs(dev.cpu().numpy() - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))
    E = g.energy()
    Eo = orc.energy(s)
    assert abs(E["total"] - Eo["total"]) < 1e-13 * Eo["total"]
    assert E["gauss"] < 1e-13


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_FP32])
@pytest.mark.parametrize("k", [2, 3, 5])
def test_deposits(k, precision):
    w = small(k=k, M=40, npart=5003)
    orc, s, g = setup(w, precision, az_seed=2)
    tol = 1e-13 if precision == pic.PIC_FP64 else 2e-6
    out = torch.zeros(2 * w.nx, dtype=torch.float64, device="cuda")
    g.deposit(pic.PIC_DEP_CHARGE, None, out)
    rho = orc.charge(s.x)
    assert np.max(np.abs(out[: w.nx].cpu().numpy() - rho)) < tol * np.max(rho) * 10
    # path-integrated current for displacements that cross 0..6 knots, both ways
    rng = np.random.default_rng(k)
    disp = rng.uniform(-6.5, 6.5, w.np) * w.dx * (rng.random(w.np) < 0.5)
    disp[:7] = [0.0, w.dx, -w.dx, 1e-12, -1e-12, 3 * w.dx, -2 * w.dx]
    # a handle with dt large enough that 6.5-cell displacements lie inside its halo
    g2 = pic.Pic(pic.Config(w.L, w.nx, k, w.np, w.weight, 8 * w.dx, precision=precision),
                 s.x, s.p, s.ay, s.az)
    g2.deposit(pic.PIC_DEP_CURRENT, torch.from_numpy(disp).cuda(), out)
    ref = np.zeros(w.nx)
    for a in range(w.np):
        ref += w.weight * O.path_integral(k, w.nx, w.dx, s.x[a], s.x[a] + disp[a])[1]
    scale = w.weight * np.sum(np.abs(disp))
    assert np.max(np.abs(out[: w.nx].cpu().numpy() - ref)) < tol * scale
    # susceptibility deposit of subsystem II with A^* = a^n + perturbation
    astar = np.concatenate([s.ay + 0.01 * rng.normal(size=w.nx), s.az + 0.02 * rng.normal(size=w.nx)])
    g.deposit(pic.PIC_DEP_SUSCEPT, torch.from_numpy(astar).cuda(), out)
    sy, sz = np.zeros(w.nx), np.zeros(w.nx)
    L = O.lib()
    L.orc_sweep2(k, w.nx, w.dx, w.weight, w.np, O._p(s.x), O._p(s.p), O._p(s.ay), O._p(s.az),
                 O._p(np.ascontiguousarray(astar[: w.nx])), O._p(np.ascontiguousarray(astar[w.nx:])),
                 O._p(sy), O._p(sz))
    o = out.cpu().numpy()
    assert np.max(np.abs(o[: w.nx] - sy)) < tol * 10 * np.max(np.abs(sy))
    assert np.max(np.abs(o[w.nx:] - sz)) < tol * 10 * np.max(np.abs(sz))


@pytest.mark.parametrize("k", [2, 3, 5])
def test_substeps_fp64(k):
    w = small(k=k, M=32, npart=4099, vth=0.3, pump=0.3)
    orc, s, g = setup(w, az_seed=4)
    s1, i1 = orc.substep1(s)
    gi1 = g.substep(pic.PIC_SUBSYSTEM_I)
    assert abs(gi1 - i1) <= 1
    compare_state(g, s1, w.L, 1e-13, 1e-12, 1e-12)
    s2, i2 = orc.substep2(s1)
    gi2 = g.substep(pic.PIC_SUBSYSTEM_II)
    assert abs(gi2 - i2) <= 1
    compare_state(g, s2, w.L, 1e-13, 1e-12, 1e-12)


def test_c1_fifty_steps_fp64():
    """The plain FP64 workload, 50 steps: relative 1e-10 in state and fields,
    energy conserved to the iteration tolerance, Gauss law to rounding."""
    w = I.workload("C1")
    orc, s, g = setup(w)
    H0 = g.energy()["total"]
    for n in range(w.steps):
        s = orc.step(s)
        g.step(1)
        if n % 10 == 9:
            E = g.energy()
            assert abs(E["total"] - H0) / H0 < 1e-12
            assert E["gauss"] < 1e-13
    compare_state(g, s, w.L, 1e-10, 1e-10, 1e-10)


@pytest.mark.parametrize("npart", [1, 2, 31, 257])
def test_ragged_and_tiny_marker_counts(npart):
    w = small(M=16, npart=npart, vth=0.5, pump=0.2)
    orc, s, g = setup(w)
    for _ in range(3):
        s = orc.step(s)
    g.step(3)
    compare_state(g, s, w.L, 1e-12, 1e-11, 1e-11)


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_FP32])
def test_all_markers_in_one_cell(precision):
    """Degenerate distribution: every marker in one cell (all warps on the same
    deposit window, heavy same-address accumulation), moving both ways."""
    w = small(M=32, npart=5003, vth=0.3, pump=0.2)
    x = 7.0 * w.dx + 0.999 * w.dx * np.random.default_rng(12).random(w.np)
    p = np.random.default_rng(13).normal(0.0, w.vth, w.np)
    ay, az, ey, ez = I.fields(w)
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, w.tol, w.max_iter)
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    g = pic.Pic(pic.Config.from_workload(w, precision=precision, sort_every=1), x, p, ay, az, ey, ez)
    for _ in range(3):
        s = orc.step(s)
    g.step(3)
    if precision == pic.PIC_FP64:
        compare_state(g, s, w.L, 1e-12, 1e-11, 1e-11)
    else:
        compare_state(g, s, w.L, 1e-6, 1e-5, 1e-5)


def test_grid_too_large_for_shared_memory_is_rejected():
    """nx = 8192 with quintic splines cannot be staged in shared memory: pic_init
    refuses it with PIC_ERR_INVALID and a message, and the library stays usable."""
    w = I.Workload("big", nx=8192, degree=5, np=1000)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    with pytest.raises(pic.PicError) as e:
        pic.Pic(pic.Config.from_workload(w, precision=pic.PIC_FP32), x, p, ay, az, ey, ez)
    assert e.value.code == pic.PIC_ERR_INVALID and "shared memory" in str(e.value)
    w2 = small(M=16, npart=100)
    x2, p2 = I.particles(w2)
    ay2, az2, ey2, ez2 = I.fields(w2)
    g = pic.Pic(pic.Config.from_workload(w2), x2, p2, ay2, az2, ey2, ez2)
    g.step(1)
    g.close()


@pytest.mark.parametrize("M", [16, 128])
def test_edge_markers_on_knots_at_rest_and_crossing_the_boundary(M):
    """Markers exactly on knots, at rest, and crossing x = 0 and x = L; with
    M = 128 and dt = 0.3 fast markers cross up to three knots per step."""
    k = 3
    w = small(M=M, npart=64, dt=0.3)
    x, p = I.particles(w)
    x[:8] = np.arange(8) * w.dx            # exactly on knots
    p[:8] = 0.0                            # at rest
    x[8:16] = w.L - 1e-9 * np.arange(1, 9)  # just left of the periodic boundary
    p[8:16] = 2.0                          # moving right, across x = L
    x[16:24] = 1e-9 * np.arange(8)
    p[16:24] = -3.0                        # moving left, across x = 0
    ay, az, ey, ez = I.fields(w)
    orc = O.Oracle(w.L, M, k, w.weight, w.dt, w.tol)
    s = O.initial_state(orc, x, p, ay, az)
    g = pic.Pic(pic.Config.from_workload(w), x, p, ay, az, ey, ez)
    for _ in range(4):
        s = orc.step(s)
    g.step(4)
    compare_state(g, s, w.L, 1e-12, 1e-11, 1e-11)


def test_fp32_form_against_oracle():
    """FP32 particle arithmetic: state within float resolution of the FP64
    oracle after a few steps; energy and Gauss law still conserved to the
    accuracy of float positions and momenta."""
    w = small(M=64, npart=20011, vth=0.1, pump=0.2)
    orc, s, g = setup(w, pic.PIC_FP32, az_seed=5)
    H0 = g.energy()["total"]
    for _ in range(5):
        s = orc.step(s)
    g.step(5)
    compare_state(g, s, w.L, 2e-7, 2e-5, 2e-5)
    E = g.energy()
    assert abs(E["total"] - H0) / H0 < 1e-9
    # Gauss law: each marker's path integral is formed in float (relative error
    # eps ~ 1.2e-7) on a current w v dt; per node and step the residual grows by
    # about eps w v dt sqrt(k Np / M) / dx, a random walk over steps.  Allow 20x.
    est = 1.2e-7 * w.weight * w.vth * w.dt * math.sqrt(3 * w.np / w.nx) / w.dx * math.sqrt(5)
    print(f"\nFP32 vs oracle, 5 steps: energy {abs(E['total'] - H0) / H0:.3e}, Gauss {E['gauss']:.3e} = "
          f"{E['gauss'] / est:.3f} x estimate")
    assert E["gauss"] < 20 * est


def test_noconvergence_is_reported():
    w = small(M=16, npart=100)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    cfg = pic.Config.from_workload(w, max_iter=1, tol=1e-30)
    g = pic.Pic(cfg, x, p, ay, az, ey, ez)
    with pytest.raises(pic.NoConvergence):
        g.substep(pic.PIC_SUBSYSTEM_I)


def test_timing_counts_match_sweeps():
    """Kernel timing (events recorded without host synchronisation, read back by
    pic_timing_read): one timed launch per sweep and per solve, positive times,
    and a fresh enable starts from zero."""
    w = small(M=64, npart=20000, seed=9)
    for warm in (pic.PIC_WARM_NONE, pic.PIC_WARM_EXPLICIT):
        _, _, g = setup(w, precision=pic.PIC_FP32, warm_start=warm, sort_every=2)
        g.step(1)
        g.timing_enable(True)
        i1, i2 = g.step(3)
        t = g.timing_read()
        assert t["sweep1_launches"] == i1 and t["sweep2_launches"] == i2
        assert t["solve_launches"] == i1 + i2
        assert t["sweep1_ms"] > 0 and t["sweep2_ms"] > 0 and t["solve_ms"] > 0
        assert t["marker_sweeps1"] == i1 * w.np
        g.timing_enable(True)
        t = g.timing_read()
        assert t["sweep1_launches"] == 0 and t["sweep1_ms"] == 0
        g.close()
