"""Subsystem I of the two-dimensional scheme (Sec. 4.3) on the GPU against the 2D
oracle, through the C ABI (include/pic2d.h): the same markers and fields stepped by
both, positions, momenta and both e_xy components compared at 1e-10 relative;
energy conservation and the Gauss-law identity on the GPU's own result; the
one-cell reduction; invalid configurations refused."""
import numpy as np
import pytest

from oracle import oracle2d as O2
from paper_2203_06513_gb300 import pic
from paper_2203_06513_gb300 import pic2d as P2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _case(seed, M1, M2, k, npart, L1=4.0, L2=3.0, amp=0.3, vth=0.2, dt=0.1):
    rng = np.random.default_rng(seed)
    x = np.column_stack([rng.uniform(0, L1, npart), rng.uniform(0, L2, npart)])
    p = rng.normal(0, vth, (npart, 2))
    n = M1 * M2
    a = amp * rng.normal(0, 1, n)
    ex = 0.05 * rng.normal(0, 1, n)
    ey = 0.05 * rng.normal(0, 1, n)
    cfg = P2.Config2D(L1, L2, M1, M2, k, npart, L1 * L2 / npart, dt)
    orc = O2.Oracle2D(L1, L2, M1, M2, k, w=L1 * L2 / npart, dt=dt)
    return cfg, orc, x, p, ex, ey, a


def _close(a, b, L, tol):
    d = np.abs(np.mod(a - b + 0.5 * L, L) - 0.5 * L)
    return float(np.max(d) / L) < tol


@pytest.mark.parametrize("k,M1,M2", [(2, 6, 5), (3, 7, 6), (4, 8, 5)])
def test_2d_substep_matches_oracle(k, M1, M2):
    cfg, orc, x, p, ex, ey, a = _case(40 + k, M1, M2, k, 60)
    g = P2.Pic2D(cfg, x, p, ex, ey, a)
    sx, sp, sex, sey = x, p, ex, ey
    for step in range(2):
        sx, sp, sex, sey, it = orc.substep1(sx, sp, sex, sey, a)
        it_gpu = g.substep1()
        assert abs(it_gpu - it) <= 1
        st = g.state()
        assert _close(st["x"][:, 0], sx[:, 0], cfg.L1, 1e-10)
        assert _close(st["x"][:, 1], sx[:, 1], cfg.L2, 1e-10)
        assert np.max(np.abs(st["p"] - sp)) <= 1e-10 * np.max(np.abs(sp))
        assert np.max(np.abs(st["ex"] - sex)) <= 1e-10 * np.max(np.abs(sex))
        assert np.max(np.abs(st["ey"] - sey)) <= 1e-10 * np.max(np.abs(sey))
    E = g.energy()
    Eo = orc.energy(sx, sp, sex, sey, a)
    assert abs(E["total"] - Eo["total"]) < 1e-12 * abs(Eo["total"])
    g.close()


def test_2d_energy_and_gauss_law_on_gpu():
    cfg, orc, x, p, ex, ey, a = _case(77, 12, 10, 3, 4000, L1=6.0, L2=5.0, vth=0.3)
    g = P2.Pic2D(cfg, x, p, ex, ey, a)
    H0 = g.energy()["total"]
    st0 = g.state()
    for _ in range(5):
        g.substep1()
    H1 = g.energy()["total"]
    st1 = g.state()
    g.close()
    assert abs(H1 - H0) < 1e-12 * abs(H0)
    # G^T M1 (e^{n+1} - e^n) = -(rho^{n+1} - rho^n), charges by the oracle's basis
    gr = orc.g
    lhs = gr.Gx.T @ (gr.M1x @ (st1["ex"] - st0["ex"])) + gr.Gy.T @ (gr.M1y @ (st1["ey"] - st0["ey"]))
    rhs = -(gr.charge(st1["x"], cfg.weight) - gr.charge(st0["x"], cfg.weight))
    assert np.max(np.abs(lhs - rhs)) < 1e-11 * np.max(np.abs(gr.charge(st0["x"], cfg.weight)))


def test_2d_one_cell_across_matches_oracle():
    """M2 = 1: the grid degenerates to one dimension along x1 (the oracle's
    reduction to the 1D scheme is pinned on the CPU); the GPU follows the oracle."""
    cfg, orc, x, p, ex, ey, a = _case(5, 9, 1, 3, 50)
    p[:, 1] = 0.0
    ey[:] = 0.0
    g = P2.Pic2D(cfg, x, p, ex, ey, a)
    sx, sp, sex, sey, it = orc.substep1(x, p, ex, ey, a)
    g.substep1()
    st = g.state()
    g.close()
    assert _close(st["x"][:, 0], sx[:, 0], cfg.L1, 1e-10)
    assert np.max(np.abs(st["x"][:, 1] - x[:, 1])) == 0.0
    assert np.max(np.abs(st["p"] - sp)) <= 1e-10 * np.max(np.abs(sp))
    assert np.max(np.abs(st["ex"] - sex)) <= 1e-10 * np.max(np.abs(sex))


def test_2d_invalid_configurations():
    cfg, orc, x, p, ex, ey, a = _case(1, 4, 4, 3, 10)
    bad = P2.Config2D(cfg.L1, cfg.L2, 100, 100, 3, 10, 0.1, 0.1)        # M1 * M2 > 4096
    with pytest.raises(pic.PicError):
        P2.Pic2D(bad, x, p, np.zeros(10000), np.zeros(10000), np.zeros(10000))
    xo = x.copy()
    xo[0, 0] = cfg.L1 + 1.0                                            # outside the box
    with pytest.raises(pic.PicError):
        P2.Pic2D(cfg, xo, p, ex, ey, a)


def _spins(seed, npart, n, amp=0.3):
    rng = np.random.default_rng(seed)
    s = rng.normal(0, 1, (npart, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    return s, amp * rng.normal(0, 1, n)


@pytest.mark.parametrize("k,M1,M2", [(2, 6, 5), (3, 7, 6), (4, 8, 5)])
def test_2d_spin_substep_matches_oracle(k, M1, M2):
    """hbar = 0.1: the Zeeman quotients (second differences of A_z, first of b_z)
    on the GPU against the oracle; the Zeeman energy and the total likewise."""
    cfg, orc, x, p, ex, ey, a = _case(60 + k, M1, M2, k, 40)
    cfg.hbar = orc.hbar = 0.1
    s, bz = _spins(90 + k, 40, M1 * M2)
    g = P2.Pic2D(cfg, x, p, ex, ey, a)
    g.set_spin(s, bz)
    E0 = g.energy()
    E0o = orc.energy(x, p, ex, ey, a, s, bz)
    assert abs(E0["zeeman"] - E0o["zeeman"]) < 1e-12 * abs(E0o["total"])
    assert abs(E0o["zeeman"]) > 1e-3 * abs(E0o["total"])
    sx, sp, sex, sey = x, p, ex, ey
    for step in range(2):
        sx, sp, sex, sey, it = orc.substep1(sx, sp, sex, sey, a, s=s, bz=bz)
        it_gpu = g.substep1()
        assert abs(it_gpu - it) <= 1
        st = g.state()
        assert _close(st["x"][:, 0], sx[:, 0], cfg.L1, 1e-10)
        assert _close(st["x"][:, 1], sx[:, 1], cfg.L2, 1e-10)
        assert np.max(np.abs(st["p"] - sp)) <= 1e-10 * np.max(np.abs(sp))
        assert np.max(np.abs(st["ex"] - sex)) <= 1e-10 * np.max(np.abs(sex))
        assert np.max(np.abs(st["ey"] - sey)) <= 1e-10 * np.max(np.abs(sey))
    E = g.energy()
    Eo = orc.energy(sx, sp, sex, sey, a, s, bz)
    assert abs(E["zeeman"] - Eo["zeeman"]) < 1e-12 * abs(Eo["total"])
    assert abs(E["total"] - Eo["total"]) < 1e-12 * abs(Eo["total"])
    g.close()


def test_2d_spin_energy_conserved_on_gpu():
    cfg, orc, x, p, ex, ey, a = _case(78, 12, 10, 3, 4000, L1=6.0, L2=5.0, vth=0.3)
    cfg.hbar = 0.1
    s, bz = _spins(79, 4000, 120)
    g = P2.Pic2D(cfg, x, p, ex, ey, a)
    g.set_spin(s, bz)
    E0 = g.energy()
    for _ in range(5):
        g.substep1()
    E1 = g.energy()
    g.close()
    assert abs(E1["zeeman"] - E0["zeeman"]) > 1e-6 * abs(E0["total"])     # the term does work
    assert abs(E1["total"] - E0["total"]) < 1e-12 * abs(E0["total"])


def test_2d_spin_required_when_hbar_set():
    cfg, orc, x, p, ex, ey, a = _case(3, 5, 4, 3, 10)
    cfg.hbar = 0.1
    g = P2.Pic2D(cfg, x, p, ex, ey, a)
    with pytest.raises(pic.PicError):
        g.substep1()
    g.close()


@pytest.mark.parametrize("k,M1,M2,spin", [(2, 6, 5, False), (3, 7, 6, False), (3, 7, 6, True)])
def test_2d_predicted_start_same_fixed_point(k, M1, M2, spin):
    """warm = 1 starts the fixed point at the explicit predictor with its consistent
    field: the same fixed point (the oracle's result, started from x^n, at 1e-10)
    in no more sweeps than the start at x^n."""
    cfg, orc, x, p, ex, ey, a = _case(80 + k, M1, M2, k, 60)
    s, bz = _spins(81 + k, 60, M1 * M2)
    if spin:
        cfg.hbar = orc.hbar = 0.1
    cfg.warm = 1
    g = P2.Pic2D(cfg, x, p, ex, ey, a)
    if spin:
        g.set_spin(s, bz)
    sx, sp, sex, sey = x, p, ex, ey
    for step in range(2):
        sx, sp, sex, sey, it = orc.substep1(sx, sp, sex, sey, a, s=s if spin else None, bz=bz if spin else None)
        it_gpu = g.substep1()
        print(f"step {step}: sweeps oracle (from x^n) {it}, GPU predicted start {it_gpu}")
        assert it_gpu <= it
        st = g.state()
        assert _close(st["x"][:, 0], sx[:, 0], cfg.L1, 1e-10)
        assert _close(st["x"][:, 1], sx[:, 1], cfg.L2, 1e-10)
        assert np.max(np.abs(st["p"] - sp)) <= 1e-10 * np.max(np.abs(sp))
        assert np.max(np.abs(st["ex"] - sex)) <= 1e-10 * np.max(np.abs(sex))
        assert np.max(np.abs(st["ey"] - sey)) <= 1e-10 * np.max(np.abs(sey))
    g.close()


def test_2d_predicted_start_energy_and_gauss():
    cfg, orc, x, p, ex, ey, a = _case(88, 12, 10, 3, 4000, L1=6.0, L2=5.0, vth=0.3)
    cfg.warm = 1
    g = P2.Pic2D(cfg, x, p, ex, ey, a)
    H0 = g.energy()["total"]
    st0 = g.state()
    sweeps = [g.substep1() for _ in range(5)]
    H1 = g.energy()["total"]
    st1 = g.state()
    g.close()
    print("sweeps with the predicted start:", sweeps)
    assert abs(H1 - H0) < 1e-12 * abs(H0)
    gr = orc.g
    lhs = gr.Gx.T @ (gr.M1x @ (st1["ex"] - st0["ex"])) + gr.Gy.T @ (gr.M1y @ (st1["ey"] - st0["ey"]))
    rhs = -(gr.charge(st1["x"], cfg.weight) - gr.charge(st0["x"], cfg.weight))
    assert np.max(np.abs(lhs - rhs)) < 1e-11 * np.max(np.abs(gr.charge(st0["x"], cfg.weight)))
