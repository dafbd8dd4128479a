"""CUDA path (through the C ABI) against the FP64 oracle for the step variants:
the symmetric splitting Phi_I(dt/2) o Phi_II(dt) o Phi_I(dt/2), the path-average
gather of E_x (Sec. 4.2, subsystem I), and the deposit accumulations of the FP32
form (plain float, compensated float pair, double lane sums)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_06513_gb300 import inputs as I
from paper_2203_06513_gb300 import pic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def pdist(a, b, L):
    return np.abs(np.mod(a - b + 0.5 * L, L) - 0.5 * L)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _inputs(w, az_seed=None):
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    if az_seed is not None:
        az = 0.05 * np.random.default_rng(az_seed).normal(size=w.nx)
    return x, p, ay, az, ey, ez


@pytest.mark.parametrize("k", [3, 5])
def test_strang_steps_fp64_vs_oracle(k):
    w = I.Workload("s", nx=48, degree=k, np=6007, seed=21, vth=0.2, pump=0.3)
    x, p, ay, az, ey, ez = _inputs(w, az_seed=6)
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, w.tol, w.max_iter, splitting="strang")
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    g = pic.Pic(pic.Config.from_workload(w, splitting=pic.PIC_SPLIT_STRANG, sort_every=2), x, p, ay, az, ey, ez)
    H0 = g.energy()["total"]
    for _ in range(8):
        s = orc.step(s)
    g.step(8)
    st = g.state_numpy()
    assert np.max(pdist(st["x"], s.x, w.L)) / w.L < 1e-12
    assert rel(st["p"], s.p) < 1e-11
    for key in ("ex", "ey", "ez", "ay", "az"):
        assert rel(st[key], getattr(s, key)) < 1e-11, key
    E = g.energy()
    assert abs(E["total"] - H0) / H0 < 1e-12
    assert E["gauss"] < 1e-13
    g.close()


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_FP32])
@pytest.mark.parametrize("k", [2, 3, 5])
def test_path_average_gather_vs_oracle(k, precision):
    w = I.Workload("g", nx=40, degree=k, np=3001, seed=5)
    x, p, ay, az, ey, ez = _inputs(w)
    # a handle whose dt puts 3-cell displacements inside its halo
    g = pic.Pic(pic.Config(w.L, w.nx, k, w.np, w.weight, 4 * w.dx, precision=precision), x, p, ay, az, ey, ez)
    st = g.state_numpy()
    rng = np.random.default_rng(k)
    disp = rng.uniform(-3.0, 3.0, w.np) * w.dx
    disp[:4] = [0.0, w.dx, -w.dx, 1e-9 * w.dx]
    out = torch.from_numpy(disp.copy()).cuda()
    g.gather(pic.PIC_FIELD_EX_PATHAVG, out)
    got = out.cpu().numpy()
    # the handle's marker positions (float offsets in the FP32 form) and its e_x
    xs, ex = st["x"], st["ex"]
    want = np.empty(w.np)
    for a in range(w.np):
        mean, _ = O.path_integral(k, w.nx, w.dx, xs[a], xs[a] + disp[a])
        want[a] = mean @ ex
    scale = np.max(np.abs(ex))
    # both forms evaluate the path mean in double from the stored positions
    assert np.max(np.abs(got - want)) < 1e-12 * scale
    # zero displacement: the point value E_x,h(x_a)
    pt = torch.empty(w.np, dtype=torch.float64, device="cuda")
    g.gather(pic.PIC_FIELD_EX, pt)
    assert abs(got[0] - pt[0].item()) < 1e-13 * scale
    # a displacement beyond the halo is reported
    bad = torch.from_numpy(disp.copy()).cuda()
    bad[7] = 50 * w.dx
    with pytest.raises(pic.PicError) as e:
        g.gather(pic.PIC_FIELD_EX_PATHAVG, bad)
    assert e.value.code == pic.PIC_ERR_NUMERIC
    g.close()


@pytest.mark.parametrize("deposit", [pic.PIC_ACC_FLOAT, pic.PIC_ACC_COMPENSATED, pic.PIC_ACC_DOUBLE])
@pytest.mark.parametrize("k", [3, 5])
def test_fp32_deposit_accumulations_vs_oracle(k, deposit):
    """FP32 form with each lane accumulation: state within float resolution of the
    oracle, energy conserved, and the Gauss residual within its rounding estimate."""
    w = I.Workload("a", nx=64, degree=k, np=20011, seed=31, vth=0.1, pump=0.2)
    x, p, ay, az, ey, ez = _inputs(w, az_seed=5)
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, w.tol, w.max_iter)
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    g = pic.Pic(pic.Config.from_workload(w, precision=pic.PIC_FP32, deposit=deposit, sort_every=2),
                x, p, ay, az, ey, ez)
    H0 = g.energy()["total"]
    for _ in range(5):
        s = orc.step(s)
    g.step(5)
    st = g.state_numpy()
    assert np.max(pdist(st["x"], s.x, w.L)) / w.L < 2e-7
    assert rel(st["p"], s.p) < 2e-5
    for key in ("ex", "ey", "ay"):
        assert rel(st[key], getattr(s, key)) < 2e-5, key
    E = g.energy()
    assert abs(E["total"] - H0) / H0 < 1e-9
    # Gauss law: the sweep deposits each marker's path integral as a difference of
    # float cumulative basis sums at its two ends, each value rounded to about
    # eps K! in units of w dx / K!; per node and step the residual then grows by
    # about eps w sqrt(2 (k+1) Np / M), a random walk over steps
    est = 1.2e-7 * w.weight * math.sqrt(2 * (k + 1) * w.np / w.nx) * math.sqrt(5)
    print(f"deposit={deposit} k={k}: gauss {E['gauss']:.3e} (estimate {est:.3e}), "
          f"energy {abs(E['total'] - H0) / H0:.3e}")
    assert E["gauss"] < est
    g.close()


def test_unsupported_deposit_accumulation_is_rejected():
    w = I.Workload("a", nx=32, degree=4, np=100)
    x, p, ay, az, ey, ez = _inputs(w)
    with pytest.raises(pic.PicError) as e:
        pic.Pic(pic.Config.from_workload(w, precision=pic.PIC_FP32, deposit=pic.PIC_ACC_FLOAT),
                x, p, ay, az, ey, ez)
    assert e.value.code == pic.PIC_ERR_INVALID
    with pytest.raises(pic.PicError):
        pic.Pic(pic.Config.from_workload(w, precision=pic.PIC_FP64, deposit=pic.PIC_ACC_COMPENSATED),
                x, p, ay, az, ey, ez)
