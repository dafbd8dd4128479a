"""CUDA path with spin (hbar != 0, FP64 form) against the FP64 oracle: the
discrete gradient of the Zeeman energy in subsystem I, its source in subsystem
II, the exact spin rotation of subsystem III (Eq. spin_rodrigue), and whole
Lie--Trotter steps Phi_III o Phi_II o Phi_I (Sec. 4.2, Sec. 5)."""
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


def _spin_workload(M=64, k=3, npart=4001, seed=7, random_spin=True):
    w = I.workload("P2", nx=M, degree=k, np=npart, seed=seed)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    if random_spin:
        s = np.random.default_rng(seed).normal(size=(3, npart))
        s /= np.linalg.norm(s, axis=0)
        spin = (s[0].copy(), s[1].copy(), s[2].copy())
    else:
        spin = I.spins(w)
    return w, x, p, ay, az, ey, ez, spin


def _pair(w, x, p, ay, az, ey, ez, spin):
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, w.tol, w.max_iter, hbar=w.hbar)
    s = O.initial_state(orc, x, p, ay, az, ey, ez, spin=spin)
    g = pic.Pic(pic.Config.from_workload(w, sort_every=2), x, p, ay, az, ey, ez, spin=spin)
    return orc, s, g


def _compare(g, s, L, tol):
    st = g.state_numpy()
    assert np.max(pdist(st["x"], s.x, L)) / L < tol
    assert rel(st["p"], s.p) < tol
    for key in ("ex", "ey", "ez", "ay", "az"):
        assert rel(st[key], getattr(s, key)) < tol, key
    for key in ("sx", "sy", "sz"):
        assert np.max(np.abs(st[key] - getattr(s, key))) < tol, key
    return st


@pytest.mark.parametrize("k", [2, 3, 5])
def test_spin_substeps_vs_oracle(k):
    w, x, p, ay, az, ey, ez, spin = _spin_workload(M=48, k=k, npart=3001)
    orc, s, g = _pair(w, x, p, ay, az, ey, ez, spin)
    E0 = g.energy()
    Eo = orc.energy(s)
    assert abs(E0["spin"] - Eo["spin"]) < 1e-13 * abs(Eo["total"])
    assert abs(E0["total"] - Eo["total"]) < 1e-13 * abs(Eo["total"])
    s1, i1 = orc.substep1(s)
    assert abs(g.substep(pic.PIC_SUBSYSTEM_I) - i1) <= 1
    _compare(g, s1, w.L, 1e-12)
    s2, i2 = orc.substep2(s1)
    assert abs(g.substep(pic.PIC_SUBSYSTEM_II) - i2) <= 1
    _compare(g, s2, w.L, 1e-12)
    s3 = orc.substep3(s2)
    g.substep(pic.PIC_SUBSYSTEM_III)
    st = _compare(g, s3, w.L, 1e-12)
    n = st["sx"] ** 2 + st["sy"] ** 2 + st["sz"] ** 2
    assert np.max(np.abs(n - 1.0)) < 1e-14
    g.close()


def test_spin_twenty_steps_vs_oracle():
    """Relative 1e-10 in particle state, spins and fields over 20 steps; the
    energy with its Zeeman term conserved to the iteration tolerance."""
    w, x, p, ay, az, ey, ez, spin = _spin_workload(M=64, npart=4001, random_spin=False)
    orc, s, g = _pair(w, x, p, ay, az, ey, ez, spin)
    H0 = g.energy()["total"]
    for n in range(20):
        s = orc.step(s)
        g.step(1)
        if n % 5 == 4:
            E = g.energy()
            assert abs(E["total"] - H0) / abs(H0) < 1e-12
            assert E["gauss"] < 1e-13
    _compare(g, s, w.L, 1e-10)
    g.close()


def test_spin_configuration_checks():
    w, x, p, ay, az, ey, ez, spin = _spin_workload(M=32, npart=100)
    with pytest.raises(pic.PicError) as e:       # spin needs the spin arrays
        pic.Pic(pic.Config.from_workload(w), x, p, ay, az, ey, ez)
    assert e.value.code == pic.PIC_ERR_INVALID
    with pytest.raises(pic.PicError):            # and the FP64 form
        pic.Pic(pic.Config.from_workload(w, precision=pic.PIC_FP32), x, p, ay, az, ey, ez, spin=spin)
    g = pic.Pic(pic.Config.from_workload(w, hbar=0.0), x, p, ay, az, ey, ez)
    with pytest.raises(pic.PicError):            # no subsystem III without spin
        g.substep(pic.PIC_SUBSYSTEM_III)
    g.close()
