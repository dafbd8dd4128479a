"""One plasma split by markers over two processes (gloo, CPU): the host logic of
split runs (paper_2203_06513_gb300/split.py) driving the oracle's step, whose
marker sums and maxima go through the processes' all-reduce.  The two halves
together must reproduce the single-process step: the same fields, the same
markers, the same sweep counts and the same energy, up to the order of the
additions."""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_06513_gb300 import inputs as I
from paper_2203_06513_gb300 import split

torch = pytest.importorskip("torch")

W = I.Workload("split", nx=32, degree=3, np=3001, dt=0.05, vth=0.15, pump=0.3, seed=13)
STEPS = 3


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir, hbar):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, p = I.particles(W)
        ay, az, ey, ez = I.fields(W)
        lo, hi = split.shard(W.np, rank, world)
        sp = None
        if hbar:
            rng = np.random.default_rng(3)
            s = rng.normal(size=(3, W.np))
            s /= np.linalg.norm(s, axis=0)
            sp = (s[0][lo:hi], s[1][lo:hi], s[2][lo:hi])
        orc = O.Oracle(W.L, W.nx, W.degree, W.weight, W.dt, W.tol, W.max_iter, comm=split.TorchComm(), hbar=hbar)
        st = O.initial_state(orc, x[lo:hi], p[lo:hi], ay, az, ey, ez, spin=sp)
        H0 = orc.energy(st)["total"]
        iters = []
        for _ in range(STEPS):
            st = orc.step(st)
            iters.append(orc.last_iters)
        H = orc.energy(st)["total"]
        gauss = float(np.max(np.abs(orc.gauss_residual(st.x, st.ex))))
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), x=st.x, p=st.p, ex=st.ex, ey=st.ey, ez=st.ez,
                 ay=st.ay, az=st.az, iters=np.array(iters), H0=H0, H=H, gauss=gauss,
                 sz=st.sz if st.sz is not None else np.zeros(0))
    finally:
        dist.destroy_process_group()


def _serial(hbar):
    x, p = I.particles(W)
    ay, az, ey, ez = I.fields(W)
    sp = None
    if hbar:
        rng = np.random.default_rng(3)
        s = rng.normal(size=(3, W.np))
        s /= np.linalg.norm(s, axis=0)
        sp = (s[0], s[1], s[2])
    orc = O.Oracle(W.L, W.nx, W.degree, W.weight, W.dt, W.tol, W.max_iter, hbar=hbar)
    st = O.initial_state(orc, x, p, ay, az, ey, ez, spin=sp)
    H0 = orc.energy(st)["total"]
    iters = []
    for _ in range(STEPS):
        st = orc.step(st)
        iters.append(orc.last_iters)
    return st, np.array(iters), H0, orc.energy(st)["total"]


def test_shard_covers_all_markers_once():
    for n in (1, 7, 3001, 10 ** 6):
        for world in (1, 2, 3, 8):
            ranges = [split.shard(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    with pytest.raises(ValueError):
        split.shard(10, 2, 2)


@pytest.mark.parametrize("hbar", [0.0, 0.1])
def test_two_processes_reproduce_one(tmp_path, hbar):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), hbar), nprocs=world, join=True)
    ref, iters, H0, H = _serial(hbar)
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    x = np.concatenate([q["x"] for q in parts])
    p = np.concatenate([q["p"] for q in parts])
    d = np.abs(np.mod(x - ref.x + 0.5 * W.L, W.L) - 0.5 * W.L)
    assert np.max(d) < 1e-13 * W.L
    assert np.max(np.abs(p - ref.p)) < 1e-13 * np.max(np.abs(ref.p))
    for q in parts:
        for key in ("ex", "ey", "ez", "ay", "az"):
            r = getattr(ref, key)
            assert np.max(np.abs(q[key] - r)) <= 1e-12 * max(np.max(np.abs(r)), 1e-300), key
        np.testing.assert_array_equal(q["iters"], iters)
        assert abs(float(q["H"]) - H) < 1e-13 * abs(H)
        assert abs(float(q["H0"]) - H0) < 1e-13 * abs(H0)
        assert float(q["gauss"]) < 1e-13
    if hbar:
        sz = np.concatenate([q["sz"] for q in parts])
        assert np.max(np.abs(sz - ref.sz)) < 1e-13
