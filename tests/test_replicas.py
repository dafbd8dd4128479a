"""The N>1 path on CPU: world-size-2 `gloo` ranks, each advancing its own replica.

Each rank reads its rank from the torchrun-style environment, draws its plasma
from its own seed, advances it with the oracle (no data crosses ranks), then
takes the barrier and the max-over-ranks of its timed duration exactly as the
bench does. The parent checks that every rank agreed on the slowest time, that
the whole-job rate counts both ranks' markers, that the replicas differ, and that
each replica's result equals the same seed run alone (no cross-rank coupling).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2203_06513_gb300 import inputs as I  # noqa: E402
from paper_2203_06513_gb300 import replicas as R  # noqa: E402

NP = 2000
STEPS = 1


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(seed: int):
    """One replica of the small workload (M=128, k=3, NP markers), advanced STEPS steps by the oracle."""
    w = I.workload("C1", np=NP, seed=seed)
    orc = O.Oracle(w.L, w.nx, w.degree, w.weight, w.dt, w.tol)
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    s = O.initial_state(orc, x, p, ay, az, ey, ez)
    H0 = orc.energy(s)["total"]
    s = orc.run(s, STEPS)
    return x, s, H0, orc.energy(s)["total"]


def _rank_main(rank, ws, port, durations, out_dir):
    os.environ.update({"WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    ws_, rank_, _ = R.dist_env()
    dist.init_process_group("gloo", rank=rank_, world_size=ws_)
    try:
        R.barrier(ws_)
        x0, s, H0, H1 = _replica(R.replica_seed(5, rank_))
        R.barrier(ws_)
        slowest = R.max_over_ranks(durations[rank_], ws_)
        rate = R.whole_job_rate(NP, ws_, STEPS, slowest)
        np.savez(os.path.join(out_dir, f"rank{rank_}.npz"), x0=x0, x=s.x, p=s.p, ex=s.ex, ay=s.ay,
                 H=np.array([H0, H1]), slowest=slowest, rate=rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_are_independent_replicas(tmp_path):
    ws = 2
    durations = [0.75, 1.25]            # stand-in timed durations (seconds) per rank
    tmp.start_processes(_rank_main, args=(ws, _free_port(), durations, str(tmp_path)), nprocs=ws,
                        join=True, start_method="spawn")
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(ws)]
    for r in res:
        assert float(r["slowest"]) == max(durations)
        assert float(r["rate"]) == pytest.approx(ws * NP * STEPS / max(durations), rel=1e-15)
    # distinct seeds: distinct plasmas
    assert not np.array_equal(res[0]["x0"], res[1]["x0"])
    # no coupling: each rank's step equals the same seed advanced alone
    for rank, r in enumerate(res):
        x0, s, H0, H1 = _replica(R.replica_seed(5, rank))
        np.testing.assert_array_equal(r["x0"], x0)
        for name in ("x", "p", "ex", "ay"):
            np.testing.assert_array_equal(r[name], getattr(s, name))
        assert abs(H1 - H0) / H0 < 1e-12


def test_rank_environment_and_rate():
    old = {k: os.environ.get(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    try:
        for k in old:
            os.environ.pop(k, None)
        assert R.dist_env() == (1, 0, 0)
        os.environ.update({"WORLD_SIZE": "4", "RANK": "3", "LOCAL_RANK": "3"})
        assert R.dist_env() == (4, 3, 3)
        os.environ["RANK"] = "4"
        with pytest.raises(ValueError):
            R.dist_env()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    assert R.replica_seed(0, 0) == 0 and R.replica_seed(0, 1) == 1
    assert R.max_over_ranks(2.5, 1) == 2.5
    assert R.whole_job_rate(1e8, 8, 20, 2.0) == 8e9
    with pytest.raises(ValueError):
        R.whole_job_rate(1e8, 1, 1, 0.0)
