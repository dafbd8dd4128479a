"""Split runs through the C ABI (pic_init_split) on one GPU: two handles of one
process, each holding half the markers of one plasma, stepped from two host
threads; the reduction callback adds (or maxes) their buffers on the host, the
stand-in here for the all-reduce between processes.  Only host threads wait for
each other; every kernel runs on its own handle's stream without waiting on the
other's.  Together the halves must reproduce the handle that holds all markers,
up to the order of the additions."""
import threading

import numpy as np
import pytest

from paper_2203_06513_gb300 import inputs as I
from paper_2203_06513_gb300 import pic
from paper_2203_06513_gb300 import split

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


class PairReducer:
    """The reduction of a split run over two handles of this process."""

    def __init__(self):
        self.barrier = threading.Barrier(2, timeout=120)
        self.slots = [None, None]
        self.calls = [0, 0]

    def member(self, rank):
        outer = self

        class _M:
            def _call(self, ctx, op, ptr, n, stream):
                try:
                    s = torch.cuda.ExternalStream(int(stream)) if stream else torch.cuda.default_stream()
                    t = torch.as_tensor(split._DeviceArray(ptr, n), device="cuda")
                    s.synchronize()
                    outer.slots[rank] = t.cpu().numpy().copy()
                    outer.calls[rank] += 1
                    outer.barrier.wait()
                    a, b = outer.slots
                    r = a + b if op == split.PIC_REDUCE_SUM else np.maximum(a, b)
                    outer.barrier.wait()
                    with torch.cuda.stream(s):
                        t.copy_(torch.from_numpy(r).cuda(non_blocking=False))
                    s.synchronize()
                    return 0
                except Exception:
                    self.error = True
                    try:
                        outer.barrier.abort()
                    except Exception:
                        pass
                    return 1

        m = _M()
        m.error = False
        m.cfunc = split.REDUCE_FN(m._call)
        return m


def _halves(w, precision, steps, spin=None, **kw):
    x, p = I.particles(w)
    ay, az, ey, ez = I.fields(w)
    red = PairReducer()
    members = [red.member(r) for r in range(2)]
    results, errors = [None, None], []

    def run(r):
        try:
            lo, hi = split.shard(w.np, r, 2)
            cfg = pic.Config.from_workload(w, precision=precision, **kw)
            cfg.np = hi - lo
            sp = None if spin is None else tuple(c[lo:hi].copy() for c in spin)
            stream = torch.cuda.Stream()
            g = pic.Pic(cfg, x[lo:hi].copy(), p[lo:hi].copy(), ay, az, ey, ez, stream=stream.cuda_stream,
                        spin=sp, reducer=members[r])
            it = g.step(steps)
            E = g.energy()
            results[r] = (g.state_numpy(), it, E)
            g.close()
        except Exception as e:
            errors.append(e)
            try:
                red.barrier.abort()
            except Exception:
                pass

    th = [threading.Thread(target=run, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errors, errors
    assert red.calls[0] == red.calls[1] > 0
    whole = pic.Pic(pic.Config.from_workload(w, precision=precision, **kw), x, p, ay, az, ey, ez,
                    spin=spin)
    it = whole.step(steps)
    ref = (whole.state_numpy(), it, whole.energy())
    whole.close()
    return results, ref


@pytest.mark.parametrize("precision", [pic.PIC_FP64, pic.PIC_FP32])
def test_two_halves_reproduce_the_whole(precision):
    w = I.Workload("sp", nx=64, degree=3, np=20011, seed=17, vth=0.15, pump=0.3)
    res, (st, it, E) = _halves(w, precision, 4, sort_every=2)
    x = np.concatenate([r[0]["x"] for r in res])
    p = np.concatenate([r[0]["p"] for r in res])
    d = np.abs(np.mod(x - st["x"] + 0.5 * w.L, w.L) - 0.5 * w.L)
    tol = 1e-12 if precision == pic.PIC_FP64 else 1e-6
    assert np.max(d) / w.L < tol
    assert np.max(np.abs(p - st["p"])) < tol * np.max(np.abs(st["p"]))
    for r in res:
        assert r[1] == it                      # the same sweep counts
        for key in ("ex", "ey", "ez", "ay", "az"):
            ref = st[key]
            if np.max(np.abs(ref)) > 0:
                assert np.max(np.abs(r[0][key] - ref)) < tol * np.max(np.abs(ref)), key
        assert abs(r[2]["total"] - E["total"]) < (1e-13 if precision == pic.PIC_FP64 else 1e-9) * E["total"]
        assert abs(r[2]["gauss"] - E["gauss"]) < 1e-12 or precision == pic.PIC_FP32


def test_two_halves_with_spin():
    w = I.workload("P2", nx=64, np=6001, seed=5)
    s = np.random.default_rng(2).normal(size=(3, w.np))
    s /= np.linalg.norm(s, axis=0)
    spin = (s[0].copy(), s[1].copy(), s[2].copy())
    res, (st, it, E) = _halves(w, pic.PIC_FP64, 5, spin=spin)
    sz = np.concatenate([r[0]["sz"] for r in res])
    assert np.max(np.abs(sz - st["sz"])) < 1e-12
    for r in res:
        assert r[1] == it
        assert abs(r[2]["total"] - E["total"]) < 1e-13 * abs(E["total"])
        assert abs(r[2]["spin"] - E["spin"]) < 1e-13 * abs(E["total"])
