"""Oracle particle loops over very large marker sets, split into chunks and run
in a pool of spawned processes (test infrastructure: full-size checks).

Each function takes one chunk of markers and returns the chunk's part of a sum
(kinetic energy, charge, susceptibility deposit); the caller adds the parts.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import multiprocessing as mp
import os

import numpy as np


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _kinetic(job):
    from oracle import oracle as O
    k, M, dx, w, x, p, ay, az = job
    return O.lib().orc_kinetic(k, M, dx, x.shape[0], _p(x), _p(p), w, _p(ay), _p(az))


def _charge(job):
    from oracle import oracle as O
    k, M, dx, w, x = job
    rho = np.zeros(M)
    O.lib().orc_charge(k, M, dx, x.shape[0], _p(x), w, _p(rho))
    return rho


def _sweep2(job):
    from oracle import oracle as O
    k, M, dx, w, x, p, ayn, azn, ayk, azk = job
    sy, sz = np.zeros(M), np.zeros(M)
    O.lib().orc_sweep2(k, M, dx, w, x.shape[0], _p(x), _p(p), _p(ayn), _p(azn), _p(ayk), _p(azk),
                       _p(sy), _p(sz))
    return np.stack([sy, sz])


class Pool:
    """A pool of spawned worker processes (safe to start after CUDA is in use)."""

    def __init__(self, workers: int | None = None):
        n = workers or max(1, min(16, os.cpu_count() or 1))
        self.ex = cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))
        self.n = n

    def close(self):
        self.ex.shutdown()

    def _chunks(self, n):
        size = max(1, -(-n // (4 * self.n)))
        return [(s, min(n, s + size)) for s in range(0, n, size)]

    def kinetic(self, k, M, dx, w, x, p, ay, az) -> float:
        jobs = [(k, M, dx, w, x[a:b], p[a:b], ay, az) for a, b in self._chunks(x.shape[0])]
        return float(sum(self.ex.map(_kinetic, jobs)))

    def charge(self, k, M, dx, w, x) -> np.ndarray:
        jobs = [(k, M, dx, w, x[a:b]) for a, b in self._chunks(x.shape[0])]
        return np.sum(list(self.ex.map(_charge, jobs)), axis=0)

    def sweep2(self, k, M, dx, w, x, p, ayn, azn, ayk, azk) -> np.ndarray:
        jobs = [(k, M, dx, w, x[a:b], p[a:b], ayn, azn, ayk, azk) for a, b in self._chunks(x.shape[0])]
        return np.sum(list(self.ex.map(_sweep2, jobs)), axis=0)
