"""Thin ctypes binding of the two-dimensional subsystem I (include/pic2d.h):
argument marshalling only; every step runs in libpic's kernels."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import pic as P

_dp = ctypes.POINTER(ctypes.c_double)


class pic2d_config(ctypes.Structure):
    _fields_ = [("L1", ctypes.c_double), ("L2", ctypes.c_double), ("M1", ctypes.c_int32), ("M2", ctypes.c_int32),
                ("degree", ctypes.c_int32), ("np", ctypes.c_int64), ("weight", ctypes.c_double),
                ("dt", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("hbar", ctypes.c_double), ("warm", ctypes.c_int32)]


_ready = False


def _lib():
    global _ready
    L = P.load()
    if not _ready:
        L.pic2d_init.argtypes = [ctypes.POINTER(pic2d_config), _dp, _dp, _dp, _dp, _dp, ctypes.c_int32,
                                 ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
        L.pic2d_set_spin.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_int32]
        L.pic2d_substep1.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
        L.pic2d_energy.argtypes = [ctypes.c_void_p, _dp]
        L.pic2d_get_state.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp, ctypes.c_int32]
        L.pic2d_destroy.argtypes = [ctypes.c_void_p]
        L.pic2d_last_error.argtypes = [ctypes.c_void_p]
        L.pic2d_last_error.restype = ctypes.c_char_p
        _ready = True
    return L


@dataclass
class Config2D:
    L1: float
    L2: float
    M1: int
    M2: int
    degree: int
    np: int
    weight: float
    dt: float
    tol: float = 1e-13
    max_iter: int = 100
    hbar: float = 0.0
    warm: int = 0

    def c(self) -> pic2d_config:
        return pic2d_config(self.L1, self.L2, self.M1, self.M2, self.degree, self.np, self.weight, self.dt,
                            self.tol, self.max_iter, self.hbar, self.warm)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Pic2D:
    """Subsystem I of the 2D scheme on one GPU (host arrays in and out)."""

    def __init__(self, cfg: Config2D, x, p, ex, ey, az, stream=None):
        self.L = _lib()
        self.cfg = cfg
        x, p, ex, ey, az = (_f64(v) for v in (x, p, ex, ey, az))
        assert x.shape == (cfg.np, 2) and p.shape == (cfg.np, 2)
        n = cfg.M1 * cfg.M2
        assert ex.shape == (n,) and ey.shape == (n,) and az.shape == (n,)
        c = cfg.c()
        h = ctypes.c_void_p()
        rc = self.L.pic2d_init(ctypes.byref(c), x.ctypes.data_as(_dp), p.ctypes.data_as(_dp),
                               ex.ctypes.data_as(_dp), ey.ctypes.data_as(_dp), az.ctypes.data_as(_dp),
                               P.PIC_MEM_HOST, ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if rc:
            raise P.PicError(rc, self.L.pic2d_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc:
            msg = self.L.pic2d_last_error(self.h).decode()
            raise (P.NoConvergence if rc == P.PIC_ERR_NOCONVERGE else P.PicError)(rc, msg)

    def set_spin(self, s, bz):
        """Spins (np x 3) and b_z (M1 * M2) for the Zeeman terms (hbar != 0)."""
        c = self.cfg
        s, bz = _f64(s), _f64(bz)
        assert s.shape == (c.np, 3) and bz.shape == (c.M1 * c.M2,)
        self._check(self.L.pic2d_set_spin(self.h, s.ctypes.data_as(_dp), bz.ctypes.data_as(_dp), P.PIC_MEM_HOST))

    def substep1(self) -> int:
        it = ctypes.c_int32()
        self._check(self.L.pic2d_substep1(self.h, ctypes.byref(it)))
        return it.value

    def energy(self) -> dict:
        out = np.zeros(4)
        self._check(self.L.pic2d_energy(self.h, out.ctypes.data_as(_dp)))
        return {"kinetic": out[0], "field": out[1], "zeeman": out[2], "total": out[3]}

    def state(self) -> dict:
        c = self.cfg
        x, p = np.zeros((c.np, 2)), np.zeros((c.np, 2))
        n = c.M1 * c.M2
        ex, ey = np.zeros(n), np.zeros(n)
        self._check(self.L.pic2d_get_state(self.h, x.ctypes.data_as(_dp), p.ctypes.data_as(_dp),
                                           ex.ctypes.data_as(_dp), ey.ctypes.data_as(_dp), P.PIC_MEM_HOST))
        return {"x": x, "p": p, "ex": ex, "ey": ey}

    def close(self):
        if self.h:
            self.L.pic2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
