"""Thin ctypes binding of libpic (include/pic.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy
arrays / torch tensors to pointers and status codes to exceptions.  Loading
fails loudly when the built library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "_build", "libpic.so")
HEADER = os.path.join(ROOT, "include", "pic.h")

PIC_OK, PIC_ERR_INVALID, PIC_ERR_NOCONVERGE, PIC_ERR_CUDA, PIC_ERR_NOMEM, PIC_ERR_NUMERIC = range(6)
PIC_FP64, PIC_FP32 = 0, 1
PIC_MEM_HOST, PIC_MEM_DEVICE = 0, 1
PIC_WARM_NONE, PIC_WARM_EXPLICIT, PIC_WARM_MLP = 0, 1, 2
PIC_DEP_CHARGE, PIC_DEP_CURRENT, PIC_DEP_SUSCEPT = 0, 1, 2
PIC_FIELD_EX, PIC_FIELD_EY, PIC_FIELD_EZ, PIC_FIELD_AY, PIC_FIELD_AZ, PIC_FIELD_EX_PATHAVG = range(6)
PIC_ACC_DEFAULT, PIC_ACC_FLOAT, PIC_ACC_COMPENSATED, PIC_ACC_DOUBLE = range(4)
PIC_SPLIT_LIE, PIC_SPLIT_STRANG = 0, 1
PIC_SUBSYSTEM_I, PIC_SUBSYSTEM_II, PIC_SUBSYSTEM_III = 1, 2, 3


class PicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libpic error {code}: {msg}")
        self.code = code


class NoConvergence(PicError):
    pass


class pic_config(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("nx", ctypes.c_int32), ("degree", ctypes.c_int32),
                ("np", ctypes.c_int64), ("weight", ctypes.c_double), ("dt", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("sort_every", ctypes.c_int32), ("deposit", ctypes.c_int32),
                ("splitting", ctypes.c_int32), ("hbar", ctypes.c_double), ("warm_field", ctypes.c_int32)]


_dp = ctypes.POINTER(ctypes.c_double)


class pic_arrays(ctypes.Structure):
    _fields_ = [("x", _dp), ("p", _dp), ("ex", _dp), ("ey", _dp), ("ez", _dp),
                ("ay", _dp), ("az", _dp), ("sx", _dp), ("sy", _dp), ("sz", _dp)]


_lib = None


def declared_symbols() -> list[str]:
    """Entry points declared in include/*.h (pic.h, pic2d.h)."""
    names = set()
    inc = os.path.dirname(HEADER)
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pic(?:2d)?_\w+)\s*\(", txt, re.M))
    return sorted(names)


def load(path: str | None = None):
    """Load libpic; raises if it has not been built (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libpic not built ({path} missing): run paper_2203_06513_gb300/build.py")
    L = ctypes.CDLL(path)
    H = ctypes.POINTER(ctypes.c_void_p)
    L.pic_init.argtypes = [ctypes.POINTER(pic_config), ctypes.POINTER(pic_arrays), ctypes.c_int32,
                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    if hasattr(L, "pic_init_split"):
        L.pic_init_split.argtypes = [ctypes.POINTER(pic_config), ctypes.POINTER(pic_arrays), ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_void_p)]
    L.pic_get_state.argtypes = [ctypes.c_void_p, ctypes.POINTER(pic_arrays), ctypes.c_int32]
    L.pic_deposit.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    L.pic_gather.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    L.pic_substep.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    L.pic_step.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(ctypes.c_int64)]
    L.pic_energy.argtypes = [ctypes.c_void_p, _dp]
    L.pic_timing_enable.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    L.pic_timing_read.argtypes = [ctypes.c_void_p, _dp]
    L.pic_destroy.argtypes = [ctypes.c_void_p]
    L.pic_last_error.argtypes = [ctypes.c_void_p]
    L.pic_last_error.restype = ctypes.c_char_p
    L.pic_version.restype = ctypes.c_char_p
    del H
    _lib = L
    return L


def _ptr(a) -> _dp:
    """Pointer to a float64 numpy array or torch tensor (host or device)."""
    if a is None:
        return _dp()
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data_as(_dp)
    # torch tensor
    assert a.dtype.__repr__() == "torch.float64" and a.is_contiguous()
    return ctypes.cast(ctypes.c_void_p(a.data_ptr()), _dp)


def _vptr(a) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if a is None else (a.data_ptr() if not isinstance(a, np.ndarray)
                                                else a.ctypes.data))


@dataclass
class Config:
    L: float
    nx: int
    degree: int
    np: int
    weight: float
    dt: float
    tol: float = 1e-13
    max_iter: int = 100
    precision: int = PIC_FP64
    warm_start: int = PIC_WARM_NONE
    sort_every: int = 0
    deposit: int = PIC_ACC_DEFAULT
    splitting: int = PIC_SPLIT_LIE
    hbar: float = 0.0
    warm_field: int = 0

    def c(self) -> pic_config:
        return pic_config(self.L, self.nx, self.degree, self.np, self.weight, self.dt, self.tol,
                          self.max_iter, self.precision, self.warm_start, self.sort_every,
                          self.deposit, self.splitting, self.hbar, self.warm_field)

    @staticmethod
    def from_workload(w, precision=PIC_FP64, warm_start=PIC_WARM_NONE, sort_every=0,
                      tol=None, max_iter=None, deposit=PIC_ACC_DEFAULT,
                      splitting=PIC_SPLIT_LIE, hbar=None, warm_field=0) -> "Config":
        return Config(w.L, w.nx, w.degree, w.np, w.weight, w.dt,
                      w.tol if tol is None else tol,
                      w.max_iter if max_iter is None else max_iter,
                      precision, warm_start, sort_every, deposit, splitting,
                      getattr(w, "hbar", 0.0) if hbar is None else hbar, warm_field)


class Pic:
    """One simulation handle.  Arrays are float64 numpy (host) or torch (device)."""

    def __init__(self, cfg: Config, x, p, ay, az, ey=None, ez=None, stream=None, spin=None, reducer=None):
        """spin: (sx, sy, sz) marker spins, required when cfg.hbar != 0.  reducer: an
        object whose `cfunc` is the reduction callback of a split run (see split.py);
        None: all markers are in this handle."""
        L = load()
        self._lib = L
        self.cfg = cfg
        host = isinstance(x, np.ndarray)
        sx, sy, sz = spin if spin is not None else (None, None, None)
        arrs = pic_arrays(_ptr(x), _ptr(p), _dp(), _ptr(ey), _ptr(ez), _ptr(ay), _ptr(az),
                          _ptr(sx), _ptr(sy), _ptr(sz))
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(0 if stream is None else int(stream))
        self._reducer = reducer
        if reducer is None:
            rc = L.pic_init(ctypes.byref(cfg.c()), ctypes.byref(arrs),
                            PIC_MEM_HOST if host else PIC_MEM_DEVICE, s, ctypes.byref(h))
        else:
            fn = ctypes.cast(reducer.cfunc, ctypes.c_void_p)
            rc = L.pic_init_split(ctypes.byref(cfg.c()), ctypes.byref(arrs),
                                  PIC_MEM_HOST if host else PIC_MEM_DEVICE, s, fn, None, ctypes.byref(h))
        if rc != PIC_OK:
            raise PicError(rc, L.pic_last_error(None).decode())
        self._h = h
        self._owned = True

    @classmethod
    def _borrow(cls, lib, handle, cfg: Config) -> "Pic":
        """A view of a handle owned elsewhere (a run of an Ensemble)."""
        obj = cls.__new__(cls)
        obj._lib, obj._h, obj.cfg, obj._owned = lib, handle, cfg, False
        return obj

    # ------------------------------------------------------------------
    def _check(self, rc: int):
        if rc != PIC_OK:
            msg = self._lib.pic_last_error(self._h).decode()
            if rc == PIC_ERR_NOCONVERGE:
                raise NoConvergence(rc, msg)
            raise PicError(rc, msg)

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                self._lib.pic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------
    def substep(self, which: int) -> int:
        it = ctypes.c_int32()
        self._check(self._lib.pic_substep(self._h, which, ctypes.byref(it)))
        return it.value

    def step(self, nsteps: int = 1):
        i1, i2 = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.pic_step(self._h, nsteps, ctypes.byref(i1), ctypes.byref(i2)))
        return i1.value, i2.value

    def energy(self) -> dict:
        out = (ctypes.c_double * 7)()
        self._check(self._lib.pic_energy(self._h, out))
        return {"kinetic": out[0], "ex": out[1], "eperp": out[2], "aperp": out[3],
                "total": out[4], "gauss": out[5], "spin": out[6]}

    def get_state(self, x=None, p=None, ex=None, ey=None, ez=None, ay=None, az=None,
                  sx=None, sy=None, sz=None):
        arrays = [a for a in (x, p, ex, ey, ez, ay, az, sx, sy, sz) if a is not None]
        host = isinstance(arrays[0], np.ndarray) if arrays else True
        arrs = pic_arrays(_ptr(x), _ptr(p), _ptr(ex), _ptr(ey), _ptr(ez), _ptr(ay), _ptr(az),
                          _ptr(sx), _ptr(sy), _ptr(sz))
        self._check(self._lib.pic_get_state(self._h, ctypes.byref(arrs),
                                            PIC_MEM_HOST if host else PIC_MEM_DEVICE))

    def state_numpy(self):
        n, M = self.cfg.np, self.cfg.nx
        out = {k: np.empty(n) for k in ("x", "p")}
        out.update({k: np.empty(M) for k in ("ex", "ey", "ez", "ay", "az")})
        if self.cfg.hbar != 0.0:
            out.update({k: np.empty(n) for k in ("sx", "sy", "sz")})
        self.get_state(**out)
        return out

    def deposit(self, kind: int, aux, out):
        """aux / out: torch float64 CUDA tensors (see pic_deposit)."""
        self._check(self._lib.pic_deposit(self._h, kind, _vptr(aux), _vptr(out)))

    def gather(self, field: int, out):
        """out: torch float64 CUDA tensor (N_p); for PIC_FIELD_EX_PATHAVG it holds the
        displacements on entry (see pic_gather)."""
        self._check(self._lib.pic_gather(self._h, field, _vptr(out)))

    def timing_enable(self, on: bool = True):
        self._check(self._lib.pic_timing_enable(self._h, 1 if on else 0))

    def timing_read(self) -> dict:
        out = (ctypes.c_double * 10)()
        self._check(self._lib.pic_timing_read(self._h, out))
        return {"sweep1_ms": out[0], "sweep1_launches": int(out[1]), "sweep2_ms": out[2],
                "sweep2_launches": int(out[3]), "solve_ms": out[4], "solve_launches": int(out[5]),
                "launches": int(out[6]), "marker_sweeps1": out[7], "warm_ms": out[8],
                "warm_launches": int(out[9])}


def version() -> str:
    return load().pic_version().decode()


class Ensemble:
    """Independent runs advanced together (see pic_ensemble_* in include/pic.h).
    cfgs: list of Config; inputs: list of (x, p, ay, az, ey, ez) float64 numpy
    arrays (ey, ez may be None)."""

    def __init__(self, cfgs, inputs, use_graph: bool = True, stream=None):
        L = load()
        self._lib = L
        vp = ctypes.c_void_p
        L.pic_ensemble_create.argtypes = [ctypes.POINTER(pic_config), ctypes.POINTER(pic_arrays), ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, vp, ctypes.POINTER(vp)]
        L.pic_ensemble_step.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int32)]
        L.pic_ensemble_tune.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32)]
        L.pic_ensemble_set_schedule.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
        L.pic_ensemble_run.argtypes = [vp, ctypes.c_int32]
        L.pic_ensemble_run.restype = vp
        L.pic_ensemble_launches.argtypes = [vp]
        L.pic_ensemble_launches.restype = ctypes.c_int64
        L.pic_ensemble_destroy.argtypes = [vp]
        L.pic_ensemble_last_error.argtypes = [vp]
        L.pic_ensemble_last_error.restype = ctypes.c_char_p
        n = len(cfgs)
        assert len(inputs) == n
        self.cfgs = list(cfgs)
        self.nruns = n
        carr = (pic_config * n)(*[c.c() for c in cfgs])
        self._keep = [tuple(np.ascontiguousarray(a, dtype=np.float64) if a is not None else None for a in inp)
                      for inp in inputs]
        aarr = (pic_arrays * n)(*[pic_arrays(_ptr(x), _ptr(p), _dp(), _ptr(ey), _ptr(ez), _ptr(ay), _ptr(az),
                                             _dp(), _dp(), _dp())
                                  for (x, p, ay, az, ey, ez) in self._keep])
        h = vp()
        s = vp(0 if stream is None else int(stream))
        rc = L.pic_ensemble_create(carr, aarr, n, PIC_MEM_HOST, 1 if use_graph else 0, s, ctypes.byref(h))
        if rc != PIC_OK:
            raise PicError(rc, L.pic_last_error(None).decode())
        self._h = h
        self._keep = None

    def _check(self, rc: int):
        if rc != PIC_OK:
            msg = self._lib.pic_ensemble_last_error(self._h).decode()
            if rc == PIC_ERR_NOCONVERGE:
                raise NoConvergence(rc, msg)
            raise PicError(rc, msg)

    def step(self, nsteps: int = 1, check: bool = True):
        """Returns (sweeps[nruns, 2], status[nruns]); raises on a run's error if check."""
        sw = np.zeros((self.nruns, 2), dtype=np.int64)
        st = np.zeros(self.nruns, dtype=np.int32)
        rc = self._lib.pic_ensemble_step(self._h, nsteps, sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if check:
            self._check(rc)
        return sw, st

    def tune(self, cache_path: str | None = None):
        ch = (ctypes.c_int32 * 3)()
        self._check(self._lib.pic_ensemble_tune(self._h, None if cache_path is None else cache_path.encode(), ch))
        return int(ch[0]), int(ch[1]), bool(ch[2])

    def set_schedule(self, item_markers: int, blocks_per_sm: int):
        self._check(self._lib.pic_ensemble_set_schedule(self._h, item_markers, blocks_per_sm))

    def run(self, r: int) -> Pic:
        h = self._lib.pic_ensemble_run(self._h, r)
        if not h:
            raise IndexError(r)
        return Pic._borrow(self._lib, ctypes.c_void_p(h), self.cfgs[r])

    @property
    def launches(self) -> int:
        return int(self._lib.pic_ensemble_launches(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pic_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


N_MLP_PARAMS = 8898


class Mlp:
    """The warm-start network (see pic_mlp_* in include/pic.h).  X, T, Y are torch
    float32 CUDA tensors of shape (B, 6), (B, 2), (B, 2)."""

    def __init__(self, norm, params=None, stream=None):
        L = load()
        self._lib = L
        fp = ctypes.POINTER(ctypes.c_float)
        L.pic_mlp_create.argtypes = [fp, fp, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
        L.pic_mlp_destroy.argtypes = [ctypes.c_void_p]
        L.pic_mlp_get_params.argtypes = [ctypes.c_void_p, fp]
        L.pic_mlp_grad.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
        L.pic_mlp_train_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
        L.pic_mlp_infer.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L.pic_set_warm_mlp.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        norm = np.ascontiguousarray(norm, dtype=np.float32)
        assert norm.size == 14
        self.norm = norm
        pr = None
        if params is not None:
            pr = np.ascontiguousarray(params, dtype=np.float32)
            assert pr.size == N_MLP_PARAMS
        h = ctypes.c_void_p()
        rc = L.pic_mlp_create(None if pr is None else pr.ctypes.data_as(fp), norm.ctypes.data_as(fp),
                              ctypes.c_void_p(0 if stream is None else int(stream)), ctypes.byref(h))
        if rc != PIC_OK:
            raise PicError(rc, L.pic_last_error(None).decode())
        self._h = h

    def _check(self, rc):
        if rc != PIC_OK:
            raise PicError(rc, self._lib.pic_last_error(None).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pic_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(N_MLP_PARAMS, dtype=np.float32)
        self._check(self._lib.pic_mlp_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def grad(self, X, T, grad_out=None) -> float:
        loss = ctypes.c_double()
        self._check(self._lib.pic_mlp_grad(self._h, _vptr(X), _vptr(T), X.shape[0], _vptr(grad_out),
                                           ctypes.byref(loss)))
        return loss.value

    def train_step(self, X, T, lr: float) -> float:
        loss = ctypes.c_double()
        self._check(self._lib.pic_mlp_train_step(self._h, _vptr(X), _vptr(T), X.shape[0], lr,
                                                 ctypes.byref(loss)))
        return loss.value

    def infer(self, X, Y):
        self._check(self._lib.pic_mlp_infer(self._h, _vptr(X), X.shape[0], _vptr(Y)))

    def attach(self, sim: "Pic"):
        self._check(self._lib.pic_set_warm_mlp(sim._h, self._h))
