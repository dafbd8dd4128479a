"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/pic.h declares (no compute call: this runs without a GPU)."""
import ctypes

import pytest

from paper_2203_06513_gb300 import build as B
from paper_2203_06513_gb300 import pic


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_boundary():
    names = pic.declared_symbols()
    for required in ["pic_init", "pic_deposit", "pic_gather", "pic_substep", "pic_step",
                     "pic_energy", "pic_destroy", "pic_get_state", "pic_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in pic.declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_null_handle_errors(libpath):
    L = pic.load(libpath)
    assert b"sm_103a" in L.pic_version()
    assert L.pic_destroy(None) == 0
    assert L.pic_substep(None, 1, None) == pic.PIC_ERR_INVALID
    assert L.pic_energy(None, None) == pic.PIC_ERR_INVALID


def test_invalid_config_rejected_before_device_work(libpath):
    L = pic.load(libpath)
    cfg = pic.Config(L=1.0, nx=4, degree=3, np=10, weight=0.1, dt=0.1).c()   # nx < 8
    h = ctypes.c_void_p()
    arrs = pic.pic_arrays()
    rc = L.pic_init(ctypes.byref(cfg), ctypes.byref(arrs), 0, None, ctypes.byref(h))
    assert rc == pic.PIC_ERR_INVALID
    assert L.pic_last_error(None)
