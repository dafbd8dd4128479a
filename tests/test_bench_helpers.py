"""Host arithmetic of bench.py (CPU): the roofline and issue-slot entries of the
JSON line, from a stand-in timing record, and the peak fallback."""
import importlib
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    return importlib.import_module("bench")


def timing(sweep1_ms=20.0, n1=10, sweep2_ms=10.0, n2=10, warm_ms=50.0, nw=10):
    return {"sweep1_ms": sweep1_ms, "sweep1_launches": n1, "sweep2_ms": sweep2_ms, "sweep2_launches": n2,
            "warm_ms": warm_ms, "warm_launches": nw}


def test_roofline_entries(bench):
    np_ = 100_000_000
    ks = bench.kernel_rooflines(timing(), np_, 6000.0, 1700.0, "measured", sms=152, sm_mhz=2070.0)
    by = {k["kernel"]: k for k in ks}
    s1 = by["k_sweep1<3,float>"]
    # 28 bytes a marker (x^n 8, p^n 4, x^(k) 8 read; x^(k+1) 8 written) in 2 ms a launch
    assert s1["launch_ms"] == pytest.approx(2.0)
    assert s1["achieved"] == pytest.approx(28 * np_ / 2e-3 / 1e9)
    assert s1["frac"] == pytest.approx(s1["achieved"] / 6000.0)
    assert s1["algorithmic_per_launch"] == 28 * np_
    assert s1["traffic"] == pytest.approx(bench.NCU_DRAM_PER_MARKER["k_sweep1<3,float>"] * np_)
    # issue slots: instructions / 32 per marker against SMs x 4 x clock
    inst = bench.NCU_INST_PER_MARKER["k_sweep1<3,float>"]
    assert s1["issue"]["peak"] == pytest.approx(152 * 4 * 2.07)
    assert s1["issue"]["achieved"] == pytest.approx(inst / 32 * np_ / 2e-3 / 1e9)
    mlp = by["k_warm_mlp<3,float>"]
    assert mlp["bound"] == "tensor" and mlp["unit"] == "TFLOP/s"
    assert mlp["achieved"] == pytest.approx(bench.FLOP_MLP * np_ / 5e-3 / 1e12)
    assert bench.FLOP_MLP == 2 * (6 * 64 + 64 * 64 + 64 * 64 + 64 * 2)
    json.dumps(ks)                       # the entries go into the JSON line as they are


def test_kernels_without_launches_or_clock(bench):
    ks = bench.kernel_rooflines(timing(warm_ms=0.0, nw=0), 1000, 6000.0, 1700.0, "fallback")
    names = [k["kernel"] for k in ks]
    assert "k_warm_mlp<3,float>" not in names
    assert all("issue" not in k for k in ks)     # no SM count / clock: no issue entry


def test_peaks_read_the_measured_file_or_fall_back(bench, tmp_path, monkeypatch):
    hbm, tf, kind = bench.peaks()
    assert hbm > 0 and tf > 0 and kind in ("measured", "fallback")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, 1700.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5, "bf16_tflops": 1900.0,
                                                              "bf16_tflops_sustained": 1720.0}))
    assert bench.peaks() == (7000.5, 1720.0, "measured")
