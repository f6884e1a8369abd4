"""The bench line's roofline arithmetic (host logic of bench.py) on a fake profile whose
answers are worked by hand: the bound is the larger of bytes / bandwidth and algorithmic
flops / peak, the fraction divides achieved by peak, traffic scales bytes per launch."""
import importlib.util
import os

import pytest


def _bench(monkeypatch):
    spec = importlib.util.spec_from_file_location("bench", os.path.join(os.path.dirname(__file__), "..", "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops_sustained": 1700.0}
    monkeypatch.setattr(mod, "_measured", lambda key, default: peaks.get(key, default))
    return mod


class FakeZ:
    PREC_FP64, PREC_MIXED = 0, 1


def _gp(tc_bytes):
    return {"gemm_ms": 2000.0, "tc_ms": 1000.0, "gemm_flops": 2.0e14, "tc_flops": 1.2e14, "tc_bytes": tc_bytes,
            "gemm_bytes": 3.0e12, "tc_launches": 100, "launches": 1000, "gemm_launches": 200}


def test_tensor_bound_launches(monkeypatch):
    """Algorithmic / executed flops = 1.6e14 / 2e14 = 0.8, so the tensor-core jobs did
    1.2e14 x 0.8 = 9.6e13 algorithmic flops in 1 s; the 3xTF32 peak is 1700 x 1.1/2.25 / 3
    = 277.04 TF/s, so flops take 0.3465 s at peak and 2e12 bytes take 0.294 s at 6.8 TB/s:
    tensor-bound, 96 TF/s, frac 0.3465; HBM view 2000 GB/s = 0.294."""
    B = _bench(monkeypatch)
    r = B.roofline(FakeZ, FakeZ.PREC_MIXED, _gp(2.0e12), {}, 1.6e14, 10000.0)
    peak = 1700.0 * 1.1 / 2.25 / 3.0
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(96.0) and r["peak"] == pytest.approx(peak)
    assert r["frac"] == pytest.approx(96.0 / peak)
    assert r["hbm_view"]["frac"] == pytest.approx(2000.0 / 6800.0)
    assert r["traffic"] == pytest.approx(2.0e12 / 100 * B.TC_DRAM_OVER_ALG)
    assert r["algorithmic_over_executed"] == pytest.approx(0.8)
    assert r["breakdown_ms"]["gemm_fma"] == pytest.approx(1000.0) and r["breakdown_ms"]["other"] == pytest.approx(8000.0)


def test_hbm_bound_launches(monkeypatch):
    """Twice the bytes (4e12 in 1 s): 0.588 s at 6.8 TB/s > 0.3465 s of flops -> HBM-bound,
    4000 GB/s, frac 4000 / 6800."""
    B = _bench(monkeypatch)
    r = B.roofline(FakeZ, FakeZ.PREC_MIXED, _gp(4.0e12), {}, 1.6e14, 10000.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(4000.0) and r["frac"] == pytest.approx(4000.0 / 6800.0)
    assert r["t_roof_over_t"] == pytest.approx(4.0e12 / 6.8e12)


def test_fp64_launches_are_alu_bound(monkeypatch):
    """complex128: the FMA GEMMs' algorithmic flops (2e14 - 1.2e14) x 0.8 = 6.4e13 over their
    1 s, against the FP64 peak (1.10 TF/s when no measured figure exists)."""
    B = _bench(monkeypatch)
    r = B.roofline(FakeZ, FakeZ.PREC_FP64, _gp(2.0e12), {}, 1.6e14, 10000.0)
    assert r["bound"] == "alu" and r["traffic"] is None
    assert r["achieved"] == pytest.approx(64.0) and r["peak"] == pytest.approx(1.10)
