"""Host-side arithmetic of bench.py (no GPU): the algorithmic flop counts, the
roofline of the tensor-core forms as the slowest of three floors, and the
rule that a stored DRAM-traffic figure is used only for the source it was
measured on."""

import importlib.util
import json
import math
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _FakeLib:
    """compressed_bytes of the FP32 layout for every form (only the HBM floor uses it)."""

    @staticmethod
    def compressed_bytes(N, T, H, Q, fp):
        return N * T * H * (Q // 2) * 8


def test_flops_per_pair_counts_contraction_fft_and_reduction(bench):
    H, Q = 12, 256
    # 8 flops per complex multiply-add over Q/2+1 frequencies, 2.5 Q log2 Q for the C2R FFT, 2 per score
    assert bench._alg_flops_per_pair(H, Q) == 8 * 12 * 129 + 2.5 * 256 * 8 + 2 * 256
    assert bench._alg_flops_per_pair(16, 512) == 8 * 16 * 257 + 2.5 * 512 * 9 + 2 * 512


def test_form_roofline_takes_the_slowest_floor(bench, monkeypatch):
    monkeypatch.setattr(bench, "_peaks", lambda: {"bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0})
    N_A, N_B, T, H, Q, sms = 8192, 1024, 9, 12, 256, 152
    r = bench._form_roofline(_FakeLib, "bf16", N_A, N_B, T, H, Q, 28.0, sms)
    pairs = N_A * T * N_B
    alu_peak = sms * 128 * 2 * 2.07e9
    alu_ms = pairs * (2.5 * Q * math.log2(Q) + 2 * Q) / alu_peak * 1e3
    tensor_ms = pairs * 8 * H * (Q // 2 + 1) / 1700e12 * 1e3
    assert r["bound"] == "alu" and alu_ms > tensor_ms > r["floors_ms"]["hbm"]
    assert r["floors_ms"]["alu"] == pytest.approx(alu_ms, rel=1e-3)
    assert r["floors_ms"]["tensor"] == pytest.approx(tensor_ms, rel=1e-3)
    assert r["frac"] == pytest.approx(alu_ms / 28.0, rel=1e-3)
    # three operand terms triple the tensor floor and the tensor pipe's own work
    r3 = bench._form_roofline(_FakeLib, "bf16x3", N_A, N_B, T, H, Q, 28.0, sms)
    assert r3["floors_ms"]["tensor"] == pytest.approx(3 * r["floors_ms"]["tensor"], rel=1e-3)
    assert r3["tensor"]["mma_per_launch"] == 3 * r["tensor"]["mma_per_launch"]
    # a slow enough tensor peak makes the contraction the bound
    monkeypatch.setattr(bench, "_peaks", lambda: {"bf16_tflops_sustained": 50.0, "hbm_gbs": 6800.0})
    r4 = bench._form_roofline(_FakeLib, "bf16", N_A, N_B, T, H, Q, 28.0, sms)
    assert r4["bound"] == "tensor" and r4["unit"] == "TFLOP/s"


def test_stored_traffic_only_for_the_measured_source(bench, tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel source A")
    import hashlib

    entry = {"bytes_per_launch": 123, "sources": [str(src)], "sha256": hashlib.sha256(b"kernel source A").hexdigest()}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k@w": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._load_traffic("k@w") == 123
    assert bench._load_traffic("other@w") is None
    src.write_text("kernel source B")  # the kernel changed since the counters were taken
    assert bench._load_traffic("k@w") is None

