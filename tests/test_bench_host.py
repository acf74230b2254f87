"""Host-side logic of bench.py on the CPU: the oracle timing modes (all
cores and one thread) and the algorithmic byte model of the fused RK sweep
that the roofline figure divides by."""
import pytest

import bench
from paper_2006_07964_gb300 import workloads as W


def test_oracle_report_times_all_cores_and_one_thread(monkeypatch):
    monkeypatch.setattr(bench, "ORACLE_REPORT_WORKLOADS", ["vortex32"])
    rep = bench.oracle_report(W, steps=2)
    row = rep["workloads"]["vortex32"]
    assert rep["report"] == "oracle" and rep["steps"] == 2
    assert row["nodes"] == 32 ** 3
    assert row["one_thread"]["threads"] == 1
    assert row["all_cores"]["threads"] >= 1
    for label in ("all_cores", "one_thread"):
        r = row[label]
        assert r["mpts"] > 0 and r["seconds"] > 0
        assert r["mpts"] == pytest.approx(row["nodes"] * 3 * 2 / r["seconds"] / 1e6)


def test_cpu_baseline_adds_the_single_thread_figure():
    out = bench.cpu_baseline(W.vortex(16), seconds_target=0.2)
    assert out["kind"] == "oracle" and out["unit"] == "Mpts/s" and out["value"] > 0
    st = out["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and st["unit"] == "Mpts/s"


def test_rk_sweep_byte_model():
    """Per node, averaged over the three stages as the launch time is.
    FP64: A read instead of read + write (-5 words), Q^n, J, Q^(k+1) (+11).
    Mixed: -5 FP32 words; Q^n, Q^(k+1) and, in two stages of three, Q^(k)
    in FP64; J, the FP32 copy and A_ref in FP32; for Navier-Stokes the FP32
    primitives of the output in two stages of three."""
    assert bench.rk_extra_bytes_per_node("fp64", False) == -5 * 8 + 11 * 8
    assert bench.rk_extra_bytes_per_node("fp64", True) == bench.rk_extra_bytes_per_node("fp64", False)
    euler = -5 * 4 + (5 + 5 * 2 / 3 + 5) * 8 + 4 + 5 * 4 + 5 * 4
    assert bench.rk_extra_bytes_per_node("mixed", False) == pytest.approx(euler)
    assert bench.rk_extra_bytes_per_node("mixed", True) == pytest.approx(euler + 16 * 2 / 3)
