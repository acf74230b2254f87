"""Host-side logic of bench.py on the CPU: the oracle timing modes (all
cores and one thread), the algorithmic byte model of an RK stage that the
roofline figure divides by, and the traffic table's source check."""
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


def test_cpu_baseline_times_two_whole_steps_on_all_cores_and_one_thread():
    out = bench.cpu_baseline(W.vortex(16), steps=2, single_thread_w=W.vortex(12))
    assert out["kind"] == "oracle" and out["unit"] == "Mpts/s" and out["value"] > 0
    assert out["sample"].startswith("2 full RK3 steps of the 4096-node workload")
    st = out["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and st["unit"] == "Mpts/s"
    assert st["sample"].startswith("2 full RK3 steps of vortex12 (1728 nodes)")


def test_stage_byte_model_is_the_compulsory_traffic():
    """Per node and RK stage, the compulsory HBM traffic of Eq. (20) with
    FP64 metrics: stage 1 reads the 9 metrics and J and Q^n and writes
    Q^(1) (20 words = 160 B); stages 2 and 3 also read their input Q^(k)
    (25 words = 200 B); the mixed form adds an FP32 copy of the state read
    and written (10 x 4 B), 240 B in stages 2 and 3."""
    assert bench.stage_bytes_per_node("fp64") == pytest.approx((160 + 200 + 200) / 3)
    assert bench.stage_bytes_per_node("mixed") == pytest.approx((200 + 240 + 240) / 3)


def test_traffic_is_null_unless_the_sources_match(monkeypatch):
    """The roofline's DRAM traffic comes from an ncu capture keyed by the
    kernel sources' hash; another hash reports null."""
    sha = bench.kernel_sources_sha()
    assert len(sha) == 16 and sha == bench.kernel_sources_sha()
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES_SHA", "0" * 16)
    monkeypatch.setattr(bench, "TRAFFIC_PER_NODE", {("fp64", "flux_xi"): 100.0})

    class Ctx:
        def profile_step(self, steps, dt):
            return {"flux_xi": (6, 6.0), "prep": (6, 1.0)}

        def tuning(self):
            return {}

    class Wl:
        npts = 1000
        viscous = True

    peaks = {"hbm_gbs": 6800.0, "src": "fallback", "fp64_tflops": 1.0, "fp32_tflops": 64.0, "alu_src": "x"}
    out = bench.roofline_for(Ctx(), Wl(), "fp64", 2, 1e-3, peaks, 9.0)
    assert out["traffic"] is None and out["bound"] == "alu"
    monkeypatch.setattr(bench, "TRAFFIC_SOURCES_SHA", sha)
    out = bench.roofline_for(Ctx(), Wl(), "fp64", 2, 1e-3, peaks, 9.0)
    assert out["traffic"] == pytest.approx(100.0 * 1000)
    assert out["traffic_view"]["achieved"] == pytest.approx(100.0 * 1000 / 1e-3 / 1e9)
    # achieved flops per launch over the launch time (1 ms)
    flops = (bench.FLUX_FLOPS_INV + bench.FLUX_FLOPS_VISC - bench.FLUX_FLOPS_STATIC_FP64) * 1000
    assert out["achieved"] == pytest.approx(flops / 1e-3 / 1e12)
    assert out["frac"] == pytest.approx(out["achieved"] / 1.0)
    # the stage's algorithmic bytes over this launch, and over the stage
    assert out["hbm_view"]["achieved"] == pytest.approx(bench.stage_bytes_per_node("fp64") * 1000 / 1e-3 / 1e9)
    assert out["stage_view"]["stage_ms"] == pytest.approx(3.0)
    assert out["stage_view"]["hbm_achieved"] == pytest.approx(bench.stage_bytes_per_node("fp64") * 1000 / 3e-3 / 1e9)
