"""Host logic of bench.py (no GPU): the roofline object of the dominant kernel, every kernel's
fraction of its own bound, the measured-traffic lookup, and the profiling case that cuts the
workload's blocks while keeping their number."""
import numpy as np
import pytest

import bench

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1600.0, "sm_max_mhz": 2000.0}


def _prof():
    # ms totals over 10 launches; work totals over the same launches
    return {
        "bwd_dx_bf16": {"launches": 10, "ms": 0.5, "flops": 10 * 1.6e9, "bytes": 0.0},
        "update_adam": {"launches": 10, "ms": 0.4, "flops": 0.0, "bytes": 10 * 3.0e8},
        "fwd_hidden_static_fp8": {"launches": 10, "ms": 0.2, "flops": 10 * 2.0e9, "bytes": 0.0},
        "fwd_hidden_dm": {"launches": 10, "ms": 0.1, "flops": 10 * 1.0e9, "bytes": 0.0},
        "count_step": {"launches": 10, "ms": 0.1, "flops": 0.0, "bytes": 0.0},
    }


def test_dominant_kernel_and_its_bound():
    r, per = bench.roofline(_prof(), PEAKS, "measured")
    assert r["kernel"] == "bwd_dx_bf16" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    # 1.6 GFLOP per launch in 0.05 ms = 32 TFLOP/s against the sustained BF16 peak
    assert r["achieved"] == pytest.approx(32.0)
    assert r["frac"] == pytest.approx(32.0 / 1600.0)
    assert r["work_per_launch"] == pytest.approx(1.6e9)
    assert r["traffic"] is None  # no capture of this kernel
    assert sum(v["share"] for v in per.values()) == pytest.approx(1.0)


def test_fused_update_is_hbm_bound_and_its_traffic_scales_with_its_bytes(monkeypatch):
    """The dW2 GEMM with the optimiser in its epilogue: HBM-bound (its 26 bytes per parameter take
    longer than its FLOPs); without a capture of the kernel as it stands its traffic is null, and with
    one it is the captured DRAM bytes per algorithmic byte times the launch's algorithmic bytes (here
    the figures of its last capture)."""
    alg = 1024 * 256 * 4096 * 26.0
    prof = {"bwd_dw2_adam_bf16": {"launches": 2, "ms": 2 * 5.0, "flops": 2 * 2.0 * 131072 * 256 * 4096,
                                  "bytes": 2 * alg}}
    r, _ = bench.roofline(prof, PEAKS, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(alg / 5e-3 / 1e9)
    assert r["traffic"] is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, "bwd_dw2_adam_bf16", (876706304 + 877779968, 64 * 256 * 4096 * 26))
    r, _ = bench.roofline(prof, PEAKS, "measured")
    dram, alg64 = bench.NCU_TRAFFIC["bwd_dw2_adam_bf16"]
    assert r["traffic"] == pytest.approx(dram / alg64 * alg)
    assert 0.99 < dram / alg64 < 1.1  # the capture moved its algorithmic bytes, no re-reads


def test_every_kernel_against_its_own_bound():
    _, per = bench.roofline(_prof(), PEAKS, "measured")
    # HBM-bound optimiser: 300 MB per launch in 0.04 ms = 7500 GB/s against 6000
    assert per["update_adam"]["bound"] == "hbm"
    assert per["update_adam"]["frac"] == pytest.approx(7500.0 / 6000.0)
    # E4M3 kernels against twice the BF16 figure
    assert per["fwd_hidden_static_fp8"]["bound"] == "tensor"
    assert per["fwd_hidden_static_fp8"]["frac"] == pytest.approx(100.0 / 3200.0)
    # FP32 form: ALU peak = 152 SMs x 128 lanes x 2 x 2.0 GHz
    alu = 152 * 128 * 2 * 2000e6 / 1e12
    assert per["fwd_hidden_dm"]["bound"] == "alu"
    assert per["fwd_hidden_dm"]["frac"] == pytest.approx(100.0 / alu)
    assert per["count_step"]["frac"] == 0.0


def test_no_profile_gives_no_roofline():
    assert bench.roofline({}, PEAKS, "measured") == (None, {})


def test_profiling_case_keeps_blocks_and_cuts_them():
    w, kw = bench.load_workload("plain", 1 << 12)
    assert len(w.block_lens) == 64 and np.all(w.block_lens == (1 << 12))
    assert w.seq.size == 64 << 12
    full, _ = bench.load_workload("plain")
    assert np.array_equal(w.seq, full.seq[: 64 << 12])  # the blocks' leading bases
    assert kw["k"] == 4 and kw["lanes_per_block"] == 64
    name = bench.workload_name("plain", w, kw)
    assert "262144 bases" in name and "64 blocks" in name and "(s,k)=(2,4)" in name


def test_job_throughput_is_whole_job():
    assert bench.job_throughput(4, 1 << 24, 1000.0) == pytest.approx(4 * (1 << 24) / 1e6)


def test_reference_arm_runs_the_oracle_alone(monkeypatch, capsys):
    """--impl reference times the oracle on the host cores and loads nothing of the library."""
    import json
    import sys
    monkeypatch.delitem(sys.modules, "paper_2507_12805_gb300", raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "plain", "--steps", "1",
                                      "--warmup", "0", "--block-bases", "2048"])
    bench.main()
    assert "paper_2507_12805_gb300" not in sys.modules
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "MB/s"
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "MB/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "1024 bases" in line["cpu_baseline"]["sample"]
    # the same config object the GPU arm prints: the workload and the L2 policy, no model keys
    w, kw = bench.load_workload("plain", 2048)
    assert line["config"] == bench.bench_config("plain", w, kw)
    assert set(line["config"]) == {"workload", "l2"} and line["details"]["model"] == kw


def test_throttle_detection():
    assert not bench.throttled({"reasons": []})
    assert not bench.throttled({"reasons": ["sw_power_cap"]})
    assert not bench.throttled({"reasons": ["unsampled"]})
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.throttled({"reasons": ["sw_power_cap", r]})


def test_autotune_candidates_start_at_the_plain_forms_lanes():
    _, kw = bench.load_workload("plain", 1 << 12)
    assert bench.lane_candidates(kw)[0] == kw["lanes_per_block"] == 64
    assert bench.lane_candidates(dict(bench.WORKLOADS["human"][1]))[0] == 128
