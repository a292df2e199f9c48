"""Host logic of bench.py that needs no GPU: the clock-record summary and
the gate that reports recorded ncu traffic only for the kernel source it was
measured on."""
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))
import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons():
    rows = [
        "0, 2070 MHz, 2070 MHz, 900.10 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055 MHz, 2070 MHz, 1390.00 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2040 MHz, 2070 MHz, 1398.50 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070 MHz, 1.0 W, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = bench.parse_clock_samples(rows)
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = rows[:1] + ["0, 1500 MHz, 2070 MHz, 1.0 W, 0x8, Active, Not Active, Active, Not Active"]
    assert bench.parse_clock_samples(hot)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.parse_clock_samples(["nothing here"]) is None


def test_recorded_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2506_09242_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "lbm_kernels.cuh").write_text("// kernel v1\n")
    (csrc / "lbm_internal.cuh").write_text("// internals\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    h = bench.kernel_source_hash()
    (tmp_path / "profiles" / "k.md").write_text(
        f"workload: tgv3d_64_d3q19_f32\ntraffic_bytes_per_launch: 1.5e9\nkernel_source_sha256_16: {h}\n")
    assert bench.recorded_traffic("tgv3d_64_d3q19_f32") == 1.5e9
    assert bench.recorded_traffic("tgv3d_128_d3q19_f32") is None
    (csrc / "lbm_kernels.cuh").write_text("// kernel v2\n")
    assert bench.recorded_traffic("tgv3d_64_d3q19_f32") is None


def test_clock_sampler_runs_a_sampling_process(tmp_path, monkeypatch):
    """start/stop around a stand-in nvidia-smi that prints two rows and
    waits: the rows are parsed and the temporary record is removed."""
    import os
    import time

    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 2070 MHz, 2070 MHz, 800.00 W, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 2040 MHz, 2070 MHz, 1390.00 W, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    s = bench.ClockSampler(0)
    s.start()
    assert s.proc is not None
    time.sleep(0.5)
    summary = s.stop()
    assert summary == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}
    assert not os.path.exists(s.path)


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    import os
    monkeypatch.setenv("PATH", str(tmp_path))  # an empty directory: no nvidia-smi
    s = bench.ClockSampler(0)
    s.start()
    assert s.proc is None and not os.path.exists(s.path)
    assert s.stop() is None


def test_cpu_baseline_reports_cores_per_core_rate_and_host(monkeypatch):
    """The CPU baseline times the oracle on every host core and on one, and
    reports the threads used, a per-core rate and the host it ran on (here on
    tiny lattices)."""
    monkeypatch.setitem(bench.CPU_PLANS, "tiny", [(19, 256, 0, 1, 1, 2), (27, 12, 1, 1, 2, 2)])
    monkeypatch.setattr(bench, "tgv_tau", lambda n, u0, re: 0.6)
    import lbm_inputs as inp
    monkeypatch.setattr(inp, "tgv3d", lambda n, u0, _real=inp.tgv3d: _real(12 if n == 256 else n, u0))
    import oracle
    calls = []
    real_problem = oracle.Problem

    def small_problem(Q, nx, ny, nz, *a, **k):
        calls.append((Q, nx, k.get("openmp")))
        m = 12 if nx == 256 else nx
        return real_problem(Q, m, m, m, *a, **k)
    monkeypatch.setattr(oracle, "Problem", small_problem)
    cb = bench.cpu_baseline("tiny")
    assert cb["kind"] == "oracle" and cb["unit"] == "GLUPS"
    import os
    assert cb["cores"] == os.cpu_count()
    assert cb["value"] > 0 and abs(cb["per_core"] * cb["cores"] - cb["value"]) < 1e-12 * cb["value"] + 1e-15
    assert set(cb["host"]) == {"nproc", "cpu_model", "arch"} and cb["host"]["nproc"] >= 1
    assert [r["threads"] for r in cb["table"]][1] == 1
    assert all(openmp for _, _, openmp in calls)
