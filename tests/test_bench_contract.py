"""bench.py's reference arm runs on the host (the FP64 oracle): its JSON line
keeps the contract's keys, for the sampling and the gradient workloads."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--cpu-budget", "2",
                        *args], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("workload,unit", [("n12", "samples/s"), ("grad3reg", "gradients/s")])
def test_reference_arm_line(workload, unit):
    if workload == "grad3reg":
        import paper_2510_24218_gb300 as mod
        from paper_2510_24218_gb300 import build as B
        if not os.path.exists(mod.library_path()):
            B.build()
    d = _run("--workload", workload, "--steps", "2", "--warmup", "1")
    assert d["impl"] == "reference" and d["unit"] == unit and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1
    for key in ("metric", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "vs_baseline", "dtype",
                "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    if workload == "n12":
        # the steps were run (a bounded sample each), and the config is the GPU arm's
        sys.path.insert(0, ROOT)
        import argparse
        import bench
        assert d["chains_timed"] >= 2 and d["extrapolated"] is False
        ns = argparse.Namespace(workload="n12", samples=0, precision="fp64")
        assert d["config"] == bench.workload_config(ns, 1)


def test_profiled_traffic_follows_the_kernel_sources(monkeypatch):
    """roofline.traffic comes from a profile summary only while the kernel
    sources hash to the captured value and the launch has the captured size."""
    sys.path.insert(0, ROOT)
    import bench
    text = open(os.path.join(ROOT, "profiles", bench.PROFILE_OF["grid6x6"])).read()
    captured = text.split("kernel-sources-sha256:")[1].split()[0]
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda *a: captured)
    assert bench.profiled_traffic("grid6x6", 4096) > 0
    assert bench.profiled_traffic("grid6x6", 4095) is None
    assert bench.profiled_traffic("n12", 256) is None            # no FP32 summary mapped
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda *a: "0" * 64)
    assert bench.profiled_traffic("grid6x6", 4096) is None


def test_dense_pass_traffic_scales_with_the_timed_launches(monkeypatch, tmp_path):
    """The dense passes' summary gives DRAM bytes per algorithmic byte; the
    bench scales it to the algorithmic bytes of its own launches, and drops
    it when the dense sources no longer hash to the captured value."""
    sys.path.insert(0, ROOT)
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "d.md").write_text(
        "    kernel-sources-sha256: abc\n    dram-bytes-per-algorithmic-byte: 1.25\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "PROFILE_OF", {"w_hbm": "d.md"})
    seen = []
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda files=bench.KERNEL_SOURCES: seen.append(files) or "abc")
    assert bench.profiled_traffic("w_hbm", 8192, 1000.0) == 1250.0
    assert seen[-1] == bench.DENSE_SOURCES
    assert bench.profiled_traffic("w_hbm", 8192, None) is None
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda files=None: "def")
    assert bench.profiled_traffic("w_hbm", 8192, 1000.0) is None
