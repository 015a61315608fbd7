"""bench.py host logic on CPU: the reference arm (the FP64 oracle on the
host cores) prints one JSON line with the contract's keys, a non-zero rank
prints nothing, and the profiled-traffic lookup is keyed by the kernel
source without its comments.  No GPU is touched."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    p = _run(["--impl", "reference", "--workload", "sphere40", "--steps", "3", "--warmup", "1"])
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["steps"] == 3 and d["warmup"] == 1 and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "3 of the 3 requested" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_print_nothing():
    p = _run(["--impl", "reference", "--workload", "sphere40", "--steps", "1", "--warmup", "1"], {"RANK": "1"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_traffic_lookup_ignores_comments(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    csrc = tmp_path / "paper_1312_3426_gb300" / "csrc"
    csrc.mkdir(parents=True)
    code = "int f(int x) {\n    return x + 1;\n}\n"
    (csrc / "fluid_core.cuh").write_text("// header\n" + code)
    (csrc / "fluid.cu").write_text(code)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    (csrc / "fluid_core.cuh").write_text("// another header\n\n" + code.replace("+ 1;", "+ 1;  // add one"))
    assert bench.kernel_source_hash() == h0
    (csrc / "fluid.cu").write_text(code.replace("+ 1", "+ 2"))
    assert bench.kernel_source_hash() != h0
    prof = tmp_path / "profiles"
    prof.mkdir()
    h1 = bench.kernel_source_hash()
    (prof / "k_fluid_dram_traffic.md").write_text(
        f"traffic: workload=rbc256 precision=f32 source_hash={h1} dram_bytes_per_cell=150.0\n"
        f"traffic: workload=rbc256 precision=f16s source_hash={h0} dram_bytes_per_cell=75.0\n")
    assert bench.profiled_traffic("rbc256", "f32", 10) == 1500
    assert bench.profiled_traffic("rbc256", "f16s", 10) is None   # taken on other code
    assert bench.profiled_traffic("rbc512", "f32", 10) is None


def test_clock_sampler_with_a_fake_nvidia_smi(tmp_path, monkeypatch):
    """The sampler's parse of `nvidia-smi --query-gpu` lines: median SM clock,
    max clock, active throttle reasons, only the GPU asked for; its temporary
    file is removed."""
    sys.path.insert(0, ROOT)
    import bench
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo 'GPU-aaa, 1980, 2070, 900.1, Not Active, Not Active, Not Active, Active'\n"
                    "echo 'GPU-aaa, 2070, 2070, 910.2, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo 'GPU-aaa, 2070, 2070, 905.0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo 'GPU-bbb, 300, 2070, 100.0, Active, Not Active, Not Active, Not Active'\n"
                    "echo 'garbage line'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    c = bench.ClockSampler("GPU-aaa")
    c.start()
    out = c.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(c.path)


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(None)
    c.start()
    assert c.stop() is None
    assert c.path is None or not os.path.exists(c.path)


def test_e2e_record_keys():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.e2e_record(4_000_000, 100, 0.02, 0.025, 1, 200)
    assert set(r) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert r["unit"] == "MLUPS" and r["h2d_bytes_per_step"] == 2400 and r["d2h_bytes_per_step"] == 22404
    assert r["value"] == round(bench.whole_job_mlups(4_000_000, 100, 20.0, 1), 2)
    assert r["synchronous_value"] < r["value"]


def test_profile_sampling_gives_eight_fluid_launches():
    """The per-kernel events sample every n-th step with n = steps / 8 (at
    most 16): the fluid kernel's mean rests on at least 8 launches from 8
    steps on, whatever step count the timed region starts at."""
    sys.path.insert(0, ROOT)
    import bench
    for steps in (8, 10, 20, 64, 127, 128, 129, 1000, 4000):
        n = bench.profile_every(steps)
        assert 1 <= n <= 16
        for start in range(n):
            sampled = sum(1 for t in range(start, start + steps) if t % n == 0)
            assert sampled >= 8, (steps, n, start, sampled)
    assert bench.profile_every(4000) == 16 and bench.profile_every(20) == 2


def test_poiseuille_reference_profile_is_readable():
    """The bench's Poiseuille reference is the committed oracle profile:
    256 values, zero at the walls, peak near 0.184."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    u = np.loadtxt(bench.GOLDEN_PROFILE)
    assert u.shape == (256,) and u[0] == 0.0 and u[-1] == 0.0
    assert 0.18 < u.max() < 0.19
