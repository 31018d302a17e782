"""bench.py's host-side parts on CPU: the reference arm (the oracle timed on
the host cores, on the full instance of the workload it names, here 40^3)
prints one JSON line with the contract's keys and the steps it ran, from rank 0
only when launched as two ranks with torch.distributed.run (the other rank
exits 0 without work); the clock sampler parses nvidia-smi's samples (a
stand-in script here)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_two_ranks_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3", "--grid", "40"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["ms_per_step"] == d["value"] and d["n_gpus"] == 2
    assert d["steps"] == 2 and d["steps_requested"] == 2 and d["warmup"] == 3
    assert d["timed_wall_ms"] >= d["steps"] * d["ms_per_step"] * 0.999
    assert d["config"]["workload"].startswith("poisson3d_40^3")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["host_cores"] >= 1 and "not scaled" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_clock_sampler_parses_smi_samples(tmp_path, monkeypatch):
    # a stand-in nvidia-smi on PATH prints three samples, one of them with a
    # power-cap reason active; the sampler reports their median and maximum
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 1965, 2070, 900.5, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 2070, 2070, 940.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    sys.path.insert(0, ROOT)
    import bench
    import time
    with bench.ClockSampler(0) as clk:
        time.sleep(1.0)
    s = clk.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not os.path.exists(clk.path)
