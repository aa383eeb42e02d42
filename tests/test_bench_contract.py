"""bench.py's command-line contract, on the CPU.

- The reference arm (the FP64 oracle on the host) prints one JSON line with
  the contract's keys.  Under torchrun with two ranks only rank 0 prints it,
  and both ranks exit 0.
- Our arm has no CPU path: without a CUDA device it exits non-zero with a
  message and prints no result line.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"}


def _json_lines(text):
    out = []
    for line in text.splitlines():
        line = line.strip()
        if line.startswith("{"):
            out.append(json.loads(line))
    return out


def _check_reference_line(line, steps, warmup, gpus):
    assert KEYS <= set(line), KEYS - set(line)
    assert line["impl"] == "reference" and line["metric"] == "MLUPS" and line["unit"] == "MLUPS"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["dtype"] == "f64"
    assert (line["steps"], line["warmup"], line["n_gpus"]) == (steps, warmup, gpus)
    assert line["vs_baseline"] is None and line["data"] == "synthetic"
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    assert cb["cpu"] and cb["host_cores"] >= 1
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, BENCH, "--impl", "reference", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 2, 1, 1)


def test_reference_arm_under_torchrun_prints_on_rank_0_only():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port), BENCH, "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1
    _check_reference_line(lines[0], 1, 1, 2)


def test_our_arm_has_no_cpu_path():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    out = subprocess.run([sys.executable, BENCH, "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode != 0
    assert "no CUDA device" in out.stderr
    assert not _json_lines(out.stdout)


def test_dram_traffic_entries_describe_the_current_kernels():
    """Each DRAM-traffic factor bench.py reports (from a committed ncu capture)
    is tagged with the hash of the kernel sources it was measured on; a stale
    tag would silently drop `roofline.traffic`, so every tag must match the
    sources as they stand, and each entry must name a committed profile."""
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    sha = bench.kernel_source_sha()
    src = open(BENCH).read()
    for key, entry in bench.NCU_TRAFFIC.items():
        assert entry["src_sha"] == sha, (key, entry["src_sha"], sha)
        assert 0.8 < entry["dram_per_alg_byte"] < 1.2, key
    for name in ("k_bulk_batch_fp32_sweep320_launches.md", "k_bulk_batch_fp16_sweep_half_full.md",
                 "k_bulk_fp32_pipe4096x8192_launches.md"):
        assert name in src and os.path.exists(os.path.join(ROOT, "profiles", name)), name
