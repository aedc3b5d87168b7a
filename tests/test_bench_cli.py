"""The benchmark's command line on CPU.  The reference arm (the oracle timed on
a bounded sample) prints exactly one JSON line with every key the contract
names; under a two-rank launch only rank 0 prints it and the other rank exits
0 without work.  The CUDA arm and the binding refuse to run without a device
instead of falling back to anything."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--impl", "reference", "--steps", "1", "--warmup", "3", "--cpu-log2n", "14"]


def _run(cmd, env=None, timeout=300):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=e)


def _json_lines(out: str):
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_reference_arm_prints_one_contract_line():
    r = _run([sys.executable, "bench.py", *SMALL])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "Gkeys/s" and d["higher_is_better"] is True
    assert d["dtype"] == "u32" and d["data"] == "synthetic" and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_names_the_duplicate_workload():
    r = _run([sys.executable, "bench.py", *SMALL, "--dup", "8"])
    assert r.returncode == 0, r.stderr[-2000:]
    (d,) = _json_lines(r.stdout)
    assert "[1 .. N/8]" in d["config"]["workload"]


def test_reference_arm_two_ranks_rank0_prints():
    port = _free_port()
    r = _run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
              "--master-addr=127.0.0.1", f"--master-port={port}", "bench.py", *SMALL, "--gpus", "2"],
             env={"OMP_NUM_THREADS": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def test_cuda_arm_fails_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    r = _run([sys.executable, "bench.py", "--steps", "1", "--warmup", "3", "--log2n", "12", "--no-cpu-baseline"])
    assert r.returncode != 0
    assert _json_lines(r.stdout) == []


def test_binding_rejects_host_tensors():
    import torch
    import paper_1907_02900_gb300 as hg
    with pytest.raises(ValueError):
        hg.build(torch.arange(10, dtype=torch.int32).view(torch.uint32), 16)
