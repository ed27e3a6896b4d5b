"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps
the one-JSON-line contract, alone and under torchrun with two ranks (rank 0
prints, the other exits without work).  CPU only: the small FP64 Toeplitz
workload (n = 2000)."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--workload", "toeplitz2k", "--steps", "1", "--warmup", "0"]
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check(line, n_gpus, workload="toeplitz2k"):
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["n_gpus"] == n_gpus
    assert line["metric"] == "HSS compress s" and line["unit"] == "s"
    assert line["higher_is_better"] is False and line["value"] > 0
    assert line["config"]["workload"] == workload
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == "s"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def _env():
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    return env


def test_reference_arm_prints_one_line():
    r = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, env=_env(),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0], 1)


def test_reference_arm_under_torchrun_two_ranks():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(port), "bench.py", *ARGS, "--gpus", "2"],
                       cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0], 2)


def test_reference_arm_of_the_matvec_and_solve_workload():
    """ops80k (HSS matvec and ULV solve of QChemToeplitz): the oracle's
    compress + factor + solve on a bounded sample, in the same line format."""
    args = ["--impl", "reference", "--workload", "ops80k", "--steps", "1", "--warmup", "0"]
    r = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, env=_env(),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check(lines[0], 1, "ops80k")
