"""bench.py --impl reference (the oracle timed on the host cores) keeps the
JSON-line contract on CPU, alone and under torchrun with two ranks (rank 0
alone runs and prints; the other rank exits 0 without work)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--workload", "l3_nt8", "--steps", "1", "--warmup", "0",
        "--cpu-sample-s", "0.2"]


def json_lines(text):
    return [json.loads(s) for s in text.splitlines() if s.startswith("{")]


def check_line(line, n_gpus):
    assert line["impl"] == "reference"
    assert line["unit"] == "trajectories/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["n_gpus"] == n_gpus and line["steps"] == 1
    assert line["config"]["workload"] == "l3_nt8"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_one_process():
    r = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    check_line(lines[0], 1)


def test_reference_arm_under_torchrun_two_ranks():
    port = 29600 + os.getpid() % 1000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2",
           *ARGS]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1                      # rank 0 only
    check_line(lines[0], 2)


def test_reference_arm_apply_mode():
    """--mode apply: the oracle's M-applications/s on the workload's lattice."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--mode", "apply",
                        "--workload", "l3_nt8", "--steps", "1", "--warmup", "0",
                        "--cpu-sample-s", "0.2"], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    (line,) = json_lines(r.stdout)
    assert line["impl"] == "reference" and line["unit"] == "M-applications/s"
    assert line["value"] > 0 and line["config"]["mode"] == "apply"
    assert line["cpu_baseline"]["unit"] == "M-applications/s"
